"""The opt-in convergence check of the mass solve (felbm_solver_check).

The solve runs a fixed number of steps; with the check on, each time step
also measures ||b - M x|| / ||b|| before the last step of its solve.  These
tests run through the C ABI: the check leaves the trajectory bit for bit as
it is, reports a small residual for the default step counts, and flags a solve
capped at two steps as not converged -- a failure made on the host through
the step-count parameter, with no fault on the GPU.
"""
import math

import numpy as np
import pytest

from paper_1708_04678_gb300 import felbm as F
from paper_1708_04678_gb300 import inputs as I
from parity_util import gpu_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_04678_gb300 import build
    build.build()


def _w():
    return I.small_sessile(nx=40, ny=20, R=9.0, theta=60.0)


@pytest.mark.parametrize("precision,bound", [(F.FP64, 1e-9), (F.FP32_DEV, 5e-3)])
def test_check_reports_a_small_residual_and_leaves_the_trajectory(precision, bound):
    w = _w()
    a = gpu_state(w, precision=precision)
    b = gpu_state(w, precision=precision)
    b.solver_check(True, 1e-2)
    a.step(25)
    b.step(25)
    ga, ha = a.get_state()
    gb, hb = b.get_state()
    np.testing.assert_array_equal(ga, gb)
    np.testing.assert_array_equal(ha, hb)
    d = b.diagnostics()
    assert d["status"] == 0
    assert d["solver_sweeps"] == (14 * 3 if precision == F.FP64 else 10)
    assert 0.0 < d["solver_residual"] < bound, d["solver_residual"]
    assert math.isnan(a.diagnostics()["solver_residual"])


def test_capped_solve_is_reported_not_converged():
    w = _w()
    st = gpu_state(w, precision=F.FP32_DEV, solver_iters=2)
    st.solver_check(True, 1e-6)
    st.step(3)
    d = st.diagnostics()
    assert d["status"] == -7 and d["solver_residual"] > 1e-6, d
    slots = np.zeros(F.DIAG_SLOTS)
    st.diagnostics_enqueue(slots)
    st.stream.synchronize()
    assert st.diag_finish(slots)["status"] == -7
    with pytest.raises(F.FelbmError) as e:
        F._check(F.lib().felbm_solver_check(st.handle, 1, -1.0))
    assert e.value.code == -1
    st.solver_check(False)
    st.step(1)
    d = st.diagnostics()
    assert d["status"] == 0 and math.isnan(d["solver_residual"])


def test_check_is_unsupported_for_the_fp64_solver_mode():
    st = gpu_state(_w(), solver_mode=F.SOLVER_FP64)
    with pytest.raises(F.FelbmError) as e:
        st.solver_check(True, 1e-6)
    assert e.value.code == -6
