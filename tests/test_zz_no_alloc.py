"""felbm_mass_solve_static: the mass solve for callers that cannot allocate.

Some callers must not allocate device memory at the point where they solve
(a plugin whose host application owns all device memory, a section that must
not synchronise) and cannot lend the state's workspace because a time step
may be using it.  The static entry point keeps its iterates in a
library-owned static device array instead.  This file checks, through the C
ABI, that it returns what the ordinary workspace-backed solve returns, on two
calls in a row (the array keeps the previous call's contents), for a full and
a partial set of right-hand sides, and that a mesh too large for the array is
refused before anything runs.  It is collected last so that a failure here
cannot stop the other GPU tests.
"""
import numpy as np
import pytest

from paper_1708_04678_gb300 import felbm as F
from paper_1708_04678_gb300 import inputs as I
from parity_util import gpu_state, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_04678_gb300 import build
    build.build()


@pytest.mark.parametrize("mode", [F.SOLVER_MIXED, F.SOLVER_FP64])
def test_static_solve_matches_workspace_solve(mode):
    import torch
    w = I.sessile_droplet_64x32()
    gst = gpu_state(w, solver_mode=mode)
    rng = np.random.default_rng(7)
    for k in (18, 5):
        B = rng.standard_normal((k, gst.N))
        X_ref = gst.mass_solve(B)                       # workspace scratch, host buffers
        d_B = torch.from_numpy(B).cuda()
        for call in range(2):                           # the array keeps the last call's contents
            d_X = torch.full_like(d_B, float("nan"))
            gst.mass_solve_static(d_B, d_X)
            torch.cuda.synchronize()
            X = d_X.cpu().numpy()
            for q in range(k):
                assert rel_err(X[q], X_ref[q]) < 1e-13, (k, call, q)


def test_static_solve_rejects_meshes_beyond_its_array():
    import torch
    w = I.free_droplet_256()                            # 131,072 nodes > ~103,000
    gst = gpu_state(w)
    d_B = torch.zeros((1, gst.N), dtype=torch.float64, device="cuda")
    d_X = torch.zeros_like(d_B)
    with pytest.raises(F.FelbmError) as e:
        gst.mass_solve_static(d_B, d_X)
    assert e.value.code == -4 and "static array" in str(e.value)


def test_static_solve_overlapping_another_states_steps():
    """Static solves of one state on its stream while another state takes
    time steps on a second stream: neither touches the other's memory, so
    both results are bit for bit those of the same work run one after the
    other."""
    import torch
    w = I.sessile_droplet_64x32()
    s_step, s_solve = torch.cuda.Stream(), torch.cuda.Stream()
    a = gpu_state(w, stream=s_step)                     # takes the steps
    b = gpu_state(w, stream=s_solve)                    # runs the static solves
    ref = gpu_state(w)
    ref.step(40)
    g_ref, h_ref = ref.get_state()
    rng = np.random.default_rng(11)
    B = torch.from_numpy(rng.standard_normal((18, b.N))).cuda()
    X_ref = torch.empty_like(B)
    b.mass_solve_static(B, X_ref)
    torch.cuda.synchronize()
    X = [torch.full_like(B, float("nan")) for _ in range(8)]
    torch.cuda.synchronize()
    a.step(40)                                          # queued on s_step
    for k in range(8):                                  # queued on s_solve meanwhile, one after another
        b.mass_solve_static(B, X[k])
    torch.cuda.synchronize()
    g, h = a.get_state()
    np.testing.assert_array_equal(g, g_ref)
    np.testing.assert_array_equal(h, h_ref)
    for k in range(8):
        assert torch.equal(X[k], X_ref), k
