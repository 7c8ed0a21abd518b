"""3D path (D3Q19 on tetrahedra) against the 3D FP64 oracle.

FP64 storage: g, h and C agree with the oracle to a max relative error of
1e-11 after the run, for both solvers, both patch-Laplacian modes, walled
and periodic meshes, at sizes spanning many thread blocks with a ragged
tail.  FP32-deviation storage: FP32-level agreement on short runs and the
method's own measures (mass drift, contact angle) on long runs.  The
262,144-node static droplet, too large for the oracle's global matrices, is
held to the properties that hold at any size.
"""
import math

import numpy as np
import pytest

from oracle.felbm_oracle3d import OracleMesh3D, OracleSim3D, params_from_physical3d
from paper_1708_04678_gb300 import felbm as F
from paper_1708_04678_gb300 import felbm3d as F3
from paper_1708_04678_gb300 import inputs3d as I3

pytestmark = pytest.mark.gpu

LAP = {"consistent": F.LAP_CONSISTENT, "paper": F.LAP_PAPER}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_04678_gb300 import build
    build.build()


def rel_err(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


def oracle3d(w, lap="consistent"):
    m = w["mesh"]
    om = OracleMesh3D(m["xyz"], m["tet"], m["wall_faces"], m["wall_id"], m["period"])
    return OracleSim3D(om, params_from_physical3d(w["phys"], lap), w["C0"])


def gpu3d(w, lap="consistent", precision=F.FP64, solver_mode=F.SOLVER_MIXED, iters=0):
    prm = F.params_derive(w["phys"], LAP[lap], solver_iters=iters, precision=precision, solver_mode=solver_mode)
    return F3.State3D(F3.Mesh3D.from_dict(w["mesh"]), prm, w["C0"])


def compare(osim, st):
    g, h = st.get_state()
    return {"g": rel_err(g, osim.g), "h": rel_err(h, osim.h), "C": rel_err(h.sum(0), osim.h.sum(0))}


CASES = {
    "sessile60": lambda: I3.small_sessile_3d(),
    "sessile120": lambda: I3.small_sessile_3d(n=12, nz=7, R=4.5, seed=12, theta=120.0),
    "free": lambda: I3.small_free_droplet_3d(),
    "free_ratio10": lambda: I3.small_free_droplet_3d(n=11, R=3.5, seed=13, rho_v=0.1),
}


def test_fields_after_init():
    w = CASES["sessile60"]()
    st = gpu3d(w)
    f = st.get_fields()
    assert rel_err(f["C"], w["C0"]) < 1e-15
    assert np.abs(f["p"]).max() == 0.0 and np.abs(f["ux"]).max() == 0.0
    g, h = st.get_state()
    osim = oracle3d(w)
    assert rel_err(h, osim.h) < 1e-15 and np.abs(g).max() == 0.0


@pytest.mark.parametrize("name", sorted(CASES))
def test_single_step(name):
    w = CASES[name]()
    osim, st = oracle3d(w), gpu3d(w)
    osim.step(1)
    st.step(1)
    err = compare(osim, st)
    assert max(err.values()) < 1e-12, err


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("mode", [F.SOLVER_MIXED, F.SOLVER_FP64])
def test_multi_step(name, mode):
    w = CASES[name]()
    osim, st = oracle3d(w), gpu3d(w, solver_mode=mode)
    osim.step(20)
    st.step(20)
    err = compare(osim, st)
    assert max(err.values()) < 1e-11, err


def test_paper_laplacian_mode():
    w = CASES["sessile60"]()
    osim, st = oracle3d(w, "paper"), gpu3d(w, "paper")
    osim.step(10)
    st.step(10)
    err = compare(osim, st)
    assert max(err.values()) < 1e-11, err


def test_ragged_mid_size_periodic():
    """15^3 periodic mesh (3,375 nodes, 20,250 tetrahedra): many blocks and a
    ragged last block in every kernel."""
    w = I3.small_free_droplet_3d(n=15, R=4.5, seed=14)
    osim, st = oracle3d(w), gpu3d(w)
    osim.step(5)
    st.step(5)
    err = compare(osim, st)
    assert max(err.values()) < 1e-11, err


def test_diagnostics_match_oracle():
    w = CASES["sessile60"]()
    osim, st = oracle3d(w), gpu3d(w)
    osim.step(15)
    st.step(15)
    do = osim.diagnostics(w["centre"], w["R"], 2.0, substrate=0)
    dg = st.diagnostics(w["centre"], w["R"], 2.0, substrate=0)
    assert dg["status"] == 0 and dg["step"] == 15
    for k in ("mass", "kinetic_energy", "max_u", "p_in", "p_out", "interface_rho_uu", "wetted_area",
              "height", "base_diameter", "theta_deg"):
        assert math.isclose(dg[k], do[k], rel_tol=1e-9, abs_tol=1e-14), (k, dg[k], do[k])
    assert abs(dg["mass_drift_rel"]) < 1e-13


def test_state_roundtrip_and_determinism():
    w = CASES["free"]()
    a, b = gpu3d(w), gpu3d(w)
    a.step(7)
    g, h = a.get_state()
    b.set_state(g, h)
    g2, h2 = b.get_state()
    np.testing.assert_array_equal(g, g2)
    np.testing.assert_array_equal(h, h2)
    a.step(5)
    b.step(5)
    ga, ha = a.get_state()
    gb, hb = b.get_state()
    np.testing.assert_array_equal(ga, gb)
    np.testing.assert_array_equal(ha, hb)


def test_timing_and_launch_count():
    w = CASES["free"]()
    st = gpu3d(w)
    st.timing_enable(True)
    st.step(1)
    t = st.timing_get()
    assert t["total_ms"] > 0 and all(v >= 0 for v in t.values())
    assert st.launches() == 5 + 3 * 15 + 2


# ------------------------------------------------------------ FP32 dev ----
@pytest.mark.parametrize("name", ["sessile60", "free_ratio10"])
def test_fp32_dev_matches_oracle_at_fp32_level(name):
    w = CASES[name]()
    osim, st = oracle3d(w), gpu3d(w, precision=F.FP32_DEV)
    osim.step(20)
    st.step(20)
    err = compare(osim, st)
    assert err["C"] < 1e-6, err
    assert err["h"] < 1e-5 and err["g"] < 1e-3, err


def test_fp32_dev_state_roundtrip():
    w = CASES["sessile60"]()
    a = gpu3d(w)
    a.step(10)
    g, h = a.get_state()
    b = gpu3d(w, precision=F.FP32_DEV)
    b.set_state(g, h)
    g2, h2 = b.get_state()
    assert rel_err(h2, h) < 1e-6 and rel_err(g2, g) < 1e-5
    assert rel_err(b.get_fields()["C"], h.sum(0)) < 1e-14


# ------------------------------------------------------- full size (64^3) ----
def test_static_droplet_64_properties():
    """262k nodes / 1.57M tetrahedra: FP64 mass conservation to round-off,
    FP32-deviation storage within 1e-6 mass drift and close to FP64 on the
    spurious-current and Laplace-pressure measures after 200 steps."""
    w = I3.static_droplet_64()
    a = gpu3d(w)
    b = gpu3d(w, precision=F.FP32_DEV)
    a.step(200)
    b.step(200)
    da = a.diagnostics(w["centre"], w["R"], w["phys"]["xi"], substrate=-1)
    db = b.diagnostics(w["centre"], w["R"], w["phys"]["xi"], substrate=-1)
    assert da["status"] == 0 and db["status"] == 0
    assert abs(da["mass_drift_rel"]) < 1e-12
    assert abs(db["mass_drift_rel"]) < 1e-6
    assert math.isclose(da["delta_p"], db["delta_p"], rel_tol=0.02)
    assert math.isclose(da["max_u"], db["max_u"], rel_tol=0.05, abs_tol=1e-6)


@pytest.mark.parametrize("precision", [F.FP64, F.FP32_DEV])
def test_pipelined_inputs_and_async_diagnostics(precision):
    """As in 2D: distinct states streamed through one pinned host buffer pair
    that is overwritten as soon as set_state returns, a step each, and the
    diagnostics queued with felbm3d_diagnostics_enqueue and finished after one
    synchronisation give, bit for bit, the synchronous sequence's results."""
    import torch
    w = CASES["sessile60"]()
    src = gpu3d(w, precision=precision)
    states = []
    for _ in range(5):
        src.step(3)
        states.append(src.get_state())
    req = dict(centre=w["centre"], radius=w["R"], band=2.0, substrate=0)

    a = gpu3d(w, precision=precision)
    seq = []
    for g, h in states:
        a.set_state(g, h)
        a.step(2)
        seq.append(a.diagnostics(**req))
    ga, ha = a.get_state()

    b = gpu3d(w, precision=precision)
    gp = torch.empty(states[0][0].shape, dtype=torch.float64).pin_memory()
    hp = torch.empty(states[0][1].shape, dtype=torch.float64).pin_memory()
    slots = torch.zeros((len(states), F.DIAG_SLOTS), dtype=torch.float64).pin_memory()
    for k, (g, h) in enumerate(states):
        gp.copy_(torch.from_numpy(g))
        hp.copy_(torch.from_numpy(h))
        b.set_state(gp, hp)
        gp.fill_(float("nan"))
        hp.fill_(float("nan"))
        b.step(2)
        b.diagnostics_enqueue(slots[k], **req)
    torch.cuda.synchronize()
    pip = [b.diag_finish(slots[k], **req) for k in range(len(states))]
    for d1, d2 in zip(pip, seq):
        assert d1.keys() == d2.keys()
        for key in d1:
            v1, v2 = d1[key], d2[key]
            assert v1 == v2 or (math.isnan(v1) and math.isnan(v2)), (key, v1, v2)
    assert all(d["status"] == 0 for d in pip)
    gb, hb = b.get_state()
    np.testing.assert_array_equal(ga, gb)
    np.testing.assert_array_equal(ha, hb)
