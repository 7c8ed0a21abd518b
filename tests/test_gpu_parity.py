"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Tolerance: the FP64 path must match the oracle to a maximum relative error of
1e-11 in g, h and C after the run (normwise, see parity_util.rel_err).
Single operators are held to tighter bounds.  Sizes span many thread blocks
with ragged tails (node and triangle counts are not multiples of the block
sizes), the smallest legal mesh (two triangles), walls with wetting, periodic
meshes and the body-fitted rough wall; the 131,072-node free droplet is run
at full size in the same launch configuration the benchmark times.
"""
import math

import numpy as np
import pytest

from paper_1708_04678_gb300 import felbm as F
from paper_1708_04678_gb300 import inputs as I
from parity_util import compare_states, elementwise_c_err, gpu_state, oracle_sim, rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_04678_gb300 import build
    build.build()


def _rough_small(theta=60.0):
    return I.rough_wall_droplet(width=192, height=64, rows=49, R=20.0, theta=theta, steps=50)


@pytest.mark.parametrize("mode", [F.SOLVER_MIXED, F.SOLVER_FP64])
def test_mass_solve_matches_oracle_pcg(mode):
    w = I.sessile_droplet_64x32()
    osim = oracle_sim(w)
    gst = gpu_state(w, solver_mode=mode)
    rng = np.random.default_rng(0)
    B = rng.standard_normal((18, gst.N))
    X = gst.mass_solve(B)
    Xo = osim.solve_mass(B.T).T
    for k in range(18):
        assert rel_err(X[k], Xo[k]) < 1e-13
    X5 = gst.mass_solve(B[:5])
    np.testing.assert_array_equal(X5, X[:5])


@pytest.mark.parametrize("lap", ["consistent", "paper"])
def test_fields_after_init(lap):
    w = I.small_sessile(nx=40, ny=20, R=9.0, theta=60.0)
    osim = oracle_sim(w, lap)
    gst = gpu_state(w, lap)
    f = gst.get_fields()
    C, p, u, rho = osim.moments()
    mu = osim.chemical_potential(C)
    assert rel_err(f["C"], C) < 1e-15
    assert rel_err(f["mu"], mu) < 1e-13


WORKLOADS = {
    "sessile60": lambda: I.small_sessile(nx=40, ny=20, R=9.0, theta=60.0),
    "sessile120_paper": lambda: I.small_sessile(nx=36, ny=18, R=8.0, theta=120.0),
    "free_droplet": lambda: I.small_free_droplet(n=24, R=6.0),
    "rough_wall": _rough_small,
    # internal walls with re-entrant corners (a block with a channel through it)
    "channel": lambda: I.capillary_channel(H=6, length_factor=6, reservoir=2, theta=56.0, l0_factor=1.0,
                                           liquid_factor=1.5, dt=0.1, xi=2.0),
}


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_single_step(name):
    w = WORKLOADS[name]()
    lap = "paper" if name.endswith("paper") else "consistent"
    osim = oracle_sim(w, lap)
    gst = gpu_state(w, lap)
    osim.step(1)
    gst.step(1)
    err = compare_states(osim, gst)
    assert max(err.values()) < 1e-13, err


@pytest.mark.parametrize("name,steps", [("sessile60", 300), ("free_droplet", 300),
                                        ("rough_wall", 150), ("sessile120_paper", 200), ("channel", 150)])
def test_multi_step(name, steps):
    w = WORKLOADS[name]()
    lap = "paper" if name.endswith("paper") else "consistent"
    osim = oracle_sim(w, lap)
    gst = gpu_state(w, lap)
    osim.step(steps)
    gst.step(steps)
    err = compare_states(osim, gst)
    assert max(err.values()) < TOL, err


@pytest.mark.parametrize("mode", [F.SOLVER_MIXED, F.SOLVER_FP64])
def test_solver_modes_multi_step(mode):
    w = WORKLOADS["sessile60"]()
    osim = oracle_sim(w)
    gst = gpu_state(w, solver_mode=mode)
    osim.step(200)
    gst.step(200)
    err = compare_states(osim, gst)
    assert max(err.values()) < TOL, err


def test_sessile_droplet_64x32_full_run():
    """The 64x32 sessile droplet (2,145 grid points) for its full 2,000 steps."""
    w = I.sessile_droplet_64x32()
    osim = oracle_sim(w)
    gst = gpu_state(w)
    osim.step(w["steps"])
    gst.step(w["steps"])
    err = compare_states(osim, gst)
    assert max(err.values()) < TOL, err
    ce = elementwise_c_err(osim, gst)
    print(f"elementwise relative C error over C >= 0.05: {ce:.2e}")
    assert ce < TOL, ce
    dg = gst.diagnostics(w["centre"], w["R"], 4.0, 0)
    do = osim.diagnostics(w["centre"], w["R"], 4.0, 0)
    assert abs(dg["mass_drift_rel"]) < 1e-12 and abs(do["mass_drift_rel"]) < 1e-12
    for key in ("mass", "kinetic_energy", "max_u", "delta_p", "interface_rho_uu",
                "wetted_length", "height", "theta_deg"):
        assert math.isclose(dg[key], do[key], rel_tol=1e-9, abs_tol=1e-14), (key, dg[key], do[key])


def test_free_droplet_256_full_size():
    """The 256x256 free droplet (131,585 grid points) at full size, 20 steps,
    in the configuration the benchmark times."""
    w = I.free_droplet_256()
    osim = oracle_sim(w)
    gst = gpu_state(w)
    osim.step(20)
    gst.step(20)
    err = compare_states(osim, gst)
    assert max(err.values()) < TOL, err
    ce = elementwise_c_err(osim, gst)
    print(f"elementwise relative C error over C >= 0.05: {ce:.2e}")
    assert ce < TOL, ce


def test_rough_wall_full_size_properties():
    """2048 x 1017-node rough-wall droplet (2.08M nodes): too large for the
    oracle, so check what holds at any size -- finite state, mass conserved to
    round-off, and diagnostics consistent with the initial cap."""
    w = I.rough_wall_droplet()
    gst = gpu_state(w)
    d0 = gst.diagnostics(w["centre"], w["R"], 4.0, 0)
    gst.step(20)
    d1 = gst.diagnostics(w["centre"], w["R"], 4.0, 0)
    assert d1["status"] == 0
    assert abs(d1["mass_drift_rel"]) < 1e-12
    assert abs(d1["wetted_length"] - d0["wetted_length"]) < 1.0
    assert d1["max_u"] < 0.1


def test_two_triangle_mesh():
    xy = np.array([[0.0, 0.0], [3.0, 0.0], [3.0, 2.5], [0.0, 2.5]])
    mesh = {"xy": xy, "tri": np.array([[0, 1, 2], [0, 2, 3]], np.int32),
            "wall_edges": np.array([[0, 1], [1, 2], [2, 3], [3, 0]], np.int32),
            "wall_id": np.array([0, 0, 1, 1], np.int32), "period": (0.0, 0.0)}
    phys = dict(dt=0.1, tau_l=0.8, tau_v=0.8, rho_l=1.0, rho_v=0.1, sigma=0.01, xi=4.0,
                mobility=0.02, theta_deg=(60.0, 120.0))
    w = {"mesh": mesh, "phys": phys, "C0": np.array([0.9, 0.2, 0.4, 0.7])}
    osim = oracle_sim(w)
    gst = gpu_state(w)
    osim.step(10)
    gst.step(10)
    err = compare_states(osim, gst)
    assert max(err.values()) < TOL, err


def test_zero_steps_roundtrip_and_determinism():
    w = WORKLOADS["sessile60"]()
    a = gpu_state(w)
    g0, h0 = a.get_state()
    a.step(0)
    g1, h1 = a.get_state()
    np.testing.assert_array_equal(g0, g1)
    a.step(25)
    ga, ha = a.get_state()
    b = gpu_state(w)
    b.step(25)
    gb, hb = b.get_state()
    np.testing.assert_array_equal(ga, gb)          # bitwise: no atomics, fixed orders
    np.testing.assert_array_equal(ha, hb)
    b.set_state(g0, h0)
    b.step(25)
    gc, hc = b.get_state()
    np.testing.assert_array_equal(ga, gc)


def test_nonfinite_state_is_reported():
    w = WORKLOADS["free_droplet"]()
    gst = gpu_state(w)
    g, h = gst.get_state()
    h[3, 17] = np.nan                               # planted on the host
    gst.set_state(g, h)
    d = gst.diagnostics()
    assert d["status"] == -5


def test_bad_workspace_is_rejected():
    import torch
    w = WORKLOADS["free_droplet"]()
    mesh = F.Mesh.from_dict(w["mesh"])
    prm = F.params_derive(w["phys"])
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(ValueError):
        F.State(mesh, prm, w["C0"], workspace=small)


@pytest.mark.parametrize("precision", [F.FP64, F.FP32_DEV])
def test_pipelined_inputs_and_async_diagnostics(precision):
    """Streaming distinct states through one state object: set_state from one
    pinned host buffer pair that the caller overwrites as soon as the call
    returns (the copy overlaps the previous step on its own stream, into two
    input buffers used in turn), a step, and the diagnostics queued with
    felbm_diagnostics_enqueue and finished after one synchronisation.  Every
    result equals, bit for bit, the synchronous set_state / step /
    felbm_diagnostics sequence."""
    import torch
    w = WORKLOADS["sessile60"]()
    src = gpu_state(w, precision=precision)
    states = []
    for _ in range(6):
        src.step(4)
        states.append(src.get_state())
    req = dict(centre=w["centre"], radius=w["R"], band=2.0, substrate=0)

    a = gpu_state(w, precision=precision)
    seq = []
    for g, h in states:
        a.set_state(g, h)
        a.step(3)
        seq.append(a.diagnostics(**req))
    ga, ha = a.get_state()

    b = gpu_state(w, precision=precision)
    gp = torch.empty(states[0][0].shape, dtype=torch.float64).pin_memory()
    hp = torch.empty(states[0][1].shape, dtype=torch.float64).pin_memory()
    slots = torch.zeros((len(states), F.DIAG_SLOTS), dtype=torch.float64).pin_memory()
    for k, (g, h) in enumerate(states):
        gp.copy_(torch.from_numpy(g))
        hp.copy_(torch.from_numpy(h))
        b.set_state(gp, hp)
        gp.fill_(float("nan"))                    # the host arrays are free once set_state returns
        hp.fill_(float("nan"))
        b.step(3)
        b.diagnostics_enqueue(slots[k], **req)
    torch.cuda.synchronize()
    pip = [b.diag_finish(slots[k], **req) for k in range(len(states))]

    def same(d):   # NaN marks "not measured" (solver_residual without the check)
        return {k: ("nan" if isinstance(v, float) and math.isnan(v) else v) for k, v in d.items()}
    assert [same(d) for d in pip] == [same(d) for d in seq]
    assert all(d["status"] == 0 for d in pip)
    gb, hb = b.get_state()
    np.testing.assert_array_equal(ga, gb)
    np.testing.assert_array_equal(ha, hb)
    with pytest.raises(ValueError):
        b.diagnostics_enqueue(torch.zeros(4, dtype=torch.float64))


@pytest.mark.parametrize("precision", [F.FP64, F.FP32_DEV])
def test_initial_pressure_and_velocity_fields(precision):
    """felbm_init with p0 and u0: the state starts at the equilibria of the
    given fields (their moments come back from felbm_get_fields) and evolves
    as the oracle started from the same fields -- a sheared flow crossing a
    wetting droplet on the walled mesh, 40 steps."""
    w = I.small_sessile(nx=40, ny=20, R=9.0, theta=60.0)
    N = len(w["mesh"]["xy"])
    rng = np.random.default_rng(12)
    y = w["mesh"]["xy"][:, 1]
    p0 = rng.uniform(-1e-3, 1e-3, N)
    u0 = np.stack([0.02 * y / 20.0, 0.005 * np.sin(w["mesh"]["xy"][:, 0] * 2 * np.pi / 40)], axis=1)
    m = w["mesh"]
    from oracle import OracleMesh, OracleSim, params_from_physical
    osim = OracleSim(OracleMesh(m["xy"], m["tri"], m["wall_edges"], m["wall_id"], m["period"]),
                     params_from_physical(w["phys"]), w["C0"], p0=p0, u0=u0)
    gst = F.State(F.Mesh.from_dict(m), F.params_derive(w["phys"], precision=precision), w["C0"], p0=p0, u0=u0)
    f = gst.get_fields()
    # p is a small difference of O(rho cs2) terms: FP64 round-off relative to max|p0| = 1e-3 is ~1e-13
    tol0 = 1e-12 if precision == F.FP64 else 1e-7
    assert rel_err(f["C"], w["C0"]) < 1e-14
    assert rel_err(f["p"], p0) < tol0 and rel_err(f["ux"], u0[:, 0]) < tol0 and rel_err(f["uy"], u0[:, 1]) < tol0
    osim.step(40)
    gst.step(40)
    err = compare_states(osim, gst)
    if precision == F.FP64:
        assert max(err.values()) < TOL, err
    else:
        assert err["C"] < 1e-6 and err["h"] < 1e-5 and err["g"] < 1e-3, err
