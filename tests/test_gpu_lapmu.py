"""The element Laplacian of mu in its two forms (felbm_params.lapmu_mode).

FELBM_LAPMU_FACE is the paper's (Sec. II.D) and the default; everything else
in the suite runs it.  FELBM_LAPMU_NODAL (the patch Laplacian applied to mu
with zero wall flux, averaged over the element) is checked here: FP64
parity with the oracle in the same mode (2D and 3D, walled and periodic),
FP32 deviation storage at FP32 level, the batch CTA schedule against the
tiled one, the adjoint refusing it, and bounded long runs on the meshes
where the face form grows (the 64x32 sessile droplet of the contact-angle
case, whose FACE run leaves [0, 1] after ~4,000 steps).
"""
import math

import numpy as np
import pytest

from oracle import OracleMesh, OracleSim, params_from_physical
from oracle.felbm_oracle3d import OracleMesh3D, OracleSim3D, params_from_physical3d
from paper_1708_04678_gb300 import felbm as F
from paper_1708_04678_gb300 import felbm3d as F3
from paper_1708_04678_gb300 import inputs as I
from paper_1708_04678_gb300 import inputs3d as I3

pytestmark = pytest.mark.gpu

NODAL = F.LAPMU_NODAL


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_04678_gb300 import build
    build.build()


def rel_err(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


def _pair2d(w, precision=F.FP64):
    m = w["mesh"]
    osim = OracleSim(OracleMesh(m["xy"], m["tri"], m["wall_edges"], m["wall_id"], m["period"]),
                     params_from_physical(w["phys"], lapmu="nodal"), w["C0"])
    st = F.State(F.Mesh.from_dict(m), F.params_derive(w["phys"], precision=precision, lapmu_mode=NODAL), w["C0"])
    return osim, st


def _pair3d(w, precision=F.FP64):
    m = w["mesh"]
    osim = OracleSim3D(OracleMesh3D(m["xyz"], m["tet"], m["wall_faces"], m["wall_id"], m["period"]),
                       params_from_physical3d(w["phys"], lapmu="nodal"), w["C0"])
    st = F3.State3D(F3.Mesh3D.from_dict(m), F.params_derive(w["phys"], precision=precision, lapmu_mode=NODAL),
                    w["C0"])
    return osim, st


@pytest.mark.parametrize("name", ["sessile", "free"])
def test_nodal_2d_fp64_matches_oracle(name):
    w = {"sessile": lambda: I.small_sessile(nx=32, ny=16, R=7.0, theta=60.0),
         "free": lambda: I.small_free_droplet(n=24, R=6.0)}[name]()
    osim, st = _pair2d(w)
    osim.step(20)
    st.step(20)
    g, h = st.get_state()
    assert max(rel_err(g, osim.g), rel_err(h, osim.h), rel_err(h.sum(0), osim.h.sum(0))) < 1e-11


def test_nodal_2d_fp32_matches_oracle_at_fp32_level():
    w = I.small_sessile(nx=40, ny=20, R=9.0, theta=60.0)
    osim, st = _pair2d(w, F.FP32_DEV)
    osim.step(20)
    st.step(20)
    g, h = st.get_state()
    assert rel_err(h.sum(0), osim.h.sum(0)) < 1e-6 and rel_err(h, osim.h) < 1e-5 and rel_err(g, osim.g) < 1e-3


@pytest.mark.parametrize("name", ["sessile", "free"])
def test_nodal_3d_fp64_matches_oracle(name):
    w = {"sessile": lambda: I3.small_sessile_3d(),
         "free": lambda: I3.small_free_droplet_3d(n=11, R=3.5, seed=13, rho_v=0.1)}[name]()
    osim, st = _pair3d(w)
    osim.step(20)
    st.step(20)
    g, h = st.get_state()
    assert max(rel_err(g, osim.g), rel_err(h, osim.h), rel_err(h.sum(0), osim.h.sum(0))) < 1e-11


def test_nodal_3d_fp32_matches_oracle_at_fp32_level():
    w = I3.small_sessile_3d()
    osim, st = _pair3d(w, F.FP32_DEV)
    osim.step(20)
    st.step(20)
    g, h = st.get_state()
    assert rel_err(h.sum(0), osim.h.sum(0)) < 1e-6 and rel_err(h, osim.h) < 1e-5 and rel_err(g, osim.g) < 1e-3


def test_nodal_batch_cta_schedule_matches_tiled():
    ws = [I.small_sessile(nx=32, ny=16, seed=21, R=6.4, theta=45.0),
          I.small_sessile(nx=48, ny=24, seed=24, R=9.6, theta=100.0)]
    b = I.batch(ws)
    prm = F.params_derive(b["phys"], precision=F.FP32_DEV, lapmu_mode=NODAL)
    a = F.State(F.Mesh.batch(b["meshes"]), prm, b["C0"])
    c = F.State(F.Mesh.batch(b["meshes"]), prm, b["C0"])
    c.batch_schedule(10 ** 6)
    a.step(100)
    c.step(100)
    ga, ha = a.get_state()
    gc, hc = c.get_state()
    assert rel_err(gc, ga) < 1e-6 and rel_err(hc, ha) < 1e-6


def test_adjoint_refuses_nodal_mode():
    w = I.small_sessile(nx=12, ny=6, R=3.0, theta=60.0)
    st = F.State(F.Mesh.from_dict(w["mesh"]), F.params_derive(w["phys"], lapmu_mode=NODAL), w["C0"])
    g, h = st.get_state()
    with pytest.raises(F.FelbmError) as e:
        st.adjoint_seed(g, h)
    assert e.value.code == -6


def test_nodal_long_run_stays_bounded_2d():
    """The 64x32 sessile droplet, 10,000 steps (2,500 time units): C stays in
    [-0.01, 1.01], mass drift below 1e-12, the angle settles near 90 deg."""
    w = I.sessile_droplet_64x32()
    st = F.State(F.Mesh.from_dict(w["mesh"]), F.params_derive(w["phys"], lapmu_mode=NODAL), w["C0"])
    for _ in range(5):
        st.step(2000)
        C = st.get_fields()["C"]
        assert np.isfinite(C).all() and -0.01 < C.min() and C.max() < 1.01, (C.min(), C.max())
    d = st.diagnostics(w["centre"], w["R"], 4.0, 0)
    assert abs(d["mass_drift_rel"]) < 1e-12
    assert abs(d["theta_deg"] - 90.0) < 2.0, d["theta_deg"]


def test_nodal_long_run_stays_bounded_3d():
    """3D static droplet 40^3, sigma 0.01: the face form diverges after
    ~3,500 steps; the nodal form runs 8,000 steps with C in [-0.02, 1.02]
    and the Laplace jump within 5% of 2 sigma / R."""
    mesh = I3.kuhn_box(40, 40, 40, 0.15, 21, walls=False)
    C0 = I3.droplet_C0_3d(mesh["xyz"], (20, 20, 20), 10.0, 4.0, mesh["period"])
    phys = I3._phys(theta_deg=())
    st = F3.State3D(F3.Mesh3D.from_dict(mesh), F.params_derive(phys, precision=F.FP32_DEV, lapmu_mode=NODAL), C0)
    for _ in range(4):
        st.step(2000)
        C = st.get_fields()["C"]
        assert np.isfinite(C).all() and -0.02 < C.min() and C.max() < 1.02, (C.min(), C.max())
    d = st.diagnostics((20, 20, 20), 10.0, 4.0, substrate=-1)
    R = (3 * d["mass"] / (4 * math.pi)) ** (1 / 3)
    assert abs(d["delta_p"] / (2 * phys["sigma"] / R) - 1) < 0.05, d["delta_p"]
    assert abs(d["mass_drift_rel"]) < 1e-6


@pytest.mark.parametrize("theta", [60.0, 90.0, 120.0])
def test_nodal_3d_young_law(theta):
    """Sec. III.B in 3D: a hemisphere R=12 on the substrate of a 48x48x24
    box, sigma 0.01, density ratio 2, 20,000 FP32 steps; the angle from
    height and wetted area settles within 2.5 degrees of Young's angle (the
    paper reports 5 degrees for 45-135)."""
    w = I3._sessile(f"sessile {theta}", 48, 24, 12.0, 22, 0.15, theta, 20000)
    st = F3.State3D(F3.Mesh3D.from_dict(w["mesh"]),
                    F.params_derive(w["phys"], precision=F.FP32_DEV, lapmu_mode=NODAL), w["C0"])
    st.step(20000)
    d = st.diagnostics(w["centre"], w["R"], 4.0, substrate=0)
    assert d["status"] == 0 and abs(d["mass_drift_rel"]) < 1e-6
    assert abs(d["theta_deg"] - theta) < 2.5, d["theta_deg"]
