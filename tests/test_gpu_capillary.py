"""Capillary intrusion (Sec. III.C) in its 2D form: liquid drawn into a
channel between parallel plates, against the Washburn law as corrected
(the column length l obeys l-weighted, not constant, speed: the viscous
resistance of the column grows with l).

Between plates a distance H apart a meniscus of contact angle theta carries
the Laplace pressure 2 sigma cos(theta) / H; Poiseuille flow through the
liquid column (length l, viscosity eta_l) and the vapour ahead of it in the
channel (length L - l, eta_v) in series gives

    dl/dt = H sigma cos(theta) / (6 (eta_l l + eta_v (L - l))),

eta = rho cs2 tau dt for this scheme.  With eta_v = 0 this is the
parallel-plate analogue of y dy/dt = H sigma cos(theta) / (8 eta_l) for a
tube of diameter H.  The law leaves out the entrance losses, inertia and
the dissipation of the diffuse contact line, so the simulated speed
approaches it from below once the start-up transient has passed; the
checks are that the ratio of measured to predicted speed settles between
0.75 and 1.05, stays constant as l doubles (so the speed falls with l as
the corrected law says, where the printed constant-speed form would keep it
fixed), and that the column's advance is ordered by cos(theta).

The workload (``inputs.capillary_intrusion``) runs with the nodal element
Laplacian of mu; its FP64 step is checked against the oracle first.
"""
import math

import numpy as np
import pytest

from oracle import OracleMesh, OracleSim, params_from_physical
from paper_1708_04678_gb300 import felbm as F
from paper_1708_04678_gb300 import inputs as I
from parity_util import rel_err

pytestmark = pytest.mark.gpu

CS2 = 1.0 / 3.0


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_04678_gb300 import build
    build.build()


def meniscus(xy, C, w):
    """Distance from the channel entrance to the C = 1/2 crossing on the
    channel's centre line (linear between the last liquid node and the next)."""
    x_in, L, yc = w["x_in"], w["length"], w["y_c"]
    sel = (np.abs(xy[:, 1] - yc) < 0.25) & (xy[:, 0] >= x_in - 1.0) & (xy[:, 0] <= x_in + L + 1.0)
    x, c = xy[sel, 0], C[sel]
    o = np.argsort(x)
    x, c = x[o], c[o]
    j = np.nonzero(c > 0.5)[0][-1]
    return float(x[j] + (c[j] - 0.5) / (c[j] - c[j + 1]) * (x[j + 1] - x[j]) - x_in)


def washburn_speed(w, l):
    ph = w["phys"]
    eta_l = ph["rho_l"] * CS2 * ph["tau_l"] * ph["dt"]
    eta_v = ph["rho_v"] * CS2 * ph["tau_v"] * ph["dt"]
    H, L = w["H"], w["length"]
    return H * ph["sigma"] * math.cos(math.radians(ph["theta_deg"][0])) / (6.0 * (eta_l * l + eta_v * (L - l)))


def run_column(w, T, precision=F.FP32_DEV, every=100.0):
    """l(t) sampled every `every` time units up to T."""
    st = F.State(F.Mesh.from_dict(w["mesh"]), F.params_derive(w["phys"], precision=precision,
                                                              lapmu_mode=F.LAPMU_NODAL), w["C0"])
    n = int(round(every / w["phys"]["dt"]))
    xy = w["mesh"]["xy"]
    t, l = [0.0], [meniscus(xy, st.get_fields()["C"], w)]
    while t[-1] < T - 1e-9:
        st.step(n)
        t.append(t[-1] + every)
        l.append(meniscus(xy, st.get_fields()["C"], w))
    d = st.diagnostics()
    st.close()
    assert d["status"] == 0
    return np.array(t), np.array(l), d


def window_ratio(w, t, l, t0, t1):
    """Measured mean speed over [t0, t1] and its ratio to the corrected law
    at the window's mean length."""
    a, b = np.searchsorted(t, t0), np.searchsorted(t, t1)
    v = (l[b] - l[a]) / (t[b] - t[a])
    lm = 0.5 * (l[a] + l[b])
    return v, v / washburn_speed(w, lm), lm


def test_intrusion_step_matches_oracle():
    """The workload's physics (xi 4, M 1, dt 0.05, nodal Laplacian of mu) on a
    small channel: FP64 to 1e-11 and FP32 deviation storage at FP32 level
    after 100 steps."""
    w = I.capillary_channel(H=6, length_factor=6, reservoir=2, theta=56.0, l0_factor=1.0, liquid_factor=1.5,
                            dt=0.05, xi=4.0, mobility=1.0)
    m = w["mesh"]
    for prec in (F.FP64, F.FP32_DEV):
        osim = OracleSim(OracleMesh(m["xy"], m["tri"], m["wall_edges"], m["wall_id"], m["period"]),
                         params_from_physical(w["phys"], lapmu="nodal"), w["C0"])
        st = F.State(F.Mesh.from_dict(m), F.params_derive(w["phys"], precision=prec, lapmu_mode=F.LAPMU_NODAL),
                     w["C0"])
        osim.step(100)
        st.step(100)
        g, h = st.get_state()
        st.close()
        err = {"g": rel_err(g, osim.g), "h": rel_err(h, osim.h), "C": rel_err(h.sum(0), osim.h.sum(0))}
        if prec == F.FP64:
            assert max(err.values()) < 1e-11, err
        else:
            assert err["C"] < 1e-6 and err["h"] < 1e-5 and err["g"] < 1e-3, err


def test_column_follows_corrected_washburn_law():
    """H = 16, theta = 56 degrees, 20,000 time units (400,000 steps)."""
    w = I.capillary_intrusion(H=16, theta=56.0)
    t, l, d = run_column(w, 20000.0)
    assert np.all(np.diff(l[t >= 2000.0]) > 0.0)                  # advancing throughout after start-up
    rows = [window_ratio(w, t, l, a, a + 2000.0) for a in (6000.0, 9000.0, 12000.0, 15000.0, 18000.0)]
    for v, r, lm in rows:
        print(f"l {lm:7.2f}  dl/dt {v:.5f}  ratio to the corrected law {r:.3f}")
    late = [r for _, r, _ in rows[2:]]
    assert all(0.75 <= r <= 1.05 for r in late), late
    assert max(late) - min(late) < 0.05, late
    # the speed falls as the column lengthens, as the corrected law says
    (v0, r0, l0), (v1, r1, l1) = rows[0], rows[-1]
    assert l1 > 1.6 * l0 and v1 / v0 < 0.8
    assert abs((v1 / v0) / (washburn_speed(w, l1) / washburn_speed(w, l0)) - 1.0) < 0.15
    assert abs(d["mass_drift_rel"]) < 1e-6


def test_advance_is_ordered_by_cos_theta():
    """theta = 30, 56, 75 and 90 degrees, 8,000 time units each: the column
    advances further the more the wall wets, each at a comparable fraction of
    its own corrected-law speed, and at 90 degrees (no Laplace pressure) it
    does not advance."""
    res = {}
    for theta in (30.0, 56.0, 75.0, 90.0):
        w = I.capillary_intrusion(H=16, theta=theta)
        t, l, _ = run_column(w, 8000.0)
        v, r, lm = window_ratio(w, t, l, 6000.0, 8000.0) if theta < 90.0 else (0.0, float("nan"), l[-1])
        res[theta] = (l[-1] - l[0], r)
        print(f"theta {theta:5.1f}: advance {l[-1] - l[0]:7.2f} in 8,000 time units, ratio to the corrected law "
              f"{r:.3f}")
    assert res[30.0][0] > res[56.0][0] > res[75.0][0] > 2.0
    assert abs(res[90.0][0]) < 2.0
    for theta in (30.0, 56.0, 75.0):
        assert 0.5 <= res[theta][1] <= 1.05, res


def test_fp32_column_matches_fp64():
    """The column length of the FP32-deviation form against FP64 over the
    first 2,000 time units (40,000 steps)."""
    w = I.capillary_intrusion(H=16, theta=56.0)
    t32, l32, d32 = run_column(w, 2000.0, F.FP32_DEV)
    t64, l64, d64 = run_column(w, 2000.0, F.FP64)
    print(f"max |l32 - l64| = {np.abs(l32 - l64).max():.2e}; l(2000) {l32[-1]:.4f} / {l64[-1]:.4f}")
    assert np.abs(l32 - l64).max() < 0.05
    assert abs(d64["mass_drift_rel"]) < 1e-11 and abs(d32["mass_drift_rel"]) < 1e-6
