"""The tiny PyTorch re-implementation used as the adjoint's gradient
reference follows the oracle step for step, and its autograd gradient agrees
with central finite differences of the oracle itself."""
import numpy as np
import torch

from oracle import D2Q9_W, OracleMesh, OracleSim, params_from_physical
from paper_1708_04678_gb300 import inputs as I
from torch_reference import TorchStep


def _case():
    w = I.small_sessile(nx=12, ny=6, seed=31, R=3.0, theta=60.0)
    w["phys"]["xi"] = 2.0
    m = w["mesh"]
    om = OracleMesh(m["xy"], m["tri"], m["wall_edges"], m["wall_id"], m["period"])
    prm = params_from_physical(w["phys"])
    C0 = I.droplet_C0(m["xy"], w["centre"], w["R"], 2.0, m["period"])
    return w, om, prm, C0


def test_torch_step_matches_oracle():
    w, om, prm, C0 = _case()
    sim = OracleSim(om, prm, C0)
    ts = TorchStep(om, prm)
    g = torch.zeros((9, om.N), dtype=torch.float64)
    h = torch.as_tensor(sim.h.copy())
    phi = torch.as_tensor(np.array(prm.phi_c))
    for _ in range(5):
        sim.step()
        g, h = ts.step(g, h, phi)
    assert np.abs(g.numpy() - sim.g).max() < 1e-13 * max(1.0, np.abs(sim.g).max())
    assert np.abs(h.numpy() - sim.h).max() < 1e-13


def test_torch_gradient_matches_oracle_finite_differences():
    w, om, prm, C0 = _case()
    ts = TorchStep(om, prm)
    rng = np.random.default_rng(0)
    wts = rng.standard_normal((9, om.N))

    def oracle_loss(phi0):
        p2 = params_from_physical(w["phys"])
        p2.phi_c = (phi0,) + tuple(prm.phi_c[1:])
        sim = OracleSim(om, p2, C0)
        sim.step(4)
        return float(np.sum(wts * sim.h))

    phi = torch.tensor(np.array(prm.phi_c), dtype=torch.float64, requires_grad=True)
    g = torch.zeros((9, om.N), dtype=torch.float64)
    h = torch.as_tensor(np.asarray(D2Q9_W)[:, None] * C0[None, :])
    for _ in range(4):
        g, h = ts.step(g, h, phi)
    (h * torch.as_tensor(wts)).sum().backward()
    eps = 1e-6
    fd = (oracle_loss(prm.phi_c[0] + eps) - oracle_loss(prm.phi_c[0] - eps)) / (2 * eps)
    assert abs(phi.grad[0].item() - fd) < 1e-6 * max(1.0, abs(fd))

