"""The hand-written adjoint of the FP64 step (felbm_adjoint_*) behind
torch.autograd with checkpointed recomputation.

Checks: the full gradient (initial composition and wetting potentials) equals
torch autograd of the tiny PyTorch re-implementation (itself pinned to the
oracle); the gradient of the wetted-length loss agrees with central finite
differences of the forward run (relative error 1e-5); and on the 128x64
sessile droplet, 3,000 steps with a checkpoint every 100, the gradients with
respect to the wall wetting parameter and a 16-mode Fourier perturbation of
the initial C field agree with finite differences (eps = 1e-6, FP64).
"""
import math

import numpy as np
import pytest
import torch

from oracle import OracleMesh, params_from_physical
from paper_1708_04678_gb300 import adjoint as ADJ
from paper_1708_04678_gb300 import felbm as F
from paper_1708_04678_gb300 import inputs as I
from parity_util import gpu_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_04678_gb300 import build
    build.build()


def _tiny():
    w = I.small_sessile(nx=12, ny=6, seed=31, R=3.0, theta=60.0)
    w["phys"]["xi"] = 2.0
    w["C0"] = I.droplet_C0(w["mesh"]["xy"], w["centre"], w["R"], 2.0, w["mesh"]["period"])
    return w


def test_adjoint_matches_torch_autograd_of_the_reference_step():
    from torch_reference import TorchStep
    w = _tiny()
    m = w["mesh"]
    n_steps = 7
    rng = np.random.default_rng(1)
    wg = torch.as_tensor(rng.standard_normal((9, len(m["xy"]))))
    wh = torch.as_tensor(rng.standard_normal((9, len(m["xy"]))))
    prm = params_from_physical(w["phys"])
    phi0 = np.array(prm.phi_c)
    # library: forward + hand-written adjoint
    st = gpu_state(w)
    C0 = torch.tensor(w["C0"], dtype=torch.float64, requires_grad=True)
    phi = torch.tensor(phi0, dtype=torch.float64, requires_grad=True)
    g, h = ADJ.run(st, C0, phi, n_steps, every=3)
    ((g * wg).sum() + (h * wh).sum()).backward()
    # reference: torch autograd through the PyTorch step
    om = OracleMesh(m["xy"], m["tri"], m["wall_edges"], m["wall_id"], m["period"])
    ts = TorchStep(om, prm)
    C0r = torch.tensor(w["C0"], dtype=torch.float64, requires_grad=True)
    phir = torch.tensor(phi0, dtype=torch.float64, requires_grad=True)
    gr = torch.zeros((9, om.N), dtype=torch.float64)
    hr = torch.as_tensor(ADJ.D2Q9_W)[:, None] * C0r[None, :]
    for _ in range(n_steps):
        gr, hr = ts.step(gr, hr, phir)
    ((gr * wg).sum() + (hr * wh).sum()).backward()
    assert torch.allclose(g, gr.detach(), rtol=0, atol=1e-12)
    scale_c = C0r.grad.abs().max().item()
    assert (C0.grad - C0r.grad).abs().max().item() < 1e-9 * scale_c
    assert (phi.grad - phir.grad).abs().max().item() < 1e-9 * phir.grad.abs().max().item()


def _loss_fn(w, target):
    edges = ADJ.wall_edge_table(w["mesh"], 0)

    def loss(g, h):
        return (ADJ.wetted_length(h, edges) - target) ** 2
    return loss


def test_wetted_length_matches_library_diagnostic():
    w = I.small_sessile(nx=32, ny=16, R=7.0, theta=60.0)
    st = gpu_state(w)
    st.step(40)
    g, h = st.get_state()
    b = ADJ.wetted_length(torch.as_tensor(h), ADJ.wall_edge_table(w["mesh"], 0)).item()
    assert math.isclose(b, st.diagnostics()["wetted_length"], rel_tol=1e-12)


def test_adjoint_gradient_matches_finite_differences():
    w = I.small_sessile(nx=32, ny=16, R=7.0, theta=60.0)
    n_steps, every = 60, 25
    st = gpu_state(w)
    loss = _loss_fn(w, 13.0)
    prm = F.params_derive(w["phys"])
    phi0 = np.array(prm.phi_c[:2])
    rng = np.random.default_rng(3)
    v = rng.standard_normal(len(w["C0"])) * 1e-2
    C0 = torch.tensor(w["C0"], dtype=torch.float64, requires_grad=True)
    phi = torch.tensor(phi0, dtype=torch.float64, requires_grad=True)
    L = loss(*ADJ.run(st, C0, phi, n_steps, every))
    L.backward()

    def L_at(C0n, phin):
        with torch.no_grad():
            return loss(*ADJ.run(st, torch.as_tensor(C0n), torch.as_tensor(phin), n_steps, every)).item()

    eps = 1e-6
    # the substrate's wetting potential (the top wall does not reach the
    # wetted length within these steps: its derivative is round-off)
    dp = np.array([eps, 0.0])
    fd = (L_at(w["C0"], phi0 + dp) - L_at(w["C0"], phi0 - dp)) / (2 * eps)
    assert abs(phi.grad[0].item() - fd) <= 1e-5 * abs(fd), (phi.grad[0].item(), fd)
    assert abs(phi.grad[1].item()) < 1e-6 * abs(phi.grad[0].item())
    fd = (L_at(w["C0"] + eps * v, phi0) - L_at(w["C0"] - eps * v, phi0)) / (2 * eps)
    ad = float(C0.grad.numpy() @ v)
    assert abs(ad - fd) <= 1e-5 * abs(fd), (ad, fd)


def test_sessile_128x64_3000_steps_wetting_and_fourier_gradients():
    """Loss (b(3000) - 40)^2; parameters: the bottom wall's phi_c and the 16
    amplitudes a_m of R(phi) = R0 (1 + sum_m a_m cos(m phi)) of the initial
    cap; checkpoint every 100 steps."""
    w = I.sessile_droplet_128x64()
    m = w["mesh"]
    n_steps, every = w["steps"], 100
    st = gpu_state(w)
    loss = _loss_fn(w, 40.0)
    xy = torch.as_tensor(m["xy"])
    dx = xy[:, 0] - w["centre"][0]
    dy = xy[:, 1] - w["centre"][1]
    r = torch.sqrt(dx * dx + dy * dy)
    ang = torch.atan2(dy, dx)
    xi = w["phys"]["xi"]
    modes = torch.arange(1, 17, dtype=torch.float64)

    def C0_of(a):
        R = w["R"] * (1.0 + (a[:, None] * torch.cos(modes[:, None] * ang[None, :])).sum(0))
        return 0.5 + 0.5 * torch.tanh(2.0 * (R - r) / xi)

    prm = F.params_derive(w["phys"])
    phi0 = np.array(prm.phi_c[:2])
    a = torch.zeros(16, dtype=torch.float64, requires_grad=True)
    phi = torch.tensor(phi0, dtype=torch.float64, requires_grad=True)
    L = loss(*ADJ.run(st, C0_of(a), phi, n_steps, every))
    L.backward()

    def L_at(an, phin):
        with torch.no_grad():
            return loss(*ADJ.run(st, C0_of(torch.as_tensor(an)), torch.as_tensor(phin), n_steps, every)).item()

    eps = 1e-6
    dp = np.array([eps, 0.0])
    fd = (L_at(np.zeros(16), phi0 + dp) - L_at(np.zeros(16), phi0 - dp)) / (2 * eps)
    assert abs(phi.grad[0].item() - fd) <= 1e-5 * abs(fd), (phi.grad[0].item(), fd)
    for k in range(16):
        da = np.zeros(16)
        da[k] = eps
        fd = (L_at(da, phi0) - L_at(-da, phi0)) / (2 * eps)
        g = a.grad[k].item()
        assert abs(g - fd) <= 1e-5 * max(abs(fd), 1e-3 * a.grad.abs().max().item()), (k, g, fd)
