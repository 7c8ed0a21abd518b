"""Gradients through many FE-LBM time steps: a torch.autograd.Function over
the library's forward step and its hand-written adjoint (felbm_adjoint_*),
with checkpointed recomputation.

``run(state, C0, phi_c, n_steps, every)`` returns the final distributions
(g, h) as float64 tensors whose backward pass yields dL/dC0 and dL/dphi_c:
the forward pass saves a device checkpoint every ``every`` steps; the
backward pass walks the segments from the last to the first, recomputes each
segment's states from its checkpoint into a device ring, and applies the
adjoint step in reverse order.  The initial state is the rest state of C0
(g = 0, h = w C0), so dL/dC0 = sum_a w_a dL/dh^0_a.  FP64 states only.

``wetted_length(h, edges)`` is the substrate wetted length of Sec. III.B as a
differentiable torch function of h (C linear along each wall edge).
"""
from __future__ import annotations

import numpy as np
import torch

D2Q9_W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


class _Run(torch.autograd.Function):
    @staticmethod
    def forward(ctx, C0, phi_c, state, n_steps, every):
        st = state
        dev = st.workspace.device
        st.set_wetting(phi_c.detach().cpu().numpy())
        C0n = C0.detach().cpu().numpy().astype(np.float64)
        g0 = np.zeros((9, st.N))
        h0 = D2Q9_W[:, None] * C0n[None, :]
        st.set_state(g0, h0)
        nbytes = st.checkpoint_bytes()
        n_ck = (n_steps + every - 1) // every
        ck = torch.empty((max(n_ck, 1), nbytes), dtype=torch.uint8, device=dev)
        for k in range(n_steps):
            if k % every == 0:
                st.checkpoint_save(ck[k // every])
            st.step(1)
        g, h = st.get_state()
        ctx.st, ctx.ck, ctx.n_steps, ctx.every = st, ck, n_steps, every
        ctx.n_ids = int(phi_c.numel())
        return torch.from_numpy(g), torch.from_numpy(h)

    @staticmethod
    def backward(ctx, grad_g, grad_h):
        st, ck, n_steps, every = ctx.st, ctx.ck, ctx.n_steps, ctx.every
        dev = ck.device
        gg = np.zeros((9, st.N)) if grad_g is None else grad_g.detach().cpu().numpy().astype(np.float64)
        gh = np.zeros((9, st.N)) if grad_h is None else grad_h.detach().cpu().numpy().astype(np.float64)
        st.adjoint_seed(gg, gh)
        ring = torch.empty((every, ck.shape[1]), dtype=torch.uint8, device=dev)
        n_seg = (n_steps + every - 1) // every
        for s in reversed(range(n_seg)):
            start, end = s * every, min((s + 1) * every, n_steps)
            st.checkpoint_load(ck[s])
            for j in range(end - start):
                st.checkpoint_save(ring[j])
                if j < end - start - 1:
                    st.step(1)
            for j in reversed(range(end - start)):
                st.checkpoint_load(ring[j])
                st.adjoint_step()
        dg0, dh0, dphi = st.adjoint_get(ctx.n_ids)
        dC0 = (D2Q9_W[:, None] * dh0).sum(axis=0)
        return torch.from_numpy(dC0), torch.from_numpy(dphi), None, None, None


def run(state, C0, phi_c, n_steps, every=100):
    """Final (g, h) of ``n_steps`` steps from the rest state of C0 with wetting
    potentials phi_c; differentiable with respect to C0 and phi_c."""
    return _Run.apply(C0, phi_c, state, int(n_steps), int(every))


def wall_edge_table(mesh, wall_id=0):
    """(a, b, length) of the wall edges with the given id, from a mesh dict."""
    we = np.asarray(mesh["wall_edges"])
    sel = np.asarray(mesh["wall_id"]) == wall_id
    a, b = we[sel, 0], we[sel, 1]
    d = mesh["xy"][b] - mesh["xy"][a]
    for k in range(2):
        L = mesh["period"][k]
        if L > 0:
            d[:, k] -= L * np.round(d[:, k] / L)
    return torch.from_numpy(a.astype(np.int64)), torch.from_numpy(b.astype(np.int64)), \
        torch.from_numpy(np.hypot(d[:, 0], d[:, 1]))


def wetted_length(h, edges):
    """Length of the wall edges where C = sum h >= 1/2, C linear along each."""
    a, b, L = edges
    C = h.sum(dim=0)
    Ca, Cb = C[a], C[b]
    hi, lo = torch.maximum(Ca, Cb), torch.minimum(Ca, Cb)
    full = (lo >= 0.5).to(C.dtype)
    part = ((hi >= 0.5) & (lo < 0.5)).to(C.dtype)
    frac = torch.where(part > 0, (hi - 0.5) / torch.where(part > 0, hi - lo, torch.ones_like(hi)), torch.zeros_like(hi))
    return (L * (full + part * frac)).sum()
