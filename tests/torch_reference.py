"""A tiny PyTorch re-implementation of the FE-LBM step (test infrastructure).

The same step as the oracle -- moments, patch Laplacian with the wetting
flux, element Laplacian of mu, P0 forces, collision, weak-form right-hand
side, consistent-mass solve -- written with torch operations on dense
matrices taken from the oracle's mesh, so that torch autograd differentiates
it.  Its gradients are the reference for the library's hand-written adjoint
on tiny meshes.  Dense matrices: meant for a few hundred nodes.
"""
import numpy as np
import torch

from oracle.felbm_oracle import CS2, D2Q9_E, D2Q9_OPP, D2Q9_W

T64 = torch.float64


class TorchStep:
    def __init__(self, om, prm):
        self.om, self.prm = om, prm
        t = lambda a: torch.as_tensor(np.asarray(a), dtype=T64)
        self.M11 = t(om.M11.toarray())
        self.M10 = t(om.M10.toarray())
        self.Cm = [t(m.toarray()) for m in om.Cmat]
        self.Km = [t(m.toarray()) for m in om.Kmat]
        self.Dm = [t(m.toarray()) for m in om.Dmat]
        self.Bm = [t(m.toarray()) for m in om.Bmat]
        self.tri = torch.as_tensor(om.tri, dtype=torch.long)
        self.b = t(om.b)
        self.nu = t(om.nu)
        self.nbr = torch.as_tensor(om.nbr, dtype=torch.long)
        self.area = t(om.area)
        self.patch = t(om.patch_area)
        self.wall = torch.as_tensor(om.wall_edges, dtype=torch.long).reshape(-1, 2)
        self.wall_id = torch.as_tensor(om.wall_id, dtype=torch.long)
        self.wall_len = t(om.wall_len)
        self.E = t(D2Q9_E)
        self.W = t(D2Q9_W)

    def grad(self, f):
        return torch.einsum("ti,tid->td", f[self.tri], self.b)

    def gamma(self, u):
        eu = u @ self.E.T                                     # (..., 9)
        uu = (u * u).sum(-1, keepdim=True)
        return self.W * (1.0 + eu / CS2 + (eu * eu - CS2 * uu) / (2 * CS2 * CS2))

    def moments(self, g, h):
        p = self.prm
        C = h.sum(0)
        pr = g.sum(0)
        rho = C * p.rho_l + (1 - C) * p.rho_v
        u = (self.E.T @ g).T / (CS2 * rho[:, None])
        return C, pr, u, rho

    def mu(self, C, phi):
        p = self.prm
        gC = self.grad(C)
        flux = torch.zeros_like(C)
        for k in range(3):
            flux = flux.index_add(0, self.tri[:, k], p.kappa * (gC * self.nu[:, k]).sum(1))
        if len(self.wall):
            Ca, Cb = C[self.wall[:, 0]], C[self.wall[:, 1]]
            s = self.wall_len * ((Ca + Cb) / 2 - (Ca * Ca + Ca * Cb + Cb * Cb) / 3)
            q = -phi[self.wall_id] * s
            flux = flux.index_add(0, self.wall[:, 0], q).index_add(0, self.wall[:, 1], q)
        return 2 * p.beta * C * (C - 1) * (2 * C - 1) - flux / (p.lap_scale * self.patch)

    def lap_mu(self, mu):
        gmu = self.grad(mu)
        out = torch.zeros_like(self.area)
        for k in range(3):
            nb = self.nbr[:, k]
            inner = nb >= 0
            avg = 0.5 * (gmu + gmu[torch.where(inner, nb, torch.zeros_like(nb))])
            out = out + torch.where(inner, (avg * self.nu[:, k]).sum(1), torch.zeros_like(out))
        return out / self.area

    def forces(self, C, pr, u, mu):
        p = self.prm
        Cb, ub, mub = C[self.tri].mean(1), u[self.tri].mean(1), mu[self.tri].mean(1)
        rhob = Cb * p.rho_l + (1 - Cb) * p.rho_v
        gC, gp = self.grad(C), self.grad(pr)
        grho = (p.rho_l - p.rho_v) * gC
        lmu = self.lap_mu(mu)
        G = self.gamma(ub)                                    # (T, 9)
        vh = gC - (Cb / (rhob * CS2))[:, None] * (gp - mub[:, None] * gC)
        Pg, Ph = [], []
        for a in range(9):
            em = self.E[a][None, :] - ub
            vg = CS2 * grho * (G[:, a] - self.W[a])[:, None] + (mub * G[:, a])[:, None] * gC
            Pg.append((em * vg).sum(1))
            Ph.append((em * vh).sum(1) * G[:, a] + p.mobility * lmu * G[:, a])
        return torch.stack(Pg), torch.stack(Ph)

    def collide(self, g, h, C, pr, u, rho):
        p = self.prm
        tau = 1.0 / (C / p.tau_l + (1 - C) / p.tau_v)
        eu = u @ self.E.T
        uu = (u * u).sum(1)
        geq = self.W[:, None] * (pr[None, :] + (rho * CS2)[None, :] *
                                 (eu.T / CS2 + (eu.T ** 2 - CS2 * uu[None, :]) / (2 * CS2 * CS2)))
        heq = self.gamma(u).T * C[None, :]
        om = 1.0 / (tau + 0.5)
        return g - om * (g - geq), h - om * (h - heq)

    def rhs(self, psi, Phi):
        dt = self.prm.dt
        out = []
        for a in range(9):
            out.append(-dt * (self.Cm[a] @ psi[a]) - dt * dt * (self.Dm[a] @ psi[a])
                       + dt * (self.M10 @ Phi[a]) + dt * dt * (self.Km[a] @ Phi[a])
                       - dt * (self.Bm[a] @ (psi[int(D2Q9_OPP[a])] - psi[a])))
        return torch.stack(out)

    def step(self, g, h, phi):
        C, pr, u, rho = self.moments(g, h)
        mu = self.mu(C, phi)
        Pg, Ph = self.forces(C, pr, u, mu)
        gh, hh = self.collide(g, h, C, pr, u, rho)
        R = torch.cat([self.rhs(gh, Pg), self.rhs(hh, Ph)])  # (18, N)
        d = torch.linalg.solve(self.M11, R.T).T
        return gh + d[:9], hh + d[9:]
