"""FP64 CPU oracle of one FE-LBM time step (TEST INFRASTRUCTURE ONLY).

Plain restatement of the characteristic-based finite-element lattice Boltzmann
scheme of arXiv:1708.04678 for the free-energy two-phase model with wetting
walls, in 2D (D2Q9 velocities, linear triangles; the paper is written for
D3Q19 and tetrahedra, every formula below is its 2D form).  It is slow on
purpose: global sparse matrices assembled from their defining integrals
(Sec. II.C, eq:fem_matrices), one loop per edge family, per-column PCG.  Only
``tests/``, ``__graft_entry__.smoke`` and the CPU-baseline leg of ``bench.py``
may use it.  It shares no code with the CUDA path.

Readings taken where the paper is silent or garbled (each one is listed with
its reason in the design notes of the repository):

* weak form (eq:galerkin_lbm): the force enters as +(dt M10 + dt^2 K) Phi; the
  printed minus sign on dt M10 contradicts the streaming step (eqn::stream)
  it is derived from and breaks the static-interface balance;
  psi^n on its right-hand side is the post-collision value.
* the patch Laplacian of C (eqn:lapl_int_mp) divides by V = s * |patch|,
  s = 2/3 ("consistent", equal to the lumped P1 Laplacian) or s = 1 (the
  literal patch area, "paper"); the wall flux uses eqn:bc2 with n the normal
  into the fluid, C linear along the wall edge.
* wall populations: weak bounce-back -- in the boundary integral of C_alpha
  the incoming population psi_alpha is replaced by psi_opposite(alpha).
* contact angle from height h and base b of the C = 1/2 contour:
  theta = atan2(b, 2 (r - h)), r = (4 h^2 + b^2) / (8 h).
* initial state: the equilibria of the initial C, p, u (g = w p, h = w C at rest).

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, brute-force quadrature, invariants or physical laws
(static-interface balance, exact mass conservation, Laplace, Young); the
element Laplacian of mu of Sec. II.D against hand-derived stencils on the
unjittered grids, the forces against their zeroth and first lattice moments;
the trajectory after many steps has no independent pin beyond those.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

# D2Q9 lattice (2D form of the velocity set of Sec. II.A): rest, four axis
# and four diagonal velocities; weights 4/9, 1/9, 1/36; c_s^2 = 1/3.
D2Q9_E = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1],
                   [1, 1], [-1, 1], [-1, -1], [1, -1]], dtype=np.float64)
D2Q9_W = np.array([4.0 / 9.0] + [1.0 / 9.0] * 4 + [1.0 / 36.0] * 4)
D2Q9_OPP = np.array([0, 3, 4, 1, 2, 7, 8, 5, 6])
CS2 = 1.0 / 3.0
Q = 9


@dataclass
class OracleParams:
    """Model constants of Sec. II (2D, lattice units)."""
    dt: float
    tau_l: float
    tau_v: float
    rho_l: float
    rho_v: float
    kappa: float
    beta: float
    mobility: float
    phi_c: tuple = field(default_factory=tuple)   # one wetting potential per wall id
    lap_scale: float = 2.0 / 3.0                  # V_k = lap_scale * |patch_k|
    lapmu: str = "face"                           # element Laplacian of mu: "face" (Sec. II.D) or "nodal"


def params_from_physical(phys, lap_mode="consistent", lapmu="face"):
    """kappa, beta and phi_c from sigma, xi and the contact angles.

    Sec. II: xi = sqrt(8 kappa / beta) and sigma = sqrt(2 kappa beta) / 6,
    so kappa = 3 sigma xi / 2 and beta = 12 sigma / xi.  Sec. II.B (Young):
    cos theta = -phi_c / sqrt(2 kappa beta)."""
    sigma, xi = phys["sigma"], phys["xi"]
    kappa = 1.5 * sigma * xi
    beta = 12.0 * sigma / xi
    root = math.sqrt(2.0 * kappa * beta)
    phi_c = tuple(-root * math.cos(math.radians(t)) for t in phys["theta_deg"])
    return OracleParams(dt=phys["dt"], tau_l=phys["tau_l"], tau_v=phys["tau_v"],
                        rho_l=phys["rho_l"], rho_v=phys["rho_v"], kappa=kappa,
                        beta=beta, mobility=phys["mobility"], phi_c=phi_c,
                        lap_scale=(2.0 / 3.0 if lap_mode == "consistent" else 1.0), lapmu=lapmu)


def gamma(u):
    """Gamma_alpha(u) = h_eq / C (eqn::f_eq), for u of shape (..., 2);
    returns shape (9, ...)."""
    eu = np.tensordot(D2Q9_E, u, axes=([1], [u.ndim - 1]))          # (9, ...)
    uu = np.sum(u * u, axis=-1)
    return D2Q9_W.reshape((9,) + (1,) * uu.ndim) * (
        1.0 + eu / CS2 + (eu * eu - CS2 * uu) / (2.0 * CS2 * CS2))


class OracleMesh:
    """Linear-triangle mesh with the FE matrices of eq:fem_matrices.

    xy: (N, 2) node coordinates; tri: (T, 3) counter-clockwise triangles;
    wall_edges: (E, 2) node pairs on solid walls; wall_id: (E,) index into
    the wetting potentials; period: (Lx, Ly), 0 = not periodic (periodic
    images are one node; edge vectors use the minimum image)."""

    def __init__(self, xy, tri, wall_edges, wall_id, period=(0.0, 0.0)):
        self.xy = np.asarray(xy, dtype=np.float64)
        self.tri = np.asarray(tri, dtype=np.int64)
        self.wall_edges = np.asarray(wall_edges, dtype=np.int64).reshape(-1, 2)
        self.wall_id = np.asarray(wall_id, dtype=np.int64).reshape(-1)
        self.period = (float(period[0]), float(period[1]))
        self.N = len(self.xy)
        self.T = len(self.tri)
        self._geometry()
        self._topology()
        self._matrices()

    def min_image(self, d):
        d = np.array(d, dtype=np.float64, copy=True)
        for k in range(2):
            L = self.period[k]
            if L > 0:
                d[..., k] -= L * np.round(d[..., k] / L)
        return d

    # -- geometry ---------------------------------------------------------
    def _geometry(self):
        tri = self.tri
        P = np.zeros((self.T, 3, 2))
        for k in (1, 2):
            P[:, k] = self.min_image(self.xy[tri[:, k]] - self.xy[tri[:, 0]])
        self.P = P                                   # vertices relative to vertex 0
        x, y = P[..., 0], P[..., 1]
        area = 0.5 * ((x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0])
                      - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0]))
        if np.any(area <= 0.0):
            raise ValueError("oracle: triangle with non-positive area")
        self.area = area
        # gradient of the linear shape function of vertex i (Sec. II.C, P1):
        # (y_j - y_k, x_k - x_j) / (2A) with (i, j, k) cyclic
        b = np.zeros((self.T, 3, 2))
        for i in range(3):
            j, k = (i + 1) % 3, (i + 2) % 3
            b[:, i, 0] = (y[:, j] - y[:, k]) / (2.0 * area)
            b[:, i, 1] = (x[:, k] - x[:, j]) / (2.0 * area)
        self.b = b
        # outward normal times length of the edge opposite vertex k
        nu = np.zeros((self.T, 3, 2))
        for k in range(3):
            t = P[:, (k + 2) % 3] - P[:, (k + 1) % 3]
            nu[:, k, 0] = t[:, 1]
            nu[:, k, 1] = -t[:, 0]
        self.nu = nu
        patch = np.zeros(self.N)
        for k in range(3):
            np.add.at(patch, tri[:, k], area)
        self.patch_area = patch

    # -- topology ---------------------------------------------------------
    def _topology(self):
        tri = self.tri
        owner = {}
        self.nbr = -np.ones((self.T, 3), dtype=np.int64)
        for t in range(self.T):
            for k in range(3):
                a, c = tri[t, (k + 1) % 3], tri[t, (k + 2) % 3]
                key = (min(a, c), max(a, c))
                if key in owner:
                    t2, k2 = owner.pop(key)
                    self.nbr[t, k] = t2
                    self.nbr[t2, k2] = t
                else:
                    owner[key] = (t, k)
        # edges left unpaired are boundary edges and must be walls
        wall_lookup = {}
        for e, (a, c) in enumerate(self.wall_edges):
            wall_lookup[(min(a, c), max(a, c))] = e
        if set(owner.keys()) != set(wall_lookup.keys()):
            raise ValueError("oracle: boundary edges and wall edges differ")
        E = len(self.wall_edges)
        self.wall_len = np.zeros(E)
        self.wall_normal = np.zeros((E, 2))           # unit normal out of the fluid
        for key, (t, k) in owner.items():
            e = wall_lookup[key]
            nu = self.nu[t, k]
            L = math.hypot(nu[0], nu[1])
            self.wall_len[e] = L
            self.wall_normal[e] = nu / L
        wall_nodes = np.unique(self.wall_edges.reshape(-1)) if E else np.zeros(0, np.int64)
        self.wall_nodes = wall_nodes

    # -- finite-element matrices (eq:fem_matrices), closed forms for P1 ----
    def _matrices(self):
        tri, A, b = self.tri, self.area, self.b
        N, T = self.N, self.T
        rows, cols, vals = [], [], []
        for i in range(3):
            for j in range(3):
                rows.append(tri[:, i]); cols.append(tri[:, j])
                vals.append(A / 12.0 * (2.0 if i == j else 1.0))
        self.M11 = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows),
                                  np.concatenate(cols))), shape=(N, N))
        self.M10 = sp.csr_matrix((np.concatenate([A / 3.0] * 3),
                                  (np.concatenate([tri[:, i] for i in range(3)]),
                                   np.concatenate([np.arange(T)] * 3))), shape=(N, T))
        self.lumped = np.asarray(self.M11.sum(axis=1)).reshape(-1)
        self.Cmat, self.Kmat, self.Dmat, self.Bmat = [], [], [], []
        for a in range(Q):
            e = D2Q9_E[a]
            eb = b[..., 0] * e[0] + b[..., 1] * e[1]                 # (T, 3): e . grad N_i
            r, c, vC, vD = [], [], [], []
            for i in range(3):
                for j in range(3):
                    r.append(tri[:, i]); c.append(tri[:, j])
                    vC.append(A / 3.0 * eb[:, j])                      # int N_i e.grad N_j
                    vD.append(A / 2.0 * eb[:, i] * eb[:, j])           # 1/2 int (e.grad N_i)(e.grad N_j)
            r = np.concatenate(r); c = np.concatenate(c)
            self.Cmat.append(sp.csr_matrix((np.concatenate(vC), (r, c)), shape=(N, N)))
            self.Dmat.append(sp.csr_matrix((np.concatenate(vD), (r, c)), shape=(N, N)))
            self.Kmat.append(sp.csr_matrix(
                (np.concatenate([A / 2.0 * eb[:, i] for i in range(3)]),      # 1/2 int e.grad N_i
                 (np.concatenate([tri[:, i] for i in range(3)]),
                  np.concatenate([np.arange(T)] * 3))), shape=(N, T)))
            # wall boundary matrix int_wall N N^T (e.n_out) ds on edges where
            # the population is incoming (e.n_out < 0)
            br, bc, bv = [], [], []
            for ed in range(len(self.wall_edges)):
                en = float(e @ self.wall_normal[ed])
                if en < 0.0:
                    na, nb = self.wall_edges[ed]
                    L = self.wall_len[ed]
                    for (p, q, w) in ((na, na, L / 3), (na, nb, L / 6), (nb, na, L / 6), (nb, nb, L / 3)):
                        br.append(p); bc.append(q); bv.append(en * w)
            self.Bmat.append(sp.csr_matrix((np.array(bv, dtype=np.float64),
                                            (np.array(br, dtype=np.int64), np.array(bc, dtype=np.int64))),
                                           shape=(N, N)))

    # -- element gradient of a nodal (P1) field ----------------------------
    def grad(self, f):
        fv = f[self.tri]                                              # (T, 3)
        return np.einsum("ti,tid->td", fv, self.b)


class OracleSim:
    """State (g, h) on an OracleMesh and the time step of Sec. II.C."""

    def __init__(self, mesh: OracleMesh, params: OracleParams, C0, p0=None, u0=None,
                 solver_tol=1e-14, solver_maxit=200):
        self.mesh = mesh
        self.prm = params
        self.tol = solver_tol
        self.maxit = solver_maxit
        N = mesh.N
        C0 = np.asarray(C0, dtype=np.float64)
        p0 = np.zeros(N) if p0 is None else np.asarray(p0, dtype=np.float64)
        u0 = np.zeros((N, 2)) if u0 is None else np.asarray(u0, dtype=np.float64).reshape(N, 2)
        # initial state: the equilibria of the initial fields (at rest, u = 0,
        # they are g = w p, h = w C)
        rho0 = C0 * params.rho_l + (1.0 - C0) * params.rho_v
        self.g, self.h = self.equilibria(C0, p0, u0, rho0)
        self.step_count = 0
        self.mass0 = self.mass()
        self.last_iters = 0

    # -- macroscopic fields (eq:velocity, eq:pressure, Sec. II) ------------
    def moments(self, g=None, h=None):
        g = self.g if g is None else g
        h = self.h if h is None else h
        pr = self.prm
        C = h.sum(axis=0)
        p = g.sum(axis=0)
        rho = C * pr.rho_l + (1.0 - C) * pr.rho_v
        mom = np.tensordot(D2Q9_E.T, g, axes=([1], [0])).T              # (N, 2)
        u = mom / (CS2 * rho[:, None])
        return C, p, u, rho

    # -- chemical potential (eqn:mp_mu) with the patch Laplacian -----------
    def kappa_lap_C(self, C):
        """kappa * nabla^2 C at the nodes (eqn:lapl_int_mp): the outward flux
        of grad C over the outer edges of the vertex patch, with the wall
        edges' flux replaced by the wetting condition eqn:bc2, divided by
        V = lap_scale * |patch|.  kappa multiplies through so that the wall
        flux kappa n_out.grad C = -phi_c (C - C^2) needs no division."""
        m, pr = self.mesh, self.prm
        gC = m.grad(C)
        flux = np.zeros(m.N)
        for k in range(3):
            np.add.at(flux, m.tri[:, k], pr.kappa * np.sum(gC * m.nu[:, k], axis=1))
        for e, (a, c) in enumerate(m.wall_edges):
            L = m.wall_len[e]
            Ca, Cc = C[a], C[c]
            int_C = L * (Ca + Cc) / 2.0
            int_C2 = L * (Ca * Ca + Ca * Cc + Cc * Cc) / 3.0
            q = -pr.phi_c[m.wall_id[e]] * (int_C - int_C2)
            flux[a] += q
            flux[c] += q
        return flux / (pr.lap_scale * m.patch_area)

    def chemical_potential(self, C):
        pr = self.prm
        return 2.0 * pr.beta * C * (C - 1.0) * (2.0 * C - 1.0) - self.kappa_lap_C(C)

    def lap_mu(self, mu):
        """Element Laplacian of mu.  "face" (Sec. II.D): flux of grad mu over
        the three edges, interior edges taking the mean of the two element
        gradients, wall edges zero (eqn:bc1), divided by the element area.
        "nodal": the patch Laplacian of eqn:lapl_int_mp applied to mu with the
        zero wall flux of eqn:bc1 (consistent volume 2/3 |patch|, i.e. the
        lumped P1 Laplacian), averaged over the element's vertices like the
        other element means."""
        if self.prm.lapmu == "nodal":
            m = self.mesh
            gmu = m.grad(mu)
            flux = np.zeros(m.N)
            for k in range(3):
                np.add.at(flux, m.tri[:, k], np.sum(gmu * m.nu[:, k], axis=1))
            return (flux / (2.0 / 3.0 * m.patch_area))[m.tri].mean(axis=1)
        m = self.mesh
        gmu = m.grad(mu)
        out = np.zeros(m.T)
        for k in range(3):
            nb = m.nbr[:, k]
            inner = nb >= 0
            avg = 0.5 * (gmu + gmu[np.where(inner, nb, 0)])
            out += np.where(inner, np.sum(avg * m.nu[:, k], axis=1), 0.0)
        return out / m.area

    # -- element forces (eq:G, eq:H, eq:intF at the barycentre) ------------
    def forces(self, C, p, u, mu):
        m, pr = self.mesh, self.prm
        tri = m.tri
        Cb = C[tri].mean(axis=1)
        ub = u[tri].mean(axis=1)
        mub = mu[tri].mean(axis=1)
        rhob = Cb * pr.rho_l + (1.0 - Cb) * pr.rho_v
        gC = m.grad(C)
        gp = m.grad(p)
        grho = (pr.rho_l - pr.rho_v) * gC
        lmu = self.lap_mu(mu)
        G = gamma(ub)                                                      # (9, T)
        Phi_g = np.zeros((Q, m.T))
        Phi_h = np.zeros((Q, m.T))
        vh = gC - (Cb / (rhob * CS2))[:, None] * (gp - mub[:, None] * gC)
        for a in range(Q):
            em = D2Q9_E[a][None, :] - ub
            vg = CS2 * grho * (G[a] - D2Q9_W[a])[:, None] + (mub * G[a])[:, None] * gC
            Phi_g[a] = np.sum(em * vg, axis=1)
            Phi_h[a] = np.sum(em * vh, axis=1) * G[a] + pr.mobility * lmu * G[a]
        return Phi_g, Phi_h

    # -- equilibria (eqn::g_eq, eqn::f_eq) ----------------------------------
    @staticmethod
    def equilibria(C, p, u, rho):
        """g_eq = w (p + rho cs2 (e.u / cs2 + ((e.u)^2 - cs2 u.u) / (2 cs2^2)))
        and h_eq = Gamma(u) C, each (9, N)."""
        eu = u @ D2Q9_E.T                                                  # (N, 9)
        uu = np.sum(u * u, axis=1)
        geq = D2Q9_W[:, None] * (p[None, :] + (rho * CS2)[None, :] * (
            eu.T / CS2 + (eu.T ** 2 - CS2 * uu[None, :]) / (2.0 * CS2 * CS2)))
        heq = gamma(u) * C[None, :]
        return geq, heq

    # -- collision (eqn::collide) ------------------------------------------
    def collide(self, g, h, C, p, u, rho):
        pr = self.prm
        inv_tau = C / pr.tau_l + (1.0 - C) / pr.tau_v
        tau = 1.0 / inv_tau
        geq, heq = self.equilibria(C, p, u, rho)
        omega = 1.0 / (tau + 0.5)
        return g - omega[None, :] * (g - geq), h - omega[None, :] * (h - heq)

    # -- streaming right-hand side (eq:galerkin_lbm, sign reading) ---------
    def rhs(self, psi_hat, Phi):
        m, dt = self.mesh, self.prm.dt
        out = np.zeros_like(psi_hat)
        for a in range(Q):
            out[a] = (-dt * (m.Cmat[a] @ psi_hat[a]) - dt * dt * (m.Dmat[a] @ psi_hat[a])
                      + dt * (m.M10 @ Phi[a]) + dt * dt * (m.Kmat[a] @ Phi[a])
                      - dt * (m.Bmat[a] @ (psi_hat[D2Q9_OPP[a]] - psi_hat[a])))
        return out

    # -- mass-matrix solve: PCG with the lumped-mass preconditioner --------
    def solve_mass(self, B):
        """Solve M11 X = B column by column (B: (N, k)); start from B / m,
        stop a column when ||r|| <= tol ||b|| + 1e-300."""
        M, mvec = self.mesh.M11, self.mesh.lumped
        X = B / mvec[:, None]
        R = B - M @ X
        Z = R / mvec[:, None]
        Pd = Z.copy()
        rz = np.sum(R * Z, axis=0)
        bn = np.linalg.norm(B, axis=0)
        active = np.linalg.norm(R, axis=0) > self.tol * bn + 1e-300
        it = 0
        while active.any() and it < self.maxit:
            AP = M @ Pd
            pap = np.sum(Pd * AP, axis=0)
            alpha = np.where(active, rz / np.where(active, pap, 1.0), 0.0)
            X += alpha[None, :] * Pd
            R -= alpha[None, :] * AP
            Z = R / mvec[:, None]
            rz_new = np.sum(R * Z, axis=0)
            beta = np.where(active, rz_new / np.where(active, rz, 1.0), 0.0)
            Pd = Z + beta[None, :] * Pd
            rz = rz_new
            active &= np.linalg.norm(R, axis=0) > self.tol * bn + 1e-300
            it += 1
        self.last_iters = it
        if active.any():
            raise RuntimeError("oracle PCG did not converge")
        return X

    # -- one time step: forces from step-n fields, collision, streaming ----
    def step(self, n=1):
        for _ in range(n):
            C, p, u, rho = self.moments()
            mu = self.chemical_potential(C)
            Phi_g, Phi_h = self.forces(C, p, u, mu)
            g_hat, h_hat = self.collide(self.g, self.h, C, p, u, rho)
            rhs = np.concatenate([self.rhs(g_hat, Phi_g), self.rhs(h_hat, Phi_h)])   # (18, N)
            delta = self.solve_mass(rhs.T).T
            self.g = g_hat + delta[:Q]
            self.h = h_hat + delta[Q:]
            self.step_count += 1

    # -- diagnostics (Sec. III) --------------------------------------------
    def mass(self):
        return float(np.sum(self.mesh.lumped * self.h.sum(axis=0)))

    def diagnostics(self, centre=None, R=None, xi=None, substrate=0):
        m = self.mesh
        C, p, u, rho = self.moments()
        uu = np.sum(u * u, axis=1)
        d = {}
        d["step"] = self.step_count
        d["mass"] = self.mass()
        d["mass_drift_rel"] = (d["mass"] - self.mass0) / self.mass0
        d["kinetic_energy"] = 0.5 * float(np.sum(rho * uu)) / m.N     # <T> of Fig. 5
        d["max_u"] = float(np.sqrt(uu.max()))
        lw = m.lumped
        inside, outside = C >= 0.95, C <= 0.05
        p_in = np.sum(lw[inside] * p[inside]) / max(np.sum(lw[inside]), 1e-300)
        p_out = np.sum(lw[outside] * p[outside]) / max(np.sum(lw[outside]), 1e-300)
        d["p_in"], d["p_out"], d["delta_p"] = float(p_in), float(p_out), float(p_in - p_out)
        if centre is not None:
            r = np.linalg.norm(m.min_image(m.xy - np.asarray(centre)[None, :]), axis=1)
            band = np.abs(r - R) <= xi
            d["interface_rho_uu"] = float(np.sum(lw[band] * rho[band] * uu[band])
                                          / max(np.sum(lw[band]), 1e-300))
        # wetted length on the substrate wall: length of wall edges with C >= 1/2
        b = 0.0
        sub = m.wall_id == substrate
        for e in np.nonzero(sub)[0]:
            a, c = m.wall_edges[e]
            Ca, Cc = C[a], C[c]
            L = m.wall_len[e]
            if Ca >= 0.5 and Cc >= 0.5:
                b += L
            elif Ca >= 0.5 or Cc >= 0.5:
                hi, lo = max(Ca, Cc), min(Ca, Cc)
                b += L * (hi - 0.5) / (hi - lo)
        d["wetted_length"] = b
        # height of the C = 1/2 contour above the mean substrate height
        ymax = -np.inf
        for k in range(3):
            ia, ic = m.tri[:, (k + 1) % 3], m.tri[:, (k + 2) % 3]
            Ca, Cc = C[ia], C[ic]
            cross = (Ca >= 0.5) != (Cc >= 0.5)
            if np.any(cross):
                t = (0.5 - Ca[cross]) / (Cc[cross] - Ca[cross])
                ya = m.xy[ia[cross], 1]
                dy = m.min_image(m.xy[ic[cross]] - m.xy[ia[cross]])[:, 1]
                ymax = max(ymax, float(np.max(ya + t * dy)))
        if np.any(sub):
            ywall = float(np.mean(m.xy[np.unique(m.wall_edges[sub].reshape(-1)), 1]))
            hgt = ymax - ywall
            d["height"] = hgt
            if hgt > 0 and b > 0:
                r = (4.0 * hgt * hgt + b * b) / (8.0 * hgt)
                d["theta_deg"] = math.degrees(math.atan2(b, 2.0 * (r - hgt)))
            else:
                d["theta_deg"] = float("nan")
        return d
