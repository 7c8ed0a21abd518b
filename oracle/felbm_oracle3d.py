"""FP64 CPU oracle of the 3D FE-LBM time step (TEST INFRASTRUCTURE ONLY).

The paper's own setting (arXiv:1708.04678, Sec. II): D3Q19 velocities on
linear tetrahedra.  The scheme and every reading are those of the 2D oracle
(``felbm_oracle.py``), restated for d = 3:

* P1 tetrahedra; the FE matrices of eq:fem_matrices in closed form,
  M11 = V/20 (1 + d_ij), M10 = V/4, C_a = V/4 e.b_j, K_a = V/2 e.b_i,
  D_a = V/2 (e.b_i)(e.b_j), wall matrix A/12 (1 + d_pq) (e.n) on faces
  where the population is incoming -- pinned against quadrature by tests;
* patch Laplacian of C (eqn:lapl_int_mp): outward flux of grad C through the
  outer faces of the vertex patch, each wall face replaced by the wetting
  flux of eqn:bc2 (C linear on the face, integral exact), divided by
  V = lap_scale |patch|, lap_scale = d/(d+1) = 3/4 ("consistent", equal to
  the lumped P1 Laplacian) or 1 ("paper");
* element Laplacian of mu through the four faces (interior faces: mean of
  the two element gradients; wall faces zero, eqn:bc1);
* weak bounce-back on wall faces; force term +(dt M10 + dt^2 K) Phi;
  consistent-mass solve by PCG with the lumped-mass preconditioner;
* contact angle from the height h and base diameter b of the C = 1/2
  surface: theta = atan2(b, 2 (r - h)), r = (4 h^2 + b^2) / (8 h) (Sec. III.B),
  b the diameter of the circle with the wetted area.

Only the test-suite, the smoke check and the CPU legs of the benchmark may
use it; it shares no code with the CUDA path.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

# D3Q19 velocity set of Sec. II.A: rest, six axis and twelve face-diagonal
# velocities; weights 1/3, 1/18, 1/36; c_s^2 = 1/3.
D3Q19_E = np.array([(0, 0, 0),
                    (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
                    (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
                    (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
                    (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)], dtype=np.float64)
D3Q19_W = np.array([1.0 / 3.0] + [1.0 / 18.0] * 6 + [1.0 / 36.0] * 12)
D3Q19_OPP = np.array([int(np.nonzero(np.all(D3Q19_E == -D3Q19_E[a], axis=1))[0][0]) for a in range(19)])
CS2 = 1.0 / 3.0
Q = 19


class Params3D:
    """Model constants of Sec. II in lattice units."""

    def __init__(self, dt, tau_l, tau_v, rho_l, rho_v, kappa, beta, mobility, phi_c, lap_scale=0.75, lapmu="face"):
        self.lapmu = lapmu                   # element Laplacian of mu: "face" (Sec. II.D) or "nodal"
        self.dt, self.tau_l, self.tau_v = dt, tau_l, tau_v
        self.rho_l, self.rho_v = rho_l, rho_v
        self.kappa, self.beta, self.mobility = kappa, beta, mobility
        self.phi_c = tuple(phi_c)
        self.lap_scale = lap_scale


def params_from_physical3d(phys, lap_mode="consistent", lapmu="face"):
    """kappa = 3 sigma xi / 2, beta = 12 sigma / xi (interface width xi and
    tension sigma of the double-well free energy, Sec. II); phi_c from
    Young's relation cos(theta) = -phi_c / sqrt(2 kappa beta)."""
    sigma, xi = phys["sigma"], phys["xi"]
    kappa, beta = 1.5 * sigma * xi, 12.0 * sigma / xi
    root = math.sqrt(2.0 * kappa * beta)
    return Params3D(phys["dt"], phys["tau_l"], phys["tau_v"], phys["rho_l"], phys["rho_v"], kappa, beta,
                    phys["mobility"], [-root * math.cos(math.radians(t)) for t in phys["theta_deg"]],
                    0.75 if lap_mode == "consistent" else 1.0, lapmu)


def gamma3(u):
    """Gamma_a(u) of eqn::f_eq for velocities u (..., 3); returns (19, ...)."""
    eu = np.tensordot(D3Q19_E, u, axes=([1], [u.ndim - 1]))
    uu = np.sum(u * u, axis=-1)
    w = D3Q19_W.reshape((Q,) + (1,) * uu.ndim)
    return w * (1.0 + eu / CS2 + (eu * eu - CS2 * uu) / (2.0 * CS2 * CS2))


class OracleMesh3D:
    """P1 tetrahedral mesh and its global FE matrices.

    xyz (N, 3); tet (T, 4) positively oriented after the minimum image;
    wall_faces (F, 3) node triples; wall_id (F,); period (3,), 0 = not
    periodic along that axis.  Every face on the boundary must be a wall
    face and vice versa.
    """

    def __init__(self, xyz, tet, wall_faces, wall_id, period=(0.0, 0.0, 0.0)):
        self.xyz = np.asarray(xyz, dtype=np.float64)
        self.tet = np.asarray(tet, dtype=np.int64)
        self.wall_faces = np.asarray(wall_faces, dtype=np.int64).reshape(-1, 3)
        self.wall_id = np.asarray(wall_id, dtype=np.int64).reshape(-1)
        self.period = tuple(float(p) for p in period)
        self.N, self.T = len(self.xyz), len(self.tet)
        self._geometry()
        self._topology()
        self._matrices()

    def min_image(self, d):
        d = np.array(d, dtype=np.float64, copy=True)
        for k in range(3):
            if self.period[k] > 0:
                d[..., k] -= self.period[k] * np.round(d[..., k] / self.period[k])
        return d

    def _geometry(self):
        tet = self.tet
        P = np.zeros((self.T, 4, 3))
        for k in (1, 2, 3):
            P[:, k] = self.min_image(self.xyz[tet[:, k]] - self.xyz[tet[:, 0]])
        self.P = P
        self.vol = np.einsum("td,td->t", P[:, 1], np.cross(P[:, 2], P[:, 3])) / 6.0
        if np.any(self.vol <= 0):
            raise ValueError("oracle3d: tetrahedron with non-positive volume")
        # shape functions N_i = a_i + b_i.x from the 4x4 interpolation system
        A = np.concatenate([np.ones((self.T, 4, 1)), P], axis=2)
        coef = np.linalg.solve(A, np.broadcast_to(np.eye(4), (self.T, 4, 4)))   # column i: (a, b) of N_i
        self.b = np.transpose(coef[:, 1:, :], (0, 2, 1))                          # (T, 4, 3)
        # area-weighted outward normal of the face opposite vertex k
        nu = np.zeros((self.T, 4, 3))
        for k in range(4):
            f = [j for j in range(4) if j != k]
            n = 0.5 * np.cross(P[:, f[1]] - P[:, f[0]], P[:, f[2]] - P[:, f[0]])
            away = np.sum(n * (P[:, f[0]] - P[:, k]), axis=1)
            nu[:, k] = np.where((away < 0)[:, None], -n, n)
        self.nu = nu
        self.patch_vol = np.zeros(self.N)
        for k in range(4):
            np.add.at(self.patch_vol, tet[:, k], self.vol)

    def _topology(self):
        """Face neighbours (nbr[t, k]: the tetrahedron across the face opposite
        vertex k, -1 on walls) and the wall faces' areas and outward normals."""
        T, N = self.T, self.N
        faces = np.stack([np.sort(np.delete(self.tet, k, axis=1), axis=1) for k in range(4)], axis=1)
        key = (faces[..., 0] * N + faces[..., 1]) * N + faces[..., 2]          # (T, 4)
        flat = key.reshape(-1)
        order = np.argsort(flat, kind="stable")
        sk = flat[order]
        _, first, counts = np.unique(sk, return_index=True, return_counts=True)
        if np.any(counts > 2):
            raise ValueError("oracle3d: a face shared by more than two tetrahedra")
        self.nbr = -np.ones((T, 4), dtype=np.int64)
        pairs = first[counts == 2]
        a, b = order[pairs], order[pairs + 1]
        nb = self.nbr.reshape(-1)
        nb[a] = b // 4
        nb[b] = a // 4
        single = order[first[counts == 1]]
        wf = np.sort(self.wall_faces, axis=1)
        wkey = (wf[:, 0] * N + wf[:, 1]) * N + wf[:, 2]
        if len(np.unique(wkey)) != len(wkey) or set(wkey.tolist()) != set(flat[single].tolist()):
            raise ValueError("oracle3d: boundary faces and wall faces differ")
        where = {int(k): int(s) for k, s in zip(flat[single], single)}
        self.wall_area = np.zeros(len(wf))
        self.wall_normal = np.zeros((len(wf), 3))
        for e, k in enumerate(wkey):
            s = where[int(k)]
            n = self.nu[s // 4, s % 4]
            A = np.linalg.norm(n)
            self.wall_area[e] = A
            self.wall_normal[e] = n / A

    def _matrices(self):
        tet, V, b = self.tet, self.vol, self.b
        N, T = self.N, self.T
        rows = np.concatenate([tet[:, i] for i in range(4) for j in range(4)])
        cols = np.concatenate([tet[:, j] for i in range(4) for j in range(4)])
        vm = np.concatenate([V / 20.0 * (2.0 if i == j else 1.0) for i in range(4) for j in range(4)])
        self.M11 = sp.csr_matrix((vm, (rows, cols)), shape=(N, N))
        ncol = np.concatenate([tet[:, i] for i in range(4)])
        tcol = np.concatenate([np.arange(T)] * 4)
        self.M10 = sp.csr_matrix((np.concatenate([V / 4.0] * 4), (ncol, tcol)), shape=(N, T))
        self.lumped = np.asarray(self.M11.sum(axis=1)).reshape(-1)
        self.Cmat, self.Kmat, self.Dmat, self.Bmat = [], [], [], []
        F = len(self.wall_faces)
        for a in range(Q):
            e = D3Q19_E[a]
            eb = b @ e                                                            # (T, 4): e . grad N_i
            vC = np.concatenate([V / 4.0 * eb[:, j] for i in range(4) for j in range(4)])
            vD = np.concatenate([V / 2.0 * eb[:, i] * eb[:, j] for i in range(4) for j in range(4)])
            self.Cmat.append(sp.csr_matrix((vC, (rows, cols)), shape=(N, N)))     # int N_i e.grad N_j
            self.Dmat.append(sp.csr_matrix((vD, (rows, cols)), shape=(N, N)))     # 1/2 int (e.gN_i)(e.gN_j)
            self.Kmat.append(sp.csr_matrix((np.concatenate([V / 2.0 * eb[:, i] for i in range(4)]),
                                            (ncol, tcol)), shape=(N, T)))         # 1/2 int e.grad N_i
            # incoming wall populations: int_face N_p N_q (e.n_out) dS, e.n_out < 0
            en = self.wall_normal @ e if F else np.zeros(0)
            inc = np.nonzero(en < 0.0)[0]
            br, bc, bv = [np.zeros(0, np.int64)], [np.zeros(0, np.int64)], [np.zeros(0)]
            for p in range(3):
                for q in range(3):
                    br.append(self.wall_faces[inc, p])
                    bc.append(self.wall_faces[inc, q])
                    bv.append(en[inc] * self.wall_area[inc] / 12.0 * (2.0 if p == q else 1.0))
            self.Bmat.append(sp.csr_matrix((np.concatenate(bv), (np.concatenate(br), np.concatenate(bc))),
                                           shape=(N, N)))

    def grad(self, f):
        """P0 gradient of the P1 interpolant of nodal values f: (T, 3)."""
        return np.einsum("ti,tid->td", f[self.tet], self.b)


class OracleSim3D:
    """State (g, h) on an OracleMesh3D and the time step of Sec. II.C."""

    def __init__(self, mesh, params, C0, p0=None, solver_tol=1e-14, solver_maxit=300):
        self.mesh, self.prm = mesh, params
        self.tol, self.maxit = solver_tol, solver_maxit
        N = mesh.N
        C0 = np.asarray(C0, dtype=np.float64)
        p0 = np.zeros(N) if p0 is None else np.asarray(p0, dtype=np.float64)
        self.g = D3Q19_W[:, None] * p0[None, :]
        self.h = D3Q19_W[:, None] * C0[None, :]
        self.step_count = 0
        self.mass0 = self.mass()

    def moments(self, g=None, h=None):
        g = self.g if g is None else g
        h = self.h if h is None else h
        p = self.prm
        C, pr = h.sum(0), g.sum(0)
        rho = C * p.rho_l + (1 - C) * p.rho_v
        u = (D3Q19_E.T @ g).T / (CS2 * rho[:, None])
        return C, pr, u, rho

    def kappa_lap_C(self, C):
        """kappa * Laplacian of C at the nodes (eqn:lapl_int_mp with the wall
        flux kappa n_out.grad C = -phi_c (C - C^2) of eqn:bc2)."""
        m, p = self.mesh, self.prm
        gC = m.grad(C)
        flux = np.zeros(m.N)
        for k in range(4):
            np.add.at(flux, m.tet[:, k], p.kappa * np.sum(gC * m.nu[:, k], axis=1))
        if len(m.wall_faces):
            Cf = C[m.wall_faces]                                          # (F, 3)
            A = m.wall_area
            int_C = A * Cf.sum(1) / 3.0
            int_C2 = A / 6.0 * (np.sum(Cf * Cf, 1) + Cf[:, 0] * Cf[:, 1] + Cf[:, 1] * Cf[:, 2]
                                + Cf[:, 2] * Cf[:, 0])
            q = -np.asarray(p.phi_c)[m.wall_id] * (int_C - int_C2)
            for k in range(3):
                np.add.at(flux, m.wall_faces[:, k], q)
        return flux / (p.lap_scale * m.patch_vol)

    def chemical_potential(self, C):
        p = self.prm
        return 2.0 * p.beta * C * (C - 1.0) * (2.0 * C - 1.0) - self.kappa_lap_C(C)

    def lap_mu(self, mu):
        """Element Laplacian of mu.  "face" (Sec. II.D): flux through the four
        faces, interior faces taking the mean of the two element gradients,
        wall faces zero (eqn:bc1).  "nodal": the patch Laplacian of
        eqn:lapl_int_mp applied to mu with the zero wall flux of eqn:bc1
        (volume 3/4 |patch|, the lumped P1 Laplacian), averaged over the
        element's vertices."""
        m = self.mesh
        if self.prm.lapmu == "nodal":
            gmu = m.grad(mu)
            flux = np.zeros(m.N)
            for k in range(4):
                np.add.at(flux, m.tet[:, k], np.sum(gmu * m.nu[:, k], axis=1))
            return (flux / (0.75 * m.patch_vol))[m.tet].mean(axis=1)
        gmu = m.grad(mu)
        out = np.zeros(m.T)
        for k in range(4):
            nb = m.nbr[:, k]
            inner = nb >= 0
            avg = 0.5 * (gmu + gmu[np.where(inner, nb, 0)])
            out += np.where(inner, np.sum(avg * m.nu[:, k], axis=1), 0.0)
        return out / m.vol

    def forces(self, C, pr, u, mu):
        """P0 forces at the element barycentre (eq:G, eq:H)."""
        m, p = self.mesh, self.prm
        tet = m.tet
        Cb, ub, mub = C[tet].mean(1), u[tet].mean(1), mu[tet].mean(1)
        rhob = Cb * p.rho_l + (1 - Cb) * p.rho_v
        gC, gp = m.grad(C), m.grad(pr)
        grho = (p.rho_l - p.rho_v) * gC
        lmu = self.lap_mu(mu)
        G = gamma3(ub)
        vh = gC - (Cb / (rhob * CS2))[:, None] * (gp - mub[:, None] * gC)
        Pg, Ph = np.zeros((Q, m.T)), np.zeros((Q, m.T))
        for a in range(Q):
            em = D3Q19_E[a][None, :] - ub
            vg = CS2 * grho * (G[a] - D3Q19_W[a])[:, None] + (mub * G[a])[:, None] * gC
            Pg[a] = np.sum(em * vg, axis=1)
            Ph[a] = np.sum(em * vh, axis=1) * G[a] + p.mobility * lmu * G[a]
        return Pg, Ph

    def collide(self, g, h, C, pr, u, rho):
        """BGK collision (eqn::collide) towards eqn::g_eq / eqn::f_eq."""
        p = self.prm
        tau = 1.0 / (C / p.tau_l + (1 - C) / p.tau_v)
        eu = u @ D3Q19_E.T
        uu = np.sum(u * u, axis=1)
        geq = D3Q19_W[:, None] * (pr[None, :] + (rho * CS2)[None, :] *
                                  (eu.T / CS2 + (eu.T ** 2 - CS2 * uu[None, :]) / (2 * CS2 * CS2)))
        heq = gamma3(u) * C[None, :]
        om = 1.0 / (tau + 0.5)
        return g - om * (g - geq), h - om * (h - heq)

    def rhs(self, psi, Phi):
        """Streaming right-hand side of eq:galerkin_lbm (sign reading as in 2D)."""
        m, dt = self.mesh, self.prm.dt
        out = np.zeros_like(psi)
        for a in range(Q):
            out[a] = (-dt * (m.Cmat[a] @ psi[a]) - dt * dt * (m.Dmat[a] @ psi[a])
                      + dt * (m.M10 @ Phi[a]) + dt * dt * (m.Kmat[a] @ Phi[a])
                      - dt * (m.Bmat[a] @ (psi[D3Q19_OPP[a]] - psi[a])))
        return out

    def solve_mass(self, B):
        """Solve M11 X = B column by column by PCG (lumped preconditioner)."""
        M, mv = self.mesh.M11, self.mesh.lumped
        X = B / mv[:, None]
        R = B - M @ X
        Z = R / mv[:, None]
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
            Z = R / mv[:, None]
            rz_new = np.sum(R * Z, axis=0)
            beta = np.where(active, rz_new / np.where(active, rz, 1.0), 0.0)
            Pd = Z + beta[None, :] * Pd
            rz = rz_new
            active &= np.linalg.norm(R, axis=0) > self.tol * bn + 1e-300
            it += 1
        if active.any():
            raise RuntimeError("oracle3d PCG did not converge")
        return X

    def step(self, n=1):
        for _ in range(n):
            C, pr, u, rho = self.moments()
            mu = self.chemical_potential(C)
            Pg, Ph = self.forces(C, pr, u, mu)
            gh, hh = self.collide(self.g, self.h, C, pr, u, rho)
            d = self.solve_mass(np.concatenate([self.rhs(gh, Pg), self.rhs(hh, Ph)]).T).T
            self.g, self.h = gh + d[:Q], hh + d[Q:]
            self.step_count += 1

    # -- diagnostics (Sec. III) --------------------------------------------
    def mass(self):
        return float(np.sum(self.mesh.lumped * self.h.sum(0)))

    def diagnostics(self, centre=None, R=None, xi=None, substrate=0):
        m = self.mesh
        C, pr, u, rho = self.moments()
        uu = np.sum(u * u, axis=1)
        lw = m.lumped
        d = {"step": self.step_count, "mass": self.mass()}
        d["mass_drift_rel"] = (d["mass"] - self.mass0) / self.mass0
        d["kinetic_energy"] = 0.5 * float(np.sum(rho * uu)) / m.N
        d["max_u"] = float(np.sqrt(uu.max()))
        inside, outside = C >= 0.95, C <= 0.05
        p_in = np.sum(lw[inside] * pr[inside]) / max(np.sum(lw[inside]), 1e-300)
        p_out = np.sum(lw[outside] * pr[outside]) / max(np.sum(lw[outside]), 1e-300)
        d["p_in"], d["p_out"], d["delta_p"] = float(p_in), float(p_out), float(p_in - p_out)
        if centre is not None:
            r = np.linalg.norm(m.min_image(m.xyz - np.asarray(centre)[None, :]), axis=1)
            band = np.abs(r - R) <= xi
            d["interface_rho_uu"] = float(np.sum(lw[band] * rho[band] * uu[band])
                                          / max(np.sum(lw[band]), 1e-300))
        sub = m.wall_id == substrate
        if not np.any(sub):
            return d
        # wetted area of the substrate: the part of each wall face where the
        # linear interpolant of C is at least 1/2
        area = 0.0
        for f in np.nonzero(sub)[0]:
            c = np.sort(C[m.wall_faces[f]])[::-1]                    # c0 >= c1 >= c2
            A = m.wall_area[f]
            if c[2] >= 0.5:
                area += A
            elif c[0] < 0.5:
                pass
            elif c[1] < 0.5:                                           # only c0 above: corner triangle
                area += A * (c[0] - 0.5) / (c[0] - c[1]) * (c[0] - 0.5) / (c[0] - c[2])
            else:                                                      # only c2 below
                area += A * (1.0 - (0.5 - c[2]) / (c[0] - c[2]) * (0.5 - c[2]) / (c[1] - c[2]))
        d["wetted_area"] = area
        # height of the C = 1/2 surface: highest crossing on a tetrahedron edge
        zmax = -np.inf
        for i in range(4):
            for j in range(i + 1, 4):
                ia, ib = m.tet[:, i], m.tet[:, j]
                Ca, Cb = C[ia], C[ib]
                cross = (Ca >= 0.5) != (Cb >= 0.5)
                if np.any(cross):
                    t = (0.5 - Ca[cross]) / (Cb[cross] - Ca[cross])
                    dz = m.min_image(m.xyz[ib[cross]] - m.xyz[ia[cross]])[:, 2]
                    zmax = max(zmax, float(np.max(m.xyz[ia[cross], 2] + t * dz)))
        zwall = float(np.mean(m.xyz[np.unique(m.wall_faces[sub].reshape(-1)), 2]))
        hgt = zmax - zwall
        b = 2.0 * math.sqrt(area / math.pi)
        d["height"], d["base_diameter"] = hgt, b
        if hgt > 0 and b > 0:
            r = (4.0 * hgt * hgt + b * b) / (8.0 * hgt)
            d["theta_deg"] = math.degrees(math.atan2(b, 2.0 * (r - hgt)))
        else:
            d["theta_deg"] = float("nan")
        return d
