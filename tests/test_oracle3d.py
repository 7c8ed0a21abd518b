"""Pins of the 3D oracle (D3Q19 on linear tetrahedra, Sec. II of the paper).

Each test checks the oracle against something fixed outside it: lattice
isotropy and the textbook equilibrium moments, brute-force quadrature of every
FE matrix, the 7-point stencil the P1 Laplacian reduces to on an unjittered
Kuhn mesh, the exact planar equilibrium profile meeting a wall at Young's
angle (which pins the wetting flux and its sign), the moment identities of
the forcing terms, the static-interface balance of Sec. II.C, exact mass
conservation, stationary uniform states and the advection speed.
"""
import math

import numpy as np
import pytest

from oracle.felbm_oracle3d import (CS2, D3Q19_E, D3Q19_OPP, D3Q19_W, OracleMesh3D, OracleSim3D,
                                   gamma3, params_from_physical3d)
from paper_1708_04678_gb300 import inputs3d as I3


def _mesh(m):
    return OracleMesh3D(m["xyz"], m["tet"], m["wall_faces"], m["wall_id"], m["period"])


def _phys(**kw):
    base = dict(dt=0.25, tau_l=0.8, tau_v=0.8, rho_l=1.0, rho_v=0.5, sigma=0.01, xi=4.0,
                mobility=0.02, theta_deg=(90.0, 90.0))
    base.update(kw)
    return base


# ---------------------------------------------------------------- lattice ---
def test_d3q19_isotropy():
    E, W = D3Q19_E, D3Q19_W
    assert len(E) == 19 and len({tuple(e) for e in E}) == 19
    assert abs(W.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(W @ E, 0.0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("a,ai,aj->ij", W, E, E), CS2 * np.eye(3), atol=1e-16)
    np.testing.assert_allclose(np.einsum("a,ai,aj,ak->ijk", W, E, E, E), 0.0, atol=1e-16)
    d = np.eye(3)
    iso4 = CS2 * CS2 * (np.einsum("ij,kl->ijkl", d, d) + np.einsum("ik,jl->ijkl", d, d)
                        + np.einsum("il,jk->ijkl", d, d))
    np.testing.assert_allclose(np.einsum("a,ai,aj,ak,al->ijkl", W, E, E, E, E), iso4, atol=1e-16)
    for a in range(19):
        np.testing.assert_array_equal(E[D3Q19_OPP[a]], -E[a])


def test_gamma_moments():
    """sum Gamma = 1, sum e Gamma = u, sum e e Gamma = cs2 I + u u."""
    rng = np.random.default_rng(0)
    u = rng.uniform(-0.1, 0.1, (7, 3))
    G = gamma3(u)
    np.testing.assert_allclose(G.sum(0), 1.0, atol=1e-15)
    np.testing.assert_allclose(np.einsum("an,ai->ni", G, D3Q19_E), u, atol=1e-16)
    np.testing.assert_allclose(np.einsum("an,ai,aj->nij", G, D3Q19_E, D3Q19_E),
                               CS2 * np.eye(3)[None] + np.einsum("ni,nj->nij", u, u), atol=1e-16)


def test_equilibrium_and_collision_moments():
    m = _mesh(I3.kuhn_box(3, 3, 3, 0.1, 0, walls=False))
    prm = params_from_physical3d(_phys(tau_l=0.5, tau_v=0.5))
    sim = OracleSim3D(m, prm, np.full(m.N, 0.5))
    rng = np.random.default_rng(1)
    N = m.N
    C = rng.uniform(0, 1, N); p = rng.uniform(-0.1, 0.1, N); u = rng.uniform(-0.1, 0.1, (N, 3))
    rho = C * prm.rho_l + (1 - C) * prm.rho_v
    geq, heq = sim.collide(rng.standard_normal((19, N)), rng.standard_normal((19, N)), C, p, u, rho)
    E = D3Q19_E
    np.testing.assert_allclose(geq.sum(0), p, atol=1e-15)
    np.testing.assert_allclose(E.T @ geq, (rho * CS2)[None] * u.T, atol=1e-15)
    np.testing.assert_allclose(heq.sum(0), C, atol=1e-15)
    np.testing.assert_allclose(E.T @ heq, C[None] * u.T, atol=1e-15)
    for a in range(3):
        for b in range(3):
            sg = np.einsum("q,qn->n", E[:, a] * E[:, b], geq)
            sh = np.einsum("q,qn->n", E[:, a] * E[:, b], heq)
            np.testing.assert_allclose(sg, CS2 * (p * (a == b) + rho * u[:, a] * u[:, b]), atol=1e-15)
            np.testing.assert_allclose(sh, C * (CS2 * (a == b) + u[:, a] * u[:, b]), atol=1e-15)
    # general tau: mass of both sets and the momentum of g are conserved
    sim.prm = params_from_physical3d(_phys(tau_l=0.7, tau_v=1.3))
    g = rng.standard_normal((19, N)) * 0.01
    h = rng.uniform(0, 0.1, (19, N))
    C, p, u, rho = sim.moments(g, h)
    gh, hh = sim.collide(g, h, C, p, u, rho)
    np.testing.assert_allclose(gh.sum(0), g.sum(0), atol=1e-15)
    np.testing.assert_allclose(hh.sum(0), h.sum(0), atol=1e-15)
    np.testing.assert_allclose(E.T @ gh, E.T @ g, atol=1e-15)


# --------------------------------------------------------------- matrices ---
def _two_tet_mesh():
    xyz = np.array([[0.0, 0.0, 0.0], [1.2, 0.1, -0.1], [0.2, 1.1, 0.1], [0.1, 0.2, 1.3], [1.0, 1.0, 1.1]])
    tet = np.array([[0, 1, 2, 3], [1, 2, 3, 4]])
    for t in tet:                                  # orient positively
        P = xyz[t[1:]] - xyz[t[0]]
        if np.linalg.det(P) < 0:
            t[1], t[2] = t[2], t[1]
    faces = [[0, 1, 2], [0, 1, 3], [0, 2, 3], [1, 2, 4], [1, 3, 4], [2, 3, 4]]
    return OracleMesh3D(xyz, tet, faces, [0, 0, 1, 1, 0, 1])


def _small_periodic_mesh():
    return _mesh(I3.kuhn_box(3, 3, 3, 0.15, 123, walls=False))


def _small_walled_mesh():
    return _mesh(I3.kuhn_box(3, 3, 2, 0.15, 321, walls=True))


# 4-point rule on the reference tetrahedron, exact for degree 2
_QA, _QB = 0.5854101966249685, 0.1381966011250105
_TET_BARY = np.array([[_QA, _QB, _QB, _QB], [_QB, _QA, _QB, _QB], [_QB, _QB, _QA, _QB], [_QB, _QB, _QB, _QA]])


def _brute_force(mesh):
    """Dense M11, M10, C_a, K_a, D_a and incoming-wall B_a by quadrature of
    the shape functions (each obtained from its own interpolation system)."""
    N, T = mesh.N, mesh.T
    M11 = np.zeros((N, N)); M10 = np.zeros((N, T))
    Cm = np.zeros((19, N, N)); Km = np.zeros((19, N, T)); Dm = np.zeros((19, N, N)); Bm = np.zeros((19, N, N))
    for t in range(T):
        ids = mesh.tet[t]
        X = np.zeros((4, 3))
        for k in (1, 2, 3):
            X[k] = mesh.min_image(mesh.xyz[ids[k]] - mesh.xyz[ids[0]])
        coef = np.linalg.solve(np.column_stack([np.ones(4), X]), np.eye(4))
        grads = coef[1:, :].T                                         # (4, 3)
        vol = abs(np.linalg.det(X[1:] - X[0])) / 6.0
        qp = _TET_BARY @ X
        Nq = np.column_stack([np.ones(4), qp]) @ coef                 # (4 points, 4 functions)
        wq = vol / 4.0
        for i in range(4):
            M10[ids[i], t] += wq * Nq[:, i].sum()
            for j in range(4):
                M11[ids[i], ids[j]] += wq * np.sum(Nq[:, i] * Nq[:, j])
        for a in range(19):
            e = D3Q19_E[a]
            for i in range(4):
                Km[a, ids[i], t] += 0.5 * vol * (e @ grads[i])
                for j in range(4):
                    Cm[a, ids[i], ids[j]] += wq * np.sum(Nq[:, i]) * (e @ grads[j])
                    Dm[a, ids[i], ids[j]] += 0.5 * vol * (e @ grads[i]) * (e @ grads[j])
    for f, face in enumerate(mesh.wall_faces):
        X = np.array([mesh.xyz[face[0]], mesh.xyz[face[0]] + mesh.min_image(mesh.xyz[face[1]] - mesh.xyz[face[0]]),
                      mesh.xyz[face[0]] + mesh.min_image(mesh.xyz[face[2]] - mesh.xyz[face[0]])])
        nrm = np.cross(X[1] - X[0], X[2] - X[0])
        A = 0.5 * np.linalg.norm(nrm)
        nrm /= np.linalg.norm(nrm)
        # outward: away from the fourth vertex of the tetrahedron owning the face
        t = next(t for t in range(T) if set(face) <= set(mesh.tet[t]))
        other = [v for v in mesh.tet[t] if v not in face][0]
        if nrm @ mesh.min_image(mesh.xyz[other] - X[0]) > 0:
            nrm = -nrm
        # edge-midpoint rule on the triangle, exact for degree 2
        mid = [(0, 1), (1, 2), (2, 0)]
        for a in range(19):
            en = D3Q19_E[a] @ nrm
            if en >= 0:
                continue
            for p in range(3):
                for q in range(3):
                    val = sum((0.5 * ((p == i) + (p == j))) * (0.5 * ((q == i) + (q == j))) for i, j in mid)
                    Bm[a, face[p], face[q]] += en * A / 3.0 * val
    return M11, M10, Cm, Km, Dm, Bm


@pytest.mark.parametrize("make", [_two_tet_mesh, _small_periodic_mesh, _small_walled_mesh])
def test_matrices_match_quadrature(make):
    m = make()
    M11, M10, Cm, Km, Dm, Bm = _brute_force(m)
    np.testing.assert_allclose(m.M11.toarray(), M11, atol=1e-13)
    np.testing.assert_allclose(m.M10.toarray(), M10, atol=1e-13)
    for a in range(19):
        np.testing.assert_allclose(m.Cmat[a].toarray(), Cm[a], atol=1e-13)
        np.testing.assert_allclose(m.Kmat[a].toarray(), Km[a], atol=1e-13)
        np.testing.assert_allclose(m.Dmat[a].toarray(), Dm[a], atol=1e-13)
        np.testing.assert_allclose(m.Bmat[a].toarray(), Bm[a], atol=1e-13)


def test_mass_row_sums_and_spectrum():
    """Row sums of M11 are the nodal volumes |patch|/4; the lumped-mass
    preconditioned spectrum lies in [1/5, 1] (element matrix (I + 1 1^T)/5
    relative to its lumped diagonal), with 1 attained by constants."""
    for m in (_small_periodic_mesh(), _small_walled_mesh()):
        np.testing.assert_allclose(m.lumped, m.patch_vol / 4.0, rtol=1e-14)
        assert abs(m.lumped.sum() - m.vol.sum()) < 1e-12 * m.vol.sum()
        Md = m.M11.toarray()
        s = 1.0 / np.sqrt(m.lumped)
        ev = np.linalg.eigvalsh(s[:, None] * Md * s[None, :])
        assert ev.min() >= 0.2 - 1e-12 and ev.max() <= 1.0 + 1e-12
        assert abs(ev.max() - 1.0) < 1e-12


def test_conservation_sums():
    """Periodic mesh: sum_i C_a[i, :] = 0 (no boundary), sum_i D_a[i, :] = 0
    and sum_i K_a[i, :] = 0 (shape-function gradients sum to zero),
    sum_i M10[i, t] = V_t."""
    m = _small_periodic_mesh()
    np.testing.assert_allclose(np.asarray(m.M10.sum(axis=0)).ravel(), m.vol, rtol=1e-14)
    for a in range(19):
        assert np.abs(np.asarray(m.Cmat[a].sum(axis=0))).max() < 1e-13
        assert np.abs(np.asarray(m.Dmat[a].sum(axis=0))).max() < 1e-13
        assert np.abs(np.asarray(m.Kmat[a].sum(axis=0))).max() < 1e-13


def test_gradient_exact_on_linear_fields():
    m = _two_tet_mesh()
    f = 0.3 + 1.5 * m.xyz[:, 0] - 2.0 * m.xyz[:, 1] + 0.7 * m.xyz[:, 2]
    np.testing.assert_allclose(m.grad(f), np.tile([1.5, -2.0, 0.7], (m.T, 1)), atol=1e-13)
    w = _small_walled_mesh()                     # z is not periodic there
    np.testing.assert_allclose(w.grad(2.0 + 3.0 * w.xyz[:, 2]), np.tile([0.0, 0.0, 3.0], (w.T, 1)), atol=1e-13)


# ------------------------------------------------------------- Laplacians ---
def test_patch_laplacian_is_seven_point_stencil_on_kuhn_mesh():
    """Unjittered Kuhn mesh: the consistent patch Laplacian of C equals the
    7-point stencil (sum of the six axis neighbours - 6 C) / h^2."""
    n = 6
    mm = I3.kuhn_box(n, n, n, 0.0, 0, walls=False)
    m = _mesh(mm)
    prm = params_from_physical3d(_phys(theta_deg=()))
    x, y, z = m.xyz.T
    C = np.cos(2 * np.pi * x / n) * np.sin(4 * np.pi * y / n) + 0.3 * np.cos(2 * np.pi * z / n)
    lap = OracleSim3D(m, prm, C).kappa_lap_C(C) / prm.kappa
    idx = np.rint(m.xyz).astype(int) % n
    grid = np.zeros((n, n, n)); grid[idx[:, 0], idx[:, 1], idx[:, 2]] = C
    seven = sum(np.roll(grid, s, axis=ax) for ax in range(3) for s in (1, -1)) - 6 * grid
    np.testing.assert_allclose(lap, seven[idx[:, 0], idx[:, 1], idx[:, 2]], atol=1e-12)


def test_paper_mode_laplacian_is_three_quarters():
    m = _mesh(I3.kuhn_box(4, 4, 3, 0.15, 1, walls=True))
    C = np.sin(2 * np.pi * m.xyz[:, 0] / 4) + 0.3 * m.xyz[:, 2]
    ph = _phys(theta_deg=(60.0, 120.0))
    a = OracleSim3D(m, params_from_physical3d(ph, "consistent"), C).kappa_lap_C(C)
    b = OracleSim3D(m, params_from_physical3d(ph, "paper"), C).kappa_lap_C(C)
    np.testing.assert_allclose(b, a * 0.75, rtol=1e-13, atol=1e-16)


def _tilted_slab(nx, nz, theta_deg, xi, xl, xr, ny=3, jitter=0.0, seed=0):
    """Liquid slab between two planar interfaces (uniform in y) meeting the
    substrate z = 0 at theta and the top wall at 180 - theta: the exact
    equilibrium of Sec. II with the wetting condition eqn:bc2."""
    mm = I3.kuhn_box(nx, ny, nz, jitter, seed, walls=True)
    x, z = mm["xyz"][:, 0], mm["xyz"][:, 2]
    th = math.radians(theta_deg)
    nxs, nzs = math.sin(th), -math.cos(th)
    sl = (x - xl) * nxs + z * nzs
    sr = -(x - xr) * nxs + z * nzs
    C = (0.5 + 0.5 * np.tanh(2 * sl / xi)) * (0.5 + 0.5 * np.tanh(2 * sr / xi))
    return mm, C


@pytest.mark.parametrize("theta", [90.0, 60.0, 120.0])
def test_chemical_potential_vanishes_on_exact_equilibria(theta):
    """Planar tanh profiles meeting the walls at Young's angle give mu = 0 up
    to discretisation error; the flipped wetting sign gives mu = O(beta), the
    literal patch volume ("paper" mode) an O(beta/10) residual."""
    xi = 8.0
    mm, C = _tilted_slab(120, 20, theta, xi, 35.0, 85.0)
    m = _mesh(mm)
    phys = _phys(xi=xi, theta_deg=(theta, 180.0 - theta))
    prm = params_from_physical3d(phys)
    mu = OracleSim3D(m, prm, C).chemical_potential(C)
    assert np.abs(mu).max() < 0.02 * prm.beta
    paper = OracleSim3D(m, params_from_physical3d(phys, "paper"), C).chemical_potential(C)
    assert np.abs(paper).max() > 0.04 * prm.beta
    if theta != 90.0:
        bad = params_from_physical3d(dict(phys, theta_deg=(180.0 - theta, theta)))
        assert np.abs(OracleSim3D(m, bad, C).chemical_potential(C)).max() > 0.5 * prm.beta


def test_chemical_potential_error_is_second_order():
    errs = []
    for xi in (4.0, 8.0):
        mm, C = _tilted_slab(120, 20, 90.0, xi, 35.0, 85.0)
        prm = params_from_physical3d(_phys(xi=xi))
        errs.append(np.abs(OracleSim3D(_mesh(mm), prm, C).chemical_potential(C)).max() / prm.beta)
    assert 3.0 < errs[0] / errs[1] < 5.0


# ----------------------------------------------------------------- forces ---
def test_force_moment_identities():
    """With the exact second moments of Gamma:
       sum_a Phi_g = cs2 u.grad(rho),  sum_a e_a Phi_g = cs2 mu grad C,
       sum_a Phi_h = M lap(mu),        sum_a e_a Phi_h = cs2 v_h + M lap(mu) u,
    v_h = grad C - C/(rho cs2) (grad p - mu grad C); the volume-weighted sum
    of lap(mu) vanishes (fluxes telescope, walls give zero)."""
    m = _mesh(I3.kuhn_box(4, 4, 3, 0.15, 5, walls=True))
    prm = params_from_physical3d(_phys(theta_deg=(60.0, 120.0)))
    sim = OracleSim3D(m, prm, np.full(m.N, 0.5))
    rng = np.random.default_rng(3)
    C = rng.uniform(0, 1, m.N); p = rng.uniform(-0.01, 0.01, m.N)
    u = rng.uniform(-0.05, 0.05, (m.N, 3))
    mu = sim.chemical_potential(C)
    Pg, Ph = sim.forces(C, p, u, mu)
    lmu = sim.lap_mu(mu)
    tet = m.tet
    Cb, ub, mub = C[tet].mean(1), u[tet].mean(1), mu[tet].mean(1)
    rhob = Cb * prm.rho_l + (1 - Cb) * prm.rho_v
    gC, gp = m.grad(C), m.grad(p)
    grho = (prm.rho_l - prm.rho_v) * gC
    vh = gC - (Cb / (rhob * CS2))[:, None] * (gp - mub[:, None] * gC)
    np.testing.assert_allclose(Pg.sum(0), CS2 * np.sum(ub * grho, 1), atol=1e-14)
    np.testing.assert_allclose(D3Q19_E.T @ Pg, (CS2 * mub[:, None] * gC).T, atol=1e-14)
    np.testing.assert_allclose(Ph.sum(0), prm.mobility * lmu, atol=1e-14)
    np.testing.assert_allclose(D3Q19_E.T @ Ph, (CS2 * vh + prm.mobility * lmu[:, None] * ub).T, atol=1e-14)
    assert abs(np.sum(m.vol * lmu)) < 1e-12 * np.sum(m.vol * np.abs(lmu))


# --------------------------------------------------------------- the step ---
def test_static_interface_balance():
    """kappa = beta = 0, u = p = 0, any C on a periodic jittered mesh: the P0
    force balances streaming of h = w C (Sec. II.C); C stays put, g zero."""
    m = _mesh(I3.kuhn_box(5, 5, 5, 0.15, 7, walls=False))
    prm = params_from_physical3d(_phys(theta_deg=()))
    prm.kappa = prm.beta = 0.0
    C0 = np.random.default_rng(4).uniform(0, 1, m.N)
    sim = OracleSim3D(m, prm, C0)
    sim.step(10)
    C, p, u, rho = sim.moments()
    assert np.abs(C - C0).max() < 1e-13
    assert np.abs(sim.g).max() < 1e-15


def _equilibria(sim, C, p, u, rho):
    prm = sim.prm
    tl, tv = prm.tau_l, prm.tau_v
    prm.tau_l = prm.tau_v = 0.5
    N = len(C)
    geq, heq = sim.collide(np.zeros((19, N)), np.zeros((19, N)), C, np.full(N, p), u, np.full(N, rho))
    prm.tau_l, prm.tau_v = tl, tv
    return geq, heq


@pytest.mark.parametrize("case", ["liquid_wetting_walls", "mixture_neutral_walls", "moving_periodic"])
def test_uniform_states_are_stationary(case):
    if case == "moving_periodic":
        m = _mesh(I3.kuhn_box(4, 4, 4, 0.15, 3, walls=False))
        prm = params_from_physical3d(_phys(theta_deg=()))
        C0 = np.full(m.N, 0.4)
        sim = OracleSim3D(m, prm, C0)
        rho = 0.4 * prm.rho_l + 0.6 * prm.rho_v
        sim.g, sim.h = _equilibria(sim, C0, 0.02, np.tile([0.03, -0.02, 0.01], (m.N, 1)), rho)
    else:
        m = _mesh(I3.kuhn_box(4, 4, 3, 0.15, 3, walls=True))
        theta = (60.0, 120.0) if case == "liquid_wetting_walls" else (90.0, 90.0)
        prm = params_from_physical3d(_phys(theta_deg=theta))
        c = 1.0 if case == "liquid_wetting_walls" else 0.3
        sim = OracleSim3D(m, prm, np.full(m.N, c), p0=np.full(m.N, 0.01))
    g0, h0 = sim.g.copy(), sim.h.copy()
    sim.step(8)
    assert np.abs(sim.g - g0).max() < 1e-13
    assert np.abs(sim.h - h0).max() < 1e-13


def test_mass_is_conserved_with_wetting_walls():
    w = I3.small_sessile_3d()
    sim = OracleSim3D(_mesh(w["mesh"]), params_from_physical3d(w["phys"]), w["C0"])
    sim.step(10)
    assert abs(sim.diagnostics()["mass_drift_rel"]) < 10 * 2e-15


def test_uniform_flow_advects_composition():
    """rho_l = rho_v, kappa = beta = 0: h carries C at the fluid velocity;
    the phase of the first Fourier mode along x moves by u t."""
    n = 8
    m = _mesh(I3.kuhn_box(n, 4, 4, 0.1, 8, walls=False))
    prm = params_from_physical3d(_phys(rho_v=1.0, theta_deg=()))
    prm.kappa = prm.beta = 0.0
    k = 2 * np.pi / n
    x = m.xyz[:, 0]
    C0 = 0.5 + 0.2 * np.cos(k * x)
    sim = OracleSim3D(m, prm, C0)
    u0 = np.array([0.05, 0.0, 0.0])
    sim.g, sim.h = _equilibria(sim, C0, 0.0, np.tile(u0, (m.N, 1)), 1.0)
    steps = 80
    sim.step(steps)
    C = sim.h.sum(0)
    w = m.lumped
    phase0 = np.angle(np.sum(w * (C0 - 0.5) * np.exp(-1j * k * x)))
    phase1 = np.angle(np.sum(w * (C - 0.5) * np.exp(-1j * k * x)))
    shift = -(phase1 - phase0) / k
    expected = u0[0] * steps * prm.dt
    assert abs(shift - expected) < 0.03 * expected


def test_contact_angle_diagnostic_of_exact_caps():
    """The height / wetted-area reading of the angle recovers a spherical
    cap's angle from its nodal tanh profile (Sec. III.B measurement)."""
    for theta in (60.0, 90.0, 120.0):
        n, nz = 40, 24
        mm = I3.kuhn_box(n, n, nz, 0.0, 0, walls=True)
        m = _mesh(mm)
        Rs = 12.0
        th = math.radians(theta)
        zc = -Rs * math.cos(th)                      # sphere centre below/above the substrate
        C0 = I3.droplet_C0_3d(mm["xyz"], (n / 2, n / 2, zc), Rs, 2.0, mm["period"])
        sim = OracleSim3D(m, params_from_physical3d(_phys(xi=2.0, theta_deg=(theta, 90.0))), C0)
        d = sim.diagnostics()
        assert abs(d["theta_deg"] - theta) < 2.0, (theta, d["theta_deg"])


def test_nodal_lapmu_is_seven_point_mean_and_has_no_growing_mode():
    """"nodal" element Laplacian of mu: on the unjittered Kuhn mesh the mean
    over the tetrahedron's vertices of the 7-point stencil; on a jittered
    mesh the Cahn-Hilliard operator M11^-1 M10 lap_mu(2 beta - kappa lap)
    has no eigenvalue with positive real part, while the paper's
    face-averaged form has some."""
    n = 6
    m = _mesh(I3.kuhn_box(n, n, n, 0.0, 0, walls=False))
    prm = params_from_physical3d(_phys(theta_deg=()), lapmu="nodal")
    sim = OracleSim3D(m, prm, np.full(m.N, 0.5))
    x, y, z = m.xyz.T
    mu = np.cos(2 * np.pi * x / n) * np.sin(4 * np.pi * y / n) + 0.3 * np.cos(2 * np.pi * z / n)
    idx = np.rint(m.xyz).astype(int) % n
    grid = np.zeros((n, n, n))
    grid[idx[:, 0], idx[:, 1], idx[:, 2]] = mu
    seven = sum(np.roll(grid, s, axis=ax) for ax in range(3) for s in (1, -1)) - 6 * grid
    node = seven[idx[:, 0], idx[:, 1], idx[:, 2]]
    np.testing.assert_allclose(sim.lap_mu(mu), node[m.tet].mean(axis=1), atol=1e-12)
    mj = _mesh(I3.kuhn_box(9, 9, 9, 0.15, 3, walls=False))
    N = mj.N
    for mode, check in (("face", lambda r: r > 1e-2), ("nodal", lambda r: r < 1e-10)):
        p = params_from_physical3d(_phys(theta_deg=()), lapmu=mode)
        s = OracleSim3D(mj, p, np.full(N, 0.5))
        lapmu, lapC = np.zeros((mj.T, N)), np.zeros((N, N))
        for j in range(N):
            e = np.zeros(N)
            e[j] = 1.0
            lapmu[:, j] = s.lap_mu(e)
            lapC[:, j] = s.kappa_lap_C(e) / p.kappa
        A = np.linalg.solve(mj.M11.toarray(), mj.M10.toarray() @ lapmu) @ (2 * p.beta * np.eye(N) - p.kappa * lapC)
        r = np.linalg.eigvals(A).real.max()
        assert check(r), (mode, r)
