"""Pins of the oracle's field operators, collision, forces and time step.

Each test checks the oracle against something fixed outside it: textbook
lattice moment identities, the 5-point stencil the P1 Laplacian reduces to on
a uniform right-triangle grid, the exact planar equilibrium profile of Sec. II
(also tilted to meet a wall at Young's angle, which pins the wetting condition
eqn:bc2 and its sign), the static-interface balance of Sec. II.C, exact mass
conservation, stationarity of uniform states, advection speed, the Laplace
law and Young's law.
"""
import math

import numpy as np
import pytest

from oracle import D2Q9_E, OracleMesh, OracleSim, params_from_physical
from oracle.felbm_oracle import CS2
from paper_1708_04678_gb300 import inputs as I


def _mesh(m):
    return OracleMesh(m["xy"], m["tri"], m["wall_edges"], m["wall_id"], m["period"])


def _params(**kw):
    base = dict(dt=0.25, tau_l=0.8, tau_v=0.8, rho_l=1.0, rho_v=0.1, sigma=0.01, xi=4.0,
                mobility=0.02, theta_deg=(90.0, 90.0))
    base.update(kw)
    return base


# ---------------------------------------------------------------- lattice ---
def test_equilibrium_moments():
    """With tau = 1/2 the collision returns the equilibria; their moments are
    the textbook ones: sum g = p, sum e g = rho cs2 u, sum e e g = cs2 (p I + rho u u),
    sum h = C, sum e h = C u, sum e e h = C (cs2 I + u u)."""
    m = _mesh(I.cross_mesh(3, 3, 0.2, 0))
    prm = params_from_physical(_params(tau_l=0.5, tau_v=0.5))
    sim = OracleSim(m, prm, np.full(m.N, 0.5))
    rng = np.random.default_rng(1)
    N = m.N
    C = rng.uniform(0, 1, N); p = rng.uniform(-0.1, 0.1, N); u = rng.uniform(-0.1, 0.1, (N, 2))
    rho = C * prm.rho_l + (1 - C) * prm.rho_v
    g0 = rng.standard_normal((9, N)); h0 = rng.standard_normal((9, N))
    geq, heq = sim.collide(g0, h0, C, p, u, rho)
    E = D2Q9_E
    np.testing.assert_allclose(geq.sum(0), p, atol=1e-15)
    np.testing.assert_allclose(E.T @ geq, (rho * CS2)[None] * u.T, atol=1e-15)
    np.testing.assert_allclose(heq.sum(0), C, atol=1e-15)
    np.testing.assert_allclose(E.T @ heq, C[None] * u.T, atol=1e-15)
    for a in range(2):
        for b in range(2):
            sg = np.einsum("q,qn->n", E[:, a] * E[:, b], geq)
            sh = np.einsum("q,qn->n", E[:, a] * E[:, b], heq)
            np.testing.assert_allclose(sg, CS2 * (p * (a == b) + rho * u[:, a] * u[:, b]), atol=1e-15)
            np.testing.assert_allclose(sh, C * (CS2 * (a == b) + u[:, a] * u[:, b]), atol=1e-15)


def test_collision_conserves_moments():
    m = _mesh(I.cross_mesh(3, 3, 0.2, 0))
    prm = params_from_physical(_params(tau_l=0.7, tau_v=1.3))
    sim = OracleSim(m, prm, np.full(m.N, 0.5))
    rng = np.random.default_rng(2)
    g = rng.standard_normal((9, m.N)) * 0.01
    h = rng.uniform(0, 0.2, (9, m.N))
    C, p, u, rho = sim.moments(g, h)
    gh, hh = sim.collide(g, h, C, p, u, rho)
    np.testing.assert_allclose(gh.sum(0), g.sum(0), atol=1e-15)
    np.testing.assert_allclose(hh.sum(0), h.sum(0), atol=1e-15)
    np.testing.assert_allclose(D2Q9_E.T @ gh, D2Q9_E.T @ g, atol=1e-15)


def test_force_moment_identities():
    """sum_a Phi_h = M lap(mu)_T ; sum_a Phi_g = cs2 u.grad(rho) ; the
    area-weighted sum of lap(mu)_T vanishes (fluxes telescope, walls give 0)."""
    m = _mesh(I.grid_mesh(8, 6, 0.2, 5))
    prm = params_from_physical(_params(theta_deg=(60.0, 120.0)))
    sim = OracleSim(m, prm, np.full(m.N, 0.5))
    rng = np.random.default_rng(3)
    C = rng.uniform(0, 1, m.N); p = rng.uniform(-0.01, 0.01, m.N)
    u = rng.uniform(-0.05, 0.05, (m.N, 2))
    mu = sim.chemical_potential(C)
    Pg, Ph = sim.forces(C, p, u, mu)
    lmu = sim.lap_mu(mu)
    np.testing.assert_allclose(Ph.sum(0), prm.mobility * lmu, atol=1e-14)
    ub = u[m.tri].mean(1)
    grho = (prm.rho_l - prm.rho_v) * m.grad(C)
    np.testing.assert_allclose(Pg.sum(0), CS2 * np.sum(ub * grho, 1), atol=1e-14)
    assert abs(np.sum(m.area * lmu)) < 1e-12 * np.sum(m.area * np.abs(lmu))


# ------------------------------------------------------------- Laplacians ---
def test_patch_laplacian_is_five_point_stencil_on_uniform_grid():
    """On the unjittered '/' grid the consistent patch Laplacian of C equals
    (C_E + C_W + C_N + C_S - 4 C) / h^2 at nodes off the walls."""
    nx, ny = 16, 10
    mm = I.grid_mesh(nx, ny, 0.0, 0)
    m = _mesh(mm)
    prm = params_from_physical(_params())
    sim = OracleSim(m, prm, np.full(m.N, 0.5))
    x, y = m.xy[:, 0], m.xy[:, 1]
    C = np.cos(2 * np.pi * x / nx) * np.cos(0.37 * y) + 0.1 * y * y
    lap = sim.kappa_lap_C(C) / prm.kappa
    for j in range(1, ny):
        for i in range(nx):
            k = j * nx + i
            five = (C[j * nx + (i + 1) % nx] + C[j * nx + (i - 1) % nx]
                    + C[(j + 1) * nx + i] + C[(j - 1) * nx + i] - 4 * C[k])
            assert abs(lap[k] - five) < 1e-12


def test_paper_mode_laplacian_is_two_thirds():
    mm = I.grid_mesh(12, 8, 0.2, 1)
    m = _mesh(mm)
    C = np.sin(2 * np.pi * m.xy[:, 0] / 12) + 0.3 * m.xy[:, 1]
    a = OracleSim(m, params_from_physical(_params(), "consistent"), C).kappa_lap_C(C)
    b = OracleSim(m, params_from_physical(_params(), "paper"), C).kappa_lap_C(C)
    np.testing.assert_allclose(b, a * 2.0 / 3.0, rtol=1e-13, atol=1e-16)


def _tilted_column(nx, ny, theta_deg, xi, xl, xr, jitter=0.0, seed=0):
    """Liquid column between two straight interfaces meeting the bottom wall at
    theta and the top wall at 180 - theta: the exact equilibrium of Sec. II
    with the wetting condition eqn:bc2 (cubic surface energy)."""
    mm = I.grid_mesh(nx, ny, jitter, seed)
    x, y = mm["xy"][:, 0], mm["xy"][:, 1]
    th = math.radians(theta_deg)
    # interface normal n_s (into the liquid) satisfies n_wall . n_s = -cos(theta)
    nxs, nys = math.sin(th), -math.cos(th)
    sl = (x - xl) * nxs + y * nys
    sr = -(x - xr) * nxs + y * nys
    C = (0.5 + 0.5 * np.tanh(2 * sl / xi)) * (0.5 + 0.5 * np.tanh(2 * sr / xi))
    return mm, C


@pytest.mark.parametrize("theta", [90.0, 60.0, 120.0, 45.0])
def test_chemical_potential_vanishes_on_exact_equilibria(theta):
    """Planar tanh profile with xi = sqrt(8 kappa/beta), meeting the walls at
    Young's angle: mu = 0 up to discretisation error (second order inside,
    first order at wall nodes).  A flipped wetting sign makes mu O(beta); the
    literal patch volume ("paper" mode) leaves an O(beta/15) residual."""
    xi = 8.0
    mm, C = _tilted_column(240, 40, theta, xi, 40.0, 200.0)
    m = _mesh(mm)
    phys = _params(xi=xi, theta_deg=(theta, 180.0 - theta))
    prm = params_from_physical(phys)
    mu = OracleSim(m, prm, C).chemical_potential(C)
    assert np.abs(mu).max() < 0.02 * prm.beta
    paper = OracleSim(m, params_from_physical(phys, "paper"), C).chemical_potential(C)
    assert np.abs(paper).max() > 0.04 * prm.beta
    if theta != 90.0:
        bad = params_from_physical(dict(phys, theta_deg=(180.0 - theta, theta)))
        mu_bad = OracleSim(m, bad, C).chemical_potential(C)
        assert np.abs(mu_bad).max() > 0.5 * prm.beta


def test_chemical_potential_error_is_second_order():
    """Doubling xi on the same grid (h/xi halved) cuts the planar-profile
    residual of mu/beta by about 4."""
    errs = []
    for xi in (4.0, 8.0):
        mm, C = _tilted_column(240, 40, 90.0, xi, 40.0, 200.0)
        m = _mesh(mm)
        prm = params_from_physical(_params(xi=xi))
        errs.append(np.abs(OracleSim(m, prm, C).chemical_potential(C)).max() / prm.beta)
    assert 3.0 < errs[0] / errs[1] < 5.0


# -------------------------------------------------------------- the step ---
def test_static_interface_balance():
    """kappa = beta = 0, u = p = 0, any C on a periodic jittered mesh: the P0
    force exactly balances streaming of h = w C (Sec. II.C), so C stays put
    and g stays zero.  With the printed sign of dt M10 it would not."""
    mm = I.cross_mesh(10, 10, 0.2, 7)
    m = _mesh(mm)
    prm = params_from_physical(_params(dt=0.1))
    prm.kappa = 0.0
    prm.beta = 0.0
    rng = np.random.default_rng(4)
    C0 = rng.uniform(0, 1, m.N)
    sim = OracleSim(m, prm, C0)
    sim.step(20)
    C, p, u, rho = sim.moments()
    assert np.abs(C - C0).max() < 1e-13
    assert np.abs(sim.g).max() < 1e-15


@pytest.mark.parametrize("case", ["liquid_wetting_walls", "mixture_neutral_walls", "moving_periodic"])
def test_uniform_states_are_stationary(case):
    if case == "moving_periodic":
        mm = I.cross_mesh(8, 8, 0.2, 3)
        m = _mesh(mm)
        prm = params_from_physical(_params(dt=0.1, theta_deg=()))
        C0 = np.full(m.N, 0.4)
        sim = OracleSim(m, prm, C0)
        u0 = np.array([0.03, -0.02])
        rho = 0.4 * prm.rho_l + 0.6 * prm.rho_v
        u = np.tile(u0, (m.N, 1))
        sim.g, sim.h = _equilibria(sim, C0, 0.02, u, rho)
    else:
        mm = I.grid_mesh(8, 6, 0.2, 3)
        m = _mesh(mm)
        theta = (60.0, 120.0) if case == "liquid_wetting_walls" else (90.0, 90.0)
        prm = params_from_physical(_params(theta_deg=theta))
        c = 1.0 if case == "liquid_wetting_walls" else 0.3
        C0 = np.full(m.N, c)
        sim = OracleSim(m, prm, C0, p0=np.full(m.N, 0.01))
    g0, h0 = sim.g.copy(), sim.h.copy()
    sim.step(10)
    assert np.abs(sim.g - g0).max() < 1e-13
    assert np.abs(sim.h - h0).max() < 1e-13


def _equilibria(sim, C, p, u, rho):
    prm = sim.prm
    tau_l, tau_v = prm.tau_l, prm.tau_v
    prm.tau_l = prm.tau_v = 0.5
    N = len(C)
    geq, heq = sim.collide(np.zeros((9, N)), np.zeros((9, N)), C, np.full(N, p), u, np.full(N, rho))
    prm.tau_l, prm.tau_v = tau_l, tau_v
    return geq, heq


def test_mass_is_conserved_with_wetting_walls():
    w = I.small_sessile(nx=32, ny=16, R=7.0, theta=60.0)
    w["phys"]["dt"] = 0.25
    m = _mesh(w["mesh"])
    sim = OracleSim(m, params_from_physical(w["phys"]), w["C0"])
    sim.step(40)
    d = sim.diagnostics()
    assert abs(d["mass_drift_rel"]) < 40 * 2e-15


def _small_channel(theta=56.0):
    return I.capillary_channel(H=4, length_factor=4, reservoir=2, theta=theta, l0_factor=1.0,
                               liquid_factor=1.5, dt=0.1, xi=2.0)


def test_channel_mesh_with_internal_walls_conserves_mass():
    """A periodic box with a solid block and a channel through it (internal
    walls, eight re-entrant and salient corners, wetting at 56 degrees):
    mass is conserved to round-off through the weak bounce-back at every
    wall edge, corners included."""
    w = _small_channel()
    m = _mesh(w["mesh"])
    sim = OracleSim(m, params_from_physical(w["phys"]), w["C0"])
    sim.step(40)
    d = sim.diagnostics()
    assert abs(d["mass_drift_rel"]) < 40 * 2e-15


def test_channel_uniform_liquid_is_stationary():
    """C = 1 everywhere, p = 0, u = 0 in the channel geometry: the wetting
    flux phi_c (C - C^2) vanishes and nothing may move, at the corners too."""
    w = _small_channel(theta=45.0)
    m = _mesh(w["mesh"])
    sim = OracleSim(m, params_from_physical(w["phys"]), np.ones(len(w["C0"])))
    g0, h0 = sim.g.copy(), sim.h.copy()
    sim.step(30)
    assert np.abs(sim.g - g0).max() < 1e-13
    assert np.abs(sim.h - h0).max() < 1e-13


def test_uniform_flow_advects_composition():
    """rho_l = rho_v, kappa = beta = 0: h carries C at the fluid velocity
    (eqn:mp_che with mu = 0).  The phase of the first Fourier mode moves by
    u t; a flipped streaming sign would move it the other way."""
    n = 24
    mm = I.cross_mesh(n, n, 0.1, 8)
    m = _mesh(mm)
    prm = params_from_physical(_params(dt=0.1, rho_v=1.0, theta_deg=()))
    prm.kappa = prm.beta = 0.0
    k = 2 * np.pi / n
    x = m.xy[:, 0]
    C0 = 0.5 + 0.2 * np.cos(k * x)
    sim = OracleSim(m, prm, C0)
    u0 = np.array([0.05, 0.0])
    sim.g, sim.h = _equilibria(sim, C0, 0.0, np.tile(u0, (m.N, 1)), 1.0)
    steps = 200
    sim.step(steps)
    C = sim.h.sum(0)
    w = m.lumped
    phase0 = np.angle(np.sum(w * (C0 - 0.5) * np.exp(-1j * k * x)))
    phase1 = np.angle(np.sum(w * (C - 0.5) * np.exp(-1j * k * x)))
    shift = -(phase1 - phase0) / k
    expected = u0[0] * steps * prm.dt
    assert abs(shift - expected) < 0.03 * expected


# ------------------------------------------------------ physical laws -------
@pytest.mark.slow
def test_laplace_law():
    """Free droplet in a box: the pressure jump is sigma / R in 2D (the 2D
    form of the Laplace drop of Sec. III.C).  The jump is averaged over the
    last 300 steps to remove the acoustic breathing mode of the start-up."""
    n, R, sigma = 36, 7.0, 0.01
    mm = I.grid_mesh(n, n, 0.2, 10)
    phys = _params(sigma=sigma, tau_l=1.0, tau_v=1.0)
    C0 = I.droplet_C0(mm["xy"], (n / 2, n / 2), R, phys["xi"], mm["period"])
    sim = OracleSim(_mesh(mm), params_from_physical(phys), C0)
    sim.step(300)
    acc = []
    for _ in range(30):
        sim.step(10)
        acc.append(sim.diagnostics()["delta_p"])
    assert abs(np.mean(acc) * R / sigma - 1.0) < 0.05


@pytest.mark.slow
@pytest.mark.parametrize("theta", [60.0, 120.0])
def test_young_law(theta):
    """A circular cap started at Young's angle stays there (within 1 degree
    after 800 steps); started at 90 degrees it moves towards theta."""
    nx, R = 48, 10.0
    w = I.small_sessile(nx=nx, ny=nx // 2, seed=0, R=R, theta=theta)
    w["phys"]["dt"] = 0.25
    mm = w["mesh"]
    m = _mesh(mm)
    prm = params_from_physical(w["phys"])
    cap = I.droplet_C0(mm["xy"], (nx / 2, -R * math.cos(math.radians(theta))), R, 4.0, mm["period"])
    sim = OracleSim(m, prm, cap)
    sim.step(800)
    assert abs(sim.diagnostics()["theta_deg"] - theta) < 1.0
    sim = OracleSim(m, prm, w["C0"])
    sim.step(500)
    moved = sim.diagnostics()["theta_deg"] - 90.0
    assert moved * (theta - 90.0) > 0 and abs(moved) > 3.0


# ------------------------------------------------------- contact angle ------
@pytest.mark.parametrize("theta", [40.0, 70.0, 90.0, 110.0, 140.0])
def test_contact_angle_of_circular_caps(theta):
    nx, R = 128, 24.0
    mm = I.grid_mesh(nx, 64, 0.2, 12)
    m = _mesh(mm)
    cap = I.droplet_C0(mm["xy"], (nx / 2, -R * math.cos(math.radians(theta))), R, 4.0, mm["period"])
    sim = OracleSim(m, params_from_physical(_params()), cap)
    d = sim.diagnostics()
    assert abs(d["theta_deg"] - theta) < 0.5


# ------------------------------------------ element Laplacian of mu modes ---
def _ch_operator(sim, m, prm):
    """Nodal rate of C per unit mobility from the h-force M lap(mu) Gamma at
    rest, linearised at C = 0: M11^-1 M10 lap_mu(2 beta C - kappa lap C)."""
    N = m.N
    lapmu, lapC = np.zeros((m.T, N)), np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        lapmu[:, j] = sim.lap_mu(e)
        lapC[:, j] = sim.kappa_lap_C(e) / prm.kappa
    return np.linalg.solve(m.M11.toarray(), m.M10.toarray() @ lapmu) @ (2 * prm.beta * np.eye(N) - prm.kappa * lapC)


def test_nodal_lapmu_is_five_point_mean_on_uniform_grid():
    """"nodal" element Laplacian of mu on the unjittered grid: the mean over
    the triangle's vertices of the 5-point stencil (walls: zero normal flux)."""
    nx, ny = 12, 8
    m = _mesh(I.grid_mesh(nx, ny, 0.0, 0))
    prm = params_from_physical(_params(), lapmu="nodal")
    sim = OracleSim(m, prm, np.full(m.N, 0.5))
    x, y = m.xy[:, 0], m.xy[:, 1]
    mu = np.cos(2 * np.pi * x / nx) * np.cos(0.3 * y)
    lap = sim.lap_mu(mu)
    node = np.zeros(m.N)
    for j in range(1, ny):
        for i in range(nx):
            k = j * nx + i
            node[k] = (mu[j * nx + (i + 1) % nx] + mu[j * nx + (i - 1) % nx]
                       + mu[(j + 1) * nx + i] + mu[(j - 1) * nx + i] - 4 * mu[k])
    inner = np.all((m.xy[m.tri][:, :, 1] > 0.5) & (m.xy[m.tri][:, :, 1] < ny - 0.5), axis=1)
    np.testing.assert_allclose(lap[inner], node[m.tri[inner]].mean(axis=1), atol=1e-12)
    assert abs(np.sum(m.area * lap)) < 1e-12 * np.sum(m.area * np.abs(lap))


def test_face_lapmu_has_growing_modes_nodal_does_not():
    """The paper's face-averaged element Laplacian of mu, fed to the nodes
    through M11^-1 M10, has eigenvalues with positive real part on a
    jittered walled mesh (an anti-diffusive Cahn-Hilliard mode: long runs
    grow at rate M dt max Re); the "nodal" form has none."""
    m = _mesh(I.grid_mesh(16, 8, 0.2, 0))
    for mode, check in (("face", lambda r: r > 0.05), ("nodal", lambda r: r < 1e-10)):
        prm = params_from_physical(_params(), lapmu=mode)
        ev = np.linalg.eigvals(_ch_operator(OracleSim(m, prm, np.full(m.N, 0.5)), m, prm))
        assert check(ev.real.max()), (mode, ev.real.max())


def test_initial_state_has_the_given_moments():
    """The initial state is the equilibrium of the given C0, p0, u0: its
    moments return them exactly (sum h = C, sum g = p, sum e g = cs2 rho u)."""
    m = _mesh(I.cross_mesh(5, 4, 0.2, 3))
    prm = params_from_physical(_params())
    rng = np.random.default_rng(8)
    C0 = rng.uniform(0, 1, m.N)
    p0 = rng.uniform(-0.01, 0.01, m.N)
    u0 = rng.uniform(-0.05, 0.05, (m.N, 2))
    sim = OracleSim(m, prm, C0, p0=p0, u0=u0)
    C, p, u, rho = sim.moments()
    np.testing.assert_allclose(C, C0, atol=1e-15)
    np.testing.assert_allclose(p, p0, atol=1e-16)
    np.testing.assert_allclose(u, u0, atol=1e-15)
