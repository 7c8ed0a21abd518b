"""Pins of the element Laplacian of mu (Sec. II.D) and of the first moments of
the P0 forces (eq:G, eq:H), with checks that planted mistakes fail them.

The element Laplacian of the paper is the flux of grad(mu) through the three
edges of a triangle, each interior edge carrying the mean of the two P0
gradients beside it and each wall edge carrying nothing (eqn:bc1), divided by
the triangle's area.  On the two unjittered grids of the workloads this
reduces to fixed integer stencils, derived by hand below (h = 1):

'/' grid, cell (i, j) split along its (i, j)-(i+1, j+1) diagonal into
L = {(i,j), (i+1,j), (i+1,j+1)} and U = {(i,j), (i+1,j+1), (i,j+1)}, area 1/2
(so 1/(2A) = 1).  With the closed-triangle identity sum_e nu_e = 0 the own
gradient drops out of an element with no wall edge, and each edge adds the
neighbour's gradient dotted with the outward normal times length:

  L(i,j) = mu(i,j-1) + mu(i+2,j+1) + 2 mu(i,j+1) - 2 mu(i+1,j+1) - 2 mu(i,j)
  U(i,j) = mu(i-1,j) + mu(i+1,j+2) + 2 mu(i+1,j) - 2 mu(i+1,j+1) - 2 mu(i,j)

On a wall edge the neighbour term is missing and the own gradient no longer
cancels, leaving -grad(mu)_T . nu_wall:

  L(i,0)    = mu(i+2,1) + 2 mu(i,1) - mu(i+1,1) - mu(i,0) - mu(i+1,0)
  U(i,ny-1) = mu(i-1,j) + 2 mu(i+1,j) - mu(i,j) - mu(i+1,j+1) - mu(i,j+1)

Both interior stencils are exact on quadratics (x^2 -> 2, y^2 -> 2, xy -> 0)
and centred one third of a cell away from the element's centroid, so the
pointwise error is first order in h.

Cross grid (corners (i,j), centre c(i,j) = (i+1/2, j+1/2), triangles
B = {(i,j),(i+1,j),c}, R = {(i+1,j),(i+1,j+1),c}, T = {(i+1,j+1),(i,j+1),c},
L = {(i,j+1),(i,j),c}, area 1/4, so 1/(2A) = 2).  For B the three
neighbours are the T of the cell below and the R and L of its own cell:

  B = 2 [2 c(i,j-1) - 2 c(i,j) + (i,j+1) + (i+1,j+1) - (i,j) - (i+1,j)]

and R, T, L follow by quarter turns.  On x^2 this gives B = T = 0 and
R = L = 4; on y^2, B = T = 4 and R = L = 0: each triangle sees twice the
second derivative across its outer edge and none along it.  The mean over a
cell's four triangles is the Laplacian (2 on both), so the form converges
only in the cell (area) average on this mesh, not pointwise.
"""
import numpy as np
import pytest

from oracle import D2Q9_E, OracleMesh, OracleSim, params_from_physical
from oracle.felbm_oracle import CS2, Q, gamma
from paper_1708_04678_gb300 import inputs as I


def _mesh(m):
    return OracleMesh(m["xy"], m["tri"], m["wall_edges"], m["wall_id"], m["period"])


PHYS = dict(dt=0.25, tau_l=0.8, tau_v=0.8, rho_l=1.0, rho_v=0.1, sigma=0.01, xi=4.0,
            mobility=0.02, theta_deg=(60.0, 120.0))


def _sim(cls, m, theta=(60.0, 120.0)):
    return cls(m, params_from_physical(dict(PHYS, theta_deg=theta)), np.full(m.N, 0.5))


# ------------------------------------------------------------ the pins ---
def slash_stencil_error(cls, nx=10, ny=6, seed=0):
    """max |lap_mu - hand stencil| over every triangle of the '/' grid (walls
    at y = 0 and y = ny, periodic x), for a random nodal mu."""
    m = _mesh(I.grid_mesh(nx, ny, 0.0, 0))
    sim = _sim(cls, m)
    mu = np.random.default_rng(seed).standard_normal(m.N)
    lap = sim.lap_mu(mu)

    def M(i, j):
        return mu[j * nx + (i % nx)]

    err = 0.0
    for j in range(ny):
        for i in range(nx):
            c = j * nx + i
            if j >= 1:
                L = M(i, j - 1) + M(i + 2, j + 1) + 2 * M(i, j + 1) - 2 * M(i + 1, j + 1) - 2 * M(i, j)
            else:
                L = M(i + 2, 1) + 2 * M(i, 1) - M(i + 1, 1) - M(i, 0) - M(i + 1, 0)
            if j <= ny - 2:
                U = M(i - 1, j) + M(i + 1, j + 2) + 2 * M(i + 1, j) - 2 * M(i + 1, j + 1) - 2 * M(i, j)
            else:
                U = M(i - 1, j) + 2 * M(i + 1, j) - M(i, j) - M(i + 1, j + 1) - M(i, j + 1)
            err = max(err, abs(lap[2 * c] - L), abs(lap[2 * c + 1] - U))
    return err


def cross_stencil_error(cls, nx=8, ny=6, seed=1):
    """max |lap_mu - hand stencil| over every triangle of the doubly periodic
    cross grid, for a random nodal mu."""
    m = _mesh(I.cross_mesh(nx, ny, 0.0, 0))
    sim = _sim(cls, m, theta=())
    mu = np.random.default_rng(seed).standard_normal(m.N)
    lap = sim.lap_mu(mu)
    nc = nx * ny

    def K(i, j):
        return mu[(j % ny) * nx + (i % nx)]

    def Cc(i, j):
        return mu[nc + (j % ny) * nx + (i % nx)]

    err = 0.0
    for j in range(ny):
        for i in range(nx):
            c = j * nx + i
            B = 2 * (2 * Cc(i, j - 1) - 2 * Cc(i, j) + K(i, j + 1) + K(i + 1, j + 1) - K(i, j) - K(i + 1, j))
            R = 2 * (2 * Cc(i + 1, j) - 2 * Cc(i, j) + K(i, j) + K(i, j + 1) - K(i + 1, j) - K(i + 1, j + 1))
            T = 2 * (2 * Cc(i, j + 1) - 2 * Cc(i, j) + K(i, j) + K(i + 1, j) - K(i + 1, j + 1) - K(i, j + 1))
            L = 2 * (2 * Cc(i - 1, j) - 2 * Cc(i, j) + K(i + 1, j) + K(i + 1, j + 1) - K(i, j + 1) - K(i, j))
            err = max(err, abs(lap[4 * c] - B), abs(lap[4 * c + 1] - R), abs(lap[4 * c + 2] - T),
                      abs(lap[4 * c + 3] - L))
    return err


def _force_case(cls, seed=3):
    m = _mesh(I.grid_mesh(8, 6, 0.2, 5))
    sim = _sim(cls, m)
    prm = sim.prm
    rng = np.random.default_rng(seed)
    C = rng.uniform(0, 1, m.N)
    p = rng.uniform(-0.01, 0.01, m.N)
    u = rng.uniform(-0.05, 0.05, (m.N, 2))
    mu = sim.chemical_potential(C)
    Pg, Ph = sim.forces(C, p, u, mu)
    return m, sim, prm, C, p, u, mu, Pg, Ph


def force_first_moment_errors(cls):
    """Deviation of sum_a e_a Phi_g from cs2 mubar grad C and of sum_a e_a Phi_h
    from cs2 v_h + M lap(mu) ubar, v_h = grad C - Cbar/(rhobar cs2)(grad p -
    mubar grad C), scaled by the size of the expected values.  Both follow
    from the D2Q9 moments sum Gamma = 1, sum e Gamma = u, sum e e Gamma =
    cs2 I + u u and sum w e = 0, sum w e e = cs2 I applied to eq:G and eq:H."""
    m, sim, prm, C, p, u, mu, Pg, Ph = _force_case(cls)
    tri = m.tri
    Cb = C[tri].mean(1)
    ub = u[tri].mean(1)
    mub = mu[tri].mean(1)
    rhob = Cb * prm.rho_l + (1 - Cb) * prm.rho_v
    gC = m.grad(C)
    gp = m.grad(p)
    want_g = CS2 * mub[:, None] * gC
    vh = gC - (Cb / (rhob * CS2))[:, None] * (gp - mub[:, None] * gC)
    want_h = CS2 * vh + prm.mobility * sim.lap_mu(mu)[:, None] * ub
    got_g = np.einsum("ad,at->td", D2Q9_E, Pg)
    got_h = np.einsum("ad,at->td", D2Q9_E, Ph)
    return (np.abs(got_g - want_g).max() / np.abs(want_g).max(),
            np.abs(got_h - want_h).max() / np.abs(want_h).max())


# ------------------------------------------------------------ tests ------
def test_face_lapmu_is_the_hand_stencil_on_the_slash_grid():
    assert slash_stencil_error(OracleSim) < 1e-12


def test_face_lapmu_is_the_hand_stencil_on_the_cross_grid():
    assert cross_stencil_error(OracleSim) < 1e-12


def test_face_lapmu_on_quadratics():
    """Closed forms: '/' grid interior elements give exactly 2 on x^2 and y^2
    and 0 on xy; on the cross grid B/T give (0, 4) and R/L (4, 0) on
    (x^2, y^2), with the cell mean exactly 2."""
    nx, ny = 10, 6
    m = _mesh(I.grid_mesh(nx, ny, 0.0, 0))
    sim = _sim(OracleSim, m)
    x, y = m.xy[:, 0], m.xy[:, 1]
    inner = (m.nbr >= 0).all(1)
    # x^2 is not periodic in x: keep the elements whose stencil stays inside one period
    i_cell = (np.arange(m.T) // 2) % nx
    away = inner & (i_cell >= 1) & (i_cell <= nx - 3)
    for f, want in ((x * x, 2.0), (y * y, 2.0), (x * y, 0.0)):
        np.testing.assert_allclose(sim.lap_mu(f)[away], want, atol=1e-10)
    nx, ny = 8, 8
    m = _mesh(I.cross_mesh(nx, ny, 0.0, 0))
    sim = _sim(OracleSim, m, theta=())
    x, y = m.xy[:, 0], m.xy[:, 1]
    cell = np.arange(m.T) // 4
    ci, cj = cell % nx, cell // nx
    away = (ci >= 1) & (ci <= nx - 3) & (cj >= 1) & (cj <= ny - 3)
    kind = np.arange(m.T) % 4                     # 0 B, 1 R, 2 T, 3 L
    lx, ly = sim.lap_mu(x * x), sim.lap_mu(y * y)
    for k, (wx, wy) in enumerate(((0.0, 4.0), (4.0, 0.0), (0.0, 4.0), (4.0, 0.0))):
        sel = away & (kind == k)
        np.testing.assert_allclose(lx[sel], wx, atol=1e-9)
        np.testing.assert_allclose(ly[sel], wy, atol=1e-9)
    cell_mean_x = lx.reshape(-1, 4).mean(1)[away[0::4]]
    np.testing.assert_allclose(cell_mean_x, 2.0, atol=1e-9)


def _centroid_x(m):
    return m.xy[m.tri[:, 0], 0] + m.P[:, :, 0].mean(1)


def test_face_lapmu_converges_pointwise_on_the_slash_grid():
    """mu = cos(2 pi x / n) on n x n/2 '/' grids: the largest error over the
    interior elements, relative to the largest exact value, halves with each
    halving of h/n (first order): 0.087, 0.044, 0.022."""
    errs = []
    for n in (24, 48, 96):
        m = _mesh(I.grid_mesh(n, n // 2, 0.0, 0))
        sim = _sim(OracleSim, m, theta=(90.0, 90.0))
        k = 2 * np.pi / n
        lap = sim.lap_mu(np.cos(k * m.xy[:, 0]))
        exact = -k * k * np.cos(k * _centroid_x(m))
        inner = (m.nbr >= 0).all(1)
        errs.append(np.abs(lap - exact)[inner].max() / np.abs(exact).max())
    assert errs[0] < 0.1
    for a, b in zip(errs, errs[1:]):
        assert 1.8 < a / b < 2.2


def test_face_lapmu_converges_only_in_the_cell_mean_on_the_cross_grid():
    """mu = cos(2 pi x / n) on n x n cross grids: B and T triangles return
    about 0 whatever n (no pointwise convergence), while the mean over each
    cell's four triangles, against the exact value at the cell centre,
    converges at second order."""
    errs = []
    for n in (16, 32, 64):
        m = _mesh(I.cross_mesh(n, n, 0.0, 0))
        sim = _sim(OracleSim, m, theta=())
        k = 2 * np.pi / n
        lap = sim.lap_mu(np.cos(k * m.xy[:, 0]))
        kind = np.arange(m.T) % 4
        peak = k * k
        assert np.abs(lap[(kind == 0) | (kind == 2)]).max() < 0.01 * peak
        xc = (np.arange(n * n) % n) + 0.5
        cell = lap.reshape(-1, 4).mean(1)
        errs.append(np.abs(cell + k * k * np.cos(k * xc)).max() / peak)
    for a, b in zip(errs, errs[1:]):
        assert a / b > 3.5


def test_force_first_moments():
    eg, eh = force_first_moment_errors(OracleSim)
    assert eg < 1e-12 and eh < 1e-12


# --------------------------------------- planted mistakes fail the pins ---
class _TwiceLap(OracleSim):
    def lap_mu(self, mu):
        return 2.0 * super().lap_mu(mu)


class _NoHalf(OracleSim):
    """Edge flux with the sum of the two gradients instead of their mean."""

    def lap_mu(self, mu):
        m = self.mesh
        gmu = m.grad(mu)
        out = np.zeros(m.T)
        for k in range(3):
            nb = m.nbr[:, k]
            inner = nb >= 0
            s = gmu + gmu[np.where(inner, nb, 0)]
            out += np.where(inner, np.sum(s * m.nu[:, k], axis=1), 0.0)
        return out / m.area


class _PatchArea(OracleSim):
    """Divides by the mean vertex patch area instead of the element area."""

    def lap_mu(self, mu):
        m = self.mesh
        return super().lap_mu(mu) * m.area / m.patch_area[m.tri].mean(1)


class _WallFlux(OracleSim):
    """Gives wall edges the element's own gradient flux instead of zero."""

    def lap_mu(self, mu):
        m = self.mesh
        gmu = m.grad(mu)
        extra = np.zeros(m.T)
        for k in range(3):
            wall = m.nbr[:, k] < 0
            extra += np.where(wall, np.sum(gmu * m.nu[:, k], axis=1), 0.0)
        return super().lap_mu(mu) + 0.5 * extra / m.area


class _FlippedMuGradC(OracleSim):
    """Phi_g with -mubar grad C Gamma instead of +mubar grad C Gamma."""

    def forces(self, C, p, u, mu):
        Pg, Ph = super().forces(C, p, u, mu)
        m = self.mesh
        ub = u[m.tri].mean(1)
        mub = mu[m.tri].mean(1)
        gC = m.grad(C)
        G = gamma(ub)
        for a in range(Q):
            em = D2Q9_E[a][None, :] - ub
            Pg[a] -= 2.0 * np.sum(em * gC, axis=1) * mub * G[a]
        return Pg, Ph


class _NoMobilityMean(OracleSim):
    """Phi_h with M lap(mu) times w_a instead of Gamma_a(ubar)."""

    def forces(self, C, p, u, mu):
        Pg, Ph = super().forces(C, p, u, mu)
        m = self.mesh
        ub = u[m.tri].mean(1)
        G = gamma(ub)
        lmu = self.lap_mu(mu)
        w = G.sum(0)                                              # = 1
        for a in range(Q):
            wa = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4
            Ph[a] += self.prm.mobility * lmu * (wa[a] * w - G[a])
        return Pg, Ph


def _pins(cls):
    eg, eh = force_first_moment_errors(cls)
    return {"slash": slash_stencil_error(cls), "cross": cross_stencil_error(cls), "force_g": eg, "force_h": eh}


@pytest.mark.parametrize("cls", [_TwiceLap, _NoHalf, _PatchArea, _WallFlux, _FlippedMuGradC, _NoMobilityMean])
def test_planted_mistakes_fail_a_pin(cls):
    errs = _pins(cls)
    assert max(errs.values()) > 1e-8, errs        # the oracle itself is at round-off (< 1e-12)
    assert max(_pins(OracleSim).values()) < 1e-12
