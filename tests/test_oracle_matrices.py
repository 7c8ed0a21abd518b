"""Pins of the oracle's finite-element matrices (eq:fem_matrices, Sec. II.C).

Each matrix is re-derived here by brute force -- shape functions from solving
the 3x3 interpolation system of each triangle, integrals by a quadrature rule
exact for the integrand's degree -- and compared with the oracle's assembled
closed forms.  Further pins: mass-matrix row sums equal nodal areas, the
lumped-mass preconditioned spectrum lies in [1/4, 1], and the row/column sums
that make the scheme conservative.
"""
import numpy as np
import pytest

from oracle import D2Q9_E, OracleMesh
from paper_1708_04678_gb300 import inputs as I


def _two_element_mesh():
    xy = np.array([[0.0, 0.0], [1.3, 0.1], [1.1, 0.9], [-0.2, 1.2]])
    tri = np.array([[0, 1, 2], [0, 2, 3]])
    walls = np.array([[0, 1], [1, 2], [2, 3], [3, 0]])
    return OracleMesh(xy, tri, walls, np.array([0, 0, 1, 1]))


def _small_periodic_mesh():
    m = I.grid_mesh(3, 3, 0.2, 123)
    return OracleMesh(m["xy"], m["tri"], m["wall_edges"], m["wall_id"], m["period"])


def _brute_force(mesh):
    """Dense M11, M10, C_a, K_a, D_a and incoming-wall B_a by quadrature."""
    N, T = mesh.N, mesh.T
    M11 = np.zeros((N, N)); M10 = np.zeros((N, T))
    Cm = np.zeros((9, N, N)); Km = np.zeros((9, N, T)); Dm = np.zeros((9, N, N))
    Bm = np.zeros((9, N, N))
    third = {}
    for t in range(T):
        ids = mesh.tri[t]
        X = np.zeros((3, 2))
        for k in (1, 2):
            X[k] = mesh.min_image(mesh.xy[ids[k]] - mesh.xy[ids[0]])
        V = np.column_stack([np.ones(3), X])
        coef = np.linalg.solve(V, np.eye(3))          # column i: (a, bx, by) of N_i
        grads = coef[1:, :].T                          # (3, 2)
        area = 0.5 * abs(np.linalg.det(np.column_stack([X[1] - X[0], X[2] - X[0]])))
        # edge-midpoint rule: exact for polynomials of degree 2 on a triangle
        qp = 0.5 * (X + np.roll(X, -1, axis=0))
        Nq = np.column_stack([np.ones(3), qp]) @ coef  # (3 points, 3 functions)
        wq = area / 3.0
        for i in range(3):
            M10[ids[i], t] += wq * Nq[:, i].sum()
            for j in range(3):
                M11[ids[i], ids[j]] += wq * np.sum(Nq[:, i] * Nq[:, j])
        for a in range(9):
            eg = grads @ D2Q9_E[a]
            for i in range(3):
                Km[a, ids[i], t] += 0.5 * area * eg[i]
                for j in range(3):
                    Cm[a, ids[i], ids[j]] += wq * np.sum(Nq[:, i]) * eg[j]
                    Dm[a, ids[i], ids[j]] += 0.5 * area * eg[i] * eg[j]
        for k in range(3):
            a_, c_ = ids[(k + 1) % 3], ids[(k + 2) % 3]
            third[(min(a_, c_), max(a_, c_))] = (X[(k + 1) % 3], X[(k + 2) % 3], X[k])
    # wall edges: 3-point Gauss-Legendre on the edge, outward normal away from the third vertex
    gl_x = np.array([-np.sqrt(0.6), 0.0, np.sqrt(0.6)])
    gl_w = np.array([5.0, 8.0, 5.0]) / 9.0
    for (p, q) in mesh.wall_edges:
        xa, xc, x3 = third[(min(p, q), max(p, q))]
        L = np.linalg.norm(xc - xa)
        t_hat = (xc - xa) / L
        n = np.array([t_hat[1], -t_hat[0]])
        if n @ (x3 - xa) > 0:
            n = -n
        s = 0.5 * (gl_x + 1.0)                         # parameter along xa -> xc
        Na, Nc = 1.0 - s, s
        w = 0.5 * L * gl_w
        # map edge endpoints (xa, xc) back to node ids
        ends = _edge_node_order(mesh, p, q, xa, xc)
        for a in range(9):
            en = D2Q9_E[a] @ n
            if en < 0:
                for (u, Nu) in ((ends[0], Na), (ends[1], Nc)):
                    for (v, Nv) in ((ends[0], Na), (ends[1], Nc)):
                        Bm[a, u, v] += en * np.sum(w * Nu * Nv)
    return M11, M10, Cm, Km, Dm, Bm


def _edge_node_order(mesh, p, q, xa, xc):
    """Return (node at xa, node at xc) for the wall edge {p, q}."""
    for t in range(mesh.T):
        ids = list(mesh.tri[t])
        if p in ids and q in ids:
            X = np.zeros((3, 2))
            for k in (1, 2):
                X[k] = mesh.min_image(mesh.xy[ids[k]] - mesh.xy[ids[0]])
            Xp, Xq = X[ids.index(p)], X[ids.index(q)]
            if np.allclose(Xp, xa) and np.allclose(Xq, xc):
                return (p, q)
            if np.allclose(Xq, xa) and np.allclose(Xp, xc):
                return (q, p)
    raise AssertionError("edge not found")


@pytest.mark.parametrize("make", [_two_element_mesh, _small_periodic_mesh])
def test_matrices_match_quadrature(make):
    mesh = make()
    M11, M10, Cm, Km, Dm, Bm = _brute_force(mesh)
    tol = 1e-13
    np.testing.assert_allclose(mesh.M11.toarray(), M11, atol=tol)
    np.testing.assert_allclose(mesh.M10.toarray(), M10, atol=tol)
    for a in range(9):
        np.testing.assert_allclose(mesh.Cmat[a].toarray(), Cm[a], atol=tol)
        np.testing.assert_allclose(mesh.Kmat[a].toarray(), Km[a], atol=tol)
        np.testing.assert_allclose(mesh.Dmat[a].toarray(), Dm[a], atol=tol)
        np.testing.assert_allclose(mesh.Bmat[a].toarray(), Bm[a], atol=tol)


def test_mass_row_sums_are_nodal_areas():
    m = I.grid_mesh(8, 6, 0.2, 3)
    mesh = OracleMesh(m["xy"], m["tri"], m["wall_edges"], m["wall_id"], m["period"])
    np.testing.assert_allclose(mesh.lumped, mesh.patch_area / 3.0, rtol=1e-14)
    assert abs(mesh.lumped.sum() - 8 * 6) < 1e-11            # total area of the box


def test_lumped_preconditioned_spectrum_in_quarter_one():
    m = I.cross_mesh(6, 6, 0.25, 9)
    mesh = OracleMesh(m["xy"], m["tri"], m["wall_edges"], m["wall_id"], m["period"])
    d = 1.0 / np.sqrt(mesh.lumped)
    S = d[:, None] * mesh.M11.toarray() * d[None, :]
    ev = np.linalg.eigvalsh(S)
    assert ev.min() >= 0.25 - 1e-12
    assert abs(ev.max() - 1.0) < 1e-12


def test_conservation_sums():
    m = I.grid_mesh(6, 5, 0.2, 4)
    mesh = OracleMesh(m["xy"], m["tri"], m["wall_edges"], m["wall_id"], m["period"])
    np.testing.assert_allclose(np.asarray(mesh.M10.sum(axis=0)).ravel(), mesh.area, rtol=1e-14)
    for a in range(9):
        # C_a 1 = int N_i e.grad(1) = 0 ; D_a 1 = 0 ; 1^T K_a = 1/2 int e.grad(sum N_i) = 0
        assert np.abs(mesh.Cmat[a] @ np.ones(mesh.N)).max() < 1e-13
        assert np.abs(mesh.Dmat[a] @ np.ones(mesh.N)).max() < 1e-13
        assert np.abs(np.asarray(mesh.Kmat[a].sum(axis=0))).max() < 1e-13


def test_gradient_exact_on_linear_fields():
    m = I.cross_mesh(5, 5, 0.25, 2)
    mesh = OracleMesh(m["xy"], m["tri"], m["wall_edges"], m["wall_id"], m["period"])
    # a linear field is not periodic; use element-local values instead
    g = np.array([0.7, -1.9])
    for t in range(mesh.T):
        vals = mesh.P[t] @ g
        grad = np.einsum("i,id->d", vals, mesh.b[t])
        np.testing.assert_allclose(grad, g, atol=1e-12)
