"""Seeded synthetic 3D inputs: tetrahedral box meshes and droplet workloads.

Like ``inputs.py`` for 2D, this module produces only inputs consumed by both
the CPU oracle tests and the CUDA path: node coordinates, tetrahedra, wall
faces, periodic lengths, initial composition and physical parameters.  It
holds none of the method's arithmetic.

Meshes: an nx x ny x nz box of unit cubes, each cut into the six Kuhn
(Freudenthal) tetrahedra around its main diagonal -- a conforming, face-to-face
triangulation -- with every node jittered uniformly by +-jitter*h from
``numpy.random.default_rng(seed)`` (wall nodes only within the wall plane).
x and y are periodic; z is periodic too ("free") or bounded by walls at
z = 0 (wall id 0, the substrate) and z = nz (wall id 1).

Workloads (the paper's 3D droplet benchmarks, Sec. III):

* ``static_droplet_64``   -- free droplet R=16 in a 64^3 periodic box
  (262,144 nodes, 1,572,864 tetrahedra: the paper's coarsest 1.5e6-element
  parasitic-current mesh), density ratio 2, equal viscosities.
* ``sessile_droplet_3d``  -- hemisphere R=16 on the substrate of a
  64x64x32 box (135,200 nodes), walls at z=0 and z=32.
* ``small_free_droplet_3d``, ``small_sessile_3d`` -- small cases for the
  oracle parity tests.
"""
from __future__ import annotations

import itertools

import numpy as np

__all__ = ["kuhn_box", "droplet_C0_3d", "static_droplet_64", "sessile_droplet_3d",
           "small_free_droplet_3d", "small_sessile_3d", "DT_KUHN"]

# the six Kuhn tetrahedra of the unit cube: paths 000 -> e_a -> e_a+e_b -> 111
_CORNERS = []
for perm in itertools.permutations(range(3)):
    c = [np.zeros(3, dtype=np.int64)]
    for ax in perm:
        nxt = c[-1].copy()
        nxt[ax] = 1
        c.append(nxt)
    M = np.array([c[1] - c[0], c[2] - c[0], c[3] - c[0]], dtype=np.float64)
    if np.linalg.det(M) < 0:                 # orient every tetrahedron positively
        c[1], c[2] = c[2], c[1]
    _CORNERS.append(np.array(c))
_CORNERS = np.array(_CORNERS)                # (6, 4, 3) offsets in {0, 1}


def kuhn_box(nx, ny, nz, jitter, seed, walls=True, h=1.0):
    """Tetrahedral mesh of an nx x ny x nz box of cubes of side h.

    Nodes are numbered i + nx (j + ny k).  With ``walls`` the box has
    nz + 1 node layers and wall faces on z = 0 (id 0) and z = nz h (id 1);
    otherwise nz layers and z is periodic too."""
    nk = nz + 1 if walls else nz
    rng = np.random.default_rng(seed)
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nk), indexing="ij")
    i, j, k = (a.transpose(2, 1, 0).reshape(-1) for a in (i, j, k))
    xyz = np.stack([i, j, k], axis=1).astype(np.float64) * h
    d = rng.uniform(-jitter * h, jitter * h, size=xyz.shape)
    if walls:
        d[(k == 0) | (k == nz), 2] = 0.0
    xyz += d
    period = (nx * h, ny * h, 0.0 if walls else nz * h)
    for ax in range(3):
        if period[ax] > 0:
            xyz[:, ax] = np.mod(xyz[:, ax], period[ax])

    def node(ii, jj, kk):
        return (ii % nx) + nx * ((jj % ny) + ny * (kk % nk))

    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ci, cj, ck = (a.transpose(2, 1, 0).reshape(-1) for a in (ci, cj, ck))
    tets = []
    for c in _CORNERS:
        tets.append(np.stack([node(ci + c[v, 0], cj + c[v, 1], ck + c[v, 2]) for v in range(4)], axis=1))
    tet = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)     # cube-major, 6 per cube
    # boundary faces: triangles of the cube faces on z = 0 and z = nz
    wf, wid = [], []
    if walls:
        bi, bj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
        bi, bj = bi.T.reshape(-1), bj.T.reshape(-1)
        for kk, wall in ((0, 0), (nz, 1)):
            a, b = node(bi, bj, kk), node(bi + 1, bj, kk)
            c, e = node(bi + 1, bj + 1, kk), node(bi, bj + 1, kk)
            wf += [np.stack([a, b, c], 1), np.stack([a, e, c], 1)]
            wid += [np.full(len(a), wall), np.full(len(a), wall)]
    wall_faces = np.concatenate(wf).astype(np.int32) if wf else np.zeros((0, 3), np.int32)
    wall_id = np.concatenate(wid).astype(np.int32) if wid else np.zeros(0, np.int32)
    return {"xyz": xyz, "tet": tet, "wall_faces": wall_faces, "wall_id": wall_id, "period": period}


def droplet_C0_3d(xyz, centre, R, xi, period=(0.0, 0.0, 0.0)):
    """Ball (or a cap cut by a wall) of radius R with the tanh profile of
    width xi across its surface; distances by the minimum image."""
    d = xyz - np.asarray(centre, dtype=np.float64)[None, :]
    for k in range(3):
        if period[k] > 0:
            d[:, k] -= period[k] * np.round(d[:, k] / period[k])
    r = np.sqrt(np.sum(d * d, axis=1))
    return 0.5 + 0.5 * np.tanh(2.0 * (R - r) / xi)


# Explicit Taylor-Galerkin streaming: dt = 0.25 keeps noisy uniform states
# bounded on the Kuhn meshes with 0.15h jitter.
DT_KUHN = 0.25


def _phys(**kw):
    base = dict(dt=DT_KUHN, tau_l=0.8, tau_v=0.8, rho_l=1.0, rho_v=0.5, sigma=0.01,
                xi=4.0, mobility=0.02, theta_deg=(90.0, 90.0))
    base.update(kw)
    base["theta_deg"] = tuple(float(t) for t in base["theta_deg"])
    return base


def _free(name, n, R, seed, jitter, steps, **phys):
    mesh = kuhn_box(n, n, n, jitter, seed, walls=False)
    centre = (n / 2.0, n / 2.0, n / 2.0)
    ph = _phys(theta_deg=(), **phys)
    C0 = droplet_C0_3d(mesh["xyz"], centre, R, ph["xi"], mesh["period"])
    return {"name": name, "mesh": mesh, "C0": C0, "phys": ph, "steps": steps,
            "centre": centre, "R": float(R)}


def _sessile(name, n, nz, R, seed, jitter, theta, steps, **phys):
    mesh = kuhn_box(n, n, nz, jitter, seed, walls=True)
    centre = (n / 2.0, n / 2.0, 0.0)
    ph = _phys(theta_deg=(theta, 90.0), **phys)
    C0 = droplet_C0_3d(mesh["xyz"], centre, R, ph["xi"], mesh["period"])
    return {"name": name, "mesh": mesh, "C0": C0, "phys": ph, "steps": steps,
            "centre": centre, "R": float(R)}


def static_droplet_64(seed=6, steps=5000):
    """Static droplet R=16, xi 4, in a 64^3 periodic Kuhn mesh (1,572,864
    tetrahedra), jitter 0.15h, density ratio 2, tau 0.8 in both phases,
    sigma 0.01, M 0.02, dt 0.25."""
    return _free("static droplet 64^3", 64, 16.0, seed, 0.15, steps)


def sessile_droplet_3d(seed=7, theta=90.0, steps=5000):
    """Hemisphere R=16 on the substrate of a 64x64x32 box with walls at
    z=0 and z=32, jitter 0.15h, density ratio 2, theta on the substrate."""
    return _sessile("sessile droplet 64x64x32", 64, 32, 16.0, seed, 0.15, theta, steps)


def small_free_droplet_3d(n=10, R=3.0, seed=8, steps=20, **phys):
    """A small periodic 3D droplet for oracle checks."""
    return _free(f"free droplet {n}^3", n, R, seed, 0.15, steps, **phys)


def small_sessile_3d(n=10, nz=6, R=4.0, seed=9, theta=60.0, steps=20, **phys):
    """A small 3D sessile droplet for oracle checks."""
    return _sessile(f"sessile droplet {n}x{n}x{nz}", n, nz, R, seed, 0.15, theta, steps, **phys)
