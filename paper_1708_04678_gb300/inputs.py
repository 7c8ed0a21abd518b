"""Seeded synthetic inputs for the FE-LBM contact-line step.

This module produces the *inputs* that both the CPU oracle tests and the CUDA
path consume: triangle meshes (node coordinates, connectivity, wall edges,
periodic lengths), initial composition fields and the physical parameters of
the droplet workloads.  It holds none of the method's arithmetic: no
geometry factors, matrices, equilibria, forces or derived model constants
(kappa, beta, phi_c are derived separately on each side from sigma, xi and
theta).

Random numbers come from ``numpy.random.default_rng`` (PCG64) and are drawn in
a fixed order, so a (generator, seed) pair fixes every mesh bit for bit.

Workloads (2D analogues of the paper's droplet benchmarks, Sec. III):

* ``sessile_droplet_64x32``  -- 64x32 box, walls at y=0,32, periodic x,
  2-triangle cells, jitter 0.2h, semicircular droplet R=12 on the bottom wall.
* ``free_droplet_256``       -- 256x256 doubly periodic box, cells split into
  4 triangles around a centre node (131,585 grid points), jitter 0.25h,
  droplet R=48 (the static-droplet / spurious-current case of Sec. III.A).
* ``droplet_sweep``          -- many independent sessile droplets of uneven
  widths 64..512 and contact angles 30..150 degrees.
* ``sessile_droplet_128x64`` -- 128x64 version of the sessile case.
* ``rough_wall_droplet``     -- droplet on a sinusoidal wall
  y = 8 + 4 sin(2 pi x / 64), body-fitted 2048 x 1017 node mesh.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "grid_mesh",
    "cross_mesh",
    "droplet_C0",
    "sessile_droplet_64x32",
    "sessile_droplet_128x64",
    "free_droplet_256",
    "droplet_sweep",
    "rough_wall_droplet",
    "rough_wall_strip",
    "small_sessile",
    "small_free_droplet",
    "batch",
]


def _triangle_areas(xy, tri, period):
    """Signed areas with minimum-image edge vectors (used only to report the
    worst triangle of a generated mesh, not by either implementation)."""
    px, py = period
    d1 = xy[tri[:, 1]] - xy[tri[:, 0]]
    d2 = xy[tri[:, 2]] - xy[tri[:, 0]]
    for d in (d1, d2):
        if px > 0:
            d[:, 0] -= px * np.round(d[:, 0] / px)
        if py > 0:
            d[:, 1] -= py * np.round(d[:, 1] / py)
    return 0.5 * (d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0])


def grid_mesh(nx, ny, jitter, seed, h=1.0, y_bottom=None, y_top=None):
    """Structured grid split into two triangles per cell along the '/' diagonal.

    Grid points (i, j), i = 0..nx, j = 0..ny; column nx is the periodic image
    of column 0, so the mesh has nx*(ny+1) unique nodes.  Rows j = 0 and
    j = ny are walls (wall id 0 bottom, 1 top) and are not jittered; every
    other node moves by U(-jitter*h, +jitter*h) in x and in y.

    ``y_bottom`` / ``y_top`` (callables of x) give a body-fitted mesh: row j
    sits at y_bottom(x) + (y_top(x) - y_bottom(x)) * j / ny.  Default: flat
    walls at 0 and ny*h.
    """
    ncol = nx
    nrow = ny + 1
    n = ncol * nrow
    i = np.tile(np.arange(ncol), nrow)
    j = np.repeat(np.arange(nrow), ncol)
    x = i * h
    if y_bottom is None:
        y = j * h
    else:
        yb = np.asarray(y_bottom(x), dtype=np.float64)
        yt = np.asarray(y_top(x), dtype=np.float64)
        y = yb + (yt - yb) * (j / ny)
    xy = np.stack([x.astype(np.float64), y.astype(np.float64)], axis=1)
    rng = np.random.default_rng(seed)
    jit = rng.uniform(-jitter * h, jitter * h, size=(n, 2))
    wall_node = (j == 0) | (j == ny)
    jit[wall_node] = 0.0
    xy = xy + jit

    def nid(ii, jj):
        return jj * ncol + (ii % ncol)

    ci = np.tile(np.arange(nx), ny)
    cj = np.repeat(np.arange(ny), nx)
    n00 = nid(ci, cj)
    n10 = nid(ci + 1, cj)
    n11 = nid(ci + 1, cj + 1)
    n01 = nid(ci, cj + 1)
    tri = np.empty((2 * nx * ny, 3), dtype=np.int32)
    tri[0::2] = np.stack([n00, n10, n11], axis=1)
    tri[1::2] = np.stack([n00, n11, n01], axis=1)

    wi = np.arange(nx)
    bottom = np.stack([nid(wi, 0), nid(wi + 1, 0)], axis=1)
    top = np.stack([nid(wi, ny), nid(wi + 1, ny)], axis=1)
    wall_edges = np.concatenate([bottom, top]).astype(np.int32)
    wall_id = np.concatenate([np.zeros(nx), np.ones(nx)]).astype(np.int32)
    period = (float(nx * h), 0.0)
    areas = _triangle_areas(xy, tri, period)
    return {
        "xy": xy,
        "tri": tri,
        "wall_edges": wall_edges,
        "wall_id": wall_id,
        "period": period,
        "n_grid_points": (nx + 1) * (ny + 1),
        "min_area": float(areas.min()),
    }


def cross_mesh(nx, ny, jitter, seed, h=1.0):
    """Doubly periodic grid whose cells are split into 4 triangles around a
    cell-centre node.  Corner nodes (i, j) and centre nodes (i+1/2, j+1/2),
    i < nx, j < ny; every node is jittered by U(-jitter*h, +jitter*h).
    Grid points counted with the periodic images: (nx+1)(ny+1) + nx*ny."""
    nc = nx * ny
    n = 2 * nc
    ci = np.tile(np.arange(nx), ny)
    cj = np.repeat(np.arange(ny), nx)
    xy = np.empty((n, 2), dtype=np.float64)
    xy[:nc, 0] = ci * h
    xy[:nc, 1] = cj * h
    xy[nc:, 0] = (ci + 0.5) * h
    xy[nc:, 1] = (cj + 0.5) * h
    rng = np.random.default_rng(seed)
    xy += rng.uniform(-jitter * h, jitter * h, size=(n, 2))

    def corner(ii, jj):
        return (jj % ny) * nx + (ii % nx)

    c00 = corner(ci, cj)
    c10 = corner(ci + 1, cj)
    c11 = corner(ci + 1, cj + 1)
    c01 = corner(ci, cj + 1)
    m = nc + cj * nx + ci
    tri = np.empty((4 * nc, 3), dtype=np.int32)
    tri[0::4] = np.stack([c00, c10, m], axis=1)
    tri[1::4] = np.stack([c10, c11, m], axis=1)
    tri[2::4] = np.stack([c11, c01, m], axis=1)
    tri[3::4] = np.stack([c01, c00, m], axis=1)
    period = (float(nx * h), float(ny * h))
    areas = _triangle_areas(xy, tri, period)
    return {
        "xy": xy,
        "tri": tri,
        "wall_edges": np.zeros((0, 2), dtype=np.int32),
        "wall_id": np.zeros((0,), dtype=np.int32),
        "period": period,
        "n_grid_points": (nx + 1) * (ny + 1) + nx * ny,
        "min_area": float(areas.min()),
    }


def droplet_C0(xy, centre, R, xi, period=(0.0, 0.0)):
    """Initial composition: a disc (or a cap cut by a wall) of radius R with
    the equilibrium tanh profile of width xi across its rim (Sec. II,
    plane-interface profile with z = R - r).  Distances use the minimum
    image along periodic directions."""
    d = xy - np.asarray(centre, dtype=np.float64)[None, :]
    for k in range(2):
        if period[k] > 0:
            d[:, k] -= period[k] * np.round(d[:, k] / period[k])
    r = np.sqrt(d[:, 0] ** 2 + d[:, 1] ** 2)
    return 0.5 + 0.5 * np.tanh(2.0 * (R - r) / xi)


# Time steps: the Taylor-Galerkin streaming step is explicit, and dt = 0.5
# (h = 1) exceeds its stability limit on these meshes (noisy uniform states
# grow at dt >= 0.35 on 2-triangle cells with 0.2h jitter, and at dt >= 0.15
# on small 4-triangle meshes with 0.25h jitter; the 256x256 4-triangle mesh,
# whose jitter leaves slivers of area 0.004 h^2, diverges at dt = 0.08 and is
# stable at dt <= 0.06).  The workloads therefore use dt = 0.25 on 2-triangle
# meshes and dt = 0.05 on the 4-triangle meshes.
DT_GRID = 0.25
DT_CROSS = 0.05
# The rough-wall droplet (density ratio 100 on 2-triangle cells): at dt = 0.25
# it grows spurious currents until it diverges (within 1,500 steps with the
# face-averaged Laplacian of mu, before 10,000 with the nodal one), and at
# dt = 0.05 too (the scheme's viscosity cs2 tau dt is then too small); at
# dt = 0.1 the nodal form runs its 10,000 steps.
DT_ROUGH = 0.1


def _phys(**kw):
    base = dict(dt=DT_GRID, tau_l=0.8, tau_v=0.8, rho_l=1.0, rho_v=0.1, sigma=0.01,
                xi=4.0, mobility=0.02, theta_deg=(90.0, 90.0))
    base.update(kw)
    base["theta_deg"] = tuple(float(t) for t in base["theta_deg"])
    return base


def _sessile(name, nx, ny, seed, R, jitter=0.2, theta=90.0, ratio=10.0, steps=2000):
    mesh = grid_mesh(nx, ny, jitter, seed)
    centre = (nx / 2.0, 0.0)
    phys = _phys(rho_v=1.0 / ratio, theta_deg=(theta, 90.0))
    C0 = droplet_C0(mesh["xy"], centre, R, phys["xi"], mesh["period"])
    return {"name": name, "mesh": mesh, "C0": C0, "phys": phys, "steps": steps,
            "centre": centre, "R": float(R)}


def sessile_droplet_64x32(seed=0):
    """Semicircular droplet R=12 on the bottom wall of a 64x32 box, 90 degree
    walls, density ratio 10, tau 0.8, sigma 0.01, M 0.02, dt 0.25, 2000 steps."""
    return _sessile("sessile droplet 64x32", 64, 32, seed, 12.0)


def sessile_droplet_128x64(seed=3):
    """The sessile case on a 128x64 box (8,385 grid points), 3000 steps."""
    return _sessile("sessile droplet 128x64", 128, 64, seed, 24.0, steps=3000)


def small_sessile(nx=32, ny=16, seed=11, R=7.0, theta=90.0, jitter=0.2, steps=50):
    """A small sessile case for quick checks."""
    return _sessile(f"sessile droplet {nx}x{ny}", nx, ny, seed, R, jitter=jitter,
                    theta=theta, steps=steps)


def free_droplet_256(seed=1, n=256, R=48.0, steps=20000):
    """Static free droplet in a doubly periodic n x n box meshed with 4
    triangles per cell (131,585 grid points at n=256), jitter 0.25h, R=48,
    xi 4, density ratio 100, tau 0.6, sigma 0.005, M 0.02, dt 0.05."""
    mesh = cross_mesh(n, n, 0.25, seed)
    centre = (n / 2.0, n / 2.0)
    phys = _phys(dt=DT_CROSS, rho_v=0.01, tau_l=0.6, tau_v=0.6, sigma=0.005, theta_deg=())
    C0 = droplet_C0(mesh["xy"], centre, R, phys["xi"], mesh["period"])
    return {"name": f"free droplet {n}x{n}", "mesh": mesh, "C0": C0, "phys": phys,
            "steps": steps, "centre": centre, "R": float(R)}


def small_free_droplet(n=24, R=6.0, seed=5, steps=50, ratio=10.0, sigma=0.01):
    """A small doubly periodic free droplet for quick checks."""
    mesh = cross_mesh(n, n, 0.25, seed)
    centre = (n / 2.0, n / 2.0)
    phys = _phys(dt=DT_CROSS, rho_v=1.0 / ratio, sigma=sigma, theta_deg=())
    C0 = droplet_C0(mesh["xy"], centre, R, phys["xi"], mesh["period"])
    return {"name": f"free droplet {n}x{n}", "mesh": mesh, "C0": C0, "phys": phys,
            "steps": steps, "centre": centre, "R": float(R)}


def droplet_sweep(seed=2, count=64, w_min=64, w_max=512, jitter=0.2, steps=5000):
    """Independent sessile droplets: widths W even in [w_min, w_max], height
    W/2, R = W/5, contact angle U(30, 150) degrees on the bottom wall, density
    ratio 10.  Widths and angles come from ``default_rng(seed)``; mesh k is
    jittered from ``default_rng([seed, k])``."""
    rng = np.random.default_rng(seed)
    widths = 2 * rng.integers(w_min // 2, w_max // 2 + 1, size=count)
    thetas = rng.uniform(30.0, 150.0, size=count)
    out = []
    for k in range(count):
        W = int(widths[k])
        H = W // 2
        mesh = grid_mesh(W, H, jitter, [seed, k])
        R = W / 5.0
        centre = (W / 2.0, 0.0)
        phys = _phys(theta_deg=(float(thetas[k]), 90.0))
        C0 = droplet_C0(mesh["xy"], centre, R, phys["xi"], mesh["period"])
        out.append({"name": f"sweep droplet {k} ({W}x{H}, {thetas[k]:.1f} deg)",
                    "mesh": mesh, "C0": C0, "phys": phys, "steps": steps,
                    "centre": centre, "R": R})
    return out


def batch(workloads):
    """Many independent sessile workloads as one batch: member k keeps its
    mesh (and periodic width) and gets wall ids 2k (bottom) and 2k+1 (top),
    so theta_deg lists the angles of all walls; C0 is concatenated.  The
    members must share every physical parameter except the contact angles.
    Returns the batch workload with ``meshes`` (for Mesh.batch) and the
    per-member ``members`` (offset, node count, centre, R)."""
    meshes, thetas, C0, members = [], [], [], []
    ref = dict(workloads[0]["phys"])
    off = 0
    for k, w in enumerate(workloads):
        m = dict(w["mesh"])
        ids = np.asarray(m["wall_id"], dtype=np.int32)
        if ids.size and ids.max() > 1:
            raise ValueError("batch members must use wall ids 0 and 1")
        m["wall_id"] = (ids + 2 * k).astype(np.int32)
        meshes.append(m)
        th = tuple(w["phys"]["theta_deg"]) + (90.0,) * (2 - len(w["phys"]["theta_deg"]))
        thetas.extend(th[:2])
        for key in ("dt", "tau_l", "tau_v", "rho_l", "rho_v", "sigma", "xi", "mobility"):
            if w["phys"][key] != ref[key]:
                raise ValueError(f"batch members differ in {key}")
        C0.append(w["C0"])
        n = len(m["xy"])
        members.append({"offset": off, "nodes": n, "centre": w.get("centre"), "R": w.get("R"),
                        "substrate": 2 * k, "name": w["name"]})
        off += n
    phys = dict(ref)
    phys["theta_deg"] = tuple(thetas)
    return {"name": f"batch of {len(workloads)} droplets", "meshes": meshes, "C0": np.concatenate(C0),
            "phys": phys, "members": members, "steps": max(w["steps"] for w in workloads)}


def rough_wall_droplet(seed=4, width=2048, height=1024, rows=1017, R=300.0,
                       theta=60.0, amp=4.0, base=8.0, wavelength=64.0, steps=10000):
    """Droplet on a sinusoidally rough wall y = base + amp*sin(2 pi x/wavelength)
    (periodic in x), top wall at y = height; body-fitted mesh of width x rows
    nodes, jitter 0.2h, density ratio 100, dt 0.1, contact angle ``theta`` at
    the rough wall, 90 degrees at the top."""

    def yb(x):
        return base + amp * np.sin(2.0 * math.pi * x / wavelength)

    def yt(x):
        return np.full_like(x, float(height), dtype=np.float64)

    mesh = grid_mesh(width, rows - 1, 0.2, seed, y_bottom=yb, y_top=yt)
    centre = (width / 2.0, base)
    phys = _phys(dt=DT_ROUGH, rho_v=0.01, theta_deg=(theta, 90.0))
    C0 = droplet_C0(mesh["xy"], centre, R, phys["xi"], mesh["period"])
    return {"name": f"rough-wall droplet {width}x{height}", "mesh": mesh, "C0": C0,
            "phys": phys, "steps": steps, "centre": centre, "R": float(R)}


def rough_wall_strip(columns=128, seed=40, **kw):
    """A periodic strip of ``columns`` columns cut from the rough-wall
    droplet's recipe (same 1017 body-fitted rows, wall profile, jitter,
    physics and droplet field, centred on the droplet's axis): a bounded
    sample of that workload for timing the CPU oracle per node-update.
    ``columns`` must be a multiple of the wall's wavelength (64) so that the
    wall stays periodic; the droplet field is symmetric about the strip's
    centre, so its periodic images match."""
    if columns % 64:
        raise ValueError("columns must be a multiple of 64")
    w = rough_wall_droplet(seed=seed, width=columns, **kw)
    w["name"] = f"rough-wall strip {columns} columns"
    return w


def capillary_channel(H=16, length_factor=20, reservoir=4, theta=56.0, l0_factor=2.0, liquid_factor=4.0,
                      ratio=10.0, dt=0.1, sigma=0.01, xi=2.0, mobility=0.02, jitter=0.0, seed=6):
    """Capillary intrusion, the 2D analogue of Sec. III.C: a box periodic in x
    and y holding one solid block with a straight channel of width H and
    length length_factor*H through it (wall id 0 on every face of the block,
    wetting angle theta); outside the channel's x-range the fluid is open and
    periodic.  Liquid fills a slab of liquid_factor*H to the left of the
    entrance and the first l0_factor*H of the channel (flat meniscus); vapour
    fills the rest.  Grid points (i, j) with h = 1, two triangles per cell;
    cells inside the block are left out.  Returns the workload dict and the
    channel geometry (x of the entrance ``x_in``, centre line ``y_c``, H)."""
    Lc = int(length_factor * H)
    res = int(reservoir * H)
    nx = Lc + 2 * res
    ny = 3 * H
    i0, i1 = res, res + Lc                 # channel x-range (cells)
    j0, j1 = H, 2 * H                      # channel y-range (cells)

    ci, cj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    solid = (ci >= i0) & (ci < i1) & ((cj < j0) | (cj >= j1))
    keep = ~solid
    # nodes used by a kept cell (periodic in both directions)
    used = np.zeros((ny, nx), dtype=bool)
    for di in (0, 1):
        for dj in (0, 1):
            used[(cj + dj) % ny, (ci + di) % nx] |= keep
    node_id = -np.ones((ny, nx), dtype=np.int64)
    node_id[used] = np.arange(int(used.sum()))
    jj, ii = np.nonzero(used)
    xy = np.stack([ii.astype(np.float64), jj.astype(np.float64)], axis=1)

    def nid(a, b):
        return node_id[b % ny, a % nx]

    kc_j, kc_i = np.nonzero(keep)
    n00, n10 = nid(kc_i, kc_j), nid(kc_i + 1, kc_j)
    n11, n01 = nid(kc_i + 1, kc_j + 1), nid(kc_i, kc_j + 1)
    tri = np.empty((2 * len(kc_i), 3), dtype=np.int32)
    tri[0::2] = np.stack([n00, n10, n11], axis=1)
    tri[1::2] = np.stack([n00, n11, n01], axis=1)

    # wall edges: cell sides between a kept cell and a solid one
    walls = []
    for a, b in zip(kc_i, kc_j):
        if solid[(b - 1) % ny, a]:
            walls.append((nid(a, b), nid(a + 1, b)))
        if solid[(b + 1) % ny, a]:
            walls.append((nid(a, b + 1), nid(a + 1, b + 1)))
        if solid[b, (a - 1) % nx]:
            walls.append((nid(a, b), nid(a, b + 1)))
        if solid[b, (a + 1) % nx]:
            walls.append((nid(a + 1, b), nid(a + 1, b + 1)))
    wall_edges = np.asarray(walls, dtype=np.int32)
    wall_id = np.zeros(len(walls), dtype=np.int32)

    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        on_wall = np.zeros(len(xy), dtype=bool)
        on_wall[wall_edges.ravel()] = True
        jit = rng.uniform(-jitter, jitter, size=xy.shape)
        jit[on_wall] = 0.0
        xy = xy + jit

    period = (float(nx), float(ny))
    phys = _phys(dt=dt, rho_v=1.0 / ratio, sigma=sigma, xi=xi, mobility=mobility, theta_deg=(theta,))
    x_in = float(i0)
    xa = x_in - liquid_factor * H
    xm = x_in + l0_factor * H
    d = np.minimum(xy[:, 0] - xa, xm - xy[:, 0])
    C0 = 0.5 + 0.5 * np.tanh(2.0 * d / xi)
    mesh = {"xy": xy, "tri": tri, "wall_edges": wall_edges, "wall_id": wall_id, "period": period,
            "n_grid_points": int(used.sum()), "min_area": float(_triangle_areas(xy, tri, period).min())}
    return {"name": f"capillary channel H={H}, theta={theta}", "mesh": mesh, "C0": C0, "phys": phys,
            "x_in": x_in, "y_c": 1.5 * H, "H": float(H), "length": float(Lc), "l0": l0_factor * H}


def capillary_intrusion(H=16, theta=56.0, length_factor=20, seed=6):
    """The capillary-intrusion workload (Sec. III.C, as a 2D channel between
    parallel plates): ``capillary_channel`` with an interface width xi = 4
    (four grid spacings), Cahn-Hilliard mobility M = 1, dt = 0.05, tau 0.8 in
    both phases, density ratio 10, sigma 0.01, run with the nodal element
    Laplacian of mu.  With xi = 2 the contact line hops from node to node
    and stalls, and with M = 0.02 it barely moves; with these values the
    column's speed approaches the two-phase parallel-plate Washburn rate
    dl/dt = H sigma cos(theta) / (6 (eta_l l + eta_v (L - l))),
    eta = rho cs2 tau dt, once the start-up transient has passed."""
    w = capillary_channel(H=H, length_factor=length_factor, theta=theta, dt=0.05, xi=4.0, mobility=1.0,
                          seed=seed)
    w["name"] = f"capillary intrusion H={H}, theta={theta}"
    return w
