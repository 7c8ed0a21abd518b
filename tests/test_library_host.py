"""Host-side checks of the C-ABI library (no GPU needed): the shared library
loads, exports every function ``include/felbm.h`` declares, validates meshes,
derives the model constants, and builds the node tables."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_1708_04678_gb300 import build as B
from paper_1708_04678_gb300 import felbm as F
from paper_1708_04678_gb300 import inputs as I

HEADERS = [os.path.join(B.INCLUDE, n) for n in sorted(os.listdir(B.INCLUDE)) if n.endswith(".h")]


@pytest.fixture(scope="module")
def lib():
    B.build()
    return F.lib()


def _declared_functions():
    names = set()
    for path in HEADERS:
        src = re.sub(r"/\*.*?\*/", "", open(path).read(), flags=re.S)
        names |= set(re.findall(r"\b(felbm(?:3d)?_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_header_symbols_are_exported(lib):
    names = _declared_functions()
    assert "felbm_step" in names and "felbm_mesh_create" in names
    assert "felbm3d_step" in names and "felbm3d_mesh_create" in names
    for name in names:
        assert hasattr(lib, name), name


def test_params_derive_closed_forms(lib):
    # xi = sqrt(8 kappa / beta), sigma = sqrt(2 kappa beta) / 6, cos(theta) = -phi_c / sqrt(2 kappa beta)
    phys = dict(dt=0.5, tau_l=0.8, tau_v=0.8, rho_l=1.0, rho_v=0.1, sigma=0.01, xi=4.0,
                mobility=0.02, theta_deg=(60.0, 90.0, 120.0))
    p = F.params_derive(phys)
    assert math.isclose(math.sqrt(8 * p.kappa / p.beta), 4.0, rel_tol=1e-14)
    assert math.isclose(math.sqrt(2 * p.kappa * p.beta) / 6, 0.01, rel_tol=1e-14)
    for k, th in enumerate((60.0, 90.0, 120.0)):
        assert math.isclose(-p.phi_c[k] / math.sqrt(2 * p.kappa * p.beta), math.cos(math.radians(th)),
                            rel_tol=1e-12, abs_tol=1e-15)
    assert p.n_wall_ids == 3


def test_mesh_tables(lib):
    w = I.sessile_droplet_64x32()
    mesh = F.Mesh.from_dict(w["mesh"])
    info = mesh.info()
    assert info["n_nodes"] == 64 * 33 and info["n_tri"] == 2 * 64 * 32
    assert info["n_wall_edges"] == 128
    assert info["max_degree"] == 7                       # 6 neighbours + itself on the '/' grid
    assert info["nnz"] == 7 * 64 * 33 - 2 * 64 * 2      # wall rows have 5 entries
    assert abs(info["total_area"] - 64 * 32) < 1e-9
    # node tiles: at most 1024 nodes each, compact (bisection), so a tile's
    # halo is a thin ring: 2,112 nodes -> 4 tiles of 528
    assert info["n_tiles"] == 4
    assert 0 < info["max_tile_halo"] < 4 * 32
    p = F.params_derive(w["phys"])
    assert mesh.workspace_bytes(p) > 18 * 8 * info["n_nodes"]


def test_mesh_validation(lib):
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    walls = np.array([[0, 1], [1, 2], [2, 3], [3, 0]])
    F.Mesh(xy, [[0, 1, 2], [0, 2, 3]], walls, [0, 0, 0, 0])           # valid square
    with pytest.raises(F.FelbmError) as e:                            # clockwise triangle
        F.Mesh(xy, [[0, 2, 1], [0, 2, 3]], walls, [0, 0, 0, 0])
    assert e.value.code == -2
    with pytest.raises(F.FelbmError) as e:                            # open edge not declared a wall
        F.Mesh(xy, [[0, 1, 2], [0, 2, 3]], walls[:3], [0, 0, 0])
    assert e.value.code == -2
    with pytest.raises(F.FelbmError) as e:                            # node id out of range
        F.Mesh(xy, [[0, 1, 7], [0, 2, 3]], walls, [0, 0, 0, 0])
    assert e.value.code == -1
    with pytest.raises(F.FelbmError) as e:                            # wall edge inside the mesh
        F.Mesh(xy, [[0, 1, 2], [0, 2, 3]], np.vstack([walls, [[0, 2]]]), [0, 0, 0, 0, 0])
    assert e.value.code == -2


def test_periodic_mesh_min_image(lib):
    m = I.cross_mesh(16, 16, 0.25, 1)
    mesh = F.Mesh.from_dict(m)
    info = mesh.info()
    assert info["n_nodes"] == 512 and info["n_wall_edges"] == 0
    assert abs(info["total_area"] - 256.0) < 1e-9
    assert abs(info["min_area"] - m["min_area"]) < 1e-12


def test_empty_and_invalid_sizes_are_rejected(lib):
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0]])
    with pytest.raises(F.FelbmError) as e:
        F.Mesh(xy, np.zeros((0, 3), np.int32))
    assert e.value.code == -1
    with pytest.raises(F.FelbmError) as e:
        F.Mesh(np.zeros((0, 2)), np.zeros((0, 3), np.int32))
    assert e.value.code == -1
    with pytest.raises(F.FelbmError) as e:                       # wall id beyond the table
        F.Mesh(xy, [[0, 1, 2]], [[0, 1], [1, 2], [2, 0]], [0, 0, F.MAX_WALL_IDS])
    assert e.value.code == -1


# ------------------------------------------------------------ 3D meshes ---
def test_mesh3d_tables(lib):
    from paper_1708_04678_gb300 import felbm3d as F3
    from paper_1708_04678_gb300 import inputs3d as I3
    w = I3.small_sessile_3d(n=10, nz=6)
    mesh = F3.Mesh3D.from_dict(w["mesh"])
    info = mesh.info()
    assert info["n_nodes"] == 10 * 10 * 7 and info["n_tet"] == 6 * 10 * 10 * 6
    assert info["n_wall_faces"] == 2 * 2 * 10 * 10
    assert info["max_degree"] == 15 and info["max_incidence"] == 24   # Kuhn: 14 neighbours, 24 tetrahedra
    assert info["nnz"] == 15 * 10 * 10 * 5 + 11 * 2 * 10 * 10        # wall rows: 10 neighbours
    assert abs(info["total_volume"] - 600.0) < 1e-9
    p = F.params_derive(w["phys"])
    assert mesh.workspace_bytes(p) > 38 * 8 * info["n_nodes"]
    periodic = F3.Mesh3D.from_dict(I3.kuhn_box(6, 5, 4, 0.15, 2, walls=False))
    assert periodic.info()["nnz"] == 15 * 6 * 5 * 4 and periodic.info()["n_wall_faces"] == 0


def test_mesh3d_validation(lib):
    from paper_1708_04678_gb300 import felbm3d as F3
    xyz = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    faces = [[0, 1, 2], [0, 1, 3], [0, 2, 3], [1, 2, 3]]
    F3.Mesh3D(xyz, [[0, 1, 2, 3]], faces, [0, 0, 0, 0])                  # valid tetrahedron
    with pytest.raises(F.FelbmError) as e:                                 # inverted
        F3.Mesh3D(xyz, [[0, 2, 1, 3]], faces, [0, 0, 0, 0])
    assert e.value.code == -2
    with pytest.raises(F.FelbmError) as e:                                 # boundary face not a wall
        F3.Mesh3D(xyz, [[0, 1, 2, 3]], faces[:3], [0, 0, 0])
    assert e.value.code == -2
    with pytest.raises(F.FelbmError) as e:                                 # node out of range
        F3.Mesh3D(xyz, [[0, 1, 2, 9]], faces, [0, 0, 0, 0])
    assert e.value.code == -1
    with pytest.raises(F.FelbmError) as e:                                 # repeated node
        F3.Mesh3D(xyz, [[0, 1, 1, 3]], faces, [0, 0, 0, 0])
    assert e.value.code == -1
    with pytest.raises(F.FelbmError) as e:                                 # wall id beyond the table
        F3.Mesh3D(xyz, [[0, 1, 2, 3]], faces, [0, 0, 0, F.MAX_WALL_IDS])
    assert e.value.code == -1


def test_diag_slot_buffers_are_validated(lib):
    """The queued-diagnostics binding takes only contiguous host float64
    buffers of at least FELBM_DIAG_SLOTS values (the library copies that many
    sums into them asynchronously)."""
    torch = pytest.importorskip("torch")
    hdr = open(os.path.join(B.INCLUDE, "felbm.h")).read()
    assert int(re.search(r"#define FELBM_DIAG_SLOTS (\d+)", hdr).group(1)) == F.DIAG_SLOTS
    F.check_slots(np.zeros(F.DIAG_SLOTS))
    F.check_slots(torch.zeros((3, F.DIAG_SLOTS), dtype=torch.float64)[1])
    for bad in (np.zeros(F.DIAG_SLOTS - 1), np.zeros(F.DIAG_SLOTS, dtype=np.float32),
                np.zeros((F.DIAG_SLOTS, 2))[:, 0], torch.zeros(F.DIAG_SLOTS, dtype=torch.float32),
                torch.zeros((F.DIAG_SLOTS, 2), dtype=torch.float64)[:, 0]):
        with pytest.raises(ValueError):
            F.check_slots(bad)


def test_channel_mesh_with_a_hole(lib):
    """The capillary-channel geometry: a periodic box with a solid block and a
    channel through it.  Every boundary edge is a declared wall (the library
    accepts the mesh), the wall count is the block's perimeter in cells (two
    channel walls of length L, two end faces of height 2H) and the fluid area
    is the box minus the block."""
    H, lf, res = 4, 4, 2
    w = I.capillary_channel(H=H, length_factor=lf, reservoir=res, xi=2.0)
    info = F.Mesh.from_dict(w["mesh"]).info()
    L = lf * H
    nx, ny = L + 2 * res * H, 3 * H
    assert info["n_wall_edges"] == 2 * L + 2 * (2 * H)
    assert abs(info["total_area"] - (nx * ny - L * 2 * H)) < 1e-9
    assert info["n_groups"] == 1


def test_capillary_intrusion_workload(lib):
    """The capillary-intrusion workload: the channel geometry at H = 16 with
    the physics that lets the contact line move (xi 4, M 1, dt 0.05), the
    liquid column ending 2H inside the channel on its centre line, and a
    mesh the library accepts with the block's perimeter as walls."""
    w = I.capillary_intrusion(H=16, theta=56.0)
    ph = w["phys"]
    assert (ph["xi"], ph["mobility"], ph["dt"], ph["theta_deg"]) == (4.0, 1.0, 0.05, (56.0,))
    xy, C0 = w["mesh"]["xy"], w["C0"]
    line = np.abs(xy[:, 1] - w["y_c"]) < 0.25
    x, c = xy[line, 0], C0[line]
    o = np.argsort(x)
    x, c = x[o], c[o]
    inside = (x > w["x_in"]) & (x < w["x_in"] + w["length"])
    j = np.nonzero(inside & (c > 0.5))[0][-1]
    cross = x[j] + (c[j] - 0.5) / (c[j] - c[j + 1]) * (x[j + 1] - x[j])
    assert abs(cross - (w["x_in"] + 2 * w["H"])) < 1e-9
    info = F.Mesh.from_dict(w["mesh"]).info()
    assert info["n_nodes"] == len(xy) == 11615
    assert info["n_wall_edges"] == 2 * int(w["length"]) + 2 * (2 * 16)


def test_node_tiles_of_the_workloads():
    """Tiles cover every node with at most 1024 nodes and a halo that fits the
    staged rows of the tiled solve step (504), on the rough-wall droplet, the
    free droplet and a batch of droplets (tiles never span members)."""
    for w, n_tiles in ((I.rough_wall_droplet(width=256, height=128, rows=129, R=40.0), 64),
                       (I.free_droplet_256(n=64), 8)):
        info = F.Mesh.from_dict(w["mesh"]).info()
        assert info["n_tiles"] == n_tiles, info
        assert info["max_tile_halo"] < 160, info
    b = I.batch(I.droplet_sweep(count=4, w_min=64, w_max=96))
    info = F.Mesh.batch(b["meshes"]).info()
    assert info["n_tiles"] >= 4 * 2 and info["max_tile_halo"] < 160, info


def test_static_solve_arguments_are_validated_before_any_launch():
    """felbm_mass_solve_static reads and writes k x n_nodes doubles through
    raw device pointers, so the binding rejects every tensor that would make
    it run past a buffer -- wrong dtype, strides, shape, k, device, or X
    overlapping B -- before the C ABI is called (the handle here is a dummy
    that a call would dereference)."""
    torch = pytest.importorskip("torch")
    n = 40
    st = F.State.__new__(F.State)
    st.torch, st.N, st.handle = torch, n, None
    st.workspace = torch.empty(16, dtype=torch.uint8)          # the state's device: cpu here
    good = torch.zeros((3, n), dtype=torch.float64)
    assert st.check_static_solve_args(good, torch.zeros_like(good)) == 3
    bad_pairs = [
        (good.float(), torch.zeros_like(good)),                               # dtype of B
        (good, torch.zeros((3, n), dtype=torch.float32)),                     # dtype of X
        (torch.zeros((n, 3), dtype=torch.float64).t(), torch.zeros_like(good)),  # strided B
        (torch.zeros((3, n - 1), dtype=torch.float64), torch.zeros((3, n - 1), dtype=torch.float64)),
        (torch.zeros((19, n), dtype=torch.float64), torch.zeros((19, n), dtype=torch.float64)),
        (torch.zeros((0, n), dtype=torch.float64), torch.zeros((0, n), dtype=torch.float64)),
        (torch.zeros(3 * n, dtype=torch.float64), torch.zeros(3 * n, dtype=torch.float64)),
        (good, torch.zeros((2, n), dtype=torch.float64)),                     # X smaller than B
        (good, good),                                                         # X aliases B
        (good, torch.zeros((3, n), dtype=torch.float64, device="meta")),      # another device
        (good.numpy(), torch.zeros_like(good)),                               # not a tensor
    ]
    buf = torch.zeros((4, n), dtype=torch.float64)
    bad_pairs.append((buf[:3], buf[1:]))                                      # partial overlap
    for B_, X_ in bad_pairs:
        with pytest.raises(ValueError):
            st.mass_solve_static(B_, X_)
