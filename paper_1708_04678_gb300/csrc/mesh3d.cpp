// Host-side preprocessing of a tetrahedral mesh for the 3D FE-LBM step:
// validation, P1 geometry of each tetrahedron (Sec. II.C: constant shape
// gradients per element), face neighbours and wall faces (Sec. II.B/II.D),
// reverse Cuthill-McKee node order, and the node-centric tables of the
// gather kernels (node-node pattern with consistent mass and P1 stiffness,
// node -> tetrahedron and node -> wall-face incidence).  Runs once per mesh.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "felbm3d_internal.h"

namespace felbm {

static double min_image3(double d, double L) {
    if (L > 0.0) d -= L * std::round(d / L);
    return d;
}

namespace {
struct FaceRec {
    int32_t a, b, c;   // sorted node ids
    int32_t tet, k;    // owning tetrahedron and the local vertex opposite the face
    bool operator<(const FaceRec& o) const {
        if (a != o.a) return a < o.a;
        if (b != o.b) return b < o.b;
        if (c != o.c) return c < o.c;
        return tet < o.tet;
    }
    bool same(const FaceRec& o) const { return a == o.a && b == o.b && c == o.c; }
};

FaceRec face_of(int32_t p, int32_t q, int32_t r, int32_t t, int32_t k) {
    int32_t v[3] = {p, q, r};
    std::sort(v, v + 3);
    return FaceRec{v[0], v[1], v[2], t, k};
}
}  // namespace

static int build_mesh3d(const double* xyz, int32_t N, const int32_t* tet_in, int32_t T, const int32_t* wf_in,
                        const int32_t* wid_in, int32_t F, const double* period, HostMesh3D& m) {
    char buf[256];
    m.N = N;
    m.T = T;
    m.F = F;
    for (int d = 0; d < 3; ++d) m.period[d] = period ? period[d] : 0.0;
    for (int64_t i = 0; i < 4 * (int64_t)T; ++i)
        if (tet_in[i] < 0 || tet_in[i] >= N) {
            set_error("felbm3d_mesh_create: tetrahedron vertex out of range");
            return FELBM_ERR_INVALID_ARG;
        }
    for (int32_t t = 0; t < T; ++t) {
        const int32_t* v = tet_in + 4 * (size_t)t;
        for (int i = 0; i < 4; ++i)
            for (int j = i + 1; j < 4; ++j)
                if (v[i] == v[j]) {
                    snprintf(buf, sizeof buf, "felbm3d_mesh_create: tetrahedron %d repeats a node", t);
                    set_error(buf);
                    return FELBM_ERR_INVALID_ARG;
                }
    }
    for (int64_t i = 0; i < 3 * (int64_t)F; ++i)
        if (wf_in[i] < 0 || wf_in[i] >= N) {
            set_error("felbm3d_mesh_create: wall-face node out of range");
            return FELBM_ERR_INVALID_ARG;
        }
    for (int32_t f = 0; f < F; ++f)
        if (wid_in[f] < 0 || wid_in[f] >= FELBM_MAX_WALL_IDS) {
            set_error("felbm3d_mesh_create: wall id out of range");
            return FELBM_ERR_INVALID_ARG;
        }

    // ---- geometry in caller order: volume and shape gradients -------------
    // With edge rows r_k = x_k - x_0 (minimum image), det = r1.(r2 x r3) = 6V
    // and grad N_1 = r2 x r3 / det, grad N_2 = r3 x r1 / det,
    // grad N_3 = r1 x r2 / det, grad N_0 = -(grad N_1 + grad N_2 + grad N_3).
    std::vector<double> vol0(T), grad0(12 * (size_t)T);
    double total = 0.0, vmin = INFINITY;
    for (int32_t t = 0; t < T; ++t) {
        const int32_t* v = tet_in + 4 * (size_t)t;
        double r[3][3];
        for (int k = 0; k < 3; ++k)
            for (int d = 0; d < 3; ++d)
                r[k][d] = min_image3(xyz[3 * (size_t)v[k + 1] + d] - xyz[3 * (size_t)v[0] + d], m.period[d]);
        auto cross = [](const double* a, const double* b, double* o) {
            o[0] = a[1] * b[2] - a[2] * b[1];
            o[1] = a[2] * b[0] - a[0] * b[2];
            o[2] = a[0] * b[1] - a[1] * b[0];
        };
        double c23[3], c31[3], c12[3];
        cross(r[1], r[2], c23);
        cross(r[2], r[0], c31);
        cross(r[0], r[1], c12);
        double det = r[0][0] * c23[0] + r[0][1] * c23[1] + r[0][2] * c23[2];
        double scale = 0.0;
        for (int k = 0; k < 3; ++k)
            for (int d = 0; d < 3; ++d) scale = std::max(scale, std::fabs(r[k][d]));
        if (!(det > 1e-12 * scale * scale * scale)) {
            snprintf(buf, sizeof buf, "felbm3d_mesh_create: tetrahedron %d has non-positive volume", t);
            set_error(buf);
            return FELBM_ERR_BAD_MESH;
        }
        vol0[t] = det / 6.0;
        total += vol0[t];
        vmin = std::min(vmin, vol0[t]);
        for (int d = 0; d < 3; ++d) {
            double g1 = c23[d] / det, g2 = c31[d] / det, g3 = c12[d] / det;
            grad0[(size_t)t * 12 + 3 + d] = g1;
            grad0[(size_t)t * 12 + 6 + d] = g2;
            grad0[(size_t)t * 12 + 9 + d] = g3;
            grad0[(size_t)t * 12 + d] = -(g1 + g2 + g3);
        }
    }
    m.total_vol = total;
    m.min_vol = vmin;

    // ---- faces: neighbours and the boundary ---------------------------------
    std::vector<FaceRec> faces;
    faces.reserve(4 * (size_t)T);
    for (int32_t t = 0; t < T; ++t) {
        const int32_t* v = tet_in + 4 * (size_t)t;
        faces.push_back(face_of(v[1], v[2], v[3], t, 0));
        faces.push_back(face_of(v[0], v[2], v[3], t, 1));
        faces.push_back(face_of(v[0], v[1], v[3], t, 2));
        faces.push_back(face_of(v[0], v[1], v[2], t, 3));
    }
    std::sort(faces.begin(), faces.end());
    std::vector<int32_t> nbr0(4 * (size_t)T, -1);
    std::vector<FaceRec> boundary;
    for (size_t i = 0; i < faces.size();) {
        size_t j = i + 1;
        while (j < faces.size() && faces[j].same(faces[i])) ++j;
        if (j - i > 2) {
            set_error("felbm3d_mesh_create: a face is shared by more than two tetrahedra");
            return FELBM_ERR_BAD_MESH;
        }
        if (j - i == 2) {
            nbr0[4 * (size_t)faces[i].tet + faces[i].k] = faces[i + 1].tet;
            nbr0[4 * (size_t)faces[i + 1].tet + faces[i + 1].k] = faces[i].tet;
        } else {
            boundary.push_back(faces[i]);
        }
        i = j;
    }
    std::vector<FaceRec> walls;
    walls.reserve(F);
    for (int32_t f = 0; f < F; ++f) walls.push_back(face_of(wf_in[3 * f], wf_in[3 * f + 1], wf_in[3 * f + 2], f, 0));
    std::vector<FaceRec> walls_sorted = walls;
    std::sort(walls_sorted.begin(), walls_sorted.end());
    bool match = walls_sorted.size() == boundary.size();
    for (size_t i = 0; match && i < boundary.size(); ++i) match = walls_sorted[i].same(boundary[i]);
    for (size_t i = 0; match && i + 1 < walls_sorted.size(); ++i) match = !walls_sorted[i].same(walls_sorted[i + 1]);
    if (!match) {
        set_error("felbm3d_mesh_create: the boundary faces and the wall faces differ");
        return FELBM_ERR_BAD_MESH;
    }
    // owner (tetrahedron, local vertex opposite) of wall face f, caller order
    std::vector<int32_t> wall_owner(F), wall_k(F);
    for (size_t i = 0; i < boundary.size(); ++i) {
        int32_t f = walls_sorted[i].tet;   // caller index of the wall face
        wall_owner[f] = boundary[i].tet;
        wall_k[f] = boundary[i].k;
    }

    // ---- node order: reverse Cuthill-McKee on the edge graph --------------
    std::vector<std::vector<int32_t>> adjl(N);
    for (int32_t t = 0; t < T; ++t) {
        const int32_t* v = tet_in + 4 * (size_t)t;
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j)
                if (i != j) adjl[v[i]].push_back(v[j]);
    }
    std::vector<int32_t> adj_ptr(N + 1, 0), adj;
    for (int32_t i = 0; i < N; ++i) {
        auto& a = adjl[i];
        std::sort(a.begin(), a.end());
        a.erase(std::unique(a.begin(), a.end()), a.end());
        adj_ptr[i + 1] = adj_ptr[i] + (int32_t)a.size();
    }
    adj.reserve(adj_ptr[N]);
    for (int32_t i = 0; i < N; ++i) adj.insert(adj.end(), adjl[i].begin(), adjl[i].end());
    adjl.clear();
    adjl.shrink_to_fit();
    m.perm = rcm_order(N, adj_ptr, adj);
    m.iperm.assign(N, 0);
    for (int32_t i = 0; i < N; ++i) m.iperm[m.perm[i]] = i;
    m.x.resize(N);
    m.y.resize(N);
    m.z.resize(N);
    for (int32_t i = 0; i < N; ++i) {
        const double* p = xyz + 3 * (size_t)m.perm[i];
        m.x[i] = p[0];
        m.y[i] = p[1];
        m.z[i] = p[2];
    }

    // ---- tetrahedra sorted by their lowest (new) node -----------------------
    std::vector<int32_t> order(T), lowest(T);
    for (int32_t t = 0; t < T; ++t) {
        const int32_t* v = tet_in + 4 * (size_t)t;
        lowest[t] = std::min(std::min(m.iperm[v[0]], m.iperm[v[1]]), std::min(m.iperm[v[2]], m.iperm[v[3]]));
    }
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return lowest[a] < lowest[b]; });
    std::vector<int32_t> tnew(T);
    for (int32_t t = 0; t < T; ++t) tnew[order[t]] = t;
    m.tet.resize(4 * (size_t)T);
    m.vol.resize(T);
    m.grad.resize(12 * (size_t)T);
    m.nbr.resize(4 * (size_t)T);
    for (int32_t t = 0; t < T; ++t) {
        int32_t o = order[t];
        m.vol[t] = vol0[o];
        for (int k = 0; k < 4; ++k) {
            m.tet[(size_t)k * T + t] = m.iperm[tet_in[4 * (size_t)o + k]];
            int32_t nb = nbr0[4 * (size_t)o + k];
            m.nbr[(size_t)k * T + t] = nb < 0 ? -1 : tnew[nb];
        }
        for (int c = 0; c < 12; ++c) m.grad[(size_t)c * T + t] = grad0[(size_t)o * 12 + c];
    }

    // ---- node-node pattern with mass and stiffness --------------------------
    m.row_ptr.assign(N + 1, 0);
    for (int32_t i = 0; i < N; ++i) m.row_ptr[i + 1] = m.row_ptr[i] + (adj_ptr[m.perm[i] + 1] - adj_ptr[m.perm[i]]) + 1;
    const int32_t nnz = m.row_ptr[N];
    m.col.resize(nnz);
    m.max_degree = 0;
    m.bandwidth = 0;
    for (int32_t i = 0; i < N; ++i) {
        int32_t o = m.perm[i], at = m.row_ptr[i];
        m.col[at++] = i;
        for (int32_t k = adj_ptr[o]; k < adj_ptr[o + 1]; ++k) m.col[at++] = m.iperm[adj[k]];
        std::sort(m.col.begin() + m.row_ptr[i], m.col.begin() + m.row_ptr[i + 1]);
        m.max_degree = std::max(m.max_degree, m.row_ptr[i + 1] - m.row_ptr[i]);
        for (int32_t k = m.row_ptr[i]; k < m.row_ptr[i + 1]; ++k)
            m.bandwidth = std::max(m.bandwidth, std::abs(m.col[k] - i));
    }
    auto slot = [&](int32_t i, int32_t j) {
        auto b = m.col.begin() + m.row_ptr[i], e = m.col.begin() + m.row_ptr[i + 1];
        return (int32_t)(std::lower_bound(b, e, j) - m.col.begin());
    };
    m.mass.assign(nnz, 0.0);
    m.stiff.assign(nnz, 0.0);
    m.patch.assign(N, 0.0);
    for (int32_t t = 0; t < T; ++t) {
        const double V = m.vol[t];
        int32_t v[4];
        double g[4][3];
        for (int k = 0; k < 4; ++k) {
            v[k] = m.tet[(size_t)k * T + t];
            for (int d = 0; d < 3; ++d) g[k][d] = m.grad[(size_t)(3 * k + d) * T + t];
        }
        for (int i = 0; i < 4; ++i) {
            m.patch[v[i]] += V;
            for (int j = 0; j < 4; ++j) {
                int32_t s = slot(v[i], v[j]);
                m.mass[s] += V / 20.0 * (i == j ? 2.0 : 1.0);
                m.stiff[s] += V * (g[i][0] * g[j][0] + g[i][1] * g[j][1] + g[i][2] * g[j][2]);
            }
        }
    }
    m.lumped.assign(N, 0.0);
    for (int32_t i = 0; i < N; ++i)
        for (int32_t k = m.row_ptr[i]; k < m.row_ptr[i + 1]; ++k) m.lumped[i] += m.mass[k];

    // ---- node -> tetrahedron incidence --------------------------------------
    m.inc_ptr.assign(N + 1, 0);
    for (int32_t t = 0; t < T; ++t)
        for (int k = 0; k < 4; ++k) ++m.inc_ptr[m.tet[(size_t)k * T + t] + 1];
    for (int32_t i = 0; i < N; ++i) {
        m.max_inc = std::max(m.max_inc, m.inc_ptr[i + 1]);
        m.inc_ptr[i + 1] += m.inc_ptr[i];
    }
    const int32_t ninc = m.inc_ptr[N];
    m.inc_tet.resize(ninc);
    m.inc_b.resize(3 * (size_t)ninc);
    {
        std::vector<int32_t> fill(m.inc_ptr.begin(), m.inc_ptr.end() - 1);
        for (int32_t t = 0; t < T; ++t)          // ascending t: each node's list is sorted
            for (int k = 0; k < 4; ++k) {
                int32_t i = m.tet[(size_t)k * T + t], at = fill[i]++;
                m.inc_tet[at] = t;
                for (int d = 0; d < 3; ++d) m.inc_b[(size_t)d * ninc + at] = m.grad[(size_t)(3 * k + d) * T + t];
            }
    }

    // ---- wall faces: outward normal and area from the owner ----------------
    // The area-weighted outward normal of the face opposite vertex k is
    // -3 V grad N_k.
    m.wall_v.resize(3 * (size_t)F);
    m.wall_id.resize(F);
    m.wall_area.resize(F);
    m.wall_n.resize(3 * (size_t)F);
    for (int32_t f = 0; f < F; ++f) {
        int32_t t = wall_owner[f], k = wall_k[f];
        double nx = -3.0 * vol0[t] * grad0[(size_t)t * 12 + 3 * k];
        double ny = -3.0 * vol0[t] * grad0[(size_t)t * 12 + 3 * k + 1];
        double nz = -3.0 * vol0[t] * grad0[(size_t)t * 12 + 3 * k + 2];
        double A = std::sqrt(nx * nx + ny * ny + nz * nz);
        m.wall_area[f] = A;
        m.wall_n[f] = nx / A;
        m.wall_n[(size_t)F + f] = ny / A;
        m.wall_n[2 * (size_t)F + f] = nz / A;
        m.wall_id[f] = wid_in[f];
        for (int c = 0; c < 3; ++c) m.wall_v[(size_t)c * F + f] = m.iperm[wf_in[3 * (size_t)f + c]];
    }
    m.winc_ptr.assign(N + 1, 0);
    for (int32_t f = 0; f < F; ++f)
        for (int c = 0; c < 3; ++c) ++m.winc_ptr[m.wall_v[(size_t)c * F + f] + 1];
    for (int32_t i = 0; i < N; ++i) m.winc_ptr[i + 1] += m.winc_ptr[i];
    m.winc_face.resize(m.winc_ptr[N]);
    {
        std::vector<int32_t> fill(m.winc_ptr.begin(), m.winc_ptr.end() - 1);
        for (int32_t f = 0; f < F; ++f)
            for (int c = 0; c < 3; ++c) m.winc_face[fill[m.wall_v[(size_t)c * F + f]]++] = f;
    }
    return FELBM_OK;
}

}  // namespace felbm

extern "C" {

int felbm3d_mesh_create(const double* xyz, int32_t n_nodes, const int32_t* tet, int32_t n_tet,
                        const int32_t* wall_faces, const int32_t* wall_id, int32_t n_wall_faces,
                        const double* period, felbm3d_mesh** out) {
    if (!out || !xyz || !tet || n_nodes <= 0 || n_tet <= 0 || n_wall_faces < 0 ||
        (n_wall_faces > 0 && (!wall_faces || !wall_id))) {
        felbm::set_error("felbm3d_mesh_create: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    if (period)
        for (int d = 0; d < 3; ++d)
            if (!(period[d] >= 0.0)) {
                felbm::set_error("felbm3d_mesh_create: negative period");
                return FELBM_ERR_INVALID_ARG;
            }
    *out = nullptr;
    felbm3d_mesh* m = new (std::nothrow) felbm3d_mesh;
    if (!m) {
        felbm::set_error("felbm3d_mesh_create: out of host memory");
        return FELBM_ERR_INVALID_ARG;
    }
    int rc;
    try {
        rc = felbm::build_mesh3d(xyz, n_nodes, tet, n_tet, wall_faces, wall_id, n_wall_faces, period, m->h);
    } catch (const std::exception& ex) {
        felbm::set_error(std::string("felbm3d_mesh_create: ") + ex.what());
        rc = FELBM_ERR_INVALID_ARG;
    }
    if (rc != FELBM_OK) {
        delete m;
        return rc;
    }
    *out = m;
    return FELBM_OK;
}

int felbm3d_mesh_info_get(const felbm3d_mesh* mesh, felbm3d_mesh_info* out) {
    if (!mesh || !out) {
        felbm::set_error("felbm3d_mesh_info_get: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    const felbm::HostMesh3D& h = mesh->h;
    out->n_nodes = h.N;
    out->n_tet = h.T;
    out->n_wall_faces = h.F;
    out->nnz = h.row_ptr[h.N];
    out->max_degree = h.max_degree;
    out->bandwidth = h.bandwidth;
    out->max_incidence = h.max_inc;
    out->min_volume = h.min_vol;
    out->total_volume = h.total_vol;
    return FELBM_OK;
}

void felbm3d_mesh_destroy(felbm3d_mesh* mesh) { delete mesh; }

}  // extern "C"
