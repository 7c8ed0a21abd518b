// Host-side mesh preprocessing for the FE-LBM library: validation, element
// geometry of the linear triangles (Sec. II.C: P1 shape functions, constant
// gradients per element), edge neighbours and wall edges (Sec. II.D, walls
// of Sec. II.B), reverse Cuthill-McKee node order, and the node-centric
// tables every gather kernel reads (node-node pattern with the consistent
// mass and P1 stiffness entries, node -> triangle and node -> wall-edge
// incidence).  Runs once per mesh.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <climits>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <numeric>
#include <string>
#include <unordered_map>
#include <vector>

#include "felbm_internal.h"

namespace felbm {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

static double min_image(double d, double L) {
    if (L > 0.0) d -= L * std::round(d / L);
    return d;
}

// Reverse Cuthill-McKee order of the node graph; returns order[new] = old.
std::vector<int32_t> rcm_order(int32_t N, const std::vector<int32_t>& adj_ptr,
                                      const std::vector<int32_t>& adj) {
    std::vector<int32_t> order;
    order.reserve(N);
    std::vector<char> seen(N, 0);
    auto degree = [&](int32_t v) { return adj_ptr[v + 1] - adj_ptr[v]; };
    // BFS levels from a root restricted to unseen nodes; returns last level
    std::vector<int32_t> level(N, -1);
    auto bfs_last = [&](int32_t root, int32_t& depth) {
        std::vector<int32_t> touched{root};
        std::deque<int32_t> q{root};
        level[root] = 0;
        int32_t maxl = 0;
        while (!q.empty()) {
            int32_t v = q.front();
            q.pop_front();
            for (int32_t k = adj_ptr[v]; k < adj_ptr[v + 1]; ++k) {
                int32_t w = adj[k];
                if (seen[w] || level[w] >= 0) continue;
                level[w] = level[v] + 1;
                maxl = std::max(maxl, level[w]);
                touched.push_back(w);
                q.push_back(w);
            }
        }
        int32_t best = root;
        for (int32_t v : touched)
            if (level[v] == maxl && (best == root || degree(v) < degree(best))) best = v;
        for (int32_t v : touched) level[v] = -1;
        depth = maxl;
        return best;
    };
    std::vector<int32_t> by_degree(N);
    std::iota(by_degree.begin(), by_degree.end(), 0);
    std::stable_sort(by_degree.begin(), by_degree.end(),
                     [&](int32_t a, int32_t b) { return degree(a) < degree(b); });
    std::vector<int32_t> nb;
    for (int32_t s : by_degree) {
        if (seen[s]) continue;
        // pseudo-peripheral start: walk to the far end of the BFS tree while it deepens
        int32_t root = s, depth = 0, d2 = 0;
        int32_t far = bfs_last(root, depth);
        for (int it = 0; it < 4; ++it) {
            int32_t far2 = bfs_last(far, d2);
            if (d2 <= depth) break;
            root = far;
            far = far2;
            depth = d2;
        }
        root = far;
        std::deque<int32_t> q{root};
        seen[root] = 1;
        while (!q.empty()) {
            int32_t v = q.front();
            q.pop_front();
            order.push_back(v);
            nb.clear();
            for (int32_t k = adj_ptr[v]; k < adj_ptr[v + 1]; ++k)
                if (!seen[adj[k]]) nb.push_back(adj[k]);
            std::stable_sort(nb.begin(), nb.end(),
                             [&](int32_t a, int32_t b) { return degree(a) < degree(b); });
            for (int32_t w : nb) {
                seen[w] = 1;
                q.push_back(w);
            }
        }
    }
    std::reverse(order.begin(), order.end());
    return order;
}

// Cut the nodes nodes[lo, hi) into tiles of at most kTileNodes by recursive
// coordinate bisection: split at the median of the longer side of their
// bounding box, recurse into both halves in turn (so consecutive tiles are
// neighbours in space), and record the end of every tile in `ends`.
static void bisect_tiles(std::vector<int32_t>& nodes, int64_t lo, int64_t hi, const double* xy,
                         std::vector<int64_t>& ends) {
    if (hi - lo <= kTileNodes) {
        ends.push_back(hi);
        return;
    }
    double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300;
    for (int64_t k = lo; k < hi; ++k) {
        const double x = xy[2 * (size_t)nodes[k]], y = xy[2 * (size_t)nodes[k] + 1];
        x0 = std::min(x0, x);
        x1 = std::max(x1, x);
        y0 = std::min(y0, y);
        y1 = std::max(y1, y);
    }
    const int axis = (x1 - x0) >= (y1 - y0) ? 0 : 1;
    const int64_t mid = lo + (hi - lo) / 2;
    std::nth_element(nodes.begin() + lo, nodes.begin() + mid, nodes.begin() + hi, [&](int32_t a, int32_t b) {
        const double ca = xy[2 * (size_t)a + axis], cb = xy[2 * (size_t)b + axis];
        return ca < cb || (ca == cb && a < b);
    });
    bisect_tiles(nodes, lo, mid, xy, ends);
    bisect_tiles(nodes, mid, hi, xy, ends);
}

// node_px / node_py: periodic lengths of the sub-mesh each node belongs to
// (one value for a single mesh; per member mesh for a batch).
static int build_mesh(const double* xy, int32_t N, const int32_t* tri_in, int32_t T,
                      const int32_t* wall_edges, const int32_t* wall_id, int32_t E,
                      const std::vector<double>& node_px, const std::vector<double>& node_py, HostMesh& m) {
    char buf[256];
    m.N = N;
    m.T = T;
    m.E = E;
    for (int64_t i = 0; i < 3LL * T; ++i)
        if (tri_in[i] < 0 || tri_in[i] >= N) {
            set_error("felbm_mesh_create: triangle node id out of range");
            return FELBM_ERR_INVALID_ARG;
        }
    for (int32_t e = 0; e < E; ++e) {
        if (wall_edges[2 * e] < 0 || wall_edges[2 * e] >= N || wall_edges[2 * e + 1] < 0 ||
            wall_edges[2 * e + 1] >= N || wall_edges[2 * e] == wall_edges[2 * e + 1]) {
            set_error("felbm_mesh_create: wall edge node id out of range");
            return FELBM_ERR_INVALID_ARG;
        }
        if (wall_id[e] < 0 || wall_id[e] >= FELBM_MAX_WALL_IDS) {
            set_error("felbm_mesh_create: wall id outside [0, FELBM_MAX_WALL_IDS)");
            return FELBM_ERR_INVALID_ARG;
        }
    }
    for (int64_t i = 0; i < 2LL * N; ++i)
        if (!std::isfinite(xy[i])) {
            set_error("felbm_mesh_create: non-finite coordinate");
            return FELBM_ERR_INVALID_ARG;
        }

    // ---- element geometry in caller numbering ----------------------------
    std::vector<double> lx(3 * (size_t)T), ly(3 * (size_t)T), area(T);
    m.min_area = 1e300;
    m.total_area = 0.0;
    for (int32_t t = 0; t < T; ++t) {
        const int32_t* v = tri_in + 3 * (size_t)t;
        lx[3 * t] = 0.0;
        ly[3 * t] = 0.0;
        const double px = node_px[v[0]], py = node_py[v[0]];
        for (int k = 1; k < 3; ++k) {
            if (node_px[v[k]] != px || node_py[v[k]] != py) {
                set_error("felbm_mesh_create_batch: triangle joins two member meshes");
                return FELBM_ERR_BAD_MESH;
            }
            lx[3 * t + k] = min_image(xy[2 * v[k]] - xy[2 * v[0]], px);
            ly[3 * t + k] = min_image(xy[2 * v[k] + 1] - xy[2 * v[0] + 1], py);
        }
        double a = 0.5 * (lx[3 * t + 1] * ly[3 * t + 2] - ly[3 * t + 1] * lx[3 * t + 2]);
        if (!(a > 0.0)) {
            snprintf(buf, sizeof buf,
                     "felbm_mesh_create: triangle %d has non-positive area %.3e (clockwise or degenerate)",
                     t, a);
            set_error(buf);
            return FELBM_ERR_BAD_MESH;
        }
        area[t] = a;
        m.min_area = std::min(m.min_area, a);
        m.total_area += a;
    }

    // ---- edges: neighbours across each edge, open edges must be walls ----
    std::vector<int32_t> nbr_old(3 * (size_t)T, -1), slot_old(3 * (size_t)T, -1);
    std::unordered_map<uint64_t, int64_t> open;
    open.reserve((size_t)T * 2);
    auto key = [](int32_t a, int32_t b) {
        uint32_t lo = (uint32_t)std::min(a, b), hi = (uint32_t)std::max(a, b);
        return ((uint64_t)lo << 32) | hi;
    };
    for (int32_t t = 0; t < T; ++t)
        for (int k = 0; k < 3; ++k) {
            int32_t a = tri_in[3 * t + (k + 1) % 3], b = tri_in[3 * t + (k + 2) % 3];
            if (a == b) {
                set_error("felbm_mesh_create: triangle with a repeated node");
                return FELBM_ERR_BAD_MESH;
            }
            uint64_t kk = key(a, b);
            auto it = open.find(kk);
            if (it == open.end()) {
                open.emplace(kk, 3LL * t + k);
            } else {
                int64_t o = it->second;
                if (o < 0) {
                    set_error("felbm_mesh_create: edge shared by more than two triangles");
                    return FELBM_ERR_BAD_MESH;
                }
                nbr_old[3 * t + k] = (int32_t)(o / 3);
                slot_old[3 * t + k] = (int32_t)(o % 3);
                nbr_old[o] = t;
                slot_old[o] = k;
                it->second = -1;  // closed
            }
        }
    std::unordered_map<uint64_t, int32_t> walls;
    walls.reserve((size_t)E * 2 + 1);
    for (int32_t e = 0; e < E; ++e) {
        if (!walls.emplace(key(wall_edges[2 * e], wall_edges[2 * e + 1]), e).second) {
            set_error("felbm_mesh_create: duplicate wall edge");
            return FELBM_ERR_BAD_MESH;
        }
    }
    std::vector<int64_t> wall_owner(E, -1);
    for (auto& kv : open) {
        if (kv.second < 0) continue;
        auto it = walls.find(kv.first);
        if (it == walls.end()) {
            set_error("felbm_mesh_create: boundary edge that is not a wall edge");
            return FELBM_ERR_BAD_MESH;
        }
        wall_owner[it->second] = kv.second;
    }
    for (int32_t e = 0; e < E; ++e)
        if (wall_owner[e] < 0) {
            set_error("felbm_mesh_create: wall edge that is not a boundary edge");
            return FELBM_ERR_BAD_MESH;
        }

    // ---- node graph and reverse Cuthill-McKee ----------------------------
    std::vector<int32_t> ip0(N + 1, 0);
    for (int64_t i = 0; i < 3LL * T; ++i) ip0[tri_in[i] + 1]++;
    for (int32_t i = 0; i < N; ++i) ip0[i + 1] += ip0[i];
    std::vector<int32_t> it0(ip0[N]);
    {
        std::vector<int32_t> fill(ip0.begin(), ip0.end() - 1);
        for (int32_t t = 0; t < T; ++t)
            for (int k = 0; k < 3; ++k) it0[fill[tri_in[3 * t + k]]++] = t;
    }
    for (int32_t i = 0; i < N; ++i)
        if (ip0[i + 1] == ip0[i]) {
            set_error("felbm_mesh_create: node used by no triangle");
            return FELBM_ERR_BAD_MESH;
        }
    std::vector<int32_t> adj_ptr(N + 1, 0), adj;
    adj.reserve((size_t)N * 8);
    {
        std::vector<int32_t> row;
        for (int32_t i = 0; i < N; ++i) {
            row.clear();
            for (int32_t k = ip0[i]; k < ip0[i + 1]; ++k)
                for (int j = 0; j < 3; ++j) {
                    int32_t v = tri_in[3 * it0[k] + j];
                    if (v != i) row.push_back(v);
                }
            std::sort(row.begin(), row.end());
            row.erase(std::unique(row.begin(), row.end()), row.end());
            adj.insert(adj.end(), row.begin(), row.end());
            adj_ptr[i + 1] = (int32_t)adj.size();
        }
    }
    m.perm = rcm_order(N, adj_ptr, adj);
    // Several components (a batch): reverse Cuthill-McKee emits each one as a
    // run; order the runs by size, largest first, keeping each run's order,
    // so that the large members form a prefix of the node and triangle
    // ranges (the tiled kernels of a hybrid batch schedule cover the prefix).
    {
        std::vector<int32_t> comp_of(N, -1), csize;
        for (int32_t s0 = 0; s0 < N; ++s0) {
            if (comp_of[s0] >= 0) continue;
            int32_t id = (int32_t)csize.size();
            csize.push_back(0);
            std::deque<int32_t> q{s0};
            comp_of[s0] = id;
            while (!q.empty()) {
                int32_t v = q.front();
                q.pop_front();
                csize[id]++;
                for (int32_t k = adj_ptr[v]; k < adj_ptr[v + 1]; ++k)
                    if (comp_of[adj[k]] < 0) {
                        comp_of[adj[k]] = id;
                        q.push_back(adj[k]);
                    }
            }
        }
        if (csize.size() > 1)
            std::stable_sort(m.perm.begin(), m.perm.end(), [&](int32_t a, int32_t b) {
                return csize[comp_of[a]] > csize[comp_of[b]];
            });
        // Node tiles within each component's run.  Recursive coordinate
        // bisection makes compact tiles, the nodes of a tile keep their
        // reverse Cuthill-McKee order; FELBM_ORDER=rcm keeps the plain
        // reverse Cuthill-McKee order and cuts it into runs of kTileNodes.
        const char* env = std::getenv("FELBM_ORDER");
        const bool plain_rcm = env && std::string(env) == "rcm";
        std::vector<int32_t> rank(N);
        for (int32_t n = 0; n < N; ++n) rank[m.perm[n]] = n;
        m.tile_ptr.assign(1, 0);
        std::vector<int64_t> ends;
        for (int64_t a = 0; a < N;) {
            int64_t b = a;
            while (b < N && comp_of[m.perm[b]] == comp_of[m.perm[a]]) ++b;
            ends.clear();
            if (plain_rcm) {
                for (int64_t e = a + kTileNodes; e < b; e += kTileNodes) ends.push_back(e);
                ends.push_back(b);
            } else {
                bisect_tiles(m.perm, a, b, xy, ends);
                int64_t s0 = a;
                for (int64_t e : ends) {
                    std::sort(m.perm.begin() + s0, m.perm.begin() + e,
                              [&](int32_t u, int32_t v) { return rank[u] < rank[v]; });
                    s0 = e;
                }
            }
            for (int64_t e : ends) m.tile_ptr.push_back((int32_t)e);
            a = b;
        }
    }
    m.iperm.assign(N, 0);
    for (int32_t n = 0; n < N; ++n) m.iperm[m.perm[n]] = n;

    m.x.resize(N);
    m.y.resize(N);
    for (int32_t n = 0; n < N; ++n) {
        m.x[n] = xy[2 * m.perm[n]];
        m.y[n] = xy[2 * m.perm[n] + 1];
    }

    // ---- triangles in the new numbering, ordered by their lowest node ----
    std::vector<int32_t> torder(T);
    std::iota(torder.begin(), torder.end(), 0);
    std::vector<int32_t> tmin(T);
    for (int32_t t = 0; t < T; ++t)
        tmin[t] = std::min({m.iperm[tri_in[3 * t]], m.iperm[tri_in[3 * t + 1]], m.iperm[tri_in[3 * t + 2]]});
    std::stable_sort(torder.begin(), torder.end(), [&](int32_t a, int32_t b) { return tmin[a] < tmin[b]; });
    std::vector<int32_t> tnew(T);
    for (int32_t t = 0; t < T; ++t) tnew[torder[t]] = t;
    m.tri.assign(3 * (size_t)T, 0);
    m.area.assign(T, 0.0);
    m.grad.assign(6 * (size_t)T, 0.0);
    m.nbr.assign(3 * (size_t)T, -1);
    m.nbr_slot.assign(3 * (size_t)T, -1);
    for (int32_t t = 0; t < T; ++t) {
        int32_t o = torder[t];
        double A = area[o];
        m.area[t] = A;
        for (int k = 0; k < 3; ++k) {
            m.tri[(size_t)k * T + t] = m.iperm[tri_in[3 * o + k]];
            int32_t nb = nbr_old[3 * o + k];
            m.nbr[(size_t)k * T + t] = nb < 0 ? -1 : tnew[nb];
            m.nbr_slot[(size_t)k * T + t] = slot_old[3 * o + k];
            // gradient of the P1 shape function of local vertex k
            int j = (k + 1) % 3, l = (k + 2) % 3;
            m.grad[(size_t)(2 * k) * T + t] = (ly[3 * o + j] - ly[3 * o + l]) / (2.0 * A);
            m.grad[(size_t)(2 * k + 1) * T + t] = (lx[3 * o + l] - lx[3 * o + j]) / (2.0 * A);
        }
    }

    // ---- node -> triangle incidence in the new numbering ----------------
    m.inc_ptr.assign(N + 1, 0);
    for (int64_t i = 0; i < 3LL * T; ++i) m.inc_ptr[m.tri[i] + 1]++;
    for (int32_t i = 0; i < N; ++i) m.inc_ptr[i + 1] += m.inc_ptr[i];
    size_t ninc = m.inc_ptr[N];
    m.inc_tri.assign(ninc, 0);
    m.inc_bx.assign(ninc, 0.0);
    m.inc_by.assign(ninc, 0.0);
    std::vector<int8_t> inc_loc(ninc, 0);
    {
        std::vector<int32_t> fill(m.inc_ptr.begin(), m.inc_ptr.end() - 1);
        for (int32_t t = 0; t < T; ++t)
            for (int k = 0; k < 3; ++k) {
                int32_t v = m.tri[(size_t)k * T + t];
                int32_t p = fill[v]++;
                m.inc_tri[p] = t;
                inc_loc[p] = (int8_t)k;
                m.inc_bx[p] = m.grad[(size_t)(2 * k) * T + t];
                m.inc_by[p] = m.grad[(size_t)(2 * k + 1) * T + t];
            }
    }

    // ---- node-node pattern with consistent mass and stiffness -----------
    m.row_ptr.assign(N + 1, 0);
    m.col.clear();
    m.mass.clear();
    m.stiff.clear();
    m.col.reserve((size_t)N * 8);
    m.lumped.assign(N, 0.0);
    m.patch.assign(N, 0.0);
    m.max_degree = 0;
    m.bandwidth = 0;
    {
        std::vector<int32_t> row;
        std::vector<double> rm, rk;
        for (int32_t i = 0; i < N; ++i) {
            row.clear();
            for (int32_t p = m.inc_ptr[i]; p < m.inc_ptr[i + 1]; ++p)
                for (int j = 0; j < 3; ++j) row.push_back(m.tri[(size_t)j * T + m.inc_tri[p]]);
            std::sort(row.begin(), row.end());
            row.erase(std::unique(row.begin(), row.end()), row.end());
            rm.assign(row.size(), 0.0);
            rk.assign(row.size(), 0.0);
            for (int32_t p = m.inc_ptr[i]; p < m.inc_ptr[i + 1]; ++p) {
                int32_t t = m.inc_tri[p];
                int li = inc_loc[p];
                double A = m.area[t];
                m.patch[i] += A;
                double bix = m.grad[(size_t)(2 * li) * T + t], biy = m.grad[(size_t)(2 * li + 1) * T + t];
                for (int j = 0; j < 3; ++j) {
                    int32_t c = m.tri[(size_t)j * T + t];
                    size_t pos = std::lower_bound(row.begin(), row.end(), c) - row.begin();
                    rm[pos] += A / 12.0 * (j == li ? 2.0 : 1.0);
                    rk[pos] += A * (bix * m.grad[(size_t)(2 * j) * T + t] + biy * m.grad[(size_t)(2 * j + 1) * T + t]);
                }
            }
            double rs = 0.0;
            for (size_t q = 0; q < row.size(); ++q) {
                rs += rm[q];
                m.bandwidth = std::max(m.bandwidth, std::abs(row[q] - i));
            }
            m.lumped[i] = rs;
            m.col.insert(m.col.end(), row.begin(), row.end());
            m.mass.insert(m.mass.end(), rm.begin(), rm.end());
            m.stiff.insert(m.stiff.end(), rk.begin(), rk.end());
            m.row_ptr[i + 1] = (int32_t)m.col.size();
            m.max_degree = std::max(m.max_degree, (int32_t)row.size());
        }
    }

    // ---- halo of every node tile ---------------------------------------
    {
        const int32_t ntile = (int32_t)m.tile_ptr.size() - 1;
        m.halo_ptr.assign(ntile + 1, 0);
        m.halo.clear();
        m.max_halo = 0;
        std::vector<int32_t> h;
        for (int32_t k = 0; k < ntile; ++k) {
            const int32_t s0 = m.tile_ptr[k], s1 = m.tile_ptr[k + 1];
            h.clear();
            for (int32_t i = s0; i < s1; ++i)
                for (int32_t p = m.row_ptr[i]; p < m.row_ptr[i + 1]; ++p)
                    if (m.col[p] < s0 || m.col[p] >= s1) h.push_back(m.col[p]);
            std::sort(h.begin(), h.end());
            h.erase(std::unique(h.begin(), h.end()), h.end());
            m.halo.insert(m.halo.end(), h.begin(), h.end());
            m.halo_ptr[k + 1] = (int32_t)m.halo.size();
            m.max_halo = std::max(m.max_halo, (int32_t)h.size());
        }
    }

    // ---- wall edges: new ids, length and unit normal out of the fluid ----
    m.wall_a.assign(E, 0);
    m.wall_b.assign(E, 0);
    m.wall_id.assign(E, 0);
    m.wall_len.assign(E, 0.0);
    m.wall_nx.assign(E, 0.0);
    m.wall_ny.assign(E, 0.0);
    for (int32_t e = 0; e < E; ++e) {
        int64_t o = wall_owner[e];
        int32_t t = (int32_t)(o / 3);
        int k = (int)(o % 3);
        int j = (k + 1) % 3, l = (k + 2) % 3;
        double tx = lx[3 * t + l] - lx[3 * t + j], ty = ly[3 * t + l] - ly[3 * t + j];
        double L = std::sqrt(tx * tx + ty * ty);
        m.wall_a[e] = m.iperm[tri_in[3 * t + j]];
        m.wall_b[e] = m.iperm[tri_in[3 * t + l]];
        m.wall_id[e] = wall_id[e];
        m.wall_len[e] = L;
        m.wall_nx[e] = ty / L;   // counter-clockwise triangle: (t_y, -t_x) points out of it
        m.wall_ny[e] = -tx / L;
    }
    m.winc_ptr.assign(N + 1, 0);
    for (int32_t e = 0; e < E; ++e) {
        m.winc_ptr[m.wall_a[e] + 1]++;
        m.winc_ptr[m.wall_b[e] + 1]++;
    }
    for (int32_t i = 0; i < N; ++i) m.winc_ptr[i + 1] += m.winc_ptr[i];
    m.winc_edge.assign(m.winc_ptr[N], 0);
    {
        std::vector<int32_t> fill(m.winc_ptr.begin(), m.winc_ptr.end() - 1);
        for (int32_t e = 0; e < E; ++e) {
            m.winc_edge[fill[m.wall_a[e]]++] = e;
            m.winc_edge[fill[m.wall_b[e]]++] = e;
        }
    }

    // ---- connected components (groups) -----------------------------------
    // Reverse Cuthill-McKee emits each component as one run of internal ids,
    // and triangles are sorted by their lowest node, so a group is a node
    // range and a triangle range.
    std::vector<int32_t> comp(N, -1);
    std::vector<int32_t> runs;   // first internal node of each run
    for (int32_t n = 0; n < N; ++n) {
        if (comp[n] >= 0) continue;
        int32_t id = (int32_t)runs.size();
        runs.push_back(n);
        std::deque<int32_t> q{n};
        comp[n] = id;
        while (!q.empty()) {
            int32_t v = q.front();
            q.pop_front();
            for (int32_t k = m.row_ptr[v]; k < m.row_ptr[v + 1]; ++k) {
                int32_t w = m.col[k];
                if (comp[w] < 0) {
                    comp[w] = id;
                    q.push_back(w);
                }
            }
        }
    }
    const int32_t G = (int32_t)runs.size();
    std::vector<int32_t> cbeg(G, N), cend(G, 0), cmin(G, INT32_MAX), ccount(G, 0);
    for (int32_t n = 0; n < N; ++n) {
        int32_t c = comp[n];
        cbeg[c] = std::min(cbeg[c], n);
        cend[c] = std::max(cend[c], n + 1);
        cmin[c] = std::min(cmin[c], m.perm[n]);
        ccount[c]++;
    }
    for (int32_t c = 0; c < G; ++c)
        if (cend[c] - cbeg[c] != ccount[c]) {
            set_error("felbm_mesh_create: internal error, component not contiguous");
            return FELBM_ERR_BAD_MESH;
        }
    std::vector<int32_t> order(G);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return cmin[a] < cmin[b]; });
    std::vector<int32_t> gid(G);
    for (int32_t g = 0; g < G; ++g) gid[order[g]] = g;
    m.G = G;
    m.grp_node_begin.assign(G, 0);
    m.grp_node_end.assign(G, 0);
    m.grp_tri_begin.assign(G, T);
    m.grp_tri_end.assign(G, 0);
    m.grp_first_caller.assign(G, 0);
    m.grp_size.assign(G, 0);
    m.grp_period_x.assign(G, 0.0);
    m.grp_period_y.assign(G, 0.0);
    for (int32_t c = 0; c < G; ++c) {
        int32_t g = gid[c];
        m.grp_node_begin[g] = cbeg[c];
        m.grp_node_end[g] = cend[c];
        m.grp_first_caller[g] = cmin[c];
        m.grp_size[g] = cend[c] - cbeg[c];
        m.grp_period_x[g] = node_px[cmin[c]];
        m.grp_period_y[g] = node_py[cmin[c]];
    }
    for (int32_t t = 0; t < T; ++t) {
        int32_t g = gid[comp[m.tri[t]]];
        m.grp_tri_begin[g] = std::min(m.grp_tri_begin[g], t);
        m.grp_tri_end[g] = std::max(m.grp_tri_end[g], t + 1);
    }
    for (int32_t g = 0; g < G; ++g)
        if (m.grp_tri_begin[g] > m.grp_tri_end[g]) m.grp_tri_begin[g] = m.grp_tri_end[g] = 0;
    m.grp_wall_ptr.assign(G + 1, 0);
    for (int32_t e = 0; e < E; ++e) m.grp_wall_ptr[gid[comp[m.wall_a[e]]] + 1]++;
    for (int32_t g = 0; g < G; ++g) m.grp_wall_ptr[g + 1] += m.grp_wall_ptr[g];
    m.grp_wall_edge.assign(E, 0);
    {
        std::vector<int32_t> fill(m.grp_wall_ptr.begin(), m.grp_wall_ptr.end() - 1);
        for (int32_t e = 0; e < E; ++e) m.grp_wall_edge[fill[gid[comp[m.wall_a[e]]]]++] = e;
    }
    return FELBM_OK;
}

}  // namespace felbm

extern "C" {

const char* felbm_last_error(void) { return felbm::g_last_error.c_str(); }

int felbm_params_derive(double sigma, double xi, const double* theta_deg, int32_t n_wall_ids,
                        felbm_params* p) {
    if (!p || !(sigma > 0.0) || !(xi > 0.0) || n_wall_ids < 0 || n_wall_ids > FELBM_MAX_WALL_IDS ||
        (n_wall_ids > 0 && !theta_deg)) {
        felbm::set_error("felbm_params_derive: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    // kappa * beta = 18 sigma^2 and kappa / beta = xi^2 / 8
    p->kappa = 1.5 * sigma * xi;
    p->beta = 12.0 * sigma / xi;
    double root = std::sqrt(2.0 * p->kappa * p->beta);  // = 6 sigma
    for (int i = 0; i < FELBM_MAX_WALL_IDS; ++i) p->phi_c[i] = 0.0;
    for (int i = 0; i < n_wall_ids; ++i) p->phi_c[i] = -root * std::cos(theta_deg[i] * M_PI / 180.0);
    p->n_wall_ids = n_wall_ids;
    return FELBM_OK;
}

int felbm_mesh_create(const double* xy, int32_t n_nodes, const int32_t* tri, int32_t n_tri,
                      const int32_t* wall_edges, const int32_t* wall_id, int32_t n_wall_edges,
                      double period_x, double period_y, felbm_mesh** out) {
    if (!out || !xy || !tri || n_nodes <= 0 || n_tri <= 0 || n_wall_edges < 0 ||
        (n_wall_edges > 0 && (!wall_edges || !wall_id)) || period_x < 0.0 || period_y < 0.0) {
        felbm::set_error("felbm_mesh_create: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    *out = nullptr;
    felbm_mesh* m = new (std::nothrow) felbm_mesh;
    if (!m) {
        felbm::set_error("felbm_mesh_create: out of host memory");
        return FELBM_ERR_INVALID_ARG;
    }
    int rc;
    try {
        std::vector<double> npx(n_nodes, period_x), npy(n_nodes, period_y);
        m->h.period[0] = period_x;
        m->h.period[1] = period_y;
        rc = felbm::build_mesh(xy, n_nodes, tri, n_tri, wall_edges, wall_id, n_wall_edges, npx, npy, m->h);
    } catch (const std::exception& ex) {
        felbm::set_error(std::string("felbm_mesh_create: ") + ex.what());
        rc = FELBM_ERR_INVALID_ARG;
    }
    if (rc != FELBM_OK) {
        delete m;
        return rc;
    }
    *out = m;
    return FELBM_OK;
}

int felbm_mesh_create_batch(int32_t n_meshes, const felbm_mesh_desc* meshes, felbm_mesh** out) {
    if (!out || !meshes || n_meshes < 1) {
        felbm::set_error("felbm_mesh_create_batch: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    *out = nullptr;
    int64_t N = 0, T = 0, E = 0;
    for (int32_t k = 0; k < n_meshes; ++k) {
        const felbm_mesh_desc& d = meshes[k];
        if (!d.xy || !d.tri || d.n_nodes <= 0 || d.n_tri <= 0 || d.n_wall_edges < 0 ||
            (d.n_wall_edges > 0 && (!d.wall_edges || !d.wall_id)) || d.period_x < 0.0 || d.period_y < 0.0) {
            felbm::set_error("felbm_mesh_create_batch: invalid member mesh");
            return FELBM_ERR_INVALID_ARG;
        }
        N += d.n_nodes;
        T += d.n_tri;
        E += d.n_wall_edges;
    }
    if (N > INT32_MAX || 3 * T > INT32_MAX) {
        felbm::set_error("felbm_mesh_create_batch: batch too large for 32-bit indices");
        return FELBM_ERR_INVALID_ARG;
    }
    std::vector<double> xy(2 * N), npx(N), npy(N);
    std::vector<int32_t> tri(3 * T), we(2 * E), wid(E);
    int64_t n0 = 0, t0 = 0, e0 = 0;
    for (int32_t k = 0; k < n_meshes; ++k) {
        const felbm_mesh_desc& d = meshes[k];
        std::copy(d.xy, d.xy + 2 * (size_t)d.n_nodes, xy.begin() + 2 * n0);
        std::fill(npx.begin() + n0, npx.begin() + n0 + d.n_nodes, d.period_x);
        std::fill(npy.begin() + n0, npy.begin() + n0 + d.n_nodes, d.period_y);
        for (int64_t i = 0; i < 3LL * d.n_tri; ++i) {
            if (d.tri[i] < 0 || d.tri[i] >= d.n_nodes) {
                felbm::set_error("felbm_mesh_create_batch: triangle node id out of range");
                return FELBM_ERR_INVALID_ARG;
            }
            tri[3 * t0 + i] = (int32_t)(d.tri[i] + n0);
        }
        for (int64_t i = 0; i < 2LL * d.n_wall_edges; ++i) {
            if (d.wall_edges[i] < 0 || d.wall_edges[i] >= d.n_nodes) {
                felbm::set_error("felbm_mesh_create_batch: wall edge node id out of range");
                return FELBM_ERR_INVALID_ARG;
            }
            we[2 * e0 + i] = (int32_t)(d.wall_edges[i] + n0);
        }
        std::copy(d.wall_id, d.wall_id + d.n_wall_edges, wid.begin() + e0);
        n0 += d.n_nodes;
        t0 += d.n_tri;
        e0 += d.n_wall_edges;
    }
    felbm_mesh* m = new (std::nothrow) felbm_mesh;
    if (!m) {
        felbm::set_error("felbm_mesh_create_batch: out of host memory");
        return FELBM_ERR_INVALID_ARG;
    }
    int rc;
    try {
        rc = felbm::build_mesh(xy.data(), (int32_t)N, tri.data(), (int32_t)T, E ? we.data() : nullptr,
                               E ? wid.data() : nullptr, (int32_t)E, npx, npy, m->h);
    } catch (const std::exception& ex) {
        felbm::set_error(std::string("felbm_mesh_create_batch: ") + ex.what());
        rc = FELBM_ERR_INVALID_ARG;
    }
    if (rc != FELBM_OK) {
        delete m;
        return rc;
    }
    *out = m;
    return FELBM_OK;
}

int felbm_mesh_info_get(const felbm_mesh* mesh, felbm_mesh_info* out) {
    if (!mesh || !out) {
        felbm::set_error("felbm_mesh_info_get: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    const felbm::HostMesh& m = mesh->h;
    out->n_nodes = m.N;
    out->n_tri = m.T;
    out->n_wall_edges = m.E;
    out->n_groups = m.G;
    out->nnz = m.row_ptr.empty() ? 0 : m.row_ptr[m.N];
    out->max_degree = m.max_degree;
    out->bandwidth = m.bandwidth;
    out->min_area = m.min_area;
    out->total_area = m.total_area;
    out->n_tiles = m.tile_ptr.empty() ? 0 : (int32_t)m.tile_ptr.size() - 1;
    out->max_tile_halo = m.max_halo;
    return FELBM_OK;
}

int felbm_mesh_groups(const felbm_mesh* mesh, int32_t* group_first_node, int32_t* group_nodes) {
    if (!mesh) {
        felbm::set_error("felbm_mesh_groups: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    const felbm::HostMesh& m = mesh->h;
    for (int32_t g = 0; g < m.G; ++g) {
        if (group_first_node) group_first_node[g] = m.grp_first_caller[g];
        if (group_nodes) group_nodes[g] = m.grp_size[g];
    }
    return FELBM_OK;
}

void felbm_mesh_destroy(felbm_mesh* mesh) { delete mesh; }

}  // extern "C"
