// Internal host-side structures of the FE-LBM library (not part of the ABI).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "felbm.h"

namespace felbm {

void set_error(const std::string& msg);

// Reverse Cuthill-McKee order of a node graph given as CSR adjacency
// (no self loops); returns order[new] = old.  Components one after another.
std::vector<int32_t> rcm_order(int32_t N, const std::vector<int32_t>& adj_ptr,
                               const std::vector<int32_t>& adj);

// Most nodes in one tile of the tiled solve step (see HostMesh::tile_ptr).
constexpr int32_t kTileNodes = 1024;

// Host mesh after preprocessing.  Node ids are the internal ids (node tiles
// of recursive coordinate bisection, reverse Cuthill-McKee order inside a
// tile); perm[new] = caller id, iperm[caller] = new.
struct HostMesh {
    int32_t N = 0, T = 0, E = 0;
    double period[2] = {0.0, 0.0};
    std::vector<int32_t> perm, iperm;
    std::vector<double> x, y;                 // node coordinates, internal order
    // triangles, structure of arrays: vertex k of triangle t at tri[k*T + t]
    std::vector<int32_t> tri;                 // [3][T]
    std::vector<double> area;                 // [T]
    std::vector<double> grad;                 // [6][T]: bx0, by0, bx1, by1, bx2, by2
    std::vector<int32_t> nbr;                 // [3][T]: triangle across the edge opposite vertex k, -1 = wall
    std::vector<int32_t> nbr_slot;            // [3][T]: that edge's local index in the neighbour
    // node-node pattern (CSR, sorted columns, diagonal included)
    std::vector<int32_t> row_ptr, col;
    std::vector<double> mass;                 // consistent mass matrix entries
    std::vector<double> stiff;                // P1 stiffness entries sum_T A_T b_i.b_j
    std::vector<double> lumped;               // row sums of the mass matrix
    std::vector<double> patch;                // area of the vertex patch
    // node -> incident triangles (CSR) with the node's shape gradient there
    std::vector<int32_t> inc_ptr, inc_tri;
    std::vector<double> inc_bx, inc_by;
    // wall edges: end nodes, id, length, unit normal out of the fluid
    std::vector<int32_t> wall_a, wall_b, wall_id;
    std::vector<double> wall_len, wall_nx, wall_ny;
    // node -> incident wall edges (CSR)
    std::vector<int32_t> winc_ptr, winc_edge;
    double min_area = 0.0, total_area = 0.0;
    int32_t max_degree = 0, bandwidth = 0;
    // node tiles: tile k holds the internal nodes [tile_ptr[k], tile_ptr[k+1]),
    // at most kTileNodes, all in one component; its halo is the sorted list
    // of nodes outside it that share a matrix row entry with one inside
    std::vector<int32_t> tile_ptr;
    std::vector<int32_t> halo_ptr, halo;
    int32_t max_halo = 0;
    // connected components ("groups"), numbered by their lowest caller node
    // id; each occupies a contiguous range of internal nodes and triangles
    int32_t G = 0;
    std::vector<int32_t> grp_node_begin, grp_node_end, grp_tri_begin, grp_tri_end;
    std::vector<int32_t> grp_wall_ptr, grp_wall_edge;   // wall edges of each group (CSR)
    std::vector<int32_t> grp_first_caller, grp_size;
    std::vector<double> grp_period_x, grp_period_y;      // periodic lengths of each group
};

}  // namespace felbm

struct felbm_mesh {
    felbm::HostMesh h;
};
