// Internal host-side structures of the 3D FE-LBM library (not part of the ABI).
#pragma once

#include <cstdint>
#include <vector>

#include "felbm3d.h"
#include "felbm_internal.h"

namespace felbm {

// Tetrahedral mesh after preprocessing.  Node ids are internal (reverse
// Cuthill-McKee) ids; perm[new] = caller id, iperm[caller] = new.
// Tetrahedra are sorted by their lowest node.
struct HostMesh3D {
    int32_t N = 0, T = 0, F = 0;
    double period[3] = {0.0, 0.0, 0.0};
    std::vector<int32_t> perm, iperm;
    std::vector<double> x, y, z;              // node coordinates, internal order
    std::vector<int32_t> tet;                 // [4][T]: vertex k of tetrahedron t at tet[k*T + t]
    std::vector<double> vol;                  // [T]
    std::vector<double> grad;                 // [12][T]: component d of grad N_k at grad[(3k+d)*T + t]
    std::vector<int32_t> nbr;                 // [4][T]: tetrahedron across the face opposite vertex k, -1 = wall
    // node-node pattern (CSR, sorted columns, diagonal included)
    std::vector<int32_t> row_ptr, col;
    std::vector<double> mass;                 // consistent mass entries sum_T V/20 (1 + d_ij)
    std::vector<double> stiff;                // P1 stiffness entries sum_T V b_i.b_j
    std::vector<double> lumped;               // row sums of the mass matrix (|patch| / 4)
    std::vector<double> patch;                // volume of the vertex patch
    // node -> incident tetrahedra (CSR) with the node's shape gradient there
    std::vector<int32_t> inc_ptr, inc_tet;
    std::vector<double> inc_b;                // [3][ninc]
    // wall faces: nodes, id, area, unit normal out of the fluid
    std::vector<int32_t> wall_v;              // [3][F]
    std::vector<int32_t> wall_id;
    std::vector<double> wall_area;
    std::vector<double> wall_n;               // [3][F]
    std::vector<int32_t> winc_ptr, winc_face; // node -> incident wall faces (CSR)
    double min_vol = 0.0, total_vol = 0.0;
    int32_t max_degree = 0, bandwidth = 0, max_inc = 0;
};

}  // namespace felbm

struct felbm3d_mesh {
    felbm::HostMesh3D h;
};
