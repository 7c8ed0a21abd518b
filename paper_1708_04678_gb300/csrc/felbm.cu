// CUDA implementation of the FE-LBM contact-line step for sm_103a (GB300).
//
// Data layout in HBM (all carved from the caller's workspace):
//  * distributions psi: double [18][Np] -- g_0..g_8 then h_0..h_8, direction
//    major, node stride Np = N rounded up to 64 (coalesced node streams);
//  * nodal fields C, p, ux, uy, mu: double [Np];
//  * triangle tables: vertices int [3][Tp], area [Tp], shape gradients
//    double [6][Tp], edge neighbours int [3][Tp] (structure of arrays);
//  * element residual R: double [T][18] (array of structures: the node gather
//    reads one triangle's 18 values as 9 contiguous 16-byte loads);
//  * node-node pattern (CSR) with the consistent mass and Laplacian
//    coefficients; node -> triangle and node -> wall-edge incidence (CSR).
// Nodes are in reverse Cuthill-McKee order and triangles sorted by their
// lowest node, so every gather reads a narrow window of the arrays.
//
// One time step (Sec. II.C of arXiv:1708.04678, D2Q9 form) is six kinds of
// kernels, captured once into a CUDA graph:
//   k_collide   moments (eq:velocity, eq:pressure), collision (eqn::collide)
//   k_mu        chemical potential with the patch Laplacian and the wetting
//               flux (eqn:mp_mu, eqn:lapl_int_mp, eqn:bc2)
//   k_gradmu    P0 gradient of mu per triangle
//   k_element   element Laplacian of mu (Sec. II.D), P0 forces at the
//               barycentre (eq:G, eq:H, eq:intF) and the element residual
//               A_T (Phi - e.grad psi_hat) of eq:galerkin_lbm
//   k_rhs       node-centric gather of the streaming right-hand side with
//               weak bounce-back on walls; first Chebyshev iterate
//   k_cheb      Chebyshev sweeps of the consistent-mass solve with the
//               lumped-mass preconditioner; the last adds the increment
// No floating-point atomics: every sum is a fixed-order loop or tree.  The one
// atomic is an integer counter that picks the block of k_diag_fused32 that
// combines the blocks' partials (in block order, whichever block it is).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <utility>
#include <new>
#include <string>
#include <vector>

#include "felbm_internal.h"

namespace felbm {

// ---------------------------------------------------------------- D2Q9 ----
__host__ __device__ constexpr int ex(int q) {
    return q == 1 || q == 5 || q == 8 ? 1 : (q == 3 || q == 6 || q == 7 ? -1 : 0);
}
__host__ __device__ constexpr int ey(int q) {
    return q == 2 || q == 5 || q == 6 ? 1 : (q == 4 || q == 7 || q == 8 ? -1 : 0);
}
__host__ __device__ constexpr double wq(int q) {
    return q == 0 ? 4.0 / 9.0 : (q <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
}
__host__ __device__ constexpr int opp(int q) {
    return q == 0 ? 0 : (q <= 4 ? (q + 1) % 4 + 1 : (q - 5 + 2) % 4 + 5);
}
static_assert(opp(1) == 3 && opp(2) == 4 && opp(3) == 1 && opp(4) == 2, "opp");
static_assert(opp(5) == 7 && opp(6) == 8 && opp(7) == 5 && opp(8) == 6, "opp");

// e.v for a compile-time direction: only additions, in the type of v (an
// FP32 caller must not be promoted to FP64 -- GB300 runs FP64 at 1/64 rate)
template <int q, class T>
__device__ __forceinline__ T edot(T vx, T vy) {
    T r = T(0);
    if (ex(q) == 1) r = vx;
    if (ex(q) == -1) r = -vx;
    if (ey(q) == 1) r = r + vy;
    if (ey(q) == -1) r = r - vy;
    return r;
}

// ------------------------------------------------------- device tables ----
struct DevMesh {
    int32_t N, T, E, Np, Tp;
    double period_y;
    const int32_t* tri;       // [3][Tp]
    const double* area;       // [Tp]
    const double* grad;       // [6][Tp]
    const float* area32;      // [Tp]   FP32 copies for the FP32-deviation path
    const float* grad32;      // [6][Tp]
    const int32_t* nbr;       // [3][Tp]
    const int32_t* nbr_slot;  // [3][Tp] local index of the shared edge in the neighbour
    const int32_t* row_ptr;   // [N+1]
    const int32_t* col;       // [nnz]
    const double* mval;       // [nnz] consistent mass
    const double* lval;       // [nnz] -2 K_ij / V_i (patch Laplacian of C)
    const double* inv_lumped; // [Np]
    const float* mval32;      // [nnz] FP32 copy of the mass entries
    int32_t ell_w;            // width of the ELL copy (max row length), 0 = none
    const int32_t* ell_col;   // [ell_w][Np] column-major ELL copy of the pattern
    const uint16_t* ell_loc;  // [ell_w][Np] the same columns as indices into the node's tile's staged row
    int32_t n_tiles;          // node tiles (contiguous id ranges, HostMesh::tile_ptr)
    int32_t tiled_ok;         // every tile and halo fits the staged rows of k_sweep_tile32
    const int32_t* tile_ptr;  // [n_tiles + 1]
    const int32_t* halo_ptr;  // [n_tiles + 1]
    const int32_t* halo;      // [halo_ptr[n_tiles]] nodes outside a tile its rows reference
    const float* ell_val;     // [ell_w][Np] FP32 mass entries (padding: own column, 0)
    const double* ell_lval;   // [ell_w][Np] patch-Laplacian coefficients of C (padding 0)
    int32_t iell_w;           // width of the ELL copy of node -> triangle incidence, 0 = none
    const int32_t* iell_tri;  // [iell_w][Np] incident triangle (padding: T, a zero residual row)
    const float* iell_bx32;   // [iell_w][Np] the node's shape gradient in that triangle
    const float* iell_by32;
    const float* inv_lumped32;// [Np]
    const double* lumped;     // [Np]
    const double* inv_vol;    // [Np] 1 / V_i
    const int32_t* inc_ptr;   // [N+1]
    const int32_t* inc_tri;   // [ninc]
    const double* inc_bx;     // [ninc]
    const double* inc_by;     // [ninc]
    const float* inc_bx32;    // [ninc]
    const float* inc_by32;    // [ninc]
    const int32_t* wall_a;    // [E]
    const int32_t* wall_b;
    const int32_t* wall_id;
    const double* wall_phi;   // [E] wetting potential phi_c of the edge's wall id
    const double* wall_len;
    const double* wall_nx;
    const double* wall_ny;
    const int32_t* winc_ptr;  // [N+1]
    const int32_t* winc_edge;
    const double* x;          // [Np]
    const double* y;
    const int32_t* perm;      // [N] new -> caller
    const int32_t* iperm;     // [N] caller -> new
};

struct Phys {
    double dt, tau_l, tau_v, rho_l, rho_v, kappa, beta, mobility;
    // element Laplacian of mu: 0 = face-averaged gradients (Sec. II.D),
    // 1 = vertex mean of the nodal patch Laplacian, lapmu_fac * sum l_ij (mu_j - mu_i)
    int lapmu_nodal;
    double lapmu_fac;
    // FP32 copies, rounded once on the host
    float dt_f, dt3_f, dt2h_f, inv_tau_l_f, inv_tau_v_f, rho_v_f, drho_f, mobility_f;
};

struct Bufs {
    double* psi;     // [18][Np]
    double* C;       // [Np]
    double* p;
    double* ux;
    double* uy;
    double* mu;
    double* gmu;     // [2][Tp]; FELBM_LAPMU_NODAL: the first N hold the nodal Laplacian of mu
    double* lmu;     // alias of gmu (nodal mode)
    double* R;       // [T][18]
    double* rhs;     // [18][Np]
    double* x0;      // [18][Np] FP64 Chebyshev iterates; in the mixed solve
    double* x1;      // [18][Np] they hold x64 (solution) and rho64 (residual)
    double* x64;     // alias of x0
    double* rho64;   // alias of x1
    float* r32;      // [18][Np] FP32 residual of the current correction
    float* e0;       // [18][Np] FP32 Chebyshev iterates
    float* e1;
    // FP32-deviation storage (precision FELBM_FP32_DEV); C above stays FP64
    float* dpsi;     // deviations from equilibrium: [Np][16] rows (q = 1..8 of g, h), then [2][Np] (q = 0)
    float* p32;      // [Np]
    float* ux32;
    float* uy32;
    float* mu32;
    float* gmu32;    // [2][Tp]; FELBM_LAPMU_NODAL: the first N hold the nodal Laplacian of mu
    float* lmu32;    // alias of gmu32 (nodal mode)
    float* R32;      // [T][18]
    double* stage;   // [18][Np] caller-order staging
    double* in0;     // [18][Np] two caller-order input buffers of felbm_set_state, used in
    double* in1;     //          turn so a copy can run while the previous input converts
    double* diag_part; // [kDiagBlocks][kDiagSlots]
    double* diag_out;  // [kDiagSlots]
    double* Cdiag;     // [Np]
    unsigned* diag_done;   // blocks of k_diag_fused32 finished (0 between launches)
    unsigned* kerr;        // error bits of the solve kernels (kErrTileWait); 0 at felbm_init
};

constexpr int kBlock = 256;
constexpr int kDiagBlocks = 608;   // fixed grid (4 x 152 SMs): the reduction order never changes
constexpr int kDiagSlots = 16;
constexpr int kDiagSums = 13;        // slots of the final reduction (k_diag_final, or k_diag_fused32's last block)
constexpr int kDiagStepSlot = 15;    // felbm_diagnostics_enqueue: the step count
constexpr int kSolveResSlot = 13;    // slots 13, 14: sum r^2 and sum b^2 of the checked solve (felbm_solver_check)

// ------------------------------------------------------ K1: collision -----
// Moments of the pre-collision state (C = sum h, p = sum g, rho u = sum e g /
// cs2) and BGK collision towards the equilibria of eqn::g_eq / eqn::f_eq,
// written in place: g_eq = w p + rho cs2 (Gamma - w), h_eq = Gamma C.
__global__ void __launch_bounds__(kBlock) k_collide(DevMesh m, Phys c, Bufs b, int do_collide) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const int Np = m.Np;
    double g[9], h[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        g[q] = b.psi[q * Np + i];
        h[q] = b.psi[(9 + q) * Np + i];
    }
    double C = 0.0, p = 0.0;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        C += h[q];
        p += g[q];
    }
    double mx = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
    double my = (g[2] - g[4]) + (g[5] + g[6]) - (g[7] + g[8]);
    double rho = c.rho_v + C * (c.rho_l - c.rho_v);
    double ux = 3.0 * mx / rho, uy = 3.0 * my / rho;
    b.C[i] = C;
    b.p[i] = p;
    b.ux[i] = ux;
    b.uy[i] = uy;
    if (!do_collide) return;
    double inv_tau = C / c.tau_l + (1.0 - C) / c.tau_v;
    double omega = 1.0 / (1.0 / inv_tau + 0.5);
    double uu15 = 1.5 * (ux * ux + uy * uy);
    double rcs2 = rho * (1.0 / 3.0);
#define FELBM_COLLIDE_Q(q)                                                            \
    {                                                                                 \
        double eu = edot<q>(ux, uy);                                                  \
        double G = wq(q) * (1.0 + 3.0 * eu + 4.5 * eu * eu - uu15);                   \
        double geq = wq(q) * p + rcs2 * (G - wq(q));                                  \
        double heq = G * C;                                                           \
        b.psi[q * Np + i] = g[q] - omega * (g[q] - geq);                              \
        b.psi[(9 + q) * Np + i] = h[q] - omega * (h[q] - heq);                        \
    }
    FELBM_COLLIDE_Q(0) FELBM_COLLIDE_Q(1) FELBM_COLLIDE_Q(2) FELBM_COLLIDE_Q(3)
    FELBM_COLLIDE_Q(4) FELBM_COLLIDE_Q(5) FELBM_COLLIDE_Q(6) FELBM_COLLIDE_Q(7)
    FELBM_COLLIDE_Q(8)
#undef FELBM_COLLIDE_Q
}

// --------------------------------------------- K2: chemical potential -----
// mu_i = 2 beta C (C-1)(2C-1) - kappa lap(C)_i with the patch Laplacian
// kappa lap(C)_i = kappa sum_j l_ij C_j + (1/V_i) sum_{wall e at i} -phi_c |e|
// [ (Ca+Cb)/2 - (Ca^2 + Ca Cb + Cb^2)/3 ]  (wall flux of eqn:bc2, C linear on e).
__global__ void __launch_bounds__(kBlock) k_mu(DevMesh m, Phys c, Bufs b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    double lap = 0.0;
    for (int k = m.row_ptr[i]; k < m.row_ptr[i + 1]; ++k) lap += m.lval[k] * b.C[m.col[k]];
    double wall = 0.0;
    for (int k = m.winc_ptr[i]; k < m.winc_ptr[i + 1]; ++k) {
        int e = m.winc_edge[k];
        double Ca = b.C[m.wall_a[e]], Cb = b.C[m.wall_b[e]];
        double s = 0.5 * (Ca + Cb) - (Ca * Ca + Ca * Cb + Cb * Cb) * (1.0 / 3.0);
        wall -= m.wall_phi[e] * m.wall_len[e] * s;
    }
    double C = b.C[i];
    b.mu[i] = 2.0 * c.beta * C * (C - 1.0) * (2.0 * C - 1.0) - (c.kappa * lap + wall * m.inv_vol[i]);
}

// ------------------------------------------------- K3: grad mu per T ------
__global__ void __launch_bounds__(kBlock) k_gradmu(DevMesh m, Bufs b) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m.T) return;
    const int Tp = m.Tp;
    double gx = 0.0, gy = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double mu = b.mu[m.tri[k * Tp + t]];
        gx += mu * m.grad[(2 * k) * Tp + t];
        gy += mu * m.grad[(2 * k + 1) * Tp + t];
    }
    b.gmu[t] = gx;
    b.gmu[Tp + t] = gy;
}

// K3' (FELBM_LAPMU_NODAL): nodal Laplacian of mu, the patch Laplacian of C
// applied to mu with zero wall flux (eqn:bc1), lumped P1 volume.
__global__ void __launch_bounds__(kBlock) k_lmu(DevMesh m, Phys c, Bufs b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const double mi = b.mu[i];
    double lap = 0.0;
    for (int k = m.row_ptr[i]; k < m.row_ptr[i + 1]; ++k) lap += m.lval[k] * (b.mu[m.col[k]] - mi);
    b.lmu[i] = c.lapmu_fac * lap;
}

// ------------------------------- K4: forces and element residual ---------
// lap(mu)_T = (1/A) sum_{interior edges} 1/2 (grad mu_T + grad mu_T').nu_k with
// nu_k = -2 A b_k (outward normal x length of the edge opposite vertex k);
// wall edges give 0 (eqn:bc1).  Forces at the barycentre:
//   Phi_g = (e-u).[cs2 grad(rho) (Gamma - w) + mu grad(C) Gamma]
//   Phi_h = [(e-u).(grad C - C/(rho cs2) (grad p - mu grad C)) + M lap(mu)] Gamma
// Residual R_a = A (Phi_a - e_a . grad psi_hat_a), psi_hat P1 on the triangle.
__global__ void __launch_bounds__(128) k_element(DevMesh m, Phys c, Bufs b) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m.T) return;
    const int Tp = m.Tp, Np = m.Np;
    int v[3];
    double bx[3], by[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        v[k] = m.tri[k * Tp + t];
        bx[k] = m.grad[(2 * k) * Tp + t];
        by[k] = m.grad[(2 * k + 1) * Tp + t];
    }
    const double A = m.area[t];
    double Cs = 0, ps = 0, uxs = 0, uys = 0, mus = 0, gCx = 0, gCy = 0, gpx = 0, gpy = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double Cv = b.C[v[k]], pv = b.p[v[k]];
        Cs += Cv;
        ps += pv;
        uxs += b.ux[v[k]];
        uys += b.uy[v[k]];
        mus += b.mu[v[k]];
        gCx += Cv * bx[k];
        gCy += Cv * by[k];
        gpx += pv * bx[k];
        gpy += pv * by[k];
    }
    const double third = 1.0 / 3.0;
    double Cb = Cs * third, ux = uxs * third, uy = uys * third, mub = mus * third;
    double lapmu = 0.0;
    if (c.lapmu_nodal) {
        lapmu = (b.lmu[v[0]] + b.lmu[v[1]] + b.lmu[v[2]]) * third;
    } else {
        double gmx = b.gmu[t], gmy = b.gmu[Tp + t];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            int nb = m.nbr[k * Tp + t];
            if (nb >= 0) lapmu -= (gmx + b.gmu[nb]) * bx[k] + (gmy + b.gmu[Tp + nb]) * by[k];
        }
    }
    double drho = c.rho_l - c.rho_v;
    double rhob = c.rho_v + Cb * drho;
    double grx = drho * gCx, gry = drho * gCy;
    double f = 3.0 * Cb / rhob;
    double vhx = gCx - f * (gpx - mub * gCx), vhy = gCy - f * (gpy - mub * gCy);
    double u_gr = ux * grx + uy * gry, u_gC = ux * gCx + uy * gCy, u_vh = ux * vhx + uy * vhy;
    double uu15 = 1.5 * (ux * ux + uy * uy);
    double Mlap = c.mobility * lapmu;
    double out[18];
#define FELBM_ELEM_Q(q)                                                                           \
    {                                                                                             \
        double eu = edot<q>(ux, uy);                                                              \
        double G = wq(q) * (1.0 + 3.0 * eu + 4.5 * eu * eu - uu15);                               \
        double phig = third * (G - wq(q)) * (edot<q>(grx, gry) - u_gr) + mub * G * (edot<q>(gCx, gCy) - u_gC); \
        double phih = ((edot<q>(vhx, vhy) - u_vh) + Mlap) * G;                                    \
        double dg = 0.0, dh = 0.0;                                                                \
        if (q != 0) {                                                                             \
            for (int k = 0; k < 3; ++k) {                                                         \
                double eb = edot<q>(bx[k], by[k]);                                                \
                dg += b.psi[q * Np + v[k]] * eb;                                                  \
                dh += b.psi[(9 + q) * Np + v[k]] * eb;                                            \
            }                                                                                     \
        }                                                                                         \
        out[q] = A * (phig - dg);                                                                 \
        out[9 + q] = A * (phih - dh);                                                             \
    }
    FELBM_ELEM_Q(0) FELBM_ELEM_Q(1) FELBM_ELEM_Q(2) FELBM_ELEM_Q(3) FELBM_ELEM_Q(4)
    FELBM_ELEM_Q(5) FELBM_ELEM_Q(6) FELBM_ELEM_Q(7) FELBM_ELEM_Q(8)
#undef FELBM_ELEM_Q
    double2* dst = reinterpret_cast<double2*>(b.R + (size_t)t * 18);
#pragma unroll
    for (int k = 0; k < 9; ++k) dst[k] = make_double2(out[2 * k], out[2 * k + 1]);
}

// ------------------------------------------- K5: streaming RHS gather -----
// RHS_{i,a} = sum_{T at i} R_{T,a} (dt/3 + dt^2/2 e_a.b_{i,T})
//           - dt sum_{wall e at i} (e_a.n) [L/3 (psi_opp - psi)_i + L/6 (psi_opp - psi)_o]
// (second sum only for incoming directions e_a.n < 0; o = other end of e).
// Also writes the first iterate of the solve x1 = first_scale * RHS / m_i
// (first_scale = 1/theta for the FP64 Chebyshev recurrence, tau_0 for the
// FP32 Richardson steps): in FP64 (FP64 Chebyshev) or, for the
// mixed-precision solve, in FP32 together with the FP32 copy of the
// right-hand side.
template <bool kMixed>
__global__ void __launch_bounds__(128) k_rhs(DevMesh m, Phys c, Bufs b, double first_scale) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const int Np = m.Np;
    double acc[18];
#pragma unroll
    for (int q = 0; q < 18; ++q) acc[q] = 0.0;
    const double c1 = c.dt * (1.0 / 3.0), c2 = 0.5 * c.dt * c.dt;
    for (int k = m.inc_ptr[i]; k < m.inc_ptr[i + 1]; ++k) {
        int t = m.inc_tri[k];
        double bxi = m.inc_bx[k], byi = m.inc_by[k];
        const double2* src = reinterpret_cast<const double2*>(b.R + (size_t)t * 18);
        double r[18];
#pragma unroll
        for (int s = 0; s < 9; ++s) {
            double2 v2 = src[s];
            r[2 * s] = v2.x;
            r[2 * s + 1] = v2.y;
        }
#define FELBM_RHS_Q(q)                                          \
        {                                                       \
            double w = c1 + c2 * edot<q>(bxi, byi);             \
            acc[q] += r[q] * w;                                 \
            acc[9 + q] += r[9 + q] * w;                         \
        }
        FELBM_RHS_Q(0) FELBM_RHS_Q(1) FELBM_RHS_Q(2) FELBM_RHS_Q(3) FELBM_RHS_Q(4)
        FELBM_RHS_Q(5) FELBM_RHS_Q(6) FELBM_RHS_Q(7) FELBM_RHS_Q(8)
#undef FELBM_RHS_Q
    }
    for (int k = m.winc_ptr[i]; k < m.winc_ptr[i + 1]; ++k) {
        int e = m.winc_edge[k];
        int o = m.wall_a[e] == i ? m.wall_b[e] : m.wall_a[e];
        double L = m.wall_len[e], nx = m.wall_nx[e], ny = m.wall_ny[e];
#define FELBM_WALL_Q(q)                                                                      \
        {                                                                                    \
            double en = edot<q>(nx, ny);                                                     \
            if (en < 0.0) {                                                                  \
                double f = -c.dt * en;                                                       \
                double dgi = b.psi[opp(q) * Np + i] - b.psi[q * Np + i];                     \
                double dgo = b.psi[opp(q) * Np + o] - b.psi[q * Np + o];                     \
                double dhi = b.psi[(9 + opp(q)) * Np + i] - b.psi[(9 + q) * Np + i];         \
                double dho = b.psi[(9 + opp(q)) * Np + o] - b.psi[(9 + q) * Np + o];         \
                acc[q] += f * (L * (1.0 / 3.0) * dgi + L * (1.0 / 6.0) * dgo);               \
                acc[9 + q] += f * (L * (1.0 / 3.0) * dhi + L * (1.0 / 6.0) * dho);           \
            }                                                                                \
        }
        FELBM_WALL_Q(1) FELBM_WALL_Q(2) FELBM_WALL_Q(3) FELBM_WALL_Q(4)
        FELBM_WALL_Q(5) FELBM_WALL_Q(6) FELBM_WALL_Q(7) FELBM_WALL_Q(8)
#undef FELBM_WALL_Q
    }
    double s = m.inv_lumped[i] * first_scale;
#pragma unroll
    for (int q = 0; q < 18; ++q) {
        b.rhs[q * Np + i] = acc[q];
        if (kMixed) {
            b.r32[q * Np + i] = (float)acc[q];
            b.e1[q * Np + i] = (float)(acc[q] * s);
        } else {
            b.x1[q * Np + i] = acc[q] * s;
        }
    }
}

// First iterate for a standalone solve: x1 = first_scale * B / m_i
// (1/theta for the FP64 recurrence, tau_0 for the FP32 steps).
template <bool kMixed>
__global__ void __launch_bounds__(kBlock) k_cheb_start(DevMesh m, Bufs b, double first_scale) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const int Np = m.Np;
    double s = m.inv_lumped[i] * first_scale;
#pragma unroll
    for (int q = 0; q < 18; ++q) {
        double r = b.rhs[q * Np + i];
        if (kMixed) {
            b.r32[q * Np + i] = (float)r;
            b.e1[q * Np + i] = (float)(r * s);
        } else {
            b.x1[q * Np + i] = r * s;
        }
    }
}

// ---------------------------------------------- K6: Chebyshev sweep -------
// x_{k+1} = x_k + a (x_k - x_{k-1}) + c m^{-1} (b - M x_k), the three-term
// Chebyshev recurrence for the lumped-mass preconditioned consistent mass
// matrix, whose spectrum lies in [1/4, 1] on any P1 triangulation.
//   cur  = x_k (gathered), prev = x_{k-1} (own node only; ignored if first),
//   the new iterate overwrites prev, or is added to psi on the last sweep.
__global__ void __launch_bounds__(128) k_cheb(DevMesh m, Bufs b, const double* __restrict__ cur,
                                              double* prev, double a, double cc, int first,
                                              int add_to_psi) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const int Np = m.Np;
    double acc[18];
#pragma unroll
    for (int q = 0; q < 18; ++q) acc[q] = 0.0;
    for (int k = m.row_ptr[i]; k < m.row_ptr[i + 1]; ++k) {
        int j = m.col[k];
        double mv = m.mval[k];
#pragma unroll
        for (int q = 0; q < 18; ++q) acc[q] += mv * cur[q * Np + j];
    }
    double s = cc * m.inv_lumped[i];
#pragma unroll
    for (int q = 0; q < 18; ++q) {
        double xk = cur[q * Np + i];
        double xm = first ? 0.0 : prev[q * Np + i];
        double xn = xk + a * (xk - xm) + s * (b.rhs[q * Np + i] - acc[q]);
        if (add_to_psi)
            b.psi[q * Np + i] += xn;
        else
            prev[q * Np + i] = xn;
    }
}

// ------------------------------- K6': mixed-precision mass solve ---------
// Iterative refinement: x <- x + e, where each correction e solves
// M11 e = rho approximately with FP32 Chebyshev sweeps (same recurrence as
// k_cheb, FP32 matrix copy), and the residual rho is carried in FP64 by the
// recurrence rho <- rho - M11 e with M11 in FP64.  GB300 runs FP32 FMA at
// ~70x the FP64 rate, so only the refinement kernels pay FP64 matvecs.
enum Final { kStore = 0, kAddPsi = 1, kAddX64 = 2, kUpdateDev = 3 };

// Programmatic dependent launch: a kernel launched with the attribute may
// start while its predecessor drains; it must wait before touching that
// kernel's outputs.  Both are no-ops in a kernel launched without it.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" :::); }

#include "felbm_dev32.cuh"
#include "felbm_adjoint.cuh"
#include "felbm_tile32.cuh"

// One step of the FP32 correction solve (CSR rows): Richardson iteration
// x_{k+1} = x_k + tau_k m^{-1} (b - M x_k) with the Chebyshev step sizes
// tau_k = 1 / lambda_k, lambda_k the roots of the degree-K Chebyshev
// polynomial on the spectrum [1/4, 1] of m^{-1} M11 (taken smallest and
// largest alternately, which keeps every partial product below 1 and the
// round-off amplification below 3).  After K steps from x_0 = 0 the error
// polynomial is the same scaled Chebyshev polynomial as for the three-term
// recurrence, but each step reads only x_k (gathered) and b.
//   cur = x_k; the new iterate goes to nxt (or to the final destination).
template <int kFinal>
__global__ void __launch_bounds__(128) k_cheb32(DevMesh m, Phys c, Bufs b, const float* __restrict__ cur,
                                                float* nxt, float tau, int have_x64) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const int Np = m.Np;
    float acc[18];
#pragma unroll
    for (int q = 0; q < 18; ++q) acc[q] = 0.0f;
    for (int k = m.row_ptr[i]; k < m.row_ptr[i + 1]; ++k) {
        int j = m.col[k];
        float mv = m.mval32[k];
#pragma unroll
        for (int q = 0; q < 18; ++q) acc[q] = fmaf(mv, cur[q * Np + j], acc[q]);
    }
    float s = tau * m.inv_lumped32[i];
    float d[18];
#pragma unroll
    for (int q = 0; q < 18; ++q) {
        float xk = cur[q * Np + i];
        float xn = fmaf(s, b.r32[q * Np + i] - acc[q], xk);
        if (kFinal == kStore) {
            nxt[q * Np + i] = xn;
        } else if (kFinal == kUpdateDev) {
            d[q] = xn;
        } else {
            double x = have_x64 ? b.x64[q * Np + i] + (double)xn : (double)xn;
            if (kFinal == kAddPsi)
                b.psi[q * Np + i] += x;
            else
                b.x64[q * Np + i] = x;
        }
    }
    if (kFinal == kUpdateDev) dev32_update(m, c, b, i, d);
}

// Programmatic dependent launch: a sweep may be scheduled while its
// predecessor drains; it loads its (read-only) matrix row first and waits for
// the predecessor's results before touching them.  Both instructions are
// no-ops for a kernel launched without the attribute.

// The FP32 step of k_cheb32 on the ELL copy of the pattern (kW entries per
// row, padded with the own column and value 0).  Row indices and values are
// loaded up front (coalesced, column-major).
// kParts threads per node, each owning 18/kParts of the node's rows (more
// threads in flight for this latency-bound gather); the field update needs
// all 18 in one thread.  The parts of one node block are consecutive blocks
// (blockIdx.x = kParts * node block + part), so they run together and share
// the block's matrix rows through L2 instead of fetching them from DRAM
// once per part.
template <int kFinal, int kW, int kParts, bool kFromRhs = false>
__global__ void __launch_bounds__(128) k_sweep32(DevMesh m, Phys c, Bufs b, const float* __restrict__ cur,
                                                 float* nxt, float tau, int have_x64, float tau0) {
    pdl_release();
    static_assert(kFinal != kUpdateDev || kParts == 1, "the field update needs the whole node");
    constexpr int NQ = 18 / kParts;
    const int nb = (int)blockIdx.x / kParts;
    const int i = nb * (int)blockDim.x + (int)threadIdx.x;
    const int q0 = NQ * ((int)blockIdx.x - nb * kParts);
    const int Np = m.Np;
    static_assert(18 % kParts == 0, "parts must divide 18");
    int col[kW];
    float val[kW];
    if (i < m.N) {
#pragma unroll
        for (int k = 0; k < kW; ++k) {
            col[k] = m.ell_col[k * Np + i];
            val[k] = m.ell_val[k * Np + i];
        }
    }
    const float s = tau * (i < m.N ? m.inv_lumped32[i] : 0.0f);
    // kFromRhs: the first step of the solve, whose iterate x_0 = tau_0 b / m
    // is formed here from the right-hand side (the RHS kernel stores b only)
    float sc[kFromRhs ? kW : 1];
    float s0 = 0.0f;
    if constexpr (kFromRhs) {
        if (i < m.N) {
#pragma unroll
            for (int k = 0; k < kW; ++k) sc[k] = m.inv_lumped32[col[k]] * tau0;
            s0 = m.inv_lumped32[i] * tau0;
        }
    }
    pdl_wait();
    if (i >= m.N) return;
    // every gathered value is loaded before the first product (more loads in
    // flight per thread for this latency-bound gather: 15 % faster sweeps on
    // the 2.08M-node rough wall than interleaving loads and products)
    float g[kW][NQ], xk[NQ], rr[NQ];
    const float* src = kFromRhs ? b.r32 : cur;
#pragma unroll
    for (int k = 0; k < kW; ++k)
#pragma unroll
        for (int q = 0; q < NQ; ++q) g[k][q] = src[(q0 + q) * Np + col[k]];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        rr[q] = b.r32[(q0 + q) * Np + i];
        xk[q] = kFromRhs ? rr[q] * s0 : cur[(q0 + q) * Np + i];
    }
    if constexpr (kFromRhs) {
#pragma unroll
        for (int k = 0; k < kW; ++k)
#pragma unroll
            for (int q = 0; q < NQ; ++q) g[k][q] *= sc[k];
    }
    float d[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        float acc = 0.0f;
#pragma unroll
        for (int k = 0; k < kW; ++k) acc = fmaf(val[k], g[k][q], acc);
        const int r = (q0 + q) * Np + i;
        float xn = fmaf(s, rr[q] - acc, xk[q]);
        if (kFinal == kStore) {
            nxt[r] = xn;
        } else if (kFinal == kUpdateDev) {
            d[q] = xn;
        } else {
            double x = have_x64 ? b.x64[r] + (double)xn : (double)xn;
            if (kFinal == kAddPsi)
                b.psi[r] += x;
            else
                b.x64[r] = x;
        }
    }
    if constexpr (kFinal == kUpdateDev) dev32_update(m, c, b, i, d);
}

// x <- x + e ; rho <- rho - M11 e (FP64) ; FP32 copy of rho and the first
// iterate of the next correction, tau_0 rho / m.
__global__ void __launch_bounds__(128) k_refine(DevMesh m, Bufs b, const float* __restrict__ e,
                                                float* next_first, int first_round, double tau0) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const int Np = m.Np;
    double acc[18];
#pragma unroll
    for (int q = 0; q < 18; ++q) acc[q] = 0.0;
    for (int k = m.row_ptr[i]; k < m.row_ptr[i + 1]; ++k) {
        int j = m.col[k];
        double mv = m.mval[k];
#pragma unroll
        for (int q = 0; q < 18; ++q) acc[q] += mv * (double)e[q * Np + j];
    }
    double s = m.inv_lumped[i] * tau0;
#pragma unroll
    for (int q = 0; q < 18; ++q) {
        double xo = first_round ? 0.0 : b.x64[q * Np + i];
        double ro = first_round ? b.rhs[q * Np + i] : b.rho64[q * Np + i];
        double rn = ro - acc[q];
        b.x64[q * Np + i] = xo + (double)e[q * Np + i];
        b.rho64[q * Np + i] = rn;
        b.r32[q * Np + i] = (float)rn;
        next_first[q * Np + i] = (float)(rn * s);
    }
}

// -------------------------------------- solve residual (opt-in check) ----
// Before the last step of the solve: sum over nodes and right-hand sides of
// r^2, r = b_k - M x (FP32 rows, as the steps form them; b_k the current
// correction's right-hand side), and of the solve's original right-hand
// side squared (FP64 rhs for the mixed solve, the FP32 copy for FP32
// storage).  Fixed grid, per-block partials, one ordered final sum: the
// result does not depend on scheduling.
template <bool kRhs64>
__global__ void __launch_bounds__(kBlock) k_solve_resid(DevMesh m, Bufs b, const float* __restrict__ x,
                                                        double* part) {
    const int Np = m.Np;
    double rr = 0.0, bb = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m.N; i += gridDim.x * blockDim.x) {
        const int k0 = m.row_ptr[i], k1 = m.row_ptr[i + 1];
        for (int q = 0; q < 18; ++q) {
            float acc = 0.0f;
            for (int k = k0; k < k1; ++k) acc = fmaf(m.mval32[k], x[q * Np + m.col[k]], acc);
            const float r = b.r32[q * Np + i] - acc;
            rr += (double)r * (double)r;
            const double bq = kRhs64 ? b.rhs[q * Np + i] : (double)b.r32[q * Np + i];
            bb += bq * bq;
        }
    }
    __shared__ double sh[2][kBlock / 32];
    for (int o = 16; o > 0; o >>= 1) {
        rr += __shfl_down_sync(0xffffffffu, rr, o);
        bb += __shfl_down_sync(0xffffffffu, bb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = rr;
        sh[1][threadIdx.x >> 5] = bb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, c = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) {
            a += sh[0][w];
            c += sh[1][w];
        }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = c;
    }
}
__global__ void k_solve_resid_final(const double* __restrict__ part, int n, double* out) {
    double a = 0.0, c = 0.0;
    for (int k = 0; k < n; ++k) {
        a += part[2 * k];
        c += part[2 * k + 1];
    }
    out[0] = a;
    out[1] = c;
}

// ----------------------------------------------- permutation kernels ------
__global__ void k_scatter_in(DevMesh m, const double* __restrict__ stage, double* dst, int rows) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    int o = m.perm[i];
    for (int q = 0; q < rows; ++q) dst[q * m.Np + i] = stage[(size_t)q * m.N + o];
}
__global__ void k_gather_out(DevMesh m, const double* __restrict__ src, double* stage, int rows) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    int o = m.perm[i];
    for (int q = 0; q < rows; ++q) stage[(size_t)q * m.N + o] = src[q * m.Np + i];
}
__global__ void k_zero_rows(DevMesh m, double* dst, int row0, int row1) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    for (int q = row0; q < row1; ++q) dst[q * m.Np + i] = 0.0;
}
// Initial state at equilibrium with the fields C0, p0, u0 (caller order in
// stage: C0 [N], then p0 [N] if has_p, then u0 [2N] as x, y if has_u; the
// missing ones are zero): g = w p + rho cs2 (Gamma(u) - w), h = Gamma(u) C
// (eqn::g_eq, eqn::f_eq), rho = C rho_l + (1 - C) rho_v.
__global__ void k_init_state(DevMesh m, Phys c, const double* __restrict__ stage, double* psi, int has_p,
                             int has_u) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const int o = m.perm[i], N = m.N;
    const double C = stage[o];
    const double p = has_p ? stage[N + o] : 0.0;
    const double* u = stage + (has_p ? 2 : 1) * (size_t)N;
    const double ux = has_u ? u[o] : 0.0, uy = has_u ? u[N + o] : 0.0;
    const double rcs2 = (c.rho_v + C * (c.rho_l - c.rho_v)) * (1.0 / 3.0);
    const double uu15 = 1.5 * (ux * ux + uy * uy);
#define FELBM_INIT_Q(q)                                                      \
    {                                                                        \
        const double eu = edot<q>(ux, uy);                                   \
        const double G = wq(q) * (1.0 + 3.0 * eu + 4.5 * eu * eu - uu15);    \
        psi[q * m.Np + i] = wq(q) * p + rcs2 * (G - wq(q));                  \
        psi[(9 + q) * m.Np + i] = G * C;                                     \
    }
    FELBM_INIT_Q(0) FELBM_INIT_Q(1) FELBM_INIT_Q(2) FELBM_INIT_Q(3) FELBM_INIT_Q(4)
    FELBM_INIT_Q(5) FELBM_INIT_Q(6) FELBM_INIT_Q(7) FELBM_INIT_Q(8)
#undef FELBM_INIT_Q
}

// ------------------------------------------------------ diagnostics -------
// Slots: 0 mass, 1 sum rho|u|^2, 2 band weight, 3 band sum m rho|u|^2,
// 4 liquid weight, 5 liquid sum m p, 6 vapour weight, 7 vapour sum m p,
// 8 unused, 9 non-finite count, 10 max |u|^2 (node pass);
// 11 wetted length, 12 max contour height (edge pass).
struct DiagReq {
    double cx, cy, R, band;
    double period_x, period_y;
    int substrate;
    int use_band;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double min_image(double d, double L) {
    return L > 0.0 ? d - L * rint(d / L) : d;
}

// Block reduction of NS sums and NM maxima to out[0 .. NS+NM), in a fixed
// order.  FP64 adds run at 1/64 of the FP32 rate on this part, so every
// value is added once: the threads' partials go to shared memory, NV x NW
// threads each combine one interleaved segment of 32, and NV threads combine
// the NW segments (a warp-shuffle tree in every lane would add each value
// five times over).
template <int NS, int NM>
__device__ void block_reduce_store(double (&s)[NS], double (&mx)[NM], double* out) {
    constexpr int NV = NS + NM, NW = kBlock / 32, L = kBlock + 2;
    __shared__ double sh[NV][L];
    __shared__ double part[NV][NW];
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k][threadIdx.x] = k < NS ? s[k] : mx[k - NS];
    __syncthreads();
    if (threadIdx.x < NV * NW) {
        const int k = threadIdx.x / NW, seg = threadIdx.x - k * NW;
        double r = sh[k][seg];
        for (int j = 1; j < 32; ++j) r = k < NS ? r + sh[k][seg + NW * j] : fmax(r, sh[k][seg + NW * j]);
        part[k][seg] = r;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        const int k = threadIdx.x;
        double r = part[k][0];
        for (int w = 1; w < NW; ++w) r = k < NS ? r + part[k][w] : fmax(r, part[k][w]);
        out[k] = r;
    }
}

// Comparisons of a double with a positive threshold on the bit patterns (the
// integer pipe; FP64 compares share the 1/64-rate FP64 pipe).  For x >= 0 the
// patterns order like the values, and every x with the sign bit set is a
// negative integer, below the pattern of t.  NaNs compare by their pattern;
// non-finite states are reported through their own slot.
__device__ __forceinline__ bool ge_pos(double x, double t) { return __double_as_longlong(x) >= __double_as_longlong(t); }
__device__ __forceinline__ bool le_pos(double x, double t) { return __double_as_longlong(x) <= __double_as_longlong(t); }
__device__ __forceinline__ bool finite_bits(double x) {
    return (__double_as_longlong(x) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
}

// Per-node contributions (slots 0..9 sums, one max); writes the node's C.
template <bool kDev32>
__device__ __forceinline__ void diag_node(const DevMesh& m, const Phys& c, const Bufs& b, const DiagReq& rq,
                                          int i, double (&s)[10], double (&mx)[1]) {
    const int Np = m.Np;
    double C = 0, p = 0, uu, ruu;
    bool finite;
    if (kDev32) {
        // FP32 fields: |u|^2 and rho |u|^2 in FP32 (FP64 runs at 1/64 rate), summed in FP64
        C = b.C[i];
        p = b.p32[i];
        const float uxf = b.ux32[i], uyf = b.uy32[i];
        const float rhof = c.rho_v_f + (float)C * c.drho_f;
        const float uuf = uxf * uxf + uyf * uyf;
        uu = uuf;
        ruu = rhof * uuf;
        float dsum = 0.0f;
#pragma unroll
        for (int q = 0; q < 18; ++q) dsum += b.dpsi[dpsi_at(Np, q, i)];
        // non-finite deviations are reported too
        finite = finite_bits(C) && isfinite(b.p32[i]) && isfinite(uuf) && isfinite(dsum);
    } else {
        double g[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            g[q] = b.psi[q * Np + i];
            p += g[q];
            C += b.psi[(9 + q) * Np + i];
        }
        double mxm = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
        double mym = (g[2] - g[4]) + (g[5] + g[6]) - (g[7] + g[8]);
        const double rho = c.rho_v + C * (c.rho_l - c.rho_v);
        const double ux = 3.0 * mxm / rho, uy = 3.0 * mym / rho;
        uu = ux * ux + uy * uy;
        ruu = rho * uu;
        finite = isfinite(C) && isfinite(p) && isfinite(uu);
    }
    double w = m.lumped[i];
    b.Cdiag[i] = C;
    if (!finite) s[9] += 1.0;
    s[0] += w * C;
    s[1] += ruu;
    if (rq.use_band) {
        double dx = min_image(m.x[i] - rq.cx, rq.period_x), dy = min_image(m.y[i] - rq.cy, rq.period_y);
        double r = sqrt(dx * dx + dy * dy);
        if (fabs(r - rq.R) <= rq.band) {
            s[2] += w;
            s[3] += w * ruu;
        }
    }
    if (ge_pos(C, 0.95)) {
        s[4] += w;
        s[5] += w * p;
    }
    if (le_pos(C, 0.05)) {
        s[6] += w;
        s[7] += w * p;
    }
    mx[0] = fmax(mx[0], uu);
}

// Wetted length of a substrate wall edge (C linear along it).
__device__ __forceinline__ void diag_wall(const DevMesh& m, const double* Cn, const DiagReq& rq, int e, double& wet) {
    if (m.wall_id[e] != rq.substrate) return;
    double Ca = Cn[m.wall_a[e]], Cb = Cn[m.wall_b[e]], L = m.wall_len[e];
    const bool a = ge_pos(Ca, 0.5), bb = ge_pos(Cb, 0.5);
    if (a && bb)
        wet += L;
    else if (a || bb) {
        double hi = fmax(Ca, Cb), lo = fmin(Ca, Cb);
        wet += L * (hi - 0.5) / (hi - lo);
    }
}

// Highest crossing of the C = 1/2 contour on the edges of a triangle.
__device__ __forceinline__ void diag_tri(const DevMesh& m, const double* Cn, const DiagReq& rq, int t, double& ymax) {
    const int Tp = m.Tp;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int ia = m.tri[((k + 1) % 3) * Tp + t], ic = m.tri[((k + 2) % 3) * Tp + t];
        double Ca = Cn[ia], Cc = Cn[ic];
        if (ge_pos(Ca, 0.5) != ge_pos(Cc, 0.5)) {
            double tt = (0.5 - Ca) / (Cc - Ca);
            double dy = min_image(m.y[ic] - m.y[ia], rq.period_y);
            ymax = fmax(ymax, m.y[ia] + tt * dy);
        }
    }
}

template <bool kDev32>
__global__ void __launch_bounds__(kBlock) k_diag_nodes(DevMesh m, Phys c, Bufs b, DiagReq rq) {
    double s[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    double mx[1] = {0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m.N; i += gridDim.x * blockDim.x)
        diag_node<kDev32>(m, c, b, rq, i, s, mx);
    block_reduce_store<10, 1>(s, mx, b.diag_part + (size_t)blockIdx.x * kDiagSlots);
}

// wetted length on substrate wall edges; highest crossing of the C = 1/2
// contour on triangle edges (both from the nodal C written by k_diag_nodes)
__global__ void __launch_bounds__(kBlock) k_diag_edges(DevMesh m, Bufs b, DiagReq rq) {
    double s[1] = {0.0};
    double mx[1] = {-1e300};
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m.E; e += gridDim.x * blockDim.x)
        diag_wall(m, b.Cdiag, rq, e, s[0]);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m.T; t += gridDim.x * blockDim.x)
        diag_tri(m, b.Cdiag, rq, t, mx[0]);
    block_reduce_store<1, 1>(s, mx, b.diag_part + (size_t)blockIdx.x * kDiagSlots + 11);
}

// Tables of the connected components (groups) of the mesh.
struct GroupTables {
    const int32_t* node_begin;   // [G] internal node range of each group
    const int32_t* node_end;
    const int32_t* tri_begin;    // [G] triangle range
    const int32_t* tri_end;
    const int32_t* wall_ptr;     // [G+1] wall edges of each group (CSR)
    const int32_t* wall_edge;
    DiagReq* reqs;               // [G] per-group request (written by the host per call)
    double* out;                 // [G][kDiagSlots]
    int32_t* cta_groups;         // [G] groups run by k_step_cta32
};

// One block per group: the same slots as k_diag_nodes/k_diag_edges, reduced
// over the group's own nodes, wall edges and triangles in a fixed order.
template <bool kDev32>
__global__ void __launch_bounds__(kBlock) k_diag_groups(DevMesh m, Phys c, Bufs b, GroupTables gt) {
    const int g = blockIdx.x;
    const DiagReq rq = gt.reqs[g];
    double s[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    double mx[1] = {0.0};
    for (int i = gt.node_begin[g] + threadIdx.x; i < gt.node_end[g]; i += blockDim.x)
        diag_node<kDev32>(m, c, b, rq, i, s, mx);
    __syncthreads();   // the group's C (Cdiag) is complete; it is read below
    double we[1] = {0.0};
    double ym[1] = {-1e300};
    for (int k = gt.wall_ptr[g] + threadIdx.x; k < gt.wall_ptr[g + 1]; k += blockDim.x)
        diag_wall(m, b.Cdiag, rq, gt.wall_edge[k], we[0]);
    for (int t = gt.tri_begin[g] + threadIdx.x; t < gt.tri_end[g]; t += blockDim.x) diag_tri(m, b.Cdiag, rq, t, ym[0]);
    block_reduce_store<10, 1>(s, mx, gt.out + (size_t)g * kDiagSlots);
    block_reduce_store<1, 1>(we, ym, gt.out + (size_t)g * kDiagSlots + 11);
}

// One warp per slot: lane l reduces blocks l, l+32, ... in order, then a
// fixed shuffle tree -- the same order on every call.
__global__ void k_diag_final(Bufs b) {
    int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (k >= kDiagSums) return;
    bool is_max = (k == 10 || k == 12);
    double r = is_max ? -1e300 : 0.0;
    // every lane's partials loaded before they are combined (in block order)
    constexpr int kPer = (kDiagBlocks + 31) / 32;
    double v[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const int blk = lane + 32 * j;
        v[j] = blk < kDiagBlocks ? b.diag_part[(size_t)blk * kDiagSlots + k] : (is_max ? -1e300 : 0.0);
    }
#pragma unroll
    for (int j = 0; j < kPer; ++j) r = is_max ? fmax(r, v[j]) : r + v[j];
    r = is_max ? warp_max(r) : warp_sum(r);
    if (lane == 0) b.diag_out[k] = r;
}

// FP32-deviation states keep C in FP64, so the edge pass needs no node pass
// before it: one kernel accumulates every slot, and the last block to finish
// (a device-scope counter after a fence; no block waits for another) combines
// the blocks' partials in block order exactly as k_diag_final does.
__global__ void __launch_bounds__(kBlock) k_diag_fused32(DevMesh m, Phys c, Bufs b, DiagReq rq) {
    double s[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    double mx[1] = {0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m.N; i += gridDim.x * blockDim.x)
        diag_node<true>(m, c, b, rq, i, s, mx);
    double we[1] = {0.0};
    double ym[1] = {-1e300};
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m.E; e += gridDim.x * blockDim.x)
        diag_wall(m, b.C, rq, e, we[0]);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m.T; t += gridDim.x * blockDim.x)
        diag_tri(m, b.C, rq, t, ym[0]);
    block_reduce_store<10, 1>(s, mx, b.diag_part + (size_t)blockIdx.x * kDiagSlots);
    block_reduce_store<1, 1>(we, ym, b.diag_part + (size_t)blockIdx.x * kDiagSlots + 11);
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(b.diag_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int lane = threadIdx.x & 31;
    for (int k = threadIdx.x >> 5; k < kDiagSums; k += kBlock / 32) {
        const bool is_max = (k == 10 || k == 12);
        constexpr int kPer = (kDiagBlocks + 31) / 32;
        double v[kPer];
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int blk = lane + 32 * j;
            v[j] = blk < kDiagBlocks ? __ldcg(b.diag_part + (size_t)blk * kDiagSlots + k) : (is_max ? -1e300 : 0.0);
        }
        double r = is_max ? -1e300 : 0.0;
#pragma unroll
        for (int j = 0; j < kPer; ++j) r = is_max ? fmax(r, v[j]) : r + v[j];
        r = is_max ? warp_max(r) : warp_sum(r);
        if (lane == 0) b.diag_out[k] = r;
    }
    if (threadIdx.x == 0) *b.diag_done = 0u;
}

// ------------------------------------------- one CTA per batch member ------
// The whole FP32-deviation step of one small batch member in one thread
// block: the member is a contiguous range of nodes and triangles (its
// group), every phase is a block-stride loop over that range, and
// __syncthreads() orders the phases -- no kernel boundary and no grid-wide
// synchronisation inside the step.  Data written in one phase is read in
// the next through plain (coherent) loads.
constexpr int kCtaThreads = 512;
constexpr int kMaxSweeps = 64;
struct ChebCoef {
    float tau[kMaxSweeps];   // Richardson step sizes of the FP32 solve (see k_cheb32)
};

__device__ __forceinline__ void sweep32_node(const DevMesh& m, const Phys& c, const Bufs& b, int i,
                                             const float* cur, float* nxt, float tau, bool update) {
    const int Np = m.Np;
    float acc[18];
#pragma unroll
    for (int q = 0; q < 18; ++q) acc[q] = 0.0f;
    if (m.ell_w > 0) {
        for (int k = 0; k < m.ell_w; ++k) {
            const int j = m.ell_col[k * Np + i];
            const float v = m.ell_val[k * Np + i];
#pragma unroll
            for (int q = 0; q < 18; ++q) acc[q] = fmaf(v, cur[q * Np + j], acc[q]);
        }
    } else {
        for (int k = m.row_ptr[i]; k < m.row_ptr[i + 1]; ++k) {
            const int j = m.col[k];
            const float v = m.mval32[k];
#pragma unroll
            for (int q = 0; q < 18; ++q) acc[q] = fmaf(v, cur[q * Np + j], acc[q]);
        }
    }
    const float s = tau * m.inv_lumped32[i];
    float d[18];
#pragma unroll
    for (int q = 0; q < 18; ++q) {
        float xk = cur[q * Np + i];
        float xn = fmaf(s, b.r32[q * Np + i] - acc[q], xk);
        if (update)
            d[q] = xn;
        else
            nxt[q * Np + i] = xn;
    }
    if (update) dev32_update(m, c, b, i, d);
}

__global__ void __launch_bounds__(kCtaThreads, 1) k_step_cta32(DevMesh m, Phys c, Bufs b, GroupTables gt,
                                                               const int32_t* __restrict__ groups, ChebCoef cf,
                                                               int sweeps, float tau0) {
    const int g = groups[blockIdx.x];
    const int n0 = gt.node_begin[g], n1 = gt.node_end[g], t0 = gt.tri_begin[g], t1 = gt.tri_end[g];
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = n0 + tid; i < n1; i += nt) mu32_node(m, c, b, i);
    __syncthreads();
    if (c.lapmu_nodal)
        for (int i = n0 + tid; i < n1; i += nt) lmu32_node(m, c, b, i);
    else
        for (int t = t0 + tid; t < t1; t += nt) gradmu32_tri(m, b, t);
    __syncthreads();
    for (int t = t0 + tid; t < t1; t += nt) element32_tri(m, c, b, t);
    __syncthreads();
    for (int i = n0 + tid; i < n1; i += nt) rhs32_node(m, c, b, i, tau0);
    __syncthreads();
    float* cur = b.e1;
    float* prv = b.e0;
    for (int k = 1; k < sweeps; ++k) {
        const bool last = k == sweeps - 1;
        for (int i = n0 + tid; i < n1; i += nt) sweep32_node(m, c, b, i, cur, prv, cf.tau[k], last);
        __syncthreads();
        float* tmp = cur;
        cur = prv;
        prv = tmp;
    }
}

// ------------------------------------------- FP64 FMA rate (instrument) --
// Eight independent FP64 FMA chains per thread: the issue rate of the FP64
// pipe, the roof of the FP64 kernels.  The result is stored only when it is
// a value the chains cannot reach, so the work is kept but nothing is written.
__device__ double g_fma_sink;
__global__ void __launch_bounds__(256) k_fp64_fma_rate(int iters, double a) {
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (double)(threadIdx.x + k) * 1e-3;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, 1e-9);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == -1.0) g_fma_sink = s;
}

// --------------------------------------------------------- host side ------
static int cuda_fail(cudaError_t e, const char* what) {
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    set_error(buf);
    return FELBM_ERR_CUDA;
}
#define FELBM_CUDA(call)                                   \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// Bump allocator over the caller's workspace (256-byte aligned pieces).
struct Carver {
    char* base;
    size_t off = 0;
    explicit Carver(void* b) : base(static_cast<char*>(b)) {}
    template <class T>
    T* take(size_t n) {
        off = (off + 255) & ~size_t(255);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += n * sizeof(T);
        return p;
    }
};

static size_t pad64(size_t n) { return (n + 63) & ~size_t(63); }

}  // namespace felbm

struct felbm_state {
    felbm::HostMesh hm;
    felbm_params prm;
    felbm::DevMesh dm{};
    felbm::Phys phys{};
    felbm::Bufs buf{};
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    cudaGraph_t graph = nullptr;
    int mode = FELBM_SOLVER_MIXED;
    int sweeps = 14;   // per correction (mixed) or in total (FP64)
    int rounds = 3;    // corrections of the mixed solve
    std::vector<double> cheb_a, cheb_c;   // three-term recurrence of the FP64 solve
    double inv_theta = 1.0;               // its first iterate x_1 = m^{-1} b / theta
    std::vector<double> tau;              // Richardson step sizes of the FP32 solves; tau[0] gives x_1
    int64_t step = 0;
    double mass0 = 0.0;
    int device = 0;
    bool timing = false;
    bool timed_step_ran = false;
    cudaEvent_t ev[7] = {};
    bool dev32 = false;   // FELBM_FP32_DEV storage
    bool use_pdl = true;  // programmatic dependent launch between solve sweeps
    int sweep_parts = 2;  // threads per node of the FP32 store sweeps (1, 2, 3, 6)
    bool sweep_tiled = false;  // store sweeps stage each node tile in shared memory (k_sweep_tile32)
    bool check = false;        // felbm_solver_check: residual of every solve before its last step
    double check_tol = 0.0;
    int n_sm = 1;              // multiprocessors of the device (grid of the persistent tiled step)
    int smem_optin = 0;        // largest dynamic shared memory a block may opt into
    felbm::GroupTables gt{};
    felbm::AdjBufs adj{};         // adjoint buffers (FP64 states)
    std::vector<double> gmass0;   // per-group mass at felbm_init
    // batch schedule (FP32_DEV): groups of at most cta_max_nodes nodes run one
    // CTA each (k_step_cta32); the rest, a prefix of the node and triangle
    // ranges, run the tiled kernels.  cta_max_nodes = 0: tiled only.
    int32_t cta_max_nodes = 0;
    int32_t n_cta = 0, tiled_N = 0, tiled_T = 0;
    int32_t* d_cta_groups = nullptr;   // [G] in the workspace
    cudaStream_t side_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev_copied = nullptr;   // set_state: the host arrays have been read
    cudaStream_t copy_stream = nullptr;     // set_state's host-to-device copies
    cudaEvent_t ev_in_free[2] = {};         // the conversion that last read buf.in0 / in1 has run
    int in_next = 0;                        // input buffer of the next set_state
};

namespace felbm {

// ELL width used by the FP32 sweeps: the longest row rounded up to one of
// the compiled widths; 0 (CSR sweeps) beyond 16.
static int ell_width(const HostMesh& h) {
    int w = h.max_degree;
    for (int c : {7, 9, 12, 16})
        if (w <= c) return c;
    return 0;
}

// Width of the incidence ELL used by the FP32 RHS gather: the most triangles
// at one node rounded up to a compiled width; 0 (CSR) beyond 12.
static int inc_width(const HostMesh& h) {
    int w = 0;
    for (int32_t i = 0; i < h.N; ++i) w = std::max(w, h.inc_ptr[i + 1] - h.inc_ptr[i]);
    for (int c : {6, 8, 12})
        if (w <= c) return c;
    return 0;
}

// Layout of the workspace; with base == nullptr only the size is computed.
static size_t carve(const HostMesh& h, bool dev32, void* base, DevMesh* dm, Bufs* b,
                    GroupTables* gtab = nullptr, AdjBufs* adj = nullptr) {
    Carver cv(base);
    size_t Np = pad64(h.N), Tp = pad64(h.T);
    size_t nnz = h.row_ptr[h.N], ninc = h.inc_ptr[h.N], nwinc = h.winc_ptr[h.N];
    size_t E = std::max<int32_t>(h.E, 1);
    DevMesh d{};
    d.tri = cv.take<int32_t>(3 * Tp);
    d.area = cv.take<double>(Tp);
    d.grad = cv.take<double>(6 * Tp);
    d.area32 = cv.take<float>(Tp);
    d.grad32 = cv.take<float>(6 * Tp);
    d.nbr = cv.take<int32_t>(3 * Tp);
    d.nbr_slot = cv.take<int32_t>(3 * Tp);
    d.row_ptr = cv.take<int32_t>(h.N + 1);
    d.col = cv.take<int32_t>(nnz);
    d.mval = cv.take<double>(nnz);
    d.lval = cv.take<double>(nnz);
    d.inv_lumped = cv.take<double>(Np);
    d.mval32 = cv.take<float>(nnz);
    const int ellw = ell_width(h);
    d.ell_w = ellw;
    d.ell_col = cv.take<int32_t>((size_t)std::max(ellw, 1) * Np);
    d.ell_loc = cv.take<uint16_t>((size_t)std::max(ellw, 1) * Np);
    d.ell_val = cv.take<float>((size_t)std::max(ellw, 1) * Np);
    d.n_tiles = (int32_t)h.tile_ptr.size() - 1;
    d.tiled_ok = ellw > 0 && h.max_halo <= kHaloMax;
    d.tile_ptr = cv.take<int32_t>(h.tile_ptr.size());
    d.halo_ptr = cv.take<int32_t>(h.halo_ptr.size());
    d.halo = cv.take<int32_t>(std::max<size_t>(h.halo.size(), 1));
    d.ell_lval = cv.take<double>((size_t)std::max(ellw, 1) * Np);
    const int iw = inc_width(h);
    d.iell_w = iw;
    d.iell_tri = cv.take<int32_t>((size_t)std::max(iw, 1) * Np);
    d.iell_bx32 = cv.take<float>((size_t)std::max(iw, 1) * Np);
    d.iell_by32 = cv.take<float>((size_t)std::max(iw, 1) * Np);
    d.inv_lumped32 = cv.take<float>(Np);
    d.lumped = cv.take<double>(Np);
    d.inv_vol = cv.take<double>(Np);
    d.inc_ptr = cv.take<int32_t>(h.N + 1);
    d.inc_tri = cv.take<int32_t>(ninc);
    d.inc_bx = cv.take<double>(ninc);
    d.inc_by = cv.take<double>(ninc);
    d.inc_bx32 = cv.take<float>(ninc);
    d.inc_by32 = cv.take<float>(ninc);
    d.wall_a = cv.take<int32_t>(E);
    d.wall_b = cv.take<int32_t>(E);
    d.wall_id = cv.take<int32_t>(E);
    d.wall_phi = cv.take<double>(E);
    d.wall_len = cv.take<double>(E);
    d.wall_nx = cv.take<double>(E);
    d.wall_ny = cv.take<double>(E);
    d.winc_ptr = cv.take<int32_t>(h.N + 1);
    d.winc_edge = cv.take<int32_t>(std::max<size_t>(nwinc, 1));
    d.x = cv.take<double>(Np);
    d.y = cv.take<double>(Np);
    d.perm = cv.take<int32_t>(h.N);
    d.iperm = cv.take<int32_t>(h.N);
    Bufs bb{};
    bb.C = cv.take<double>(Np);
    if (!dev32) {
        bb.psi = cv.take<double>(18 * Np);
        bb.p = cv.take<double>(Np);
        bb.ux = cv.take<double>(Np);
        bb.uy = cv.take<double>(Np);
        bb.mu = cv.take<double>(Np);
        bb.gmu = cv.take<double>(2 * Tp);
        bb.lmu = bb.gmu;
        bb.R = cv.take<double>(18 * (size_t)h.T);
    } else {
        bb.dpsi = cv.take<float>(18 * Np);
        bb.p32 = cv.take<float>(Np);
        bb.ux32 = cv.take<float>(Np);
        bb.uy32 = cv.take<float>(Np);
        bb.mu32 = cv.take<float>(Np);
        bb.gmu32 = cv.take<float>(2 * Tp);
        bb.lmu32 = bb.gmu32;
        bb.R32 = cv.take<float>(18 * ((size_t)h.T + 1));   // row T: zeros (incidence padding)
    }
    bb.rhs = cv.take<double>(18 * Np);
    bb.x0 = cv.take<double>(18 * Np);
    bb.x1 = cv.take<double>(18 * Np);
    bb.x64 = bb.x0;
    bb.rho64 = bb.x1;
    bb.r32 = cv.take<float>(18 * Np);
    bb.e0 = cv.take<float>(18 * Np);
    bb.e1 = cv.take<float>(18 * Np);
    bb.stage = cv.take<double>(18 * Np);
    bb.in0 = cv.take<double>(18 * Np);
    bb.in1 = cv.take<double>(18 * Np);
    bb.diag_part = cv.take<double>((size_t)kDiagBlocks * kDiagSlots);
    bb.diag_out = cv.take<double>(kDiagSlots);
    bb.Cdiag = cv.take<double>(Np);
    bb.diag_done = cv.take<unsigned>(1);
    bb.kerr = cv.take<unsigned>(1);
    GroupTables g{};
    const size_t G = std::max<int32_t>(h.G, 1);
    g.node_begin = cv.take<int32_t>(G);
    g.node_end = cv.take<int32_t>(G);
    g.tri_begin = cv.take<int32_t>(G);
    g.tri_end = cv.take<int32_t>(G);
    g.wall_ptr = cv.take<int32_t>(G + 1);
    g.wall_edge = cv.take<int32_t>(E);
    g.reqs = cv.take<DiagReq>(G);
    g.out = cv.take<double>(G * kDiagSlots);
    g.cta_groups = cv.take<int32_t>(G);
    if (gtab) *gtab = g;
    AdjBufs ad{};
    if (!dev32) {
        ad.lam = cv.take<double>(18 * Np);
        ad.lamhat = cv.take<double>(18 * Np);
        ad.lamR = cv.take<double>(18 * (size_t)h.T);
        ad.lamE = cv.take<double>(9 * (size_t)h.T);
        ad.lamG = cv.take<double>(2 * Tp);
        ad.lamMu = cv.take<double>(Np);
        ad.lamC = cv.take<double>(Np);
        ad.lamP = cv.take<double>(Np);
        ad.lamUx = cv.take<double>(Np);
        ad.lamUy = cv.take<double>(Np);
        ad.dphi = cv.take<double>(E);
        ad.kval = cv.take<double>(nnz);
    }
    if (adj) *adj = ad;
    if (dm) {
        d.N = h.N;
        d.T = h.T;
        d.E = h.E;
        d.Np = (int32_t)Np;
        d.Tp = (int32_t)Tp;
        d.period_y = h.period[1];
        *dm = d;
    }
    if (b) *b = bb;
    return cv.off + 256;
}

static int check_params(const felbm_params* p) {
    if (!p || !(p->dt > 0.0) || !(p->tau_l > 0.0) || !(p->tau_v > 0.0) || !(p->rho_l > 0.0) ||
        !(p->rho_v > 0.0) || !(p->kappa >= 0.0) || !(p->beta >= 0.0) || !(p->mobility >= 0.0) ||
        p->lap_mode < 0 || p->lap_mode > 1 || p->solver_iters < 0 || p->solver_iters == 1 ||
        p->solver_iters > 1000 || p->solver_rounds < 0 || p->solver_rounds > 20 ||
        p->solver_mode < 0 || p->solver_mode > 1 ||
        p->n_wall_ids < 0 || p->n_wall_ids > FELBM_MAX_WALL_IDS ||
        (p->lapmu_mode != FELBM_LAPMU_FACE && p->lapmu_mode != FELBM_LAPMU_NODAL)) {
        set_error("felbm: invalid params (dt, tau, rho > 0; kappa, beta, mobility >= 0; lap_mode 0/1; "
                  "solver_mode 0/1; solver_iters 0 or 2..1000; solver_rounds 0..20; lapmu_mode 0/1)");
        return FELBM_ERR_INVALID_ARG;
    }
    if (p->precision != FELBM_FP64 && p->precision != FELBM_FP32_DEV) {
        set_error("felbm: unknown precision");
        return FELBM_ERR_UNSUPPORTED;
    }
    if (p->precision == FELBM_FP32_DEV && (p->solver_mode != FELBM_SOLVER_MIXED || p->solver_rounds > 1)) {
        set_error("felbm: FELBM_FP32_DEV solves in FP32 (solver_mode MIXED, solver_rounds 0 or 1)");
        return FELBM_ERR_UNSUPPORTED;
    }
    return FELBM_OK;
}

template <class T>
static cudaError_t up(const T* dst, const std::vector<T>& src, cudaStream_t s) {
    if (src.empty()) return cudaSuccess;
    return cudaMemcpyAsync(const_cast<T*>(dst), src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s);
}

static unsigned grid_for(int n, int block) { return (unsigned)((n + block - 1) / block); }

// Launch with or without programmatic dependent launch (PDL).
template <typename... KArgs, typename... Args>
static void launch_k(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// One FP32 Chebyshev sweep: the ELL kernel of the mesh's width, else CSR.
// pdl: the previous launch on the stream is a sweep (a kernel that waits).
// parts: threads per node for the store sweeps (1, 2, 3 or 6; autotuned).
// The tiled store step (k_sweep_tile32): a persistent grid of one block per
// SM walking the (tile, part) items through its pipeline stages.
template <int kW, int kParts>
static void launch_tile_w(const felbm_state* st, const DevMesh& m, const Bufs& b, cudaStream_t s, const float* cur,
                          float* nxt, float tau, bool pdl) {
    cudaLaunchConfig_t cfg{};
    const int items = m.n_tiles * kParts;
    cfg.gridDim = dim3((unsigned)std::min(items, st->n_sm));
    cfg.blockDim = dim3(kTileThreads);
    cfg.dynamicSmemBytes = tile_stages(18 / kParts, kW) * tile_stage_bytes(18 / kParts, kW);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    if constexpr (tile_stages(18 / kParts, kW) >= 2) cudaLaunchKernelEx(&cfg, k_sweep_tile32<kW, kParts>, m, b, cur, nxt, tau);
}

// Parts of the 18 right-hand sides per work item of the tiled step: 3 if
// requested (1, 2 or 3) and two or more stages fit the shared memory of a
// block, else 6; 0 if not even that fits.
static bool tile_fits(int parts, int ell_w, int smem_optin) {
    const int nq = 18 / parts;
    return tile_stages(nq, ell_w) >= 2 &&
           tile_stages(nq, ell_w) * tile_stage_bytes(nq, ell_w) + 1024 <= (size_t)smem_optin;
}
static int tile_parts(const felbm_state* st, int ell_w) {
    for (int p : {3, 6})
        if (p >= st->sweep_parts && tile_fits(p, ell_w, st->smem_optin)) return p;
    return 0;
}

template <int kW>
static void launch_tile(const felbm_state* st, const DevMesh& m, const Bufs& b, cudaStream_t s, const float* cur,
                        float* nxt, float tau, bool pdl) {
    if (tile_parts(st, kW) == 3)
        launch_tile_w<kW, 3>(st, m, b, s, cur, nxt, tau, pdl);
    else
        launch_tile_w<kW, 6>(st, m, b, s, cur, nxt, tau, pdl);
}

// Shared memory beyond the default 48 KB for the tiled steps that fit.
template <int kW>
static cudaError_t allow_tile_smem(int smem_optin) {
    cudaError_t e = cudaSuccess;
    auto set = [&](auto kern, int parts) {
        const size_t bytes = tile_stages(18 / parts, kW) * tile_stage_bytes(18 / parts, kW);
        if (e == cudaSuccess && tile_fits(parts, kW, smem_optin))
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    };
    if constexpr (tile_stages(6, kW) >= 2) set(k_sweep_tile32<kW, 3>, 3);
    if constexpr (tile_stages(3, kW) >= 2) set(k_sweep_tile32<kW, 6>, 6);
    return e;
}

template <int kFinal, int kW>
static void launch_sweep_w(felbm_state* st, const DevMesh& m, const Bufs& b, cudaStream_t s, const float* cur,
                           float* nxt, float tau, int have_x64, bool pdl) {
    if constexpr (kFinal == kStore) {
        // the tiled form covers whole meshes (not the tiled prefix of a hybrid batch schedule)
        if (st->sweep_tiled && m.tiled_ok && m.N == st->dm.N && tile_parts(st, kW) > 0) {
            launch_tile<kW>(st, m, b, s, cur, nxt, tau, pdl);
            return;
        }
    }
    const dim3 block(128);
    const int parts = kFinal == kUpdateDev ? 1 : st->sweep_parts;
    const dim3 grid(grid_for(m.N, 128) * parts);
    switch (parts) {
        case 1:
            launch_k(pdl, k_sweep32<kFinal, kW, 1>, grid, block, s, m, st->phys, b, cur, nxt, tau, have_x64, 0.0f);
            break;
        case 3:
            if constexpr (kFinal != kUpdateDev)
                launch_k(pdl, k_sweep32<kFinal, kW, 3>, grid, block, s, m, st->phys, b, cur, nxt, tau, have_x64, 0.0f);
            break;
        case 6:
            if constexpr (kFinal != kUpdateDev)
                launch_k(pdl, k_sweep32<kFinal, kW, 6>, grid, block, s, m, st->phys, b, cur, nxt, tau, have_x64, 0.0f);
            break;
        default:
            if constexpr (kFinal != kUpdateDev)
                launch_k(pdl, k_sweep32<kFinal, kW, 2>, grid, block, s, m, st->phys, b, cur, nxt, tau, have_x64, 0.0f);
    }
}

template <int kFinal>
static void launch_sweep(felbm_state* st, const DevMesh& m, const Bufs& b, cudaStream_t s, const float* cur,
                         float* nxt, float tau, int have_x64, bool pdl) {
    pdl = pdl && st->use_pdl;
    switch (m.ell_w) {
        case 7:
            launch_sweep_w<kFinal, 7>(st, m, b, s, cur, nxt, tau, have_x64, pdl);
            break;
        case 9:
            launch_sweep_w<kFinal, 9>(st, m, b, s, cur, nxt, tau, have_x64, pdl);
            break;
        case 12:
            launch_sweep_w<kFinal, 12>(st, m, b, s, cur, nxt, tau, have_x64, pdl);
            break;
        case 16:
            launch_sweep_w<kFinal, 16>(st, m, b, s, cur, nxt, tau, have_x64, pdl);
            break;
        default:
            k_cheb32<kFinal><<<grid_for(m.N, 128), 128, 0, s>>>(m, st->phys, b, cur, nxt, tau, have_x64);
    }
}

// ELL widths with compiled gathered solve steps
static bool gathered_width(int ell_w) { return ell_w == 7 || ell_w == 9 || ell_w == 12 || ell_w == 16; }

// The first step of the FP32 time-step solve with x_0 formed from b (gathered
// ELL widths and the untiled steps only).
template <int kW>
static void launch_first_w(felbm_state* st, const DevMesh& m, const Bufs& b, cudaStream_t s, float* nxt,
                           float tau, float tau0, bool pdl) {
    const dim3 block(128);
    const int parts = st->sweep_parts;
    const dim3 grid(grid_for(m.N, 128) * parts);
    switch (parts) {
        case 1: launch_k(pdl, k_sweep32<kStore, kW, 1, true>, grid, block, s, m, st->phys, b, nullptr, nxt, tau, 0, tau0); break;
        case 3: launch_k(pdl, k_sweep32<kStore, kW, 3, true>, grid, block, s, m, st->phys, b, nullptr, nxt, tau, 0, tau0); break;
        case 6: launch_k(pdl, k_sweep32<kStore, kW, 6, true>, grid, block, s, m, st->phys, b, nullptr, nxt, tau, 0, tau0); break;
        default: launch_k(pdl, k_sweep32<kStore, kW, 2, true>, grid, block, s, m, st->phys, b, nullptr, nxt, tau, 0, tau0);
    }
}

// Only called when gathered_width(m.ell_w) (first_from_rhs checks it).
static void launch_first(felbm_state* st, const DevMesh& m, const Bufs& b, cudaStream_t s, float* nxt, float tau,
                         float tau0, bool pdl) {
    pdl = pdl && st->use_pdl;
    switch (m.ell_w) {
        case 7: launch_first_w<7>(st, m, b, s, nxt, tau, tau0, pdl); break;
        case 9: launch_first_w<9>(st, m, b, s, nxt, tau, tau0, pdl); break;
        case 12: launch_first_w<12>(st, m, b, s, nxt, tau, tau0, pdl); break;
        default: launch_first_w<16>(st, m, b, s, nxt, tau, tau0, pdl);
    }
}

// Whether the FP32 time step forms x_0 inside its first solve step (then the
// RHS kernel stores b only): one correction round, gathered steps, at least
// two steps after the first, no residual check, an ELL width with kernels.
static bool first_from_rhs(const felbm_state* st, const DevMesh& m) {
    return st->dev32 && st->rounds == 1 && st->sweeps > 2 && !st->check && !st->sweep_tiled &&
           gathered_width(m.ell_w);
}

// Enqueue the mass solve for the right-hand side in b.rhs (first iterate
// already written, unless from_rhs).  into_psi: add the increment to psi (time step); else
// leave the solution in x1/x0 (FP64 mode, returned) or x64 (mixed mode).
// bufs: the buffers the solve reads and writes (the state's own, or another
// set of scratch buffers with the same layout).
static const double* enqueue_solve(felbm_state* st, const DevMesh& m, const Bufs& b, cudaStream_t s,
                                   bool into_psi, bool after_release = false, bool from_rhs = false) {
    const unsigned grid = grid_for(m.N, 128);
    if (st->mode == FELBM_SOLVER_FP64) {
        const double* result = b.x1;
        for (int k = 1; k < st->sweeps; ++k) {
            const double* cur = (k & 1) ? b.x1 : b.x0;
            double* prev = (k & 1) ? b.x0 : b.x1;
            k_cheb<<<grid, 128, 0, s>>>(m, b, cur, prev, st->cheb_a[k], st->cheb_c[k], k == 1,
                                        into_psi && k == st->sweeps - 1);
            result = prev;
        }
        return result;
    }
    float* A = b.e1;
    float* B = b.e0;
    const int have_x64 = st->rounds > 1;
    for (int r = 0; r < st->rounds; ++r) {
        float* cur = A;
        float* prv = B;
        for (int k = 1; k < st->sweeps; ++k) {
            const float tau = (float)st->tau[k];
            const bool last = r == st->rounds - 1 && k == st->sweeps - 1;
            // the previous launch is a sweep of this round, or a kernel that released its dependents
            bool pdl = k > 1 || (k == 1 && r == 0 && after_release);
            if (last && st->check) {
                if (st->dev32)
                    k_solve_resid<false><<<kDiagBlocks, kBlock, 0, s>>>(m, b, cur, b.diag_part);
                else
                    k_solve_resid<true><<<kDiagBlocks, kBlock, 0, s>>>(m, b, cur, b.diag_part);
                k_solve_resid_final<<<1, 1, 0, s>>>(b.diag_part, kDiagBlocks, b.diag_out + kSolveResSlot);
                pdl = false;
            }
            if (from_rhs && r == 0 && k == 1)
                launch_first(st, m, b, s, prv, tau, (float)st->tau[0], pdl);
            else if (!last)
                launch_sweep<kStore>(st, m, b, s, cur, prv, tau, have_x64, pdl);
            else if (!into_psi)
                launch_sweep<kAddX64>(st, m, b, s, cur, prv, tau, have_x64, pdl);
            else if (st->dev32)
                launch_sweep<kUpdateDev>(st, m, b, s, cur, prv, tau, have_x64, pdl);
            else
                launch_sweep<kAddPsi>(st, m, b, s, cur, prv, tau, have_x64, pdl);
            std::swap(cur, prv);
        }
        if (r < st->rounds - 1) {
            k_refine<<<grid, 128, 0, s>>>(m, b, cur, prv, r == 0, st->tau[0]);
            A = prv;
            B = cur;
        }
    }
    return b.x64;
}

static int solve_launches(const felbm_state* st) {
    return st->mode == FELBM_SOLVER_FP64 ? st->sweeps - 1
                                         : st->rounds * (st->sweeps - 1) + (st->rounds - 1);
}

static int step_launches(const felbm_state* st) { return (st->dev32 ? 4 : 5) + solve_launches(st); }

int set_schedule(felbm_state* st, int32_t max_nodes);

// Enqueue the kernels of one time step on stream s (optionally with the
// phase events, recorded as external event nodes of the captured graph).
static void enqueue_step(felbm_state* st, cudaStream_t s) {
    const DevMesh& m = st->dm;
    const Bufs& b = st->buf;
    auto mark = [&](int k) {
        if (st->timing) cudaEventRecordWithFlags(st->ev[k], s, cudaEventRecordExternal);
    };
    mark(0);
    if (st->dev32) {
        // small batch members: one CTA each, on a side branch of the graph
        if (st->n_cta > 0) {
            ChebCoef cf{};
            for (int k = 1; k < st->sweeps && k < kMaxSweeps; ++k) cf.tau[k] = (float)st->tau[k];
            cudaEventRecord(st->ev_fork, s);
            cudaStreamWaitEvent(st->side_stream, st->ev_fork, 0);
            k_step_cta32<<<st->n_cta, kCtaThreads, 0, st->side_stream>>>(m, st->phys, b, st->gt, st->gt.cta_groups,
                                                                         cf, st->sweeps, (float)st->tau[0]);
            cudaEventRecord(st->ev_join, st->side_stream);
        }
        // the rest (a prefix of nodes and triangles): tiled kernels
        DevMesh mt = m;
        mt.N = st->tiled_N;
        mt.T = st->tiled_T;
        // collision is folded into the element, RHS and update kernels
        mark(1);
        if (mt.N > 0) {
            // programmatic dependent launch along the chain when no phase
            // events sit between the kernels
            const bool chain = st->use_pdl && !st->timing;
            switch (mt.ell_w) {
                case 7: k_mu32<7><<<grid_for(mt.N, kBlock), kBlock, 0, s>>>(mt, st->phys, b); break;
                case 9: k_mu32<9><<<grid_for(mt.N, kBlock), kBlock, 0, s>>>(mt, st->phys, b); break;
                case 12: k_mu32<12><<<grid_for(mt.N, kBlock), kBlock, 0, s>>>(mt, st->phys, b); break;
                case 16: k_mu32<16><<<grid_for(mt.N, kBlock), kBlock, 0, s>>>(mt, st->phys, b); break;
                default: k_mu32<0><<<grid_for(mt.N, kBlock), kBlock, 0, s>>>(mt, st->phys, b);
            }
            mark(2);
            if (st->phys.lapmu_nodal)
                launch_k(chain, k_lmu32, dim3(grid_for(mt.N, kBlock)), dim3(kBlock), s, mt, st->phys, b);
            else
                launch_k(chain, k_gradmu32, dim3(grid_for(mt.T, kBlock)), dim3(kBlock), s, mt, b);
            mark(3);
            launch_k(chain, k_element32, dim3(grid_for(mt.T, 128)), dim3(128), s, mt, st->phys, b);
            mark(4);
            const bool from_rhs = first_from_rhs(st, mt);
            const float tau0 = (float)st->tau[0];
            const dim3 gn(grid_for(mt.N, 128)), bn(128);
            switch (mt.iell_w * 2 + (from_rhs ? 1 : 0)) {
                case 12: launch_k(chain, k_rhs32<6, true>, gn, bn, s, mt, st->phys, b, tau0); break;
                case 13: launch_k(chain, k_rhs32<6, false>, gn, bn, s, mt, st->phys, b, tau0); break;
                case 16: launch_k(chain, k_rhs32<8, true>, gn, bn, s, mt, st->phys, b, tau0); break;
                case 17: launch_k(chain, k_rhs32<8, false>, gn, bn, s, mt, st->phys, b, tau0); break;
                case 24: launch_k(chain, k_rhs32<12, true>, gn, bn, s, mt, st->phys, b, tau0); break;
                case 25: launch_k(chain, k_rhs32<12, false>, gn, bn, s, mt, st->phys, b, tau0); break;
                default:
                    if (from_rhs)
                        launch_k(chain, k_rhs32<0, false>, gn, bn, s, mt, st->phys, b, tau0);
                    else
                        launch_k(chain, k_rhs32<0, true>, gn, bn, s, mt, st->phys, b, tau0);
            }
            mark(5);
            enqueue_solve(st, mt, st->buf, s, true, chain, from_rhs);
        } else {
            mark(2);
            mark(3);
            mark(4);
            mark(5);
        }
        if (st->n_cta > 0) cudaStreamWaitEvent(s, st->ev_join, 0);
        mark(6);
        return;
    }
    k_collide<<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, st->phys, b, 1);
    mark(1);
    k_mu<<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, st->phys, b);
    mark(2);
    if (st->phys.lapmu_nodal)
        k_lmu<<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, st->phys, b);
    else
        k_gradmu<<<grid_for(m.T, kBlock), kBlock, 0, s>>>(m, b);
    mark(3);
    k_element<<<grid_for(m.T, 128), 128, 0, s>>>(m, st->phys, b);
    mark(4);
    if (st->mode == FELBM_SOLVER_FP64)
        k_rhs<false><<<grid_for(m.N, 128), 128, 0, s>>>(m, st->phys, b, st->inv_theta);
    else
        k_rhs<true><<<grid_for(m.N, 128), 128, 0, s>>>(m, st->phys, b, st->tau[0]);
    mark(5);
    enqueue_solve(st, st->dm, st->buf, s, true);
    mark(6);
}

}  // namespace felbm

using namespace felbm;

extern "C" {

int felbm_workspace_bytes(const felbm_mesh* mesh, const felbm_params* params, size_t* bytes) {
    if (!mesh || !bytes) {
        set_error("felbm_workspace_bytes: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    int rc = check_params(params);
    if (rc) return rc;
    *bytes = carve(mesh->h, params->precision == FELBM_FP32_DEV, nullptr, nullptr, nullptr);
    return FELBM_OK;
}

int felbm_init(const felbm_mesh* mesh, const felbm_params* params, const double* C0, const double* p0,
               const double* u0, void* d_workspace, size_t workspace_bytes, void* stream, felbm_state** out) {
    if (!mesh || !C0 || !out) {
        set_error("felbm_init: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    *out = nullptr;
    int rc = check_params(params);
    if (rc) return rc;
    const HostMesh& h = mesh->h;
    for (int32_t e = 0; e < h.E; ++e)
        if (h.wall_id[e] >= params->n_wall_ids) {
            set_error("felbm_init: a wall id has no phi_c (n_wall_ids too small)");
            return FELBM_ERR_INVALID_ARG;
        }
    const bool dev32 = params->precision == FELBM_FP32_DEV;
    size_t need = carve(h, dev32, nullptr, nullptr, nullptr);
    if (!d_workspace || workspace_bytes < need || (reinterpret_cast<uintptr_t>(d_workspace) & 255)) {
        set_error("felbm_init: workspace missing, not 256-byte aligned or smaller than felbm_workspace_bytes");
        return FELBM_ERR_WORKSPACE;
    }
    felbm_state* st = new (std::nothrow) felbm_state;
    if (!st) {
        set_error("felbm_init: out of host memory");
        return FELBM_ERR_INVALID_ARG;
    }
    st->hm = h;
    st->prm = *params;
    st->stream = static_cast<cudaStream_t>(stream);
    st->dev32 = dev32;
    carve(h, dev32, d_workspace, &st->dm, &st->buf, &st->gt, &st->adj);
    Phys& ph = st->phys;
    ph.dt = params->dt;
    ph.tau_l = params->tau_l;
    ph.tau_v = params->tau_v;
    ph.rho_l = params->rho_l;
    ph.rho_v = params->rho_v;
    ph.kappa = params->kappa;
    ph.beta = params->beta;
    ph.mobility = params->mobility;
    ph.lapmu_nodal = params->lapmu_mode == FELBM_LAPMU_NODAL;
    // lval = -2 K_ij / (s |patch_i|); the lumped P1 Laplacian is -K_ij / (|patch_i| / 3)
    ph.lapmu_fac = (params->lap_mode == FELBM_LAP_PAPER ? 1.0 : 2.0 / 3.0) * 1.5;
    ph.dt_f = (float)params->dt;
    ph.dt3_f = (float)(params->dt / 3.0);
    ph.dt2h_f = (float)(0.5 * params->dt * params->dt);
    ph.inv_tau_l_f = (float)(1.0 / params->tau_l);
    ph.inv_tau_v_f = (float)(1.0 / params->tau_v);
    ph.rho_v_f = (float)params->rho_v;
    ph.drho_f = (float)(params->rho_l - params->rho_v);
    ph.mobility_f = (float)params->mobility;

    // Chebyshev coefficients for the spectrum [1/4, 1] of m^{-1} M11
    st->mode = params->solver_mode;
    // FP32-deviation states take 10 steps per solve (bound 2*3^-10 on the
    // increment): against the FP64 path that leaves contact angles within
    // 2e-4 degree, mass drift below 1e-8 and C within 1e-7 of the oracle
    // after 20 steps, the FP32 level of the other terms
    st->sweeps = params->solver_iters ? params->solver_iters
                                      : (st->mode == FELBM_SOLVER_FP64 ? 32 : (dev32 ? 10 : 14));
    st->rounds = st->mode == FELBM_SOLVER_FP64 ? 1 : (params->solver_rounds ? params->solver_rounds : (dev32 ? 1 : 3));
    const double lmin = 0.25, lmax = 1.0;
    const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma1 = theta / delta;
    st->inv_theta = 1.0 / theta;
    st->cheb_a.assign(st->sweeps, 0.0);
    st->cheb_c.assign(st->sweeps, 0.0);
    double rho_prev = 1.0 / sigma1;
    for (int k = 1; k < st->sweeps; ++k) {
        double rho = 1.0 / (2.0 * sigma1 - rho_prev);
        st->cheb_a[k] = rho * rho_prev;
        st->cheb_c[k] = 2.0 * rho / delta;
        rho_prev = rho;
    }
    // FP32 solves: Richardson steps 1/lambda_j at the Chebyshev roots
    // lambda_j = theta + delta cos((2j+1) pi / 2K), j = 0..K-1, in the order
    // j = 0, K-1, 1, K-2, ... (largest and smallest root alternately)
    st->tau.assign(st->sweeps, 1.0);
    {
        const int K = st->sweeps;
        for (int k = 0; k < K; ++k) {
            const int j = (k & 1) ? K - 1 - k / 2 : k / 2;
            st->tau[k] = 1.0 / (theta + delta * std::cos((2.0 * j + 1.0) * 3.14159265358979323846 / (2.0 * K)));
        }
    }

    // host-side derived tables
    const double scale = params->lap_mode == FELBM_LAP_PAPER ? 1.0 : 2.0 / 3.0;
    std::vector<double> inv_vol(h.N), inv_lumped(h.N), lval(h.row_ptr[h.N]);
    std::vector<float> inv_lumped32(h.N), mval32(h.mass.begin(), h.mass.end());
    std::vector<double> wall_phi(h.E);
    for (int32_t e = 0; e < h.E; ++e) wall_phi[e] = params->phi_c[h.wall_id[e]];
    const int ellw = st->dm.ell_w;
    std::vector<int32_t> ell_col((size_t)std::max(ellw, 1) * st->dm.Np, 0);
    std::vector<float> ell_val((size_t)std::max(ellw, 1) * st->dm.Np, 0.0f);
    std::vector<double> ell_lval((size_t)std::max(ellw, 1) * st->dm.Np, 0.0);
    if (const char* env = std::getenv("FELBM_PDL")) st->use_pdl = std::atoi(env) != 0;
    for (int32_t i = 0; i < h.N; ++i) {
        inv_vol[i] = 1.0 / (scale * h.patch[i]);
        inv_lumped[i] = 1.0 / h.lumped[i];
        inv_lumped32[i] = (float)inv_lumped[i];
        for (int32_t k = h.row_ptr[i]; k < h.row_ptr[i + 1]; ++k) lval[k] = -2.0 * h.stiff[k] * inv_vol[i];
    }
    for (int32_t i = 0; i < h.N && ellw > 0; ++i) {
        int32_t r0 = h.row_ptr[i], len = h.row_ptr[i + 1] - r0;
        for (int k = 0; k < ellw; ++k) {
            size_t at = (size_t)k * st->dm.Np + i;
            ell_col[at] = k < len ? h.col[r0 + k] : i;
            ell_val[at] = k < len ? (float)h.mass[r0 + k] : 0.0f;
            ell_lval[at] = k < len ? lval[r0 + k] : 0.0;
        }
    }
    // the ELL columns as indices into the staged row of the node's tile:
    // [0, span) the 16-byte aligned run a0 = tile start rounded down to 4,
    // then the tile's halo in its sorted order
    std::vector<uint16_t> ell_loc((size_t)std::max(ellw, 1) * st->dm.Np, 0);
    if (st->dm.tiled_ok) {
        const int32_t ntile = st->dm.n_tiles;
        for (int32_t t = 0; t < ntile; ++t) {
            const int32_t s0 = h.tile_ptr[t], s1 = h.tile_ptr[t + 1], a0 = s0 & ~3;
            const int32_t span = ((s1 + 3) & ~3) - a0;
            const int32_t* hb = h.halo.data() + h.halo_ptr[t];
            const int32_t* he = h.halo.data() + h.halo_ptr[t + 1];
            for (int32_t i = s0; i < s1; ++i)
                for (int k = 0; k < ellw; ++k) {
                    const size_t at = (size_t)k * st->dm.Np + i;
                    const int32_t c = ell_col[at];
                    int32_t loc;
                    if (c >= s0 && c < s1) {
                        loc = c - a0;
                    } else {
                        const int32_t* f = std::lower_bound(hb, he, c);
                        if (f == he || *f != c) {
                            set_error("felbm_init: internal error, a row entry outside its tile's halo");
                            delete st;
                            return FELBM_ERR_BAD_MESH;
                        }
                        loc = span + (int32_t)(f - hb);
                    }
                    ell_loc[at] = (uint16_t)loc;
                }
        }
    }
    auto pad_tri = [&](const std::vector<int32_t>& src, int rows) {
        std::vector<int32_t> outv((size_t)rows * st->dm.Tp, 0);
        for (int r = 0; r < rows; ++r)
            std::copy(src.begin() + (size_t)r * h.T, src.begin() + (size_t)(r + 1) * h.T,
                      outv.begin() + (size_t)r * st->dm.Tp);
        return outv;
    };
    auto pad_trid = [&](const std::vector<double>& src, int rows) {
        std::vector<double> outv((size_t)rows * st->dm.Tp, 0.0);
        for (int r = 0; r < rows; ++r)
            std::copy(src.begin() + (size_t)r * h.T, src.begin() + (size_t)(r + 1) * h.T,
                      outv.begin() + (size_t)r * st->dm.Tp);
        return outv;
    };
    std::vector<int32_t> tri_p = pad_tri(h.tri, 3), nbr_p = pad_tri(h.nbr, 3), slot_p = pad_tri(h.nbr_slot, 3);
    std::vector<double> grad_p = pad_trid(h.grad, 6), area_p = pad_trid(h.area, 1);
    std::vector<float> grad32_p(grad_p.begin(), grad_p.end()), area32_p(area_p.begin(), area_p.end());
    std::vector<float> inc_bx32(h.inc_bx.begin(), h.inc_bx.end()), inc_by32(h.inc_by.begin(), h.inc_by.end());
    cudaStream_t s = st->stream;
    const DevMesh& d = st->dm;
    auto fail = [&](cudaError_t e, const char* what) {
        int r = cuda_fail(e, what);
        delete st;
        return r;
    };
    cudaError_t e = cudaSuccess;
#define UP(dst, src) \
    if (e == cudaSuccess) e = up(dst, src, s)
    UP(d.tri, tri_p);
    UP(d.area, area_p);
    UP(d.grad, grad_p);
    UP(d.grad32, grad32_p);
    UP(d.area32, area32_p);
    UP(d.nbr, nbr_p);
    UP(d.nbr_slot, slot_p);
    UP(d.row_ptr, h.row_ptr);
    UP(d.col, h.col);
    UP(d.mval, h.mass);
    UP(d.lval, lval);
    UP(d.inv_lumped, inv_lumped);
    UP(d.mval32, mval32);
    UP(d.ell_col, ell_col);
    UP(d.ell_val, ell_val);
    UP(d.ell_loc, ell_loc);
    UP(d.tile_ptr, h.tile_ptr);
    UP(d.halo_ptr, h.halo_ptr);
    UP(d.halo, h.halo);
    if (e == cudaSuccess) e = cudaMemsetAsync(st->buf.kerr, 0, sizeof(unsigned), s);
    int cur_dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&cur_dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&st->n_sm, cudaDevAttrMultiProcessorCount, cur_dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&st->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, cur_dev);
    if (e == cudaSuccess && st->dm.tiled_ok) {
        switch (ellw) {
            case 7: e = allow_tile_smem<7>(st->smem_optin); break;
            case 9: e = allow_tile_smem<9>(st->smem_optin); break;
            case 12: e = allow_tile_smem<12>(st->smem_optin); break;
            case 16: e = allow_tile_smem<16>(st->smem_optin); break;
            default: break;
        }
    }
    UP(d.ell_lval, ell_lval);
    UP(d.inv_lumped32, inv_lumped32);
    UP(d.lumped, h.lumped);
    UP(d.inv_vol, inv_vol);
    UP(d.inc_ptr, h.inc_ptr);
    UP(d.inc_tri, h.inc_tri);
    UP(d.inc_bx, h.inc_bx);
    UP(d.inc_by, h.inc_by);
    UP(d.inc_bx32, inc_bx32);
    UP(d.inc_by32, inc_by32);
    {
        const int iw = st->dm.iell_w;
        const size_t Npi = st->dm.Np;
        std::vector<int32_t> itri((size_t)std::max(iw, 1) * Npi, h.T);
        std::vector<float> ibx((size_t)std::max(iw, 1) * Npi, 0.0f), iby(ibx.size(), 0.0f);
        for (int32_t i = 0; i < h.N && iw > 0; ++i)
            for (int32_t k = h.inc_ptr[i]; k < h.inc_ptr[i + 1]; ++k) {
                const size_t at = (size_t)(k - h.inc_ptr[i]) * Npi + i;
                itri[at] = h.inc_tri[k];
                ibx[at] = inc_bx32[k];
                iby[at] = inc_by32[k];
            }
        UP(d.iell_tri, itri);
        UP(d.iell_bx32, ibx);
        UP(d.iell_by32, iby);
        if (dev32 && e == cudaSuccess) e = cudaMemsetAsync(st->buf.R32 + (size_t)18 * h.T, 0, 18 * sizeof(float), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(st->buf.diag_done, 0, sizeof(unsigned), s);
    }
    UP(d.wall_a, h.wall_a);
    UP(d.wall_b, h.wall_b);
    UP(d.wall_id, h.wall_id);
    UP(d.wall_phi, wall_phi);
    UP(d.wall_len, h.wall_len);
    UP(d.wall_nx, h.wall_nx);
    UP(d.wall_ny, h.wall_ny);
    UP(d.winc_ptr, h.winc_ptr);
    UP(d.winc_edge, h.winc_edge);
    UP(d.x, h.x);
    UP(d.y, h.y);
    UP(d.perm, h.perm);
    UP(d.iperm, h.iperm);
    UP(st->gt.node_begin, h.grp_node_begin);
    UP(st->gt.node_end, h.grp_node_end);
    UP(st->gt.tri_begin, h.grp_tri_begin);
    UP(st->gt.tri_end, h.grp_tri_end);
    UP(st->gt.wall_ptr, h.grp_wall_ptr);
    UP(st->gt.wall_edge, h.grp_wall_edge);
    if (!dev32) UP(st->adj.kval, h.stiff);
#undef UP
    if (e != cudaSuccess) return fail(e, "felbm_init: upload");
    {
        double* dst = st->buf.stage;
        e = cudaMemcpyAsync(dst, C0, sizeof(double) * h.N, cudaMemcpyHostToDevice, s);
        dst += h.N;
        if (e == cudaSuccess && p0) {
            e = cudaMemcpyAsync(dst, p0, sizeof(double) * h.N, cudaMemcpyHostToDevice, s);
            dst += h.N;
        }
        if (e == cudaSuccess && u0) e = cudaMemcpyAsync(dst, u0, sizeof(double) * 2 * h.N, cudaMemcpyHostToDevice, s);
    }
    if (e != cudaSuccess) return fail(e, "felbm_init: upload C0, p0, u0");
    if (dev32)
        k_init_dev32<<<grid_for(h.N, kBlock), kBlock, 0, s>>>(st->dm, st->buf, st->buf.stage, p0 != nullptr,
                                                               u0 != nullptr);
    else
        k_init_state<<<grid_for(h.N, kBlock), kBlock, 0, s>>>(st->dm, st->phys, st->buf.stage, st->buf.psi,
                                                               p0 != nullptr, u0 != nullptr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(e, "felbm_init: launch");
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(e, "felbm_init: synchronize");
    e = cudaGetDevice(&st->device);
    if (e != cudaSuccess) return fail(e, "felbm_init: cudaGetDevice");
    // mass at t = 0 (for the drift)
    felbm_diag dg;
    *out = st;
    rc = felbm_diagnostics(st, nullptr, &dg);
    if (rc != FELBM_OK && rc != FELBM_ERR_NONFINITE) {
        *out = nullptr;
        delete st;
        return rc;
    }
    st->mass0 = dg.mass;
    st->gmass0.assign(h.G, dg.mass);
    if (h.G > 1) {   // one member: its mass is the mass
        std::vector<felbm_diag> gd(h.G);
        rc = felbm_diagnostics_groups(st, nullptr, h.G, gd.data());
        if (rc != FELBM_OK && rc != FELBM_ERR_NONFINITE) {
            *out = nullptr;
            delete st;
            return rc;
        }
        for (int32_t g = 0; g < h.G; ++g) st->gmass0[g] = gd[g].mass;
    }
    rc = set_schedule(st, 0);
    if (rc != FELBM_OK) {
        *out = nullptr;
        delete st;
        return rc;
    }
    return FELBM_OK;
}

}  // extern "C"

namespace felbm {

// Split the groups: those of at most max_nodes nodes run one CTA each.  The
// groups are laid out largest first, so the others form a prefix.
int set_schedule(felbm_state* st, int32_t max_nodes) {
    const HostMesh& h = st->hm;
    std::vector<int32_t> cta;
    int32_t tiled_N = 0, tiled_T = 0;
    for (int32_t g = 0; g < h.G; ++g) {
        if (st->dev32 && max_nodes > 0 && h.grp_size[g] <= max_nodes) {
            cta.push_back(g);
        } else {
            tiled_N = std::max(tiled_N, h.grp_node_end[g]);
            tiled_T = std::max(tiled_T, h.grp_tri_end[g]);
        }
    }
    for (int32_t g : cta)
        if (h.grp_node_begin[g] < tiled_N || h.grp_tri_begin[g] < tiled_T) {
            set_error("felbm: batch schedule needs the small members after the large ones");
            return FELBM_ERR_INVALID_ARG;
        }
    if (st->sweeps >= kMaxSweeps && !cta.empty()) {
        set_error("felbm: too many solver sweeps for the per-member CTA schedule");
        return FELBM_ERR_UNSUPPORTED;
    }
    if (!cta.empty()) {
        if (!st->side_stream) FELBM_CUDA(cudaStreamCreateWithFlags(&st->side_stream, cudaStreamNonBlocking));
        if (!st->ev_fork) FELBM_CUDA(cudaEventCreateWithFlags(&st->ev_fork, cudaEventDisableTiming));
        if (!st->ev_join) FELBM_CUDA(cudaEventCreateWithFlags(&st->ev_join, cudaEventDisableTiming));
        FELBM_CUDA(cudaMemcpyAsync(st->gt.cta_groups, cta.data(), sizeof(int32_t) * cta.size(),
                                   cudaMemcpyHostToDevice, st->stream));
        FELBM_CUDA(cudaStreamSynchronize(st->stream));
    }
    st->cta_max_nodes = cta.empty() ? 0 : max_nodes;
    st->n_cta = (int32_t)cta.size();
    st->tiled_N = tiled_N;
    st->tiled_T = tiled_T;
    return FELBM_OK;
}

}  // namespace felbm

extern "C" {

static int build_graph(felbm_state* st) {
    if (!st->cap_stream) FELBM_CUDA(cudaStreamCreateWithFlags(&st->cap_stream, cudaStreamNonBlocking));
    FELBM_CUDA(cudaStreamBeginCapture(st->cap_stream, cudaStreamCaptureModeThreadLocal));
    enqueue_step(st, st->cap_stream);
    cudaError_t e = cudaStreamEndCapture(st->cap_stream, &st->graph);
    if (e != cudaSuccess) return cuda_fail(e, "felbm_step: capture");
    FELBM_CUDA(cudaGraphInstantiate(&st->graph_exec, st->graph, 0));
    return FELBM_OK;
}

int felbm_step(felbm_state* st, int32_t n_steps) {
    if (!st || n_steps < 0) {
        set_error("felbm_step: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    if (!st->graph_exec) {
        int rc = build_graph(st);
        if (rc) return rc;
    }
    for (int32_t k = 0; k < n_steps; ++k) FELBM_CUDA(cudaGraphLaunch(st->graph_exec, st->stream));
    st->step += n_steps;
    if (n_steps > 0 && st->timing) st->timed_step_ran = true;
    return FELBM_OK;
}

static void drop_graph(felbm_state* st) {
    if (st->graph_exec) cudaGraphExecDestroy(st->graph_exec);
    if (st->graph) cudaGraphDestroy(st->graph);
    st->graph_exec = nullptr;
    st->graph = nullptr;
}

int felbm_timing_enable(felbm_state* st, int32_t enable) {
    if (!st) {
        set_error("felbm_timing_enable: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    if (enable && !st->ev[0])
        for (auto& e : st->ev) FELBM_CUDA(cudaEventCreate(&e));
    FELBM_CUDA(cudaStreamSynchronize(st->stream));
    drop_graph(st);
    st->timing = enable != 0;
    st->timed_step_ran = false;
    return FELBM_OK;
}

int felbm_fp64_fma_rate(void* stream, double* tflops) {
    if (!tflops) {
        set_error("felbm_fp64_fma_rate: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, n_sm = 0;
    FELBM_CUDA(cudaGetDevice(&dev));
    FELBM_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = n_sm * 8, iters = 4096;
    cudaEvent_t e0, e1;
    FELBM_CUDA(cudaEventCreate(&e0));
    FELBM_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {   // the first launch is a warm-up
        cudaEventRecord(e0, s);
        k_fp64_fma_rate<<<blocks, 256, 0, s>>>(iters, 0.999999);
        cudaEventRecord(e1, s);
        cudaError_t e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return cuda_fail(e, "felbm_fp64_fma_rate");
        }
        if (rep > 0) best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *tflops = 2.0 * 8.0 * iters * (double)blocks * 256.0 / (best * 1e-3) / 1e12;
    return FELBM_OK;
}

int felbm_timing_get(felbm_state* st, felbm_step_timing* out) {
    if (!st || !out || !st->timing || !st->timed_step_ran) {
        set_error("felbm_timing_get: timing is off or no timed step ran");
        return FELBM_ERR_INVALID_ARG;
    }
    FELBM_CUDA(cudaStreamSynchronize(st->stream));
    float t[6];
    for (int k = 0; k < 6; ++k) FELBM_CUDA(cudaEventElapsedTime(&t[k], st->ev[k], st->ev[k + 1]));
    out->collide_ms = t[0];
    out->mu_ms = t[1];
    out->gradmu_ms = t[2];
    out->element_ms = t[3];
    out->rhs_ms = t[4];
    out->solve_ms = t[5];
    out->total_ms = t[0] + t[1] + t[2] + t[3] + t[4] + t[5];
    out->solve_launches = solve_launches(st);
    out->launches = step_launches(st);
    return FELBM_OK;
}

}  // extern "C"

namespace felbm {

static DiagReq make_req(const felbm_state* st, const felbm_diag_request* req) {
    DiagReq rq{};
    rq.period_x = st->hm.period[0];
    rq.period_y = st->hm.period[1];
    rq.substrate = req ? req->substrate_wall_id : 0;
    rq.use_band = req && req->band > 0.0;
    if (req) {
        rq.cx = req->centre[0];
        rq.cy = req->centre[1];
        rq.R = req->radius;
        rq.band = req->band;
    }
    return rq;
}

// felbm_diag from the reduced slots; the contact angle uses the mean height
// of the substrate wall nodes among the given wall edges.
// The diagnostics reductions of the whole mesh into buf.diag_out.
static void enqueue_diag(felbm_state* st, const DiagReq& rq, cudaStream_t s) {
    if (st->dev32) {
        k_diag_fused32<<<kDiagBlocks, kBlock, 0, s>>>(st->dm, st->phys, st->buf, rq);
        return;
    }
    k_diag_nodes<false><<<kDiagBlocks, kBlock, 0, s>>>(st->dm, st->phys, st->buf, rq);
    k_diag_edges<<<kDiagBlocks, kBlock, 0, s>>>(st->dm, st->buf, rq);
    k_diag_final<<<1, kDiagSums * 32, 0, s>>>(st->buf);
}

// res: the two sums of the solve check (sum r^2, sum b^2), read when it is on.
static felbm_diag fill_diag(const felbm_state* st, const double* v, double mass0, int64_t nodes, int substrate,
                            const int32_t* edges, int32_t n_edges, int64_t step, const double* res) {
    const HostMesh& h = st->hm;
    felbm_diag d{};
    d.step = step;
    d.mass = v[0];
    d.mass0 = mass0;
    d.mass_drift_rel = mass0 != 0.0 ? (v[0] - mass0) / mass0 : 0.0;
    d.kinetic_energy = 0.5 * v[1] / (double)std::max<int64_t>(nodes, 1);
    d.max_u = std::sqrt(v[10]);
    d.interface_rho_uu = v[2] > 0.0 ? v[3] / v[2] : 0.0;
    d.p_in = v[5] / std::max(v[4], 1e-300);
    d.p_out = v[7] / std::max(v[6], 1e-300);
    d.delta_p = d.p_in - d.p_out;
    d.wetted_length = v[11];
    double ysum = 0.0;
    int ny = 0;
    std::vector<int32_t> nodes_seen;
    for (int32_t k = 0; k < n_edges; ++k) {
        int32_t e = edges ? edges[k] : k;
        if (h.wall_id[e] != substrate) continue;
        nodes_seen.push_back(h.wall_a[e]);
        nodes_seen.push_back(h.wall_b[e]);
    }
    std::sort(nodes_seen.begin(), nodes_seen.end());
    nodes_seen.erase(std::unique(nodes_seen.begin(), nodes_seen.end()), nodes_seen.end());
    for (int32_t n : nodes_seen) {
        ysum += h.y[n];
        ++ny;
    }
    d.height = ny ? v[12] - ysum / ny : std::nan("");
    double b = d.wetted_length, hh = d.height;
    if (ny && hh > 0.0 && b > 0.0) {
        double r = (4.0 * hh * hh + b * b) / (8.0 * hh);
        d.theta_deg = std::atan2(b, 2.0 * (r - hh)) * 180.0 / M_PI;
    } else {
        d.theta_deg = std::nan("");
    }
    d.status = v[9] > 0.0 ? FELBM_ERR_NONFINITE : FELBM_OK;
    d.solver_sweeps = st->mode == FELBM_SOLVER_FP64 ? st->sweeps : st->sweeps * st->rounds;
    d.solver_residual = std::nan("");
    if (st->check && res) {
        d.solver_residual = std::sqrt(res[0] / std::max(res[1], 1e-300));
        if (d.status == FELBM_OK && !(d.solver_residual <= st->check_tol)) d.status = FELBM_ERR_NOT_CONVERGED;
    }
    return d;
}

}  // namespace felbm

extern "C" {

// Error bits the solve kernels left since felbm_init (read after the stream
// has been synchronised by the caller of this check).
static int solve_status(felbm_state* st, const char* who) {
    unsigned bits = 0;
    FELBM_CUDA(cudaMemcpyAsync(&bits, st->buf.kerr, sizeof bits, cudaMemcpyDeviceToHost, st->stream));
    FELBM_CUDA(cudaStreamSynchronize(st->stream));
    if (bits & kErrTileWait) {
        set_error(std::string(who) + ": a tiled solve step gave up waiting for its tile copy");
        return FELBM_ERR_CUDA;
    }
    return FELBM_OK;
}

int felbm_diagnostics(felbm_state* st, const felbm_diag_request* req, felbm_diag* out) {
    if (!st || !out) {
        set_error("felbm_diagnostics: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    DiagReq rq = make_req(st, req);
    cudaStream_t s = st->stream;
    enqueue_diag(st, rq, s);
    FELBM_CUDA(cudaGetLastError());
    double v[kDiagSlots];
    FELBM_CUDA(cudaMemcpyAsync(v, st->buf.diag_out, sizeof v, cudaMemcpyDeviceToHost, s));
    FELBM_CUDA(cudaStreamSynchronize(s));
    if (int rc = solve_status(st, "felbm_diagnostics")) return rc;
    *out = fill_diag(st, v, st->mass0, st->hm.N, rq.substrate, nullptr, st->hm.E, st->step, v + kSolveResSlot);
    if (out->status == FELBM_ERR_NOT_CONVERGED) {
        set_error("felbm_diagnostics: the last solve's residual is above the tolerance of felbm_solver_check");
        return FELBM_ERR_NOT_CONVERGED;
    }
    if (out->status != FELBM_OK) {
        set_error("felbm_diagnostics: non-finite values in the state");
        return FELBM_ERR_NONFINITE;
    }
    return FELBM_OK;
}

int felbm_diagnostics_enqueue(felbm_state* st, const felbm_diag_request* req, double* slots) {
    if (!st || !slots) {
        set_error("felbm_diagnostics_enqueue: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    static_assert(kDiagSlots == FELBM_DIAG_SLOTS, "raw diagnostic sums");
    DiagReq rq = make_req(st, req);
    cudaStream_t s = st->stream;
    enqueue_diag(st, rq, s);
    FELBM_CUDA(cudaGetLastError());
    // the reduced sums arrive asynchronously; the step count is the host's now
    FELBM_CUDA(cudaMemcpyAsync(slots, st->buf.diag_out, sizeof(double) * (kSolveResSlot + 2), cudaMemcpyDeviceToHost,
                               s));
    slots[kDiagStepSlot] = (double)st->step;
    return FELBM_OK;
}

int felbm_diag_finish(felbm_state* st, const felbm_diag_request* req, const double* slots, felbm_diag* out) {
    if (!st || !slots || !out) {
        set_error("felbm_diag_finish: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    const DiagReq rq = make_req(st, req);
    *out = fill_diag(st, slots, st->mass0, st->hm.N, rq.substrate, nullptr, st->hm.E,
                     (int64_t)slots[kDiagStepSlot], slots + kSolveResSlot);
    if (out->status == FELBM_ERR_NOT_CONVERGED) {
        set_error("felbm_diag_finish: the last solve's residual is above the tolerance of felbm_solver_check");
        return FELBM_ERR_NOT_CONVERGED;
    }
    if (out->status != FELBM_OK) {
        set_error("felbm_diag_finish: non-finite values in the state");
        return FELBM_ERR_NONFINITE;
    }
    return FELBM_OK;
}

int felbm_diagnostics_groups(felbm_state* st, const felbm_diag_request* reqs, int32_t n_groups, felbm_diag* out) {
    if (!st || !out || n_groups != st->hm.G || n_groups < 1) {
        set_error("felbm_diagnostics_groups: invalid argument (n_groups must equal the mesh's group count)");
        return FELBM_ERR_INVALID_ARG;
    }
    const HostMesh& h = st->hm;
    std::vector<DiagReq> rq(n_groups);
    for (int32_t g = 0; g < n_groups; ++g) {
        rq[g] = make_req(st, reqs ? reqs + g : nullptr);
        rq[g].period_x = h.grp_period_x[g];
        rq[g].period_y = h.grp_period_y[g];
    }
    cudaStream_t s = st->stream;
    FELBM_CUDA(cudaMemcpyAsync(st->gt.reqs, rq.data(), sizeof(DiagReq) * n_groups, cudaMemcpyHostToDevice, s));
    if (st->dev32)
        k_diag_groups<true><<<n_groups, kBlock, 0, s>>>(st->dm, st->phys, st->buf, st->gt);
    else
        k_diag_groups<false><<<n_groups, kBlock, 0, s>>>(st->dm, st->phys, st->buf, st->gt);
    FELBM_CUDA(cudaGetLastError());
    std::vector<double> v((size_t)n_groups * kDiagSlots);
    double res[2] = {0.0, 0.0};
    FELBM_CUDA(cudaMemcpyAsync(v.data(), st->gt.out, sizeof(double) * v.size(), cudaMemcpyDeviceToHost, s));
    FELBM_CUDA(cudaMemcpyAsync(res, st->buf.diag_out + kSolveResSlot, sizeof res, cudaMemcpyDeviceToHost, s));
    FELBM_CUDA(cudaStreamSynchronize(s));
    bool bad = false, unconverged = false;
    for (int32_t g = 0; g < n_groups; ++g) {
        const double* vg = v.data() + (size_t)g * kDiagSlots;
        double m0 = g < (int32_t)st->gmass0.size() ? st->gmass0[g] : vg[0];
        out[g] = fill_diag(st, vg, m0, h.grp_size[g], rq[g].substrate, h.grp_wall_edge.data() + h.grp_wall_ptr[g],
                           h.grp_wall_ptr[g + 1] - h.grp_wall_ptr[g], st->step, res);
        bad = bad || out[g].status == FELBM_ERR_NONFINITE;
        unconverged = unconverged || out[g].status == FELBM_ERR_NOT_CONVERGED;
    }
    if (bad) {
        set_error("felbm_diagnostics_groups: non-finite values in the state");
        return FELBM_ERR_NONFINITE;
    }
    if (unconverged) {
        set_error("felbm_diagnostics_groups: the last solve's residual is above the tolerance of felbm_solver_check");
        return FELBM_ERR_NOT_CONVERGED;
    }
    return FELBM_OK;
}

int felbm_get_state(felbm_state* st, double* g, double* h) {
    if (!st || !g || !h) {
        set_error("felbm_get_state: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    cudaStream_t s = st->stream;
    const int N = st->dm.N;
    if (st->dev32)
        k_dev32_to_full<<<grid_for(N, kBlock), kBlock, 0, s>>>(st->dm, st->phys, st->buf, st->buf.stage);
    else
        k_gather_out<<<grid_for(N, kBlock), kBlock, 0, s>>>(st->dm, st->buf.psi, st->buf.stage, 18);
    FELBM_CUDA(cudaGetLastError());
    FELBM_CUDA(cudaMemcpyAsync(g, st->buf.stage, sizeof(double) * 9 * N, cudaMemcpyDeviceToHost, s));
    FELBM_CUDA(cudaMemcpyAsync(h, st->buf.stage + (size_t)9 * N, sizeof(double) * 9 * N, cudaMemcpyDeviceToHost, s));
    FELBM_CUDA(cudaStreamSynchronize(s));
    return solve_status(st, "felbm_get_state");
}

int felbm_set_state(felbm_state* st, const double* g, const double* h) {
    if (!st || !g || !h) {
        set_error("felbm_set_state: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    cudaStream_t s = st->stream;
    const int N = st->dm.N;
    if (!st->copy_stream) FELBM_CUDA(cudaStreamCreateWithFlags(&st->copy_stream, cudaStreamNonBlocking));
    if (!st->ev_copied) FELBM_CUDA(cudaEventCreateWithFlags(&st->ev_copied, cudaEventDisableTiming));
    for (auto& ev : st->ev_in_free)
        if (!ev) FELBM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    // The copy runs on its own stream into the input buffer not used by the
    // previous call, so it overlaps whatever the state's stream is running
    // (the previous step); it waits only for the conversion that last read
    // this buffer.  The conversion waits for the copy on the state's stream.
    const int k = st->in_next;
    st->in_next ^= 1;
    double* in = k ? st->buf.in1 : st->buf.in0;
    FELBM_CUDA(cudaStreamWaitEvent(st->copy_stream, st->ev_in_free[k], 0));
    FELBM_CUDA(cudaMemcpyAsync(in, g, sizeof(double) * 9 * N, cudaMemcpyHostToDevice, st->copy_stream));
    FELBM_CUDA(cudaMemcpyAsync(in + (size_t)9 * N, h, sizeof(double) * 9 * N, cudaMemcpyHostToDevice, st->copy_stream));
    FELBM_CUDA(cudaEventRecord(st->ev_copied, st->copy_stream));
    FELBM_CUDA(cudaStreamWaitEvent(s, st->ev_copied, 0));
    if (st->dev32)
        k_full_to_dev32<<<grid_for(N, kBlock), kBlock, 0, s>>>(st->dm, st->phys, st->buf, in);
    else
        k_scatter_in<<<grid_for(N, kBlock), kBlock, 0, s>>>(st->dm, in, st->buf.psi, 18);
    FELBM_CUDA(cudaGetLastError());
    FELBM_CUDA(cudaEventRecord(st->ev_in_free[k], s));
    // return once the host arrays have been read; the conversion stays queued
    FELBM_CUDA(cudaEventSynchronize(st->ev_copied));
    return FELBM_OK;
}

int felbm_get_fields(felbm_state* st, double* C, double* p, double* ux, double* uy, double* mu) {
    if (!st) {
        set_error("felbm_get_fields: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    cudaStream_t s = st->stream;
    const DevMesh& m = st->dm;
    double* outs[5] = {C, p, ux, uy, mu};
    if (st->dev32) {
        k_mu32<0><<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, st->phys, st->buf);
        FELBM_CUDA(cudaGetLastError());
        const float* srcs[5] = {nullptr, st->buf.p32, st->buf.ux32, st->buf.uy32, st->buf.mu32};
        for (int k = 0; k < 5; ++k) {
            if (!outs[k]) continue;
            if (k == 0)
                k_gather_out<<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, st->buf.C, st->buf.stage, 1);
            else
                k_gather_out_f<<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, srcs[k], st->buf.stage);
            FELBM_CUDA(cudaGetLastError());
            FELBM_CUDA(cudaMemcpyAsync(outs[k], st->buf.stage, sizeof(double) * m.N, cudaMemcpyDeviceToHost, s));
            FELBM_CUDA(cudaStreamSynchronize(s));
        }
        return FELBM_OK;
    }
    k_collide<<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, st->phys, st->buf, 0);
    k_mu<<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, st->phys, st->buf);
    FELBM_CUDA(cudaGetLastError());
    double* srcs[5] = {st->buf.C, st->buf.p, st->buf.ux, st->buf.uy, st->buf.mu};
    for (int k = 0; k < 5; ++k) {
        if (!outs[k]) continue;
        k_gather_out<<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, srcs[k], st->buf.stage, 1);
        FELBM_CUDA(cudaGetLastError());
        FELBM_CUDA(cudaMemcpyAsync(outs[k], st->buf.stage, sizeof(double) * m.N, cudaMemcpyDeviceToHost, s));
        FELBM_CUDA(cudaStreamSynchronize(s));
    }
    return FELBM_OK;
}

int felbm_mass_solve(felbm_state* st, const double* B, double* X, int32_t k) {
    if (!st || !B || !X || k < 1 || k > 18) {
        set_error("felbm_mass_solve: invalid argument (1 <= k <= 18)");
        return FELBM_ERR_INVALID_ARG;
    }
    cudaStream_t s = st->stream;
    const DevMesh& m = st->dm;
    const Bufs& b = st->buf;
    FELBM_CUDA(cudaMemcpyAsync(b.stage, B, sizeof(double) * k * m.N, cudaMemcpyHostToDevice, s));
    k_scatter_in<<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, b.stage, b.rhs, k);
    if (k < 18) k_zero_rows<<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, b.rhs, k, 18);
    if (st->mode == FELBM_SOLVER_FP64)
        k_cheb_start<false><<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, b, st->inv_theta);
    else
        k_cheb_start<true><<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, b, st->tau[0]);
    const double* result = enqueue_solve(st, st->dm, b, s, false);
    k_gather_out<<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, result, b.stage, k);
    FELBM_CUDA(cudaGetLastError());
    FELBM_CUDA(cudaMemcpyAsync(X, b.stage, sizeof(double) * k * m.N, cudaMemcpyDeviceToHost, s));
    FELBM_CUDA(cudaStreamSynchronize(s));
    return FELBM_OK;
}

}  // extern "C"

// ---------------------------------------- no-allocation mass solve -------
// The iterates of felbm_mass_solve_static live here, not in any allocation.
static __device__ __align__(256) unsigned char g_static_scratch[FELBM_STATIC_SCRATCH_BYTES];

namespace felbm {

static std::mutex g_static_mu;
static void* g_static_addr[64] = {};   // device address of g_static_scratch per device ordinal

// Device address of the scratch array on `device`, looked up once per device
// with that device current (the host-side symbol is not a device address).
static int static_scratch(int device, void** out) {
    if (device < 0 || device >= 64) {
        set_error("felbm_mass_solve_static: device ordinal out of range");
        return FELBM_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[device]) {
        int current = 0;
        FELBM_CUDA(cudaGetDevice(&current));
        if (current != device) FELBM_CUDA(cudaSetDevice(device));
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (current != device) cudaSetDevice(current);
        if (e != cudaSuccess) return cuda_fail(e, "felbm_mass_solve_static: cudaGetSymbolAddress");
        g_static_addr[device] = p;
    }
    *out = g_static_addr[device];
    return FELBM_OK;
}

}  // namespace felbm

extern "C" {

int felbm_mass_solve_static(felbm_state* st, const double* d_B, double* d_X, int32_t k) {
    if (!st || !d_B || !d_X || k < 1 || k > 18 || d_B == d_X) {
        set_error("felbm_mass_solve_static: invalid argument (device B, X distinct; 1 <= k <= 18)");
        return FELBM_ERR_INVALID_ARG;
    }
    const DevMesh& m = st->dm;
    // the solve's buffers: 18 rows of stride Np, 256-byte aligned pieces
    Carver cv(nullptr);
    const size_t rows = 18 * (size_t)m.Np;
    cv.take<double>(rows);
    cv.take<double>(rows);
    cv.take<double>(rows);
    cv.take<float>(rows);
    cv.take<float>(rows);
    cv.take<float>(rows);
    if (cv.off > FELBM_STATIC_SCRATCH_BYTES) {
        char buf[256];
        snprintf(buf, sizeof buf,
                 "felbm_mass_solve_static: %d nodes need %zu bytes of scratch, the static array holds %u",
                 m.N, cv.off, (unsigned)FELBM_STATIC_SCRATCH_BYTES);
        set_error(buf);
        return FELBM_ERR_WORKSPACE;
    }
    void* base = nullptr;
    int rc = static_scratch(st->device, &base);
    if (rc) return rc;
    Carver sc(base);
    Bufs sb = st->buf;
    sb.rhs = sc.take<double>(rows);
    sb.x0 = sc.take<double>(rows);
    sb.x1 = sc.take<double>(rows);
    sb.x64 = sb.x0;
    sb.rho64 = sb.x1;
    sb.r32 = sc.take<float>(rows);
    sb.e0 = sc.take<float>(rows);
    sb.e1 = sc.take<float>(rows);
    cudaStream_t s = st->stream;
    k_scatter_in<<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, d_B, sb.rhs, k);
    if (k < 18) k_zero_rows<<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, sb.rhs, k, 18);
    if (st->mode == FELBM_SOLVER_FP64)
        k_cheb_start<false><<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, sb, st->inv_theta);
    else
        k_cheb_start<true><<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, sb, st->tau[0]);
    const double* result = enqueue_solve(st, st->dm, sb, s, false);
    k_gather_out<<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, result, d_X, k);
    FELBM_CUDA(cudaGetLastError());
    return FELBM_OK;
}

int felbm_batch_schedule(felbm_state* st, int32_t cta_max_nodes) {
    if (!st || cta_max_nodes < 0) {
        set_error("felbm_batch_schedule: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    FELBM_CUDA(cudaStreamSynchronize(st->stream));
    int rc = set_schedule(st, cta_max_nodes);
    if (rc) return rc;
    drop_graph(st);
    return FELBM_OK;
}

int felbm_solver_check(felbm_state* st, int32_t enable, double tol) {
    if (!st || (enable != 0 && enable != 1) || (enable && !(tol > 0.0))) {
        set_error("felbm_solver_check: invalid argument (enable 0 or 1, tol > 0)");
        return FELBM_ERR_INVALID_ARG;
    }
    if (enable && st->mode == FELBM_SOLVER_FP64) {
        set_error("felbm_solver_check: needs the FP32 steps of the mixed or FP32-deviation solve");
        return FELBM_ERR_UNSUPPORTED;
    }
    FELBM_CUDA(cudaStreamSynchronize(st->stream));
    FELBM_CUDA(cudaMemsetAsync(st->buf.diag_out + kSolveResSlot, 0, 2 * sizeof(double), st->stream));
    FELBM_CUDA(cudaStreamSynchronize(st->stream));
    st->check = enable != 0;
    st->check_tol = tol;
    drop_graph(st);
    return FELBM_OK;
}

int felbm_sweep_tiled(felbm_state* st, int32_t on) {
    if (!st || (on != 0 && on != 1)) {
        set_error("felbm_sweep_tiled: invalid argument (0 or 1)");
        return FELBM_ERR_INVALID_ARG;
    }
    if (on && (!st->dm.tiled_ok || tile_parts(st, st->dm.ell_w) == 0)) {
        set_error("felbm_sweep_tiled: this mesh has no ELL copy, a tile halo beyond the staged rows, or "
                  "rows too long for two pipeline stages in shared memory");
        return FELBM_ERR_UNSUPPORTED;
    }
    FELBM_CUDA(cudaStreamSynchronize(st->stream));
    st->sweep_tiled = on != 0;
    drop_graph(st);
    return FELBM_OK;
}

int felbm_sweep_parts(felbm_state* st, int32_t parts) {
    if (!st || !(parts == 1 || parts == 2 || parts == 3 || parts == 6)) {
        set_error("felbm_sweep_parts: invalid argument (1, 2, 3 or 6)");
        return FELBM_ERR_INVALID_ARG;
    }
    FELBM_CUDA(cudaStreamSynchronize(st->stream));
    st->sweep_parts = parts;
    drop_graph(st);
    return FELBM_OK;
}

}  // extern "C"



extern "C" {

static int checkpoint_copy(felbm_state* st, void* dst_v, const void* src_v, bool save);

// Mean device time of one step over `trials` steps after one warm-up step.
static int time_steps(felbm_state* st, int32_t trials, cudaEvent_t e0, cudaEvent_t e1, float* ms) {
    int rc = felbm_step(st, 1);
    if (rc) return rc;
    FELBM_CUDA(cudaEventRecord(e0, st->stream));
    if ((rc = felbm_step(st, trials)) != FELBM_OK) return rc;
    FELBM_CUDA(cudaEventRecord(e1, st->stream));
    FELBM_CUDA(cudaEventSynchronize(e1));
    FELBM_CUDA(cudaEventElapsedTime(ms, e0, e1));
    *ms /= trials;
    return FELBM_OK;
}

int felbm_autotune(felbm_state* st, int32_t trials, felbm_tune_result* out) {
    if (!st || !out || trials < 1) {
        set_error("felbm_autotune: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    *out = felbm_tune_result{};
    const HostMesh& h = st->hm;
    FELBM_CUDA(cudaStreamSynchronize(st->stream));
    void* save = st->buf.stage;   // the state fits the staging buffer in both precisions
    int rc = checkpoint_copy(st, save, nullptr, true);
    if (rc) return rc;
    const int64_t step0 = st->step;
    const bool timing0 = st->timing;
    st->timing = false;
    cudaEvent_t e0, e1;
    FELBM_CUDA(cudaEventCreate(&e0));
    FELBM_CUDA(cudaEventCreate(&e1));
    // 1. threads per node of the FP32 sweeps (tiled schedule)
    //    and where the iterate comes from (gathered, or staged per node tile)
    const int parts_c[4] = {1, 2, 3, 6};
    int best_parts = st->sweep_parts;
    bool best_tiled = st->sweep_tiled;
    float best = 1e30f;
    if (st->mode != FELBM_SOLVER_FP64 && st->dm.ell_w > 0) {
        rc = set_schedule(st, 0);
        for (int tiled = 0; tiled < 2 && rc == FELBM_OK; ++tiled) {
            if (tiled && !st->dm.tiled_ok) break;
            for (int k = 0; k < 4 && rc == FELBM_OK; ++k) {
                st->sweep_parts = parts_c[k];
                st->sweep_tiled = tiled != 0;
                // the tiled step runs 3 or 6 parts (two stages of 1 or 2 parts do not fit)
                if (tiled && (tile_parts(st, st->dm.ell_w) != parts_c[k])) continue;
                drop_graph(st);
                float ms = 0.0f;
                if ((rc = time_steps(st, trials, e0, e1, &ms)) != FELBM_OK) break;
                (tiled ? out->tiled_ms : out->parts_ms)[k] = ms;
                if (ms < best) {
                    best = ms;
                    best_parts = parts_c[k];
                    best_tiled = tiled != 0;
                }
                rc = checkpoint_copy(st, nullptr, save, false);
            }
        }
    }
    st->sweep_parts = best_parts;
    st->sweep_tiled = best_tiled;
    drop_graph(st);
    out->sweep_parts = best_parts;
    out->sweep_tiled = best_tiled ? 1 : 0;
    // 2. batch schedule: CTA per member up to a node threshold (FP32_DEV batches)
    int32_t best_t = 0;
    if (rc == FELBM_OK && st->dev32 && h.G > 1) {
        std::vector<int32_t> cand = {0, 1 << 11, 1 << 12, 1 << 13, 1 << 14, 1 << 15, 1 << 16, 1 << 17};
        int last_n_cta = -1;
        best = 1e30f;
        for (int32_t t : cand) {
            int32_t n_cta = 0;
            for (int32_t g = 0; g < h.G; ++g) n_cta += (t > 0 && h.grp_size[g] <= t);
            if (n_cta == last_n_cta) continue;   // same split as the previous candidate
            last_n_cta = n_cta;
            if ((rc = set_schedule(st, t)) != FELBM_OK) break;
            drop_graph(st);
            float ms = 0.0f;
            if ((rc = time_steps(st, trials, e0, e1, &ms)) != FELBM_OK) break;
            if (out->n_candidates < 16) {
                out->candidates[out->n_candidates] = t;
                out->step_ms[out->n_candidates] = ms;
                out->n_candidates++;
            }
            if (ms < best) {
                best = ms;
                best_t = t;
            }
            if ((rc = checkpoint_copy(st, nullptr, save, false)) != FELBM_OK) break;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int rc2 = checkpoint_copy(st, nullptr, save, false);
    FELBM_CUDA(cudaStreamSynchronize(st->stream));
    st->step = step0;
    st->timing = timing0;
    if (rc) return rc;
    if (rc2) return rc2;
    out->cta_max_nodes = best_t;
    return felbm_batch_schedule(st, best_t);
}

// ------------------------------------------------------------- adjoint ----
int felbm_set_wetting(felbm_state* st, const double* phi_c, int32_t n_wall_ids) {
    if (!st || !phi_c || n_wall_ids < 1 || n_wall_ids > FELBM_MAX_WALL_IDS) {
        set_error("felbm_set_wetting: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    const HostMesh& h = st->hm;
    std::vector<double> wall_phi(std::max<int32_t>(h.E, 1), 0.0);
    for (int32_t e = 0; e < h.E; ++e) {
        if (h.wall_id[e] >= n_wall_ids) {
            set_error("felbm_set_wetting: a wall id has no phi_c");
            return FELBM_ERR_INVALID_ARG;
        }
        wall_phi[e] = phi_c[h.wall_id[e]];
    }
    for (int32_t k = 0; k < n_wall_ids; ++k) st->prm.phi_c[k] = phi_c[k];
    if (h.E > 0)
        FELBM_CUDA(cudaMemcpyAsync(const_cast<double*>(st->dm.wall_phi), wall_phi.data(), sizeof(double) * h.E,
                                   cudaMemcpyHostToDevice, st->stream));
    FELBM_CUDA(cudaStreamSynchronize(st->stream));
    return FELBM_OK;
}

int felbm_checkpoint_bytes(const felbm_state* st, size_t* bytes) {
    if (!st || !bytes) {
        set_error("felbm_checkpoint_bytes: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    *bytes = st->dev32 ? (size_t)st->dm.Np * (18 * sizeof(float) + sizeof(double) + 3 * sizeof(float))
                       : (size_t)st->dm.Np * 18 * sizeof(double);
    return FELBM_OK;
}

static int checkpoint_copy(felbm_state* st, void* dst_v, const void* src_v, bool save) {
    const DevMesh& m = st->dm;
    const Bufs& b = st->buf;
    char* ck = reinterpret_cast<char*>(save ? dst_v : const_cast<void*>(src_v));
    std::vector<std::pair<void*, size_t>> parts;
    if (st->dev32) {
        parts = {{b.dpsi, 18 * (size_t)m.Np * sizeof(float)}, {b.C, (size_t)m.Np * sizeof(double)},
                 {b.p32, (size_t)m.Np * sizeof(float)}, {b.ux32, (size_t)m.Np * sizeof(float)},
                 {b.uy32, (size_t)m.Np * sizeof(float)}};
    } else {
        parts = {{b.psi, 18 * (size_t)m.Np * sizeof(double)}};
    }
    size_t off = 0;
    for (auto& pr : parts) {
        void* d = save ? (void*)(ck + off) : pr.first;
        const void* sr = save ? (const void*)pr.first : (const void*)(ck + off);
        FELBM_CUDA(cudaMemcpyAsync(d, sr, pr.second, cudaMemcpyDeviceToDevice, st->stream));
        off += pr.second;
    }
    return FELBM_OK;
}

int felbm_checkpoint_save(felbm_state* st, void* d_dst) {
    if (!st || !d_dst) {
        set_error("felbm_checkpoint_save: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    return checkpoint_copy(st, d_dst, nullptr, true);
}

int felbm_checkpoint_load(felbm_state* st, const void* d_src) {
    if (!st || !d_src) {
        set_error("felbm_checkpoint_load: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    return checkpoint_copy(st, nullptr, d_src, false);
}

int felbm_adjoint_seed(felbm_state* st, const double* dL_dg, const double* dL_dh) {
    if (!st || !dL_dg || !dL_dh) {
        set_error("felbm_adjoint_seed: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    if (st->phys.lapmu_nodal) {
        set_error("felbm_adjoint_seed: the adjoint covers FELBM_LAPMU_FACE only");
        return FELBM_ERR_UNSUPPORTED;
    }
    if (st->dev32) {
        set_error("felbm_adjoint_seed: the adjoint is available for FELBM_FP64 states");
        return FELBM_ERR_UNSUPPORTED;
    }
    cudaStream_t s = st->stream;
    const int N = st->dm.N;
    FELBM_CUDA(cudaMemcpyAsync(st->buf.stage, dL_dg, sizeof(double) * 9 * N, cudaMemcpyHostToDevice, s));
    FELBM_CUDA(cudaMemcpyAsync(st->buf.stage + (size_t)9 * N, dL_dh, sizeof(double) * 9 * N, cudaMemcpyHostToDevice, s));
    k_scatter_in<<<grid_for(N, kBlock), kBlock, 0, s>>>(st->dm, st->buf.stage, st->adj.lam, 18);
    FELBM_CUDA(cudaGetLastError());
    if (st->hm.E > 0) FELBM_CUDA(cudaMemsetAsync(st->adj.dphi, 0, sizeof(double) * st->hm.E, s));
    FELBM_CUDA(cudaStreamSynchronize(s));
    return FELBM_OK;
}

int felbm_adjoint_step(felbm_state* st) {
    if (!st) {
        set_error("felbm_adjoint_step: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    if (st->phys.lapmu_nodal) {
        set_error("felbm_adjoint_step: the adjoint covers FELBM_LAPMU_FACE only");
        return FELBM_ERR_UNSUPPORTED;
    }
    if (st->dev32) {
        set_error("felbm_adjoint_step: the adjoint is available for FELBM_FP64 states");
        return FELBM_ERR_UNSUPPORTED;
    }
    cudaStream_t s = st->stream;
    const DevMesh& m = st->dm;
    Bufs& b = st->buf;
    AdjBufs& a = st->adj;
    // fields of the state psi^n (the input of the step being reversed)
    k_collide<<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, st->phys, b, 0);
    k_mu<<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, st->phys, b);
    k_gradmu<<<grid_for(m.T, kBlock), kBlock, 0, s>>>(m, b);
    // lambda_RHS = M11^{-1} lambda with the step's solver
    FELBM_CUDA(cudaMemcpyAsync(b.rhs, a.lam, sizeof(double) * 18 * m.Np, cudaMemcpyDeviceToDevice, s));
    if (st->mode == FELBM_SOLVER_FP64)
        k_cheb_start<false><<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, b, st->inv_theta);
    else
        k_cheb_start<true><<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, b, st->tau[0]);
    a.lamRHS = enqueue_solve(st, m, b, s, false);
    k_adj_elem_a<<<grid_for(m.T, 128), 128, 0, s>>>(m, st->phys, b, a);
    k_adj_elem_b<<<grid_for(m.T, kBlock), kBlock, 0, s>>>(m, a);
    k_adj_node_d<<<grid_for(m.N, 128), 128, 0, s>>>(m, st->phys, a);
    k_adj_node_e<<<grid_for(m.N, 128), 128, 0, s>>>(m, st->phys, b, a);
    FELBM_CUDA(cudaGetLastError());
    return FELBM_OK;
}

int felbm_adjoint_get(felbm_state* st, double* dL_dg, double* dL_dh, double* dL_dphi_c) {
    if (!st || (!dL_dg != !dL_dh)) {
        set_error("felbm_adjoint_get: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    if (st->phys.lapmu_nodal) {
        set_error("felbm_adjoint_get: the adjoint covers FELBM_LAPMU_FACE only");
        return FELBM_ERR_UNSUPPORTED;
    }
    if (st->dev32) {
        set_error("felbm_adjoint_get: the adjoint is available for FELBM_FP64 states");
        return FELBM_ERR_UNSUPPORTED;
    }
    cudaStream_t s = st->stream;
    const int N = st->dm.N;
    if (dL_dg) {
        k_gather_out<<<grid_for(N, kBlock), kBlock, 0, s>>>(st->dm, st->adj.lam, st->buf.stage, 18);
        FELBM_CUDA(cudaGetLastError());
        FELBM_CUDA(cudaMemcpyAsync(dL_dg, st->buf.stage, sizeof(double) * 9 * N, cudaMemcpyDeviceToHost, s));
        FELBM_CUDA(cudaMemcpyAsync(dL_dh, st->buf.stage + (size_t)9 * N, sizeof(double) * 9 * N,
                                   cudaMemcpyDeviceToHost, s));
    }
    std::vector<double> de(std::max<int32_t>(st->hm.E, 1));
    if (st->hm.E > 0)
        FELBM_CUDA(cudaMemcpyAsync(de.data(), st->adj.dphi, sizeof(double) * st->hm.E, cudaMemcpyDeviceToHost, s));
    FELBM_CUDA(cudaStreamSynchronize(s));
    if (dL_dphi_c) {
        for (int k = 0; k < st->prm.n_wall_ids; ++k) dL_dphi_c[k] = 0.0;
        for (int32_t e = 0; e < st->hm.E; ++e) dL_dphi_c[st->hm.wall_id[e]] += de[e];   // edge order: fixed
    }
    return FELBM_OK;
}

void felbm_state_destroy(felbm_state* st) {
    if (!st) return;
    drop_graph(st);
    if (st->cap_stream) cudaStreamDestroy(st->cap_stream);
    if (st->side_stream) cudaStreamDestroy(st->side_stream);
    if (st->ev_fork) cudaEventDestroy(st->ev_fork);
    if (st->ev_copied) cudaEventDestroy(st->ev_copied);
    if (st->ev_join) cudaEventDestroy(st->ev_join);
    if (st->copy_stream) cudaStreamDestroy(st->copy_stream);
    for (auto& e : st->ev_in_free)
        if (e) cudaEventDestroy(e);
    for (auto& e : st->ev)
        if (e) cudaEventDestroy(e);
    delete st;
}

}  // extern "C"
