// CUDA implementation of the 3D FE-LBM step (D3Q19 on linear tetrahedra) for
// sm_103a (GB300).
//
// Data layout in HBM (all carved from the caller's workspace):
//  * distributions psi: double [38][Np] -- g_0..g_18 then h_0..h_18,
//    direction major, node stride Np = N rounded up to 64;
//  * nodal fields C, p, ux, uy, uz, mu: double [Np];
//  * tetrahedron tables (structure of arrays): vertices int [4][Tp], volume
//    [Tp], shape gradients double [12][Tp], face neighbours int [4][Tp];
//  * element residual R: double [T][38] (array of structures: a node's
//    gather reads one tetrahedron's 19 values of a set contiguously);
//  * node-node pattern (CSR + an ELL copy for the FP32 sweeps) with the
//    consistent mass and the patch-Laplacian coefficients; node ->
//    tetrahedron and node -> wall-face incidence (CSR).
// Nodes are in reverse Cuthill-McKee order and tetrahedra sorted by their
// lowest node, so every gather reads a narrow window of the arrays.
//
// One time step (Sec. II.C of arXiv:1708.04678, D3Q19 form), captured once
// into a CUDA graph:
//   k3_collide   moments (eq:velocity, eq:pressure), collision (eqn::collide)
//   k3_mu        chemical potential with the patch Laplacian and the wetting
//                flux on wall faces (eqn:mp_mu, eqn:lapl_int_mp, eqn:bc2)
//   k3_gradmu    P0 gradient of mu per tetrahedron
//   k3_element   element Laplacian of mu (Sec. II.D), P0 forces at the
//                barycentre (eq:G, eq:H) and the element residual
//                V (Phi - e.grad psi_hat) of eq:galerkin_lbm
//   k3_rhs       node-centric gather of the streaming right-hand side with
//                weak bounce-back on wall faces; first Chebyshev iterate
//   solve        Chebyshev sweeps of the consistent-mass solve (spectrum of
//                the lumped-preconditioned matrix in [1/5, 1]): FP64, or FP32
//                sweeps with FP64 residual refinement (mixed)
// Node kernels run one thread per (node, distribution set): grid.y = 2.
// No atomics: every sum is a fixed-order loop or tree.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "felbm3d_internal.h"

namespace felbm3 {

using felbm::HostMesh3D;
using felbm::set_error;

// --------------------------------------------------------------- D3Q19 ----
__host__ __device__ constexpr int ex3(int q) {
    return (q == 1 || q == 7 || q == 9 || q == 11 || q == 13) ? 1
           : (q == 2 || q == 8 || q == 10 || q == 12 || q == 14) ? -1 : 0;
}
__host__ __device__ constexpr int ey3(int q) {
    return (q == 3 || q == 7 || q == 10 || q == 15 || q == 17) ? 1
           : (q == 4 || q == 8 || q == 9 || q == 16 || q == 18) ? -1 : 0;
}
__host__ __device__ constexpr int ez3(int q) {
    return (q == 5 || q == 11 || q == 14 || q == 15 || q == 18) ? 1
           : (q == 6 || q == 12 || q == 13 || q == 16 || q == 17) ? -1 : 0;
}
__host__ __device__ constexpr double wq3(int q) { return q == 0 ? 1.0 / 3.0 : (q <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }
__host__ __device__ constexpr int opp3(int q) { return q == 0 ? 0 : ((q & 1) ? q + 1 : q - 1); }

constexpr bool d3q19_ok() {
    double s0 = 0, sx = 0, sxx = 0, syy = 0, szz = 0, sxy = 0, sxz = 0, syz = 0;
    for (int q = 0; q < 19; ++q) {
        if (ex3(opp3(q)) != -ex3(q) || ey3(opp3(q)) != -ey3(q) || ez3(opp3(q)) != -ez3(q)) return false;
        int n = ex3(q) * ex3(q) + ey3(q) * ey3(q) + ez3(q) * ez3(q);
        if ((q == 0) != (n == 0) || (q >= 1 && q <= 6 && n != 1) || (q >= 7 && n != 2)) return false;
        for (int r = 0; r < q; ++r)
            if (ex3(r) == ex3(q) && ey3(r) == ey3(q) && ez3(r) == ez3(q)) return false;
        s0 += wq3(q);
        sx += wq3(q) * (ex3(q) + ey3(q) + ez3(q));
        sxx += wq3(q) * ex3(q) * ex3(q);
        syy += wq3(q) * ey3(q) * ey3(q);
        szz += wq3(q) * ez3(q) * ez3(q);
        sxy += wq3(q) * ex3(q) * ey3(q);
        sxz += wq3(q) * ex3(q) * ez3(q);
        syz += wq3(q) * ey3(q) * ez3(q);
    }
    auto near = [](double a, double b) { return a - b < 1e-15 && b - a < 1e-15; };
    return near(s0, 1.0) && near(sx, 0.0) && near(sxx, 1.0 / 3.0) && near(syy, 1.0 / 3.0) &&
           near(szz, 1.0 / 3.0) && near(sxy, 0.0) && near(sxz, 0.0) && near(syz, 0.0);
}
static_assert(d3q19_ok(), "D3Q19 table: distinct velocities, opposites, weights and second moments");

// e_q . v with additions only, in the type of v (FP32 stays FP32)
template <class T>
__device__ __forceinline__ T edot3(int q, T vx, T vy, T vz) {
    T r = T(0);
    if (ex3(q) == 1) r = vx;
    if (ex3(q) == -1) r = -vx;
    if (ey3(q) == 1) r = r + vy;
    if (ey3(q) == -1) r = r - vy;
    if (ez3(q) == 1) r = r + vz;
    if (ez3(q) == -1) r = r - vz;
    return r;
}

// ------------------------------------------------------- device tables ----
struct DevMesh3 {
    int32_t N, T, F, Np, Tp;
    double period[3];
    const int32_t* tet;       // [4][Tp]
    const double* vol;        // [Tp]
    const double* grad;       // [12][Tp]
    const int32_t* nbr;       // [4][Tp]
    const float* vol32;       // [Tp] FP32 copies for the FP32-deviation path
    const float* grad32;      // [12][Tp]
    const int32_t* row_ptr;   // [N+1]
    const int32_t* col;       // [nnz]
    const double* mval;       // [nnz] consistent mass
    const double* lval;       // [nnz] -3 K_ij / V_i (patch Laplacian of C)
    int32_t ell_w;            // ELL width (max row length rounded up), 0 = CSR sweeps
    const int32_t* ell_col;   // [ell_w][Np] padding: own column with value 0
    const float* ell_val;     // [ell_w][Np]
    const float* mval32;      // [nnz]
    const double* inv_lumped; // [Np]
    const float* inv_lumped32;
    const double* lumped;     // [Np]
    const double* inv_vol;    // [Np] 1 / V_i
    const int32_t* inc_ptr;   // [N+1]
    const int32_t* inc_tet;   // [ninc]
    const double* inc_b;      // [3][ninc]
    const float* inc_b32;     // [3][ninc]
    int32_t ninc;
    const int32_t* wall_v;    // [3][F]
    const int32_t* wall_id;   // [F]
    const double* wall_phi;   // [F] wetting potential phi_c of the face's wall id
    const double* wall_area;  // [F]
    const double* wall_n;     // [3][F] unit normal out of the fluid
    const int32_t* winc_ptr;  // [N+1]
    const int32_t* winc_face;
    const double* x;          // [Np]
    const double* y;
    const double* z;
    const int32_t* perm;      // [N] new -> caller
};

struct Phys3 {
    double dt, tau_l, tau_v, rho_l, rho_v, kappa, beta, mobility;
    // element Laplacian of mu: 0 = face-averaged gradients (Sec. II.D),
    // 1 = vertex mean of the nodal patch Laplacian, lapmu_fac * sum l_ij (mu_j - mu_i)
    int lapmu_nodal;
    double lapmu_fac;
    float dt_f, dt4_f, dt2h_f, inv_tau_l_f, inv_tau_v_f, rho_v_f, drho_f, mobility_f;
};

struct Bufs3 {
    double* psi;     // [38][Np]
    double* C;       // [Np]
    double* p;
    double* ux;
    double* uy;
    double* uz;
    double* mu;
    double* gmu;     // [3][Tp]; FELBM_LAPMU_NODAL: the first N hold the nodal Laplacian of mu
    double* lmu;     // alias of gmu (nodal mode)
    double* R;       // [T][38]
    double* rhs;     // [38][Np]
    double* x0;      // [38][Np] FP64 Chebyshev iterates; mixed solve: x64 and rho64
    double* x1;
    float* r32;      // [Np][kRow] FP32 residual of the current correction
    float* e0;       // [Np][kRow] FP32 Chebyshev iterates
    float* e1;
    // FP32-deviation storage (FELBM_FP32_DEV); C above stays FP64
    float* dpsi;     // [Np][kRow] deviations from equilibrium
    float* p32;
    float* ux32;
    float* uy32;
    float* uz32;
    float* mu32;
    float* gmu32;    // [3][Tp]; FELBM_LAPMU_NODAL: the first N hold the nodal Laplacian of mu
    float* lmu32;    // alias of gmu32 (nodal mode)
    float* R32;      // [T][kRow]
    double* stage;   // [38][N] caller-order staging
    double* in0;     // [38][N] two caller-order input buffers of felbm3d_set_state, used in
    double* in1;     //         turn so a copy can run while the previous input converts
    double* diag_part; // [kDiagBlocks][kDiagSlots]
    double* diag_out;  // [kDiagSlots]
};

constexpr int kBlock = 256;
constexpr int kNodeBlock = 128;
constexpr int kDiagBlocks = 304;   // fixed grid (2 x 152 SMs): the reduction order never changes
constexpr int kDiagSlots = 12;
// FP32 rows (deviations, element residuals, solve iterates): 40 floats per
// node or tetrahedron, g_q at 20*0 + q, h_q at 20*1 + q, slots 19 and 39
// zero -- each set is five 16-byte vectors.
constexpr int kRow = 40;
__host__ __device__ constexpr int slot(int s, int q) { return 20 * s + q; }

// Cooperative kernels: a group of kGroup = 5 lanes per node (or
// tetrahedron); lane c owns directions 4c..4c+3 of both sets, i.e. the
// 16-byte vectors c and 5 + c of a row, so one warp load reads whole rows
// of six items contiguously.  Lanes 30 and 31 of each warp idle.
constexpr int kGroup = 5;
constexpr int kGroupsPerWarp = 6;
constexpr int kCoopBlock = 128;
constexpr int kItemsPerBlock = kGroupsPerWarp * (kCoopBlock / 32);

struct Coop {
    int lane, grp, c, item;
    bool active;
};
__device__ __forceinline__ Coop coop_index(int n_items) {
    Coop k;
    k.lane = threadIdx.x & 31;
    k.grp = k.lane / kGroup;
    k.c = k.lane - k.grp * kGroup;
    k.item = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * kGroupsPerWarp + k.grp;
    k.active = k.grp < kGroupsPerWarp && k.item < n_items;
    return k;
}
// sum of v over the lanes of this lane's group, in lane order (identical in
// every lane of the group); every lane of the warp must call it
__device__ __forceinline__ float group_sum(float v, const Coop& k) {
    const int base = k.grp * kGroup;
    float s = __shfl_sync(0xffffffffu, v, base);
#pragma unroll
    for (int l = 1; l < kGroup; ++l) s += __shfl_sync(0xffffffffu, v, base + l);
    return s;
}
__device__ __forceinline__ void fma4(float4& acc, float w, const float4& x) {
    acc.x = fmaf(w, x.x, acc.x);
    acc.y = fmaf(w, x.y, acc.y);
    acc.z = fmaf(w, x.z, acc.z);
    acc.w = fmaf(w, x.w, acc.w);
}
__device__ __forceinline__ float comp(const float4& v, int j) { return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w; }
__device__ __forceinline__ void set_comp(float4& v, int j, float x) {
    if (j == 0) v.x = x;
    else if (j == 1) v.y = x;
    else if (j == 2) v.z = x;
    else v.w = x;
}

// ------------------------------------------------------ K1: collision -----
// Moments of the pre-collision state (C = sum h, p = sum g, rho u = sum e g /
// cs2) and BGK collision towards g_eq = w p + rho cs2 (Gamma - w),
// h_eq = Gamma C, written in place.
__global__ void __launch_bounds__(kBlock) k3_collide(DevMesh3 m, Phys3 c, Bufs3 b, int do_collide) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const int Np = m.Np;
    double g[19], h[19];
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        g[q] = b.psi[q * Np + i];
        h[q] = b.psi[(19 + q) * Np + i];
    }
    double C = 0.0, p = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        C += h[q];
        p += g[q];
        mx += edot3(q, g[q], 0.0, 0.0);
        my += edot3(q, 0.0, g[q], 0.0);
        mz += edot3(q, 0.0, 0.0, g[q]);
    }
    double rho = c.rho_v + C * (c.rho_l - c.rho_v);
    double ux = 3.0 * mx / rho, uy = 3.0 * my / rho, uz = 3.0 * mz / rho;
    b.C[i] = C;
    b.p[i] = p;
    b.ux[i] = ux;
    b.uy[i] = uy;
    b.uz[i] = uz;
    if (!do_collide) return;
    double inv_tau = C / c.tau_l + (1.0 - C) / c.tau_v;
    double omega = 1.0 / (1.0 / inv_tau + 0.5);
    double uu15 = 1.5 * (ux * ux + uy * uy + uz * uz);
    double rcs2 = rho * (1.0 / 3.0);
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        double eu = edot3(q, ux, uy, uz);
        double G = wq3(q) * (1.0 + 3.0 * eu + 4.5 * eu * eu - uu15);
        double geq = wq3(q) * p + rcs2 * (G - wq3(q));
        double heq = G * C;
        b.psi[q * Np + i] = g[q] - omega * (g[q] - geq);
        b.psi[(19 + q) * Np + i] = h[q] - omega * (h[q] - heq);
    }
}

// Wetting flux of one wall face (eqn:bc2 with C linear on the face):
// -phi_c int (C - C^2) dS, with int C = A (Ca+Cb+Cc)/3 and
// int C^2 = A/6 (Ca^2+Cb^2+Cc^2 + Ca Cb + Cb Cc + Cc Ca).
__device__ __forceinline__ double wall_flux3(const DevMesh3& m, const double* __restrict__ C, int f) {
    const int F = m.F;
    double Ca = C[m.wall_v[f]], Cb = C[m.wall_v[F + f]], Cc = C[m.wall_v[2 * F + f]];
    double s = (Ca + Cb + Cc) * (1.0 / 3.0) - (Ca * Ca + Cb * Cb + Cc * Cc + Ca * Cb + Cb * Cc + Cc * Ca) * (1.0 / 6.0);
    return -m.wall_phi[f] * m.wall_area[f] * s;
}

// --------------------------------------------- K2: chemical potential -----
// mu_i = 2 beta C (C-1)(2C-1) - kappa lap(C)_i; the patch Laplacian is
// kappa sum_j l_ij (C_j - C_i) plus the wall faces' wetting flux over V_i.
__global__ void __launch_bounds__(kBlock) k3_mu(DevMesh3 m, Phys3 c, Bufs3 b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const double Ci = b.C[i];
    double lap = 0.0;
    for (int k = m.row_ptr[i]; k < m.row_ptr[i + 1]; ++k) lap += m.lval[k] * (b.C[m.col[k]] - Ci);
    double wall = 0.0;
    for (int k = m.winc_ptr[i]; k < m.winc_ptr[i + 1]; ++k) wall += wall_flux3(m, b.C, m.winc_face[k]);
    b.mu[i] = 2.0 * c.beta * Ci * (Ci - 1.0) * (2.0 * Ci - 1.0) - (c.kappa * lap + wall * m.inv_vol[i]);
}

// ------------------------------------------------- K3: grad mu per T ------
__global__ void __launch_bounds__(kBlock) k3_gradmu(DevMesh3 m, Bufs3 b) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m.T) return;
    const int Tp = m.Tp;
    double mu0 = b.mu[m.tet[t]];
    double g[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 1; k < 4; ++k) {
        double d = b.mu[m.tet[k * Tp + t]] - mu0;
#pragma unroll
        for (int a = 0; a < 3; ++a) g[a] += d * m.grad[(3 * k + a) * Tp + t];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) b.gmu[a * Tp + t] = g[a];
}

// K3' (FELBM_LAPMU_NODAL): nodal Laplacian of mu, the patch Laplacian of C
// applied to mu with zero wall flux (eqn:bc1), lumped P1 volume.
__global__ void __launch_bounds__(kBlock) k3_lmu(DevMesh3 m, Phys3 c, Bufs3 b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const double mi = b.mu[i];
    double lap = 0.0;
    for (int k = m.row_ptr[i]; k < m.row_ptr[i + 1]; ++k) lap += m.lval[k] * (b.mu[m.col[k]] - mi);
    b.lmu[i] = c.lapmu_fac * lap;
}

// ------------------------------- K4: forces and element residual ---------
// lap(mu)_T = (1/V) sum_{interior faces k} 1/2 (grad mu_T + grad mu_T').nu_k
// with nu_k = -3 V b_k (outward normal x area of the face opposite vertex
// k); wall faces give 0 (eqn:bc1).  Forces at the barycentre:
//   Phi_g = (e-u).[cs2 grad(rho) (Gamma - w) + mu grad(C) Gamma]
//   Phi_h = [(e-u).(grad C - C/(rho cs2) (grad p - mu grad C)) + M lap(mu)] Gamma
// Residual R_a = V (Phi_a - e_a . grad psi_hat_a), psi_hat P1 on the element.
__global__ void __launch_bounds__(128) k3_element(DevMesh3 m, Phys3 c, Bufs3 b) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m.T) return;
    const int Tp = m.Tp, Np = m.Np;
    int v[4];
    double bx[4], by[4], bz[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = m.tet[k * Tp + t];
        bx[k] = m.grad[(3 * k) * Tp + t];
        by[k] = m.grad[(3 * k + 1) * Tp + t];
        bz[k] = m.grad[(3 * k + 2) * Tp + t];
    }
    const double V = m.vol[t];
    double Cs = 0, uxs = 0, uys = 0, uzs = 0, mus = 0;
    double gC[3] = {0, 0, 0}, gp[3] = {0, 0, 0};
    const double C0 = b.C[v[0]], p0 = b.p[v[0]];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double Cv = b.C[v[k]], pv = b.p[v[k]];
        Cs += Cv;
        uxs += b.ux[v[k]];
        uys += b.uy[v[k]];
        uzs += b.uz[v[k]];
        mus += b.mu[v[k]];
        if (k > 0) {
            double dC = Cv - C0, dp = pv - p0;
            gC[0] += dC * bx[k];
            gC[1] += dC * by[k];
            gC[2] += dC * bz[k];
            gp[0] += dp * bx[k];
            gp[1] += dp * by[k];
            gp[2] += dp * bz[k];
        }
    }
    const double Cb = 0.25 * Cs, ux = 0.25 * uxs, uy = 0.25 * uys, uz = 0.25 * uzs, mub = 0.25 * mus;
    double lapmu;
    if (c.lapmu_nodal) {
        lapmu = 0.25 * (b.lmu[v[0]] + b.lmu[v[1]] + b.lmu[v[2]] + b.lmu[v[3]]);
    } else {
        const double gm[3] = {b.gmu[t], b.gmu[Tp + t], b.gmu[2 * Tp + t]};
        double flux = 0.0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            int nb = m.nbr[k * Tp + t];
            if (nb >= 0)
                flux += (gm[0] + b.gmu[nb]) * bx[k] + (gm[1] + b.gmu[Tp + nb]) * by[k] + (gm[2] + b.gmu[2 * Tp + nb]) * bz[k];
        }
        lapmu = -1.5 * flux;
    }
    const double drho = c.rho_l - c.rho_v;
    const double rhob = c.rho_v + Cb * drho;
    const double gr[3] = {drho * gC[0], drho * gC[1], drho * gC[2]};
    const double f = 3.0 * Cb / rhob;
    const double vh[3] = {gC[0] - f * (gp[0] - mub * gC[0]), gC[1] - f * (gp[1] - mub * gC[1]),
                          gC[2] - f * (gp[2] - mub * gC[2])};
    const double u_gr = ux * gr[0] + uy * gr[1] + uz * gr[2];
    const double u_gC = ux * gC[0] + uy * gC[1] + uz * gC[2];
    const double u_vh = ux * vh[0] + uy * vh[1] + uz * vh[2];
    const double uu15 = 1.5 * (ux * ux + uy * uy + uz * uz);
    const double Mlap = c.mobility * lapmu;
    double* dst = b.R + (size_t)t * 38;
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        const double w = wq3(q);
        const double eu = edot3(q, ux, uy, uz);
        const double G = w * (1.0 + 3.0 * eu + 4.5 * eu * eu - uu15);
        const double phig = (1.0 / 3.0) * (G - w) * (edot3(q, gr[0], gr[1], gr[2]) - u_gr) +
                            mub * G * (edot3(q, gC[0], gC[1], gC[2]) - u_gC);
        const double phih = ((edot3(q, vh[0], vh[1], vh[2]) - u_vh) + Mlap) * G;
        double dg = 0.0, dh = 0.0;
        if (q != 0) {
            const double g0 = b.psi[q * Np + v[0]], h0 = b.psi[(19 + q) * Np + v[0]];
#pragma unroll
            for (int k = 1; k < 4; ++k) {
                const double eb = edot3(q, bx[k], by[k], bz[k]);
                dg += (b.psi[q * Np + v[k]] - g0) * eb;
                dh += (b.psi[(19 + q) * Np + v[k]] - h0) * eb;
            }
        }
        dst[q] = V * (phig - dg);
        dst[19 + q] = V * (phih - dh);
    }
}

// ------------------------------------------- K5: streaming RHS gather -----
// RHS_{i,a} = sum_{T at i} R_{T,a} (dt/4 + dt^2/2 e_a.b_{i,T})
//   - dt sum_{wall f at i} (e_a.n) [A/6 (psi_opp - psi)_i + A/12 sum_{o != i} (psi_opp - psi)_o]
// (wall term only for incoming directions e_a.n < 0).  One thread per
// (node, set); also writes the first iterate of the solve first_scale RHS / m_i
// (1/theta for the FP64 Chebyshev recurrence, tau_0 for the FP32 steps):
// FP64 (FP64 Chebyshev) or FP32 with the FP32 copy of the RHS (mixed solve).
template <bool kMixed>
__global__ void __launch_bounds__(kNodeBlock) k3_rhs(DevMesh3 m, Phys3 c, Bufs3 b, double first_scale) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const int s = blockIdx.y, Np = m.Np, ninc = m.ninc;
    double acc[19];
#pragma unroll
    for (int q = 0; q < 19; ++q) acc[q] = 0.0;
    const double c1 = 0.25 * c.dt, c2 = 0.5 * c.dt * c.dt;
    for (int k = m.inc_ptr[i]; k < m.inc_ptr[i + 1]; ++k) {
        const double* src = b.R + (size_t)m.inc_tet[k] * 38 + 19 * s;
        const double bxi = m.inc_b[k], byi = m.inc_b[ninc + k], bzi = m.inc_b[2 * ninc + k];
#pragma unroll
        for (int q = 0; q < 19; ++q) acc[q] += src[q] * (c1 + c2 * edot3(q, bxi, byi, bzi));
    }
    const double* ps = b.psi + (size_t)19 * s * Np;
    const int F = m.F;
    for (int k = m.winc_ptr[i]; k < m.winc_ptr[i + 1]; ++k) {
        const int f = m.winc_face[k];
        int o[2], n = 0;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            int vv = m.wall_v[cc * F + f];
            if (vv != i && n < 2) o[n++] = vv;
        }
        const double A = m.wall_area[f], nx = m.wall_n[f], ny = m.wall_n[F + f], nz = m.wall_n[2 * F + f];
#pragma unroll
        for (int q = 1; q < 19; ++q) {
            const double en = edot3(q, nx, ny, nz);
            if (en < 0.0) {
                const int qo = opp3(q);
                const double di = ps[qo * Np + i] - ps[q * Np + i];
                const double d1 = ps[qo * Np + o[0]] - ps[q * Np + o[0]];
                const double d2 = ps[qo * Np + o[1]] - ps[q * Np + o[1]];
                acc[q] += -c.dt * en * (A * (1.0 / 6.0) * di + A * (1.0 / 12.0) * (d1 + d2));
            }
        }
    }
    const double sc = m.inv_lumped[i] * first_scale;
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        const size_t r = (size_t)(19 * s + q) * Np + i;
        b.rhs[r] = acc[q];
        if (kMixed) {
            const size_t a = (size_t)i * kRow + slot(s, q);
            b.r32[a] = (float)acc[q];
            b.e1[a] = (float)(acc[q] * sc);
        } else {
            b.x1[r] = acc[q] * sc;
        }
    }
    if (kMixed) {
        b.r32[(size_t)i * kRow + slot(s, 19)] = 0.0f;
        b.e1[(size_t)i * kRow + slot(s, 19)] = 0.0f;
    }
}

// ---------------------------------------------- K6: Chebyshev sweeps ------
// x_{k+1} = x_k + a (x_k - x_{k-1}) + c m^{-1} (b - M x_k): the three-term
// Chebyshev recurrence for the lumped-mass preconditioned consistent mass
// matrix, spectrum in [1/5, 1] on any P1 tetrahedral mesh.
__global__ void __launch_bounds__(kNodeBlock) k3_cheb(DevMesh3 m, Bufs3 b, const double* __restrict__ cur,
                                                      double* prev, double a, double cc, int first, int add_to_psi) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const int Np = m.Np;
    const size_t off = (size_t)19 * blockIdx.y * Np;
    const double* cu = cur + off;
    double acc[19];
#pragma unroll
    for (int q = 0; q < 19; ++q) acc[q] = 0.0;
    for (int k = m.row_ptr[i]; k < m.row_ptr[i + 1]; ++k) {
        const int j = m.col[k];
        const double mv = m.mval[k];
#pragma unroll
        for (int q = 0; q < 19; ++q) acc[q] += mv * cu[q * Np + j];
    }
    const double sc = cc * m.inv_lumped[i];
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        const size_t r = off + (size_t)q * Np + i;
        double xk = cur[r];
        double xm = first ? 0.0 : prev[r];
        double xn = xk + a * (xk - xm) + sc * (b.rhs[r] - acc[q]);
        if (add_to_psi)
            b.psi[r] += xn;
        else
            prev[r] = xn;
    }
}

// Mixed-precision solve: each correction e of M11 e = rho runs FP32 sweeps
// (same recurrence, FP32 matrix copy); the residual rho is carried in FP64.
enum Final3 { kStore3 = 0, kAddPsi3 = 1, kUpdateDev3 = 2 };

template <int kFinal>
__global__ void __launch_bounds__(kNodeBlock) k3_sweep32(DevMesh3 m, Phys3 c, Bufs3 b, const float* __restrict__ cur,
                                                         float* nxt, float tau, int have_x64);

// x <- x + e ; rho <- rho - M11 e (FP64); FP32 copy of rho and the first
// iterate of the next correction, tau_0 rho / m.  x64 = x0, rho64 = x1.
__global__ void __launch_bounds__(kNodeBlock) k3_refine(DevMesh3 m, Bufs3 b, const float* __restrict__ e,
                                                        float* next_first, int first_round, double tau0) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const int Np = m.Np;
    const size_t off = (size_t)19 * blockIdx.y * Np;
    double acc[19];
#pragma unroll
    for (int q = 0; q < 19; ++q) acc[q] = 0.0;
    const int s = blockIdx.y;
    for (int k = m.row_ptr[i]; k < m.row_ptr[i + 1]; ++k) {
        const float* ej = e + (size_t)m.col[k] * kRow + slot(s, 0);
        const double mv = m.mval[k];
#pragma unroll
        for (int q = 0; q < 19; ++q) acc[q] += mv * (double)ej[q];
    }
    const double sc = m.inv_lumped[i] * tau0;
    const size_t a0 = (size_t)i * kRow + slot(s, 0);
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        const size_t r = off + (size_t)q * Np + i;
        double xo = first_round ? 0.0 : b.x0[r];
        double ro = first_round ? b.rhs[r] : b.x1[r];
        double rn = ro - acc[q];
        b.x0[r] = xo + (double)e[a0 + q];
        b.x1[r] = rn;
        b.r32[a0 + q] = (float)rn;
        next_first[a0 + q] = (float)(rn * sc);
    }
}

// ------------------------------------------------ FP32 Chebyshev sweep ----
// One group of five lanes per node; the iterates and the residual are
// node-major rows, the matrix is read from the column-major ELL copy
// (coalesced) when the mesh has one.
__device__ void dev32_update3(const DevMesh3& m, const Phys3& c, const Bufs3& b, const Coop& k, int i,
                              const float4& dg, const float4& dh);

__device__ __forceinline__ void pdl_wait3() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release3() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// One Richardson step x_{k+1} = x_k + tau_k m^{-1} (b - M x_k) of the FP32
// solve, tau_k the reciprocal Chebyshev roots of the spectrum [1/5, 1] taken
// largest and smallest alternately (after K steps: the scaled Chebyshev error
// polynomial; every partial product stays below 1).  Reads x_k (gathered)
// and b only.
// kW > 0: ELL of that width, its columns and values loaded up front (they
// do not depend on the previous sweep, so under programmatic dependent
// launch they are fetched while that sweep drains); kW = 0: CSR.
template <int kFinal, int kW>
__global__ void __launch_bounds__(kCoopBlock) k3_sweep32(DevMesh3 m, Phys3 c, Bufs3 b, const float* __restrict__ cur,
                                                         float* nxt, float tau, int have_x64) {
    pdl_release3();
    const Coop k = coop_index(m.N);
    const int i = k.active ? k.item : 0;      // idle lanes read node 0 and write nothing
    const int Np = m.Np;
    constexpr int kWr = kW > 0 ? kW : 1;
    int col[kWr];
    float val[kWr];
    if (kW > 0 && k.active) {
#pragma unroll
        for (int e = 0; e < kWr; ++e) {
            col[e] = m.ell_col[e * Np + i];
            val[e] = m.ell_val[e * Np + i];
        }
    }
    const float sc = tau * m.inv_lumped32[i];
    pdl_wait3();
    float4 ag = make_float4(0.0f, 0.0f, 0.0f, 0.0f), ah = ag;
    if (k.active) {
        if (kW > 0) {
#pragma unroll
            for (int e = 0; e < kWr; ++e) {
                const float4* row = reinterpret_cast<const float4*>(cur + (size_t)col[e] * kRow);
                fma4(ag, val[e], row[k.c]);
                fma4(ah, val[e], row[5 + k.c]);
            }
        } else {
            for (int e = m.row_ptr[i]; e < m.row_ptr[i + 1]; ++e) {
                const float4* row = reinterpret_cast<const float4*>(cur + (size_t)m.col[e] * kRow);
                const float v = m.mval32[e];
                fma4(ag, v, row[k.c]);
                fma4(ah, v, row[5 + k.c]);
            }
        }
    }
    const size_t own = (size_t)i * kRow;
    const float4* xk4 = reinterpret_cast<const float4*>(cur + own);
    const float4* r4 = reinterpret_cast<const float4*>(b.r32 + own);
    float4 xn[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int v = 5 * h + k.c;
        const float4 xk = xk4[v], rr = r4[v], acc = h ? ah : ag;
        xn[h].x = xk.x + sc * (rr.x - acc.x);
        xn[h].y = xk.y + sc * (rr.y - acc.y);
        xn[h].z = xk.z + sc * (rr.z - acc.z);
        xn[h].w = xk.w + sc * (rr.w - acc.w);
        if (kFinal == kStore3 && k.active) reinterpret_cast<float4*>(nxt + own)[v] = xn[h];
    }
    if constexpr (kFinal == kAddPsi3) {
        // FP64 storage: psi += x64 + e for this lane's directions
        if (k.active) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int q = 4 * k.c + j;
                if (q >= 19) continue;
                const size_t rg = (size_t)q * Np + i, rh = (size_t)(19 + q) * Np + i;
                b.psi[rg] += have_x64 ? b.x0[rg] + (double)comp(xn[0], j) : (double)comp(xn[0], j);
                b.psi[rh] += have_x64 ? b.x0[rh] + (double)comp(xn[1], j) : (double)comp(xn[1], j);
            }
        }
    }
    if constexpr (kFinal == kUpdateDev3) dev32_update3(m, c, b, k, i, xn[0], xn[1]);
}

// The store step with ten lanes per node (three nodes per warp): lane c of a
// node's group accumulates and writes float4 c of the 160-byte rows (c < 5:
// g, c >= 5: h), so each gathered row is one contiguous 160-byte load of the
// group -- two L1 wavefronts -- instead of two 80-byte halves loaded by five
// lanes.  Same arithmetic per component as k3_sweep32<kStore3>.  The row's
// columns and values are loaded in the loop, which keeps the kernel at 32
// registers (16 blocks of 128 per SM; 4 % faster than holding them all).
constexpr int kRowLanes = 10;
constexpr int kRowGroups = 3;                       // per warp (30 of 32 lanes)
constexpr int kRowItemsPerBlock = kRowGroups * (kCoopBlock / 32);

template <int kW>
__global__ void __launch_bounds__(kCoopBlock, 16) k3_sweep_rows32(DevMesh3 m, Phys3 c, Bufs3 b,
                                                              const float* __restrict__ cur, float* nxt, float tau) {
    pdl_release3();
    const int lane = threadIdx.x & 31, grp = lane / kRowLanes, cc = lane - grp * kRowLanes;
    const int item = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * kRowGroups + grp;
    const bool active = grp < kRowGroups && item < m.N;
    const int i = active ? item : 0;
    const int Np = m.Np;
    const float sc = tau * m.inv_lumped32[i];
    pdl_wait3();
    if (!active) return;
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
    for (int e = 0; e < kW; ++e) {
        const int cl = m.ell_col[e * Np + i];
        fma4(acc, m.ell_val[e * Np + i], reinterpret_cast<const float4*>(cur + (size_t)cl * kRow)[cc]);
    }
    const size_t own = (size_t)i * kRow;
    const float4 xk = reinterpret_cast<const float4*>(cur + own)[cc];
    const float4 rr = reinterpret_cast<const float4*>(b.r32 + own)[cc];
    float4 xn;
    xn.x = xk.x + sc * (rr.x - acc.x);
    xn.y = xk.y + sc * (rr.y - acc.y);
    xn.z = xk.z + sc * (rr.z - acc.z);
    xn.w = xk.w + sc * (rr.w - acc.w);
    reinterpret_cast<float4*>(nxt + own)[cc] = xn;
}

// ----------------------------------------------- permutation kernels ------
__global__ void k3_scatter_in(DevMesh3 m, const double* __restrict__ stage, double* dst, int rows) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    int o = m.perm[i];
    for (int q = 0; q < rows; ++q) dst[(size_t)q * m.Np + i] = stage[(size_t)q * m.N + o];
}
__global__ void k3_gather_out(DevMesh3 m, const double* __restrict__ src, double* stage, int rows) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    int o = m.perm[i];
    for (int q = 0; q < rows; ++q) stage[(size_t)q * m.N + o] = src[(size_t)q * m.Np + i];
}
// rest state from C0 (staged in caller order): g = 0, h = w C0
__global__ void k3_init_state(DevMesh3 m, const double* __restrict__ stage, double* psi) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    double C = stage[m.perm[i]];
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        psi[(size_t)q * m.Np + i] = 0.0;
        psi[(size_t)(19 + q) * m.Np + i] = wq3(q) * C;
    }
}

// ------------------------------------------------------- diagnostics ------
struct DiagReq3 {
    double cx, cy, cz, radius, band;
    int32_t substrate, use_band, dev32;
};

// Area of the part of a triangle (area A, nodal values c) where the linear
// interpolant is >= 1/2.
__device__ __forceinline__ double wet_fraction_area(double A, double c0, double c1, double c2) {
    double hi = fmax(c0, fmax(c1, c2)), lo = fmin(c0, fmin(c1, c2));
    double mid = c0 + c1 + c2 - hi - lo;
    if (lo >= 0.5) return A;
    if (hi < 0.5) return 0.0;
    if (mid < 0.5) return A * (hi - 0.5) / (hi - mid) * (hi - 0.5) / (hi - lo);
    return A * (1.0 - (0.5 - lo) / (hi - lo) * (0.5 - lo) / (mid - lo));
}

__device__ __forceinline__ double min_image_d(double d, double L) { return L > 0.0 ? d - L * rint(d / L) : d; }

// x >= t and x <= t for a positive threshold t, on the bit patterns (integer
// pipe; FP64 compares share the 1/64-rate FP64 pipe): for x >= 0 the patterns
// order like the values, and any x with the sign bit set is a negative
// integer, below the pattern of t.  NaNs compare by their pattern; non-finite
// states are counted in their own slot.
__device__ __forceinline__ bool ge_pos3(double x, double t) { return __double_as_longlong(x) >= __double_as_longlong(t); }
__device__ __forceinline__ bool le_pos3(double x, double t) { return __double_as_longlong(x) <= __double_as_longlong(t); }

// slots: 0 sum m C, 1 sum rho |u|^2, 2 max |u|^2, 3-4 sum m p / sum m over
// C >= 0.95, 5-6 the same over C <= 0.05, 7-8 sum m rho|u|^2 / sum m over the
// band, 9 wetted area, 10 max height of a C = 1/2 crossing, 11 non-finite count
__global__ void __launch_bounds__(256) k3_diag_partial(DevMesh3 m, Phys3 c, Bufs3 b, DiagReq3 rq) {
    double s[kDiagSlots];
#pragma unroll
    for (int k = 0; k < kDiagSlots; ++k) s[k] = 0.0;
    s[10] = -INFINITY;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    for (int i = tid; i < m.N; i += nth) {
        const double C = b.C[i];
        double p, ux, uy, uz;
        if (rq.dev32) {
            p = b.p32[i];
            ux = b.ux32[i];
            uy = b.uy32[i];
            uz = b.uz32[i];
        } else {
            p = b.p[i];
            ux = b.ux[i];
            uy = b.uy[i];
            uz = b.uz[i];
        }
        const double lw = m.lumped[i];
        const double rho = c.rho_v + C * (c.rho_l - c.rho_v);
        const double uu = ux * ux + uy * uy + uz * uz;
        if (!isfinite(C + p + uu)) s[11] += 1.0;
        s[0] += lw * C;
        s[1] += rho * uu;
        s[2] = fmax(s[2], uu);
        if (ge_pos3(C, 0.95)) {
            s[3] += lw * p;
            s[4] += lw;
        } else if (le_pos3(C, 0.05)) {
            s[5] += lw * p;
            s[6] += lw;
        }
        if (rq.use_band) {
            double dx = min_image_d(m.x[i] - rq.cx, m.period[0]);
            double dy = min_image_d(m.y[i] - rq.cy, m.period[1]);
            double dz = min_image_d(m.z[i] - rq.cz, m.period[2]);
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            if (fabs(r - rq.radius) <= rq.band) {
                s[7] += lw * rho * uu;
                s[8] += lw;
            }
        }
    }
    if (rq.substrate >= 0) {
        const int F = m.F, Tp = m.Tp;
        for (int f = tid; f < F; f += nth)
            if (m.wall_id[f] == rq.substrate)
                s[9] += wet_fraction_area(m.wall_area[f], b.C[m.wall_v[f]], b.C[m.wall_v[F + f]], b.C[m.wall_v[2 * F + f]]);
        for (int t = tid; t < m.T; t += nth) {
            int v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) v[k] = m.tet[k * Tp + t];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int e = a + 1; e < 4; ++e) {
                    double Ca = b.C[v[a]], Cb = b.C[v[e]];
                    if (ge_pos3(Ca, 0.5) != ge_pos3(Cb, 0.5)) {
                        double w = (0.5 - Ca) / (Cb - Ca);
                        double dz = min_image_d(m.z[v[e]] - m.z[v[a]], m.period[2]);
                        s[10] = fmax(s[10], m.z[v[a]] + w * dz);
                    }
                }
        }
    }
    // block reduction in a fixed order, every partial added once (FP64 adds
    // run at 1/64 rate): the threads' partials through shared memory, 8
    // threads per slot over interleaved segments of 32, then one per slot
    constexpr int kSeg = 8, kL = 256 + 2;
    __shared__ double sh[kDiagSlots][kL];
    __shared__ double part[kDiagSlots][kSeg];
#pragma unroll
    for (int k = 0; k < kDiagSlots; ++k) sh[k][threadIdx.x] = s[k];
    __syncthreads();
    if (threadIdx.x < kDiagSlots * kSeg) {
        const int k = threadIdx.x / kSeg, seg = threadIdx.x - k * kSeg;
        const bool is_max = k == 2 || k == 10;
        double v = sh[k][seg];
        for (int j = 1; j < 32; ++j) v = is_max ? fmax(v, sh[k][seg + kSeg * j]) : v + sh[k][seg + kSeg * j];
        part[k][seg] = v;
    }
    __syncthreads();
    if (threadIdx.x < kDiagSlots) {
        const int k = threadIdx.x;
        const bool is_max = k == 2 || k == 10;
        double v = part[k][0];
        for (int w = 1; w < kSeg; ++w) v = is_max ? fmax(v, part[k][w]) : v + part[k][w];
        b.diag_part[blockIdx.x * kDiagSlots + k] = v;
    }
}

// one warp per slot over the block partials, fixed order
__global__ void k3_diag_final(Bufs3 b) {
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (k >= kDiagSlots) return;
    const bool is_max = k == 2 || k == 10;
    double v = is_max ? -INFINITY : 0.0;
    for (int blk = lane; blk < kDiagBlocks; blk += 32) {
        double w = b.diag_part[blk * kDiagSlots + k];
        v = is_max ? fmax(v, w) : v + w;
    }
    for (int o = 16; o > 0; o >>= 1) {
        double w = __shfl_down_sync(0xffffffffu, v, o);
        v = is_max ? fmax(v, w) : v + w;
    }
    if (lane == 0) b.diag_out[k] = v;
}

#include "felbm3d_dev32.cuh"

// --------------------------------------------------------- host side ------
static int cuda_fail(cudaError_t e, const char* what) {
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    set_error(buf);
    return FELBM_ERR_CUDA;
}
#define FELBM3_CUDA(call)                                  \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// Bump allocator over the caller's workspace (256-byte aligned pieces).
struct Carver3 {
    char* base;
    size_t off = 0;
    explicit Carver3(void* b) : base(static_cast<char*>(b)) {}
    template <class T>
    T* take(size_t n) {
        off = (off + 255) & ~size_t(255);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += n * sizeof(T);
        return p;
    }
};

static size_t pad64(size_t n) { return (n + 63) & ~size_t(63); }

// ELL widths with a compiled sweep: the longest row rounded up; 0 (CSR) beyond 32.
static int ell_width3(const HostMesh3D& h) {
    for (int w : {15, 16, 24, 32})
        if (h.max_degree <= w) return w;
    return 0;
}

// Workspace layout; with base == nullptr only the size is computed.
static size_t carve3(const HostMesh3D& h, bool dev32, void* base, DevMesh3* dm, Bufs3* bo) {
    Carver3 cv(base);
    const size_t Np = pad64(h.N), Tp = pad64(h.T);
    const size_t nnz = h.row_ptr[h.N], ninc = h.inc_ptr[h.N], nwinc = std::max<size_t>(h.winc_ptr[h.N], 1);
    const size_t F = std::max<int32_t>(h.F, 1);
    DevMesh3 d{};
    d.tet = cv.take<int32_t>(4 * Tp);
    d.vol = cv.take<double>(Tp);
    d.grad = cv.take<double>(12 * Tp);
    d.nbr = cv.take<int32_t>(4 * Tp);
    d.vol32 = cv.take<float>(Tp);
    d.grad32 = cv.take<float>(12 * Tp);
    d.row_ptr = cv.take<int32_t>(h.N + 1);
    d.col = cv.take<int32_t>(nnz);
    d.mval = cv.take<double>(nnz);
    d.lval = cv.take<double>(nnz);
    d.ell_w = ell_width3(h);
    d.ell_col = cv.take<int32_t>((size_t)std::max(d.ell_w, 1) * Np);
    d.ell_val = cv.take<float>((size_t)std::max(d.ell_w, 1) * Np);
    d.mval32 = cv.take<float>(nnz);
    d.inv_lumped = cv.take<double>(Np);
    d.inv_lumped32 = cv.take<float>(Np);
    d.lumped = cv.take<double>(Np);
    d.inv_vol = cv.take<double>(Np);
    d.inc_ptr = cv.take<int32_t>(h.N + 1);
    d.inc_tet = cv.take<int32_t>(ninc);
    d.inc_b = cv.take<double>(3 * ninc);
    d.inc_b32 = cv.take<float>(3 * ninc);
    d.ninc = (int32_t)ninc;
    d.wall_v = cv.take<int32_t>(3 * F);
    d.wall_id = cv.take<int32_t>(F);
    d.wall_phi = cv.take<double>(F);
    d.wall_area = cv.take<double>(F);
    d.wall_n = cv.take<double>(3 * F);
    d.winc_ptr = cv.take<int32_t>(h.N + 1);
    d.winc_face = cv.take<int32_t>(nwinc);
    d.x = cv.take<double>(Np);
    d.y = cv.take<double>(Np);
    d.z = cv.take<double>(Np);
    d.perm = cv.take<int32_t>(h.N);
    d.N = h.N;
    d.T = h.T;
    d.F = h.F;
    d.Np = (int32_t)Np;
    d.Tp = (int32_t)Tp;
    for (int k = 0; k < 3; ++k) d.period[k] = h.period[k];
    Bufs3 b{};
    b.C = cv.take<double>(Np);
    b.mu = cv.take<double>(Np);
    if (!dev32) {
        b.psi = cv.take<double>(38 * Np);
        b.p = cv.take<double>(Np);
        b.ux = cv.take<double>(Np);
        b.uy = cv.take<double>(Np);
        b.uz = cv.take<double>(Np);
        b.gmu = cv.take<double>(3 * Tp);
        b.lmu = b.gmu;
        b.R = cv.take<double>(38 * (size_t)std::max<int32_t>(h.T, 1));
        b.rhs = cv.take<double>(38 * Np);
        b.x0 = cv.take<double>(38 * Np);
        b.x1 = cv.take<double>(38 * Np);
    } else {
        b.dpsi = cv.take<float>((size_t)kRow * Np);
        b.p32 = cv.take<float>(Np);
        b.ux32 = cv.take<float>(Np);
        b.uy32 = cv.take<float>(Np);
        b.uz32 = cv.take<float>(Np);
        b.mu32 = cv.take<float>(Np);
        b.gmu32 = cv.take<float>(3 * Tp);
        b.lmu32 = b.gmu32;
        b.R32 = cv.take<float>((size_t)kRow * std::max<int32_t>(h.T, 1));
    }
    b.r32 = cv.take<float>((size_t)kRow * Np);
    b.e0 = cv.take<float>((size_t)kRow * Np);
    b.e1 = cv.take<float>((size_t)kRow * Np);
    b.stage = cv.take<double>(38 * (size_t)h.N);
    b.in0 = cv.take<double>(38 * (size_t)h.N);
    b.in1 = cv.take<double>(38 * (size_t)h.N);
    b.diag_part = cv.take<double>(kDiagBlocks * kDiagSlots);
    b.diag_out = cv.take<double>(kDiagSlots);
    if (dm) *dm = d;
    if (bo) *bo = b;
    return cv.off + 256;
}

static unsigned grid_for(int n, int block) { return (unsigned)((n + block - 1) / block); }

template <class T>
static cudaError_t up(const T* dst, const std::vector<T>& src, cudaStream_t s) {
    if (src.empty()) return cudaSuccess;
    return cudaMemcpyAsync(const_cast<T*>(dst), src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s);
}

}  // namespace felbm3

struct felbm3d_state {
    felbm::HostMesh3D hm;
    felbm_params prm;
    felbm3::DevMesh3 dm{};
    felbm3::Phys3 phys{};
    felbm3::Bufs3 buf{};
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    int mode = FELBM_SOLVER_MIXED;
    int sweeps = 16;
    int rounds = 3;
    std::vector<double> cheb_a, cheb_c;   // three-term recurrence of the FP64 solve
    double inv_theta = 1.0;               // its first iterate x_1 = m^{-1} b / theta
    std::vector<double> tau;              // Richardson step sizes of the FP32 solves; tau[0] gives x_1
    int64_t step = 0;
    double mass0 = 0.0;
    bool dev32 = false;
    bool timing = false;
    bool timed_step_ran = false;
    bool use_pdl = true;   // programmatic dependent launch between solve sweeps (FELBM_PDL=0: off)
    cudaEvent_t ev[6] = {};
    cudaEvent_t ev_copied = nullptr;   // set_state: the host arrays have been read
    cudaStream_t copy_stream = nullptr;     // set_state's host-to-device copies
    cudaEvent_t ev_in_free[2] = {};         // the conversion that last read buf.in0 / in1 has run
    int in_next = 0;                        // input buffer of the next set_state
};

namespace felbm3 {

template <typename... KArgs, typename... Args>
static void launch3(bool pdl, void (*kern)(KArgs...), unsigned grid, unsigned block, cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// One FP32 sweep with the compiled ELL width of the mesh (else CSR); pdl:
// the previous launch on the stream is a sweep.
template <int kFinal>
static void launch_sweep3(felbm3d_state* st, cudaStream_t s, const float* cur, float* nxt, float tau,
                          int have_x64, bool pdl) {
    const DevMesh3& m = st->dm;
    const unsigned g = grid_for(m.N, kItemsPerBlock);
    pdl = pdl && st->use_pdl;
    if constexpr (kFinal == kStore3) {
        const unsigned gr = grid_for(m.N, kRowItemsPerBlock);
        switch (m.ell_w) {
            case 15: launch3(pdl, k3_sweep_rows32<15>, gr, kCoopBlock, s, m, st->phys, st->buf, cur, nxt, tau); return;
            case 16: launch3(pdl, k3_sweep_rows32<16>, gr, kCoopBlock, s, m, st->phys, st->buf, cur, nxt, tau); return;
            case 24: launch3(pdl, k3_sweep_rows32<24>, gr, kCoopBlock, s, m, st->phys, st->buf, cur, nxt, tau); return;
            case 32: launch3(pdl, k3_sweep_rows32<32>, gr, kCoopBlock, s, m, st->phys, st->buf, cur, nxt, tau); return;
            default: break;
        }
    }
    switch (m.ell_w) {
        case 15: launch3(pdl, k3_sweep32<kFinal, 15>, g, kCoopBlock, s, m, st->phys, st->buf, cur, nxt, tau, have_x64); break;
        case 16: launch3(pdl, k3_sweep32<kFinal, 16>, g, kCoopBlock, s, m, st->phys, st->buf, cur, nxt, tau, have_x64); break;
        case 24: launch3(pdl, k3_sweep32<kFinal, 24>, g, kCoopBlock, s, m, st->phys, st->buf, cur, nxt, tau, have_x64); break;
        case 32: launch3(pdl, k3_sweep32<kFinal, 32>, g, kCoopBlock, s, m, st->phys, st->buf, cur, nxt, tau, have_x64); break;
        default: launch3(pdl, k3_sweep32<kFinal, 0>, g, kCoopBlock, s, m, st->phys, st->buf, cur, nxt, tau, have_x64);
    }
}

static int solve_launches3(const felbm3d_state* st) {
    return st->mode == FELBM_SOLVER_FP64 ? st->sweeps - 1 : st->rounds * (st->sweeps - 1) + (st->rounds - 1);
}
static int step_launches3(const felbm3d_state* st) { return (st->dev32 ? 4 : 5) + solve_launches3(st); }

static void enqueue_solve3(felbm3d_state* st, cudaStream_t s, bool after_release = false);
static void enqueue_step_dev32(felbm3d_state* st, cudaStream_t s);

// phase event k of the timed step, recorded as an external event node
static void mark3(felbm3d_state* st, cudaStream_t s, int k) {
    if (st->timing) cudaEventRecordWithFlags(st->ev[k], s, cudaEventRecordExternal);
}

static void enqueue_step3(felbm3d_state* st, cudaStream_t s) {
    const DevMesh3& m = st->dm;
    const Bufs3& b = st->buf;
    auto mark = [&](int k) { mark3(st, s, k); };
    mark(0);
    if (st->dev32) {
        enqueue_step_dev32(st, s);
        return;
    }
    k3_collide<<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, st->phys, b, 1);
    k3_mu<<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, st->phys, b);
    mark(1);
    if (st->phys.lapmu_nodal)
        k3_lmu<<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, st->phys, b);
    else
        k3_gradmu<<<grid_for(m.T, kBlock), kBlock, 0, s>>>(m, b);
    mark(2);
    k3_element<<<grid_for(m.T, 128), 128, 0, s>>>(m, st->phys, b);
    mark(3);
    const dim3 g2(grid_for(m.N, kNodeBlock), 2);
    if (st->mode == FELBM_SOLVER_FP64)
        k3_rhs<false><<<g2, kNodeBlock, 0, s>>>(m, st->phys, b, st->inv_theta);
    else
        k3_rhs<true><<<g2, kNodeBlock, 0, s>>>(m, st->phys, b, st->tau[0]);
    mark(4);
    enqueue_solve3(st, s);
    mark(5);
}

// The consistent-mass solve of one step; the last sweep adds the increment
// to psi.
static void enqueue_solve3(felbm3d_state* st, cudaStream_t s, bool after_release) {
    const DevMesh3& m = st->dm;
    const Bufs3& b = st->buf;
    const dim3 g2(grid_for(m.N, kNodeBlock), 2);
    if (st->mode == FELBM_SOLVER_FP64) {
        for (int k = 1; k < st->sweeps; ++k) {
            const double* cur = (k & 1) ? b.x1 : b.x0;
            double* prev = (k & 1) ? b.x0 : b.x1;
            k3_cheb<<<g2, kNodeBlock, 0, s>>>(m, b, cur, prev, st->cheb_a[k], st->cheb_c[k], k == 1,
                                              k == st->sweeps - 1);
        }
        return;
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
            const bool pdl = k > 1 || (k == 1 && r == 0 && after_release);
            if (!last)
                launch_sweep3<kStore3>(st, s, cur, prv, tau, have_x64, pdl);
            else if (st->dev32)
                launch_sweep3<kUpdateDev3>(st, s, cur, prv, tau, have_x64, pdl);
            else
                launch_sweep3<kAddPsi3>(st, s, cur, prv, tau, have_x64, pdl);
            std::swap(cur, prv);
        }
        if (r < st->rounds - 1) {
            k3_refine<<<g2, kNodeBlock, 0, s>>>(m, b, cur, prv, r == 0, st->tau[0]);
            A = prv;
            B = cur;
        }
    }
}

static int build_graph3(felbm3d_state* st) {
    if (!st->cap_stream) FELBM3_CUDA(cudaStreamCreateWithFlags(&st->cap_stream, cudaStreamNonBlocking));
    FELBM3_CUDA(cudaStreamBeginCapture(st->cap_stream, cudaStreamCaptureModeThreadLocal));
    enqueue_step3(st, st->cap_stream);
    cudaError_t e = cudaStreamEndCapture(st->cap_stream, &st->graph);
    if (e != cudaSuccess) return cuda_fail(e, "felbm3d_step: capture");
    FELBM3_CUDA(cudaGraphInstantiate(&st->graph_exec, st->graph, 0));
    return FELBM_OK;
}

static void drop_graph3(felbm3d_state* st) {
    if (st->graph_exec) cudaGraphExecDestroy(st->graph_exec);
    if (st->graph) cudaGraphDestroy(st->graph);
    st->graph_exec = nullptr;
    st->graph = nullptr;
}

// Fields of the current state (FP64 storage: moments without collision).
static void refresh_fields(felbm3d_state* st) {
    if (!st->dev32)
        k3_collide<<<grid_for(st->dm.N, kBlock), kBlock, 0, st->stream>>>(st->dm, st->phys, st->buf, 0);
}

static int check_params3(const felbm_params* p) {
    if (!p || !(p->dt > 0.0) || !(p->tau_l > 0.0) || !(p->tau_v > 0.0) || !(p->rho_l > 0.0) || !(p->rho_v > 0.0) ||
        !(p->kappa >= 0.0) || !(p->beta >= 0.0) || !(p->mobility >= 0.0) || p->n_wall_ids < 0 ||
        p->n_wall_ids > FELBM_MAX_WALL_IDS || (p->lap_mode != FELBM_LAP_CONSISTENT && p->lap_mode != FELBM_LAP_PAPER) ||
        (p->precision != FELBM_FP64 && p->precision != FELBM_FP32_DEV) ||
        (p->solver_mode != FELBM_SOLVER_MIXED && p->solver_mode != FELBM_SOLVER_FP64) || p->solver_iters < 0 ||
        p->solver_iters == 1 || p->solver_iters > 256 || p->solver_rounds < 0 || p->solver_rounds > 8 ||
        (p->lapmu_mode != FELBM_LAPMU_FACE && p->lapmu_mode != FELBM_LAPMU_NODAL)) {
        set_error("felbm3d_init: invalid parameters");
        return FELBM_ERR_INVALID_ARG;
    }
    if (p->precision == FELBM_FP32_DEV && (p->solver_mode != FELBM_SOLVER_MIXED || p->solver_rounds > 1)) {
        set_error("felbm3d_init: FP32_DEV storage takes the MIXED solver with one correction");
        return FELBM_ERR_UNSUPPORTED;
    }
    return FELBM_OK;
}

static int init_state_from_stage(felbm3d_state* st);   // FP64 or FP32-deviation state from C0 in stage
static int diag_run(felbm3d_state* st, const DiagReq3& rq, double* out);

}  // namespace felbm3

using namespace felbm3;

extern "C" {

int felbm3d_workspace_bytes(const felbm3d_mesh* mesh, const felbm_params* params, size_t* bytes) {
    if (!mesh || !params || !bytes) {
        set_error("felbm3d_workspace_bytes: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    *bytes = carve3(mesh->h, params->precision == FELBM_FP32_DEV, nullptr, nullptr, nullptr);
    return FELBM_OK;
}

int felbm3d_init(const felbm3d_mesh* mesh, const felbm_params* params, const double* C0, void* d_workspace,
                 size_t workspace_bytes, void* stream, felbm3d_state** out) {
    if (!mesh || !C0 || !out) {
        set_error("felbm3d_init: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    *out = nullptr;
    int rc = check_params3(params);
    if (rc) return rc;
    const HostMesh3D& h = mesh->h;
    for (int32_t f = 0; f < h.F; ++f)
        if (h.wall_id[f] >= params->n_wall_ids) {
            set_error("felbm3d_init: a wall id has no phi_c (n_wall_ids too small)");
            return FELBM_ERR_INVALID_ARG;
        }
    const bool dev32 = params->precision == FELBM_FP32_DEV;
    const size_t need = carve3(h, dev32, nullptr, nullptr, nullptr);
    if (!d_workspace || workspace_bytes < need || (reinterpret_cast<uintptr_t>(d_workspace) & 255)) {
        set_error("felbm3d_init: workspace missing, not 256-byte aligned or smaller than felbm3d_workspace_bytes");
        return FELBM_ERR_WORKSPACE;
    }
    felbm3d_state* st = new (std::nothrow) felbm3d_state;
    if (!st) {
        set_error("felbm3d_init: out of host memory");
        return FELBM_ERR_INVALID_ARG;
    }
    st->hm = h;
    st->prm = *params;
    st->stream = static_cast<cudaStream_t>(stream);
    st->dev32 = dev32;
    if (const char* env = std::getenv("FELBM_PDL")) st->use_pdl = std::atoi(env) != 0;
    carve3(h, dev32, d_workspace, &st->dm, &st->buf);
    Phys3& ph = st->phys;
    ph.dt = params->dt;
    ph.tau_l = params->tau_l;
    ph.tau_v = params->tau_v;
    ph.rho_l = params->rho_l;
    ph.rho_v = params->rho_v;
    ph.kappa = params->kappa;
    ph.beta = params->beta;
    ph.mobility = params->mobility;
    ph.lapmu_nodal = params->lapmu_mode == FELBM_LAPMU_NODAL;
    // lval = -3 K_ij / (s |patch_i|); the lumped P1 Laplacian is -K_ij / (|patch_i| / 4)
    ph.lapmu_fac = (params->lap_mode == FELBM_LAP_PAPER ? 1.0 : 0.75) * 4.0 / 3.0;
    ph.dt_f = (float)params->dt;
    ph.dt4_f = (float)(0.25 * params->dt);
    ph.dt2h_f = (float)(0.5 * params->dt * params->dt);
    ph.inv_tau_l_f = (float)(1.0 / params->tau_l);
    ph.inv_tau_v_f = (float)(1.0 / params->tau_v);
    ph.rho_v_f = (float)params->rho_v;
    ph.drho_f = (float)(params->rho_l - params->rho_v);
    ph.mobility_f = (float)params->mobility;

    // Chebyshev coefficients for the spectrum [1/5, 1] of m^{-1} M11 (the
    // element matrix (I + 1 1^T) V/20 against its lumped diagonal V/4 has
    // eigenvalues 1/5 and 1)
    st->mode = params->solver_mode;
    st->sweeps = params->solver_iters ? params->solver_iters : (st->mode == FELBM_SOLVER_FP64 ? 36 : 16);
    st->rounds = st->mode == FELBM_SOLVER_FP64 ? 1 : (params->solver_rounds ? params->solver_rounds : (dev32 ? 1 : 3));
    const double lmin = 0.2, lmax = 1.0;
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
    // lambda_j = theta + delta cos((2j+1) pi / 2K), in the order j = 0, K-1,
    // 1, K-2, ... (largest and smallest root alternately)
    st->tau.assign(st->sweeps, 1.0);
    for (int k = 0; k < st->sweeps; ++k) {
        const int K = st->sweeps, j = (k & 1) ? K - 1 - k / 2 : k / 2;
        st->tau[k] = 1.0 / (theta + delta * std::cos((2.0 * j + 1.0) * 3.14159265358979323846 / (2.0 * K)));
    }

    // host-side derived tables
    const DevMesh3& d = st->dm;
    const double scale = params->lap_mode == FELBM_LAP_PAPER ? 1.0 : 0.75;
    const size_t Np = d.Np, Tp = d.Tp, nnz = h.row_ptr[h.N];
    std::vector<double> inv_vol(h.N), inv_lumped(h.N), lval(nnz), wall_phi(h.F);
    std::vector<float> inv_lumped32(h.N), mval32(h.mass.begin(), h.mass.end());
    std::vector<float> inc_b32(h.inc_b.begin(), h.inc_b.end());
    for (int32_t f = 0; f < h.F; ++f) wall_phi[f] = params->phi_c[h.wall_id[f]];
    for (int32_t i = 0; i < h.N; ++i) {
        inv_vol[i] = 1.0 / (scale * h.patch[i]);
        inv_lumped[i] = 1.0 / h.lumped[i];
        inv_lumped32[i] = (float)inv_lumped[i];
        for (int32_t k = h.row_ptr[i]; k < h.row_ptr[i + 1]; ++k) lval[k] = -3.0 * h.stiff[k] * inv_vol[i];
    }
    const int ellw = d.ell_w;
    std::vector<int32_t> ell_col((size_t)std::max(ellw, 1) * Np, 0);
    std::vector<float> ell_val((size_t)std::max(ellw, 1) * Np, 0.0f);
    for (int32_t i = 0; i < h.N && ellw > 0; ++i) {
        const int32_t r0 = h.row_ptr[i], len = h.row_ptr[i + 1] - r0;
        for (int k = 0; k < ellw; ++k) {
            const size_t at = (size_t)k * Np + i;
            ell_col[at] = k < len ? h.col[r0 + k] : i;
            ell_val[at] = k < len ? (float)h.mass[r0 + k] : 0.0f;
        }
    }
    auto pad_t = [&](const auto& src, int rows) {
        using V = typename std::decay_t<decltype(src)>::value_type;
        std::vector<V> o((size_t)rows * Tp, V(0));
        for (int r = 0; r < rows; ++r)
            std::copy(src.begin() + (size_t)r * h.T, src.begin() + (size_t)(r + 1) * h.T, o.begin() + (size_t)r * Tp);
        return o;
    };
    std::vector<int32_t> tet_p = pad_t(h.tet, 4), nbr_p = pad_t(h.nbr, 4);
    std::vector<double> grad_p = pad_t(h.grad, 12), vol_p = pad_t(h.vol, 1);
    std::vector<float> grad32_p(grad_p.begin(), grad_p.end()), vol32_p(vol_p.begin(), vol_p.end());
    std::vector<double> xp(Np, 0.0), yp(Np, 0.0), zp(Np, 0.0);
    std::copy(h.x.begin(), h.x.end(), xp.begin());
    std::copy(h.y.begin(), h.y.end(), yp.begin());
    std::copy(h.z.begin(), h.z.end(), zp.begin());
    cudaStream_t s = st->stream;
    cudaError_t e = cudaMemsetAsync(d_workspace, 0, need, s);
#define UP3(dst, src) \
    if (e == cudaSuccess) e = up(dst, src, s)
    UP3(d.tet, tet_p);
    UP3(d.vol, vol_p);
    UP3(d.grad, grad_p);
    UP3(d.nbr, nbr_p);
    UP3(d.vol32, vol32_p);
    UP3(d.grad32, grad32_p);
    UP3(d.row_ptr, h.row_ptr);
    UP3(d.col, h.col);
    UP3(d.mval, h.mass);
    UP3(d.lval, lval);
    UP3(d.ell_col, ell_col);
    UP3(d.ell_val, ell_val);
    UP3(d.mval32, mval32);
    UP3(d.inv_lumped, inv_lumped);
    UP3(d.inv_lumped32, inv_lumped32);
    UP3(d.lumped, h.lumped);
    UP3(d.inv_vol, inv_vol);
    UP3(d.inc_ptr, h.inc_ptr);
    UP3(d.inc_tet, h.inc_tet);
    UP3(d.inc_b, h.inc_b);
    UP3(d.inc_b32, inc_b32);
    UP3(d.wall_v, h.wall_v);
    UP3(d.wall_id, h.wall_id);
    UP3(d.wall_phi, wall_phi);
    UP3(d.wall_area, h.wall_area);
    UP3(d.wall_n, h.wall_n);
    UP3(d.winc_ptr, h.winc_ptr);
    UP3(d.winc_face, h.winc_face);
    UP3(d.x, xp);
    UP3(d.y, yp);
    UP3(d.z, zp);
    UP3(d.perm, h.perm);
#undef UP3
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(st->buf.stage, C0, sizeof(double) * h.N, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        rc = cuda_fail(e, "felbm3d_init: upload");
        delete st;
        return rc;
    }
    rc = init_state_from_stage(st);
    if (rc == FELBM_OK) {
        double v[kDiagSlots];
        DiagReq3 rq{};
        rq.substrate = -1;
        rq.dev32 = st->dev32;
        rc = diag_run(st, rq, v);
        st->mass0 = v[0];
    }
    if (rc != FELBM_OK) {
        delete st;
        return rc;
    }
    *out = st;
    return FELBM_OK;
}

int felbm3d_step(felbm3d_state* st, int32_t n_steps) {
    if (!st || n_steps < 0) {
        set_error("felbm3d_step: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    if (!st->graph_exec) {
        int rc = build_graph3(st);
        if (rc) return rc;
    }
    for (int32_t k = 0; k < n_steps; ++k) FELBM3_CUDA(cudaGraphLaunch(st->graph_exec, st->stream));
    st->step += n_steps;
    if (n_steps > 0 && st->timing) st->timed_step_ran = true;
    return FELBM_OK;
}

int felbm3d_step_launches(const felbm3d_state* st, int32_t* n) {
    if (!st || !n) {
        set_error("felbm3d_step_launches: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    *n = step_launches3(st);
    return FELBM_OK;
}

int felbm3d_timing_enable(felbm3d_state* st, int32_t enable) {
    if (!st) {
        set_error("felbm3d_timing_enable: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    if (enable && !st->ev[0])
        for (auto& ev : st->ev) FELBM3_CUDA(cudaEventCreate(&ev));
    FELBM3_CUDA(cudaStreamSynchronize(st->stream));
    drop_graph3(st);
    st->timing = enable != 0;
    st->timed_step_ran = false;
    return FELBM_OK;
}

int felbm3d_timing_get(felbm3d_state* st, double* ms6) {
    if (!st || !ms6 || !st->timing || !st->timed_step_ran) {
        set_error("felbm3d_timing_get: timing is off or no timed step ran");
        return FELBM_ERR_INVALID_ARG;
    }
    FELBM3_CUDA(cudaStreamSynchronize(st->stream));
    double total = 0.0;
    for (int k = 0; k < 5; ++k) {
        float t = 0.0f;
        FELBM3_CUDA(cudaEventElapsedTime(&t, st->ev[k], st->ev[k + 1]));
        ms6[k] = t;
        total += t;
    }
    ms6[5] = total;
    return FELBM_OK;
}

}  // extern "C"

namespace felbm3 {

__global__ void k3_gather_out_f(DevMesh3 m, const float* __restrict__ src, double* stage) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m.N) stage[m.perm[i]] = (double)src[i];
}

// The diagnostics reductions queued on the state's stream, their sums copied
// to out (host) asynchronously.
static int diag_enqueue(felbm3d_state* st, const DiagReq3& rq, double* out) {
    cudaStream_t s = st->stream;
    refresh_fields(st);
    k3_diag_partial<<<kDiagBlocks, 256, 0, s>>>(st->dm, st->phys, st->buf, rq);
    k3_diag_final<<<1, 32 * kDiagSlots, 0, s>>>(st->buf);
    FELBM3_CUDA(cudaGetLastError());
    FELBM3_CUDA(cudaMemcpyAsync(out, st->buf.diag_out, sizeof(double) * kDiagSlots, cudaMemcpyDeviceToHost, s));
    return FELBM_OK;
}

static int diag_run(felbm3d_state* st, const DiagReq3& rq, double* out) {
    int rc = diag_enqueue(st, rq, out);
    if (rc) return rc;
    FELBM3_CUDA(cudaStreamSynchronize(st->stream));
    return FELBM_OK;
}

// Mean height of the substrate's nodes (static geometry).
static double substrate_height(const HostMesh3D& h, int id) {
    std::vector<char> seen(h.N, 0);
    double sum = 0.0;
    int64_t n = 0;
    for (int32_t f = 0; f < h.F; ++f) {
        if (h.wall_id[f] != id) continue;
        for (int c = 0; c < 3; ++c) {
            int32_t v = h.wall_v[(size_t)c * h.F + f];
            if (!seen[v]) {
                seen[v] = 1;
                sum += h.z[v];
                ++n;
            }
        }
    }
    return n ? sum / (double)n : NAN;
}

}  // namespace felbm3

extern "C" {

}  // extern "C"

namespace felbm3 {

static DiagReq3 make_req3(const felbm3d_state* st, const felbm3d_diag_request* req) {
    DiagReq3 rq{};
    rq.substrate = req ? req->substrate_wall_id : -1;
    rq.use_band = req && req->band > 0.0;
    rq.dev32 = st->dev32;
    if (req) {
        rq.cx = req->centre[0];
        rq.cy = req->centre[1];
        rq.cz = req->centre[2];
        rq.radius = req->radius;
        rq.band = req->band;
    }
    return rq;
}

// felbm3d_diag from the reduced sums v of the step `step`.
static felbm3d_diag fill_diag3(const felbm3d_state* st, const DiagReq3& rq, const double* v, int64_t step) {
    felbm3d_diag d{};
    d.step = step;
    d.mass = v[0];
    d.mass0 = st->mass0;
    d.mass_drift_rel = (v[0] - st->mass0) / st->mass0;
    d.kinetic_energy = 0.5 * v[1] / st->hm.N;
    d.max_u = std::sqrt(v[2]);
    d.p_in = v[4] > 0.0 ? v[3] / v[4] : 0.0;
    d.p_out = v[6] > 0.0 ? v[5] / v[6] : 0.0;
    d.delta_p = d.p_in - d.p_out;
    d.interface_rho_uu = v[8] > 0.0 ? v[7] / v[8] : 0.0;
    d.wetted_area = v[9];
    d.height = NAN;
    d.base_diameter = 2.0 * std::sqrt(v[9] / M_PI);
    d.theta_deg = NAN;
    if (rq.substrate >= 0) {
        double zw = substrate_height(st->hm, rq.substrate);
        if (std::isfinite(zw) && std::isfinite(v[10])) {
            d.height = v[10] - zw;
            const double hgt = d.height, b = d.base_diameter;
            if (hgt > 0.0 && b > 0.0) {
                double r = (4.0 * hgt * hgt + b * b) / (8.0 * hgt);
                d.theta_deg = std::atan2(b, 2.0 * (r - hgt)) * 180.0 / M_PI;
            }
        }
    }
    d.status = v[11] > 0.0 ? FELBM_ERR_NONFINITE : FELBM_OK;
    return d;
}

}  // namespace felbm3

extern "C" {

int felbm3d_diagnostics(felbm3d_state* st, const felbm3d_diag_request* req, felbm3d_diag* out) {
    if (!st || !out) {
        set_error("felbm3d_diagnostics: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    const DiagReq3 rq = make_req3(st, req);
    double v[kDiagSlots];
    int rc = diag_run(st, rq, v);
    if (rc) return rc;
    *out = fill_diag3(st, rq, v, st->step);
    return FELBM_OK;
}

int felbm3d_diagnostics_enqueue(felbm3d_state* st, const felbm3d_diag_request* req, double* slots) {
    if (!st || !slots) {
        set_error("felbm3d_diagnostics_enqueue: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    static_assert(kDiagSlots < FELBM_DIAG_SLOTS, "raw diagnostic sums and the step");
    int rc = diag_enqueue(st, make_req3(st, req), slots);
    if (rc) return rc;
    slots[FELBM_DIAG_SLOTS - 1] = (double)st->step;
    return FELBM_OK;
}

int felbm3d_diag_finish(felbm3d_state* st, const felbm3d_diag_request* req, const double* slots,
                        felbm3d_diag* out) {
    if (!st || !slots || !out) {
        set_error("felbm3d_diag_finish: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    *out = fill_diag3(st, make_req3(st, req), slots, (int64_t)slots[FELBM_DIAG_SLOTS - 1]);
    return FELBM_OK;
}

int felbm3d_get_state(felbm3d_state* st, double* g, double* h) {
    if (!st || !g || !h) {
        set_error("felbm3d_get_state: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    cudaStream_t s = st->stream;
    const size_t N = st->hm.N;
    if (st->dev32)
        k3_dev32_to_stage<<<grid_for(st->dm.N, kNodeBlock), kNodeBlock, 0, s>>>(st->dm, st->phys, st->buf);
    else
        k3_gather_out<<<grid_for(st->dm.N, kBlock), kBlock, 0, s>>>(st->dm, st->buf.psi, st->buf.stage, 38);
    FELBM3_CUDA(cudaGetLastError());
    FELBM3_CUDA(cudaMemcpyAsync(g, st->buf.stage, sizeof(double) * 19 * N, cudaMemcpyDefault, s));
    FELBM3_CUDA(cudaMemcpyAsync(h, st->buf.stage + 19 * N, sizeof(double) * 19 * N, cudaMemcpyDefault, s));
    FELBM3_CUDA(cudaStreamSynchronize(s));
    return FELBM_OK;
}

int felbm3d_set_state(felbm3d_state* st, const double* g, const double* h) {
    if (!st || !g || !h) {
        set_error("felbm3d_set_state: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    cudaStream_t s = st->stream;
    const size_t N = st->hm.N;
    if (!st->copy_stream) FELBM3_CUDA(cudaStreamCreateWithFlags(&st->copy_stream, cudaStreamNonBlocking));
    if (!st->ev_copied) FELBM3_CUDA(cudaEventCreateWithFlags(&st->ev_copied, cudaEventDisableTiming));
    for (auto& ev : st->ev_in_free)
        if (!ev) FELBM3_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    // the copy runs on its own stream into the input buffer the previous call
    // did not use, overlapping the work queued on the state's stream; it waits
    // only for the conversion that last read this buffer
    const int k = st->in_next;
    st->in_next ^= 1;
    double* in = k ? st->buf.in1 : st->buf.in0;
    FELBM3_CUDA(cudaStreamWaitEvent(st->copy_stream, st->ev_in_free[k], 0));
    FELBM3_CUDA(cudaMemcpyAsync(in, g, sizeof(double) * 19 * N, cudaMemcpyDefault, st->copy_stream));
    FELBM3_CUDA(cudaMemcpyAsync(in + 19 * N, h, sizeof(double) * 19 * N, cudaMemcpyDefault, st->copy_stream));
    FELBM3_CUDA(cudaEventRecord(st->ev_copied, st->copy_stream));
    FELBM3_CUDA(cudaStreamWaitEvent(s, st->ev_copied, 0));
    if (st->dev32)
        k3_stage_to_dev32<<<grid_for(st->dm.N, kNodeBlock), kNodeBlock, 0, s>>>(st->dm, st->phys, st->buf, in);
    else
        k3_scatter_in<<<grid_for(st->dm.N, kBlock), kBlock, 0, s>>>(st->dm, in, st->buf.psi, 38);
    FELBM3_CUDA(cudaGetLastError());
    FELBM3_CUDA(cudaEventRecord(st->ev_in_free[k], s));
    refresh_fields(st);
    // return once the host arrays have been read; the conversion stays queued
    FELBM3_CUDA(cudaEventSynchronize(st->ev_copied));
    return FELBM_OK;
}

int felbm3d_get_fields(felbm3d_state* st, double* C, double* p, double* ux, double* uy, double* uz, double* mu) {
    if (!st) {
        set_error("felbm3d_get_fields: invalid argument");
        return FELBM_ERR_INVALID_ARG;
    }
    cudaStream_t s = st->stream;
    const DevMesh3& m = st->dm;
    const Bufs3& b = st->buf;
    refresh_fields(st);
    double* outs[6] = {C, p, ux, uy, uz, mu};
    const double* src64[6] = {b.C, b.p, b.ux, b.uy, b.uz, b.mu};
    const float* src32[6] = {nullptr, b.p32, b.ux32, b.uy32, b.uz32, b.mu32};
    for (int k = 0; k < 6; ++k) {
        if (!outs[k]) continue;
        double* dst = b.stage + (size_t)k * st->hm.N;
        if (st->dev32 && k > 0)
            k3_gather_out_f<<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, src32[k], dst);
        else if (st->dev32 && k == 0)
            k3_gather_out<<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, b.C, dst, 1);
        else
            k3_gather_out<<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, src64[k], dst, 1);
        FELBM3_CUDA(cudaGetLastError());
        FELBM3_CUDA(cudaMemcpyAsync(outs[k], dst, sizeof(double) * st->hm.N, cudaMemcpyDeviceToHost, s));
    }
    FELBM3_CUDA(cudaStreamSynchronize(s));
    return FELBM_OK;
}

void felbm3d_state_destroy(felbm3d_state* st) {
    if (!st) return;
    if (st->stream) cudaStreamSynchronize(st->stream);
    drop_graph3(st);
    if (st->cap_stream) cudaStreamDestroy(st->cap_stream);
    for (auto& ev : st->ev)
        if (ev) cudaEventDestroy(ev);
    if (st->ev_copied) cudaEventDestroy(st->ev_copied);
    if (st->copy_stream) cudaStreamDestroy(st->copy_stream);
    for (auto& e : st->ev_in_free)
        if (e) cudaEventDestroy(e);
    delete st;
}

}  // extern "C"

namespace felbm3 {

// One FP32-deviation step: collision is folded into the element, RHS and
// update kernels.
static void enqueue_step_dev32(felbm3d_state* st, cudaStream_t s) {
    const DevMesh3& m = st->dm;
    const Bufs3& b = st->buf;
    // programmatic dependent launch along the chain when no phase events sit
    // between the kernels
    const bool chain = st->use_pdl && !st->timing;
    k3_mu32<<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, st->phys, b);
    mark3(st, s, 1);
    if (st->phys.lapmu_nodal)
        launch3(chain, k3_lmu32, grid_for(m.N, kBlock), kBlock, s, m, st->phys, b);
    else
        launch3(chain, k3_gradmu32, grid_for(m.T, kBlock), kBlock, s, m, b);
    mark3(st, s, 2);
    launch3(chain, k3_element32, grid_for(m.T, kElemTets), kCoopBlock, s, m, st->phys, b);
    mark3(st, s, 3);
    launch3(chain, k3_rhs32, grid_for(m.N, kItemsPerBlock), kCoopBlock, s, m, st->phys, b, (float)st->tau[0]);
    mark3(st, s, 4);
    enqueue_solve3(st, s, chain);
    mark3(st, s, 5);
}

static int init_state_from_stage(felbm3d_state* st) {
    cudaStream_t s = st->stream;
    const DevMesh3& m = st->dm;
    if (st->dev32) {
        k3_init_dev32<<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, st->buf);
    } else {
        k3_init_state<<<grid_for(m.N, kBlock), kBlock, 0, s>>>(m, st->buf.stage, st->buf.psi);
        refresh_fields(st);
    }
    FELBM3_CUDA(cudaGetLastError());
    FELBM3_CUDA(cudaStreamSynchronize(s));
    return FELBM_OK;
}

}  // namespace felbm3
