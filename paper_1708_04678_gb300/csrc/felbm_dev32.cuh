// FP32 deviation storage of the FE-LBM step (included by felbm.cu).
//
// The state is split into the macroscopic fields -- C in FP64, p and u in
// FP32 -- and the FP32 deviations of the distributions from their
// equilibria, dpsi_a = psi_a - psi_a^eq(C, p, u), whose zeroth (and, for g,
// first) moments are zero.  The scheme is the same as the FP64 path
// (Sec. II.C of arXiv:1708.04678); only the storage and arithmetic differ:
//  * collision needs no pass of its own: psi_hat = psi^eq + (1 - omega) dpsi;
//  * every gradient and every difference of equilibria is formed from
//    differences of the fields (C differences taken in FP64), so nothing
//    cancels catastrophically in FP32 -- e.g. h^eq_v - h^eq_0 =
//    Gamma_v (C_v - C_0) + C_0 (Gamma_v - Gamma_0), and Gamma_v - Gamma_0 is
//    a polynomial in u_v - u_0;
//  * the chemical potential (double well near C in {0, 1} and the patch
//    Laplacian of C) is evaluated in FP64;
//  * the mass solve runs in FP32 and its last sweep updates the fields (C in
//    FP64) and the deviations in place.
#pragma once

// Layout of the deviations (18 Np floats): the moving populations q = 1..8
// of g and then of h as one 64-byte row per node (dpsi + 16 i), so that a
// gather of a vertex's 16 values is four 16-byte loads; the rest populations
// (q = 0) of g and of h after all rows, one value per node each.
// q18 = q for g, 9 + q for h.
__device__ __forceinline__ size_t dpsi_at(int Np, int q18, int i) {
    const int part = q18 >= 9 ? 1 : 0, q = q18 - 9 * part;
    return q == 0 ? (size_t)(16 + part) * Np + i : (size_t)i * 16 + part * 8 + (q - 1);
}

// omega = 1 / (tau + 1/2), 1/tau = C/tau_l + (1-C)/tau_v (Sec. II.A)
__device__ __forceinline__ float omega32(float C, const Phys& c) {
    float inv_tau = C * c.inv_tau_l_f + (1.0f - C) * c.inv_tau_v_f;
    return 1.0f / (1.0f / inv_tau + 0.5f);
}

// Gamma_q(u1) - Gamma_q(u0) as a polynomial in du = u1 - u0, su = u1 + u0.
template <int q>
__device__ __forceinline__ float dgamma32(float dux, float duy, float sux, float suy) {
    float edu = edot<q, float>(dux, duy), esu = edot<q, float>(sux, suy);
    return (float)wq(q) * (3.0f * edu + 4.5f * edu * esu - 1.5f * (dux * sux + duy * suy));
}
template <int q>
__device__ __forceinline__ float gamma32(float ux, float uy, float uu15) {
    float eu = edot<q, float>(ux, uy);
    return (float)wq(q) * (1.0f + 3.0f * eu + 4.5f * eu * eu - uu15);
}

// ------------------------------------------------- chemical potential ------
// Same arithmetic as k_mu (FP64), FP32 output.
__device__ __forceinline__ void mu32_node(const DevMesh& m, const Phys& c, const Bufs& b, int i) {
    double Ci = b.C[i];
    double lap = 0.0;
    for (int k = m.row_ptr[i]; k < m.row_ptr[i + 1]; ++k) lap += m.lval[k] * (b.C[m.col[k]] - Ci);
    double wall = 0.0;
    for (int k = m.winc_ptr[i]; k < m.winc_ptr[i + 1]; ++k) {
        int e = m.winc_edge[k];
        double Ca = b.C[m.wall_a[e]], Cb = b.C[m.wall_b[e]];
        double s = 0.5 * (Ca + Cb) - (Ca * Ca + Ca * Cb + Cb * Cb) * (1.0 / 3.0);
        wall -= m.wall_phi[e] * m.wall_len[e] * s;
    }
    b.mu32[i] = (float)(2.0 * c.beta * Ci * (Ci - 1.0) * (2.0 * Ci - 1.0) - (c.kappa * lap + wall * m.inv_vol[i]));
}

// kW > 0: the sum over the ELL copy of the row (zero padding), its columns
// and coefficients loaded up front so the gathers of C are issued together;
// kW = 0: CSR, in the difference form of the FP64 path.
template <int kW>
__global__ void __launch_bounds__(kBlock) k_mu32(DevMesh m, Phys c, Bufs b) {
    pdl_release();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    if constexpr (kW == 0) {
        mu32_node(m, c, b, i);
    } else {
        const int Np = m.Np;
        int col[kW];
        double l[kW];
#pragma unroll
        for (int k = 0; k < kW; ++k) {
            col[k] = m.ell_col[k * Np + i];
            l[k] = m.ell_lval[k * Np + i];
        }
        // The row's coefficients sum to zero (the P1 stiffness rows do), so
        // sum l_k (C_k - C_i) = sum l_k C_k: one FP64 FMA per entry instead
        // of a subtraction and an FMA on this FP64-pipe-bound kernel.  The
        // cancellation costs about 1e-15 absolute in the Laplacian, far below
        // the FP32 rounding of the stored mu.
        const double Ci = b.C[i];
        double lap = 0.0;
#pragma unroll
        for (int k = 0; k < kW; ++k) lap = fma(l[k], b.C[col[k]], lap);
        double wall = 0.0;
        for (int k = m.winc_ptr[i]; k < m.winc_ptr[i + 1]; ++k) {
            int e = m.winc_edge[k];
            double Ca = b.C[m.wall_a[e]], Cb = b.C[m.wall_b[e]];
            double s = 0.5 * (Ca + Cb) - (Ca * Ca + Ca * Cb + Cb * Cb) * (1.0 / 3.0);
            wall -= m.wall_phi[e] * m.wall_len[e] * s;
        }
        b.mu32[i] = (float)(2.0 * c.beta * Ci * (Ci - 1.0) * (2.0 * Ci - 1.0) - (c.kappa * lap + wall * m.inv_vol[i]));
    }
}

__device__ __forceinline__ void gradmu32_tri(const DevMesh& m, const Bufs& b, int t) {
    const int Tp = m.Tp;
    int v0 = m.tri[t], v1 = m.tri[Tp + t], v2 = m.tri[2 * Tp + t];
    float m0 = b.mu32[v0], d1 = b.mu32[v1] - m0, d2 = b.mu32[v2] - m0;
    b.gmu32[t] = d1 * m.grad32[2 * Tp + t] + d2 * m.grad32[4 * Tp + t];
    b.gmu32[Tp + t] = d1 * m.grad32[3 * Tp + t] + d2 * m.grad32[5 * Tp + t];
}

// FELBM_LAPMU_NODAL: nodal Laplacian of mu (patch Laplacian with zero wall
// flux), formed in FP64 from the FP32 mu like the Laplacian of C.
__device__ __forceinline__ void lmu32_node(const DevMesh& m, const Phys& c, const Bufs& b, int i) {
    const double mi = b.mu32[i];
    double lap = 0.0;
    for (int k = m.row_ptr[i]; k < m.row_ptr[i + 1]; ++k) lap += m.lval[k] * ((double)b.mu32[m.col[k]] - mi);
    b.lmu32[i] = (float)(c.lapmu_fac * lap);
}

__global__ void __launch_bounds__(kBlock) k_lmu32(DevMesh m, Phys c, Bufs b) {
    pdl_release();
    pdl_wait();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m.N) lmu32_node(m, c, b, i);
}

__global__ void __launch_bounds__(kBlock) k_gradmu32(DevMesh m, Bufs b) {
    pdl_release();
    pdl_wait();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m.T) gradmu32_tri(m, b, t);
}

// ------------------------------- forces and element residual (FP32) ------
// R_a = A (Phi_a - e_a . grad psi_hat_a), psi_hat = psi^eq + (1 - omega) dpsi,
// gradients formed from differences to vertex 0 (sum of the b_v is zero).
__device__ __forceinline__ void element32_tri(const DevMesh& m, const Phys& c, const Bufs& b, int t) {
    const int Tp = m.Tp, Np = m.Np;
    int v[3];
    float bx[3], by[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        v[k] = m.tri[k * Tp + t];
        bx[k] = m.grad32[(2 * k) * Tp + t];
        by[k] = m.grad32[(2 * k + 1) * Tp + t];
    }
    const float A = m.area32[t];
    const double C0d = b.C[v[0]], C1d = b.C[v[1]], C2d = b.C[v[2]];
    const float dC1 = (float)(C1d - C0d), dC2 = (float)(C2d - C0d);
    const float C0 = (float)C0d;
    const float Cb = C0 + (dC1 + dC2) * (1.0f / 3.0f);
    float p[3], ux[3], uy[3], om1[3];
    float mus = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        p[k] = b.p32[v[k]];
        ux[k] = b.ux32[v[k]];
        uy[k] = b.uy32[v[k]];
        mus += b.mu32[v[k]];
    }
    om1[0] = 1.0f - omega32(C0, c);
    om1[1] = 1.0f - omega32(C0 + dC1, c);
    om1[2] = 1.0f - omega32(C0 + dC2, c);
    const float third = 1.0f / 3.0f;
    const float pb = (p[0] + p[1] + p[2]) * third;
    (void)pb;
    const float ubx = (ux[0] + ux[1] + ux[2]) * third, uby = (uy[0] + uy[1] + uy[2]) * third;
    const float mub = mus * third;
    const float gCx = dC1 * bx[1] + dC2 * bx[2], gCy = dC1 * by[1] + dC2 * by[2];
    const float dp1 = p[1] - p[0], dp2 = p[2] - p[0];
    const float gpx = dp1 * bx[1] + dp2 * bx[2], gpy = dp1 * by[1] + dp2 * by[2];
    float lapmu = 0.0f;
    if (c.lapmu_nodal) {
        lapmu = (b.lmu32[v[0]] + b.lmu32[v[1]] + b.lmu32[v[2]]) * (1.0f / 3.0f);
    } else {
        const float gmx = b.gmu32[t], gmy = b.gmu32[Tp + t];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            int nb = m.nbr[k * Tp + t];
            if (nb >= 0) lapmu -= (gmx + b.gmu32[nb]) * bx[k] + (gmy + b.gmu32[Tp + nb]) * by[k];
        }
    }
    const float drho = c.drho_f;
    const float rhob = c.rho_v_f + Cb * drho;
    const float rho0 = c.rho_v_f + C0 * drho;
    const float grx = drho * gCx, gry = drho * gCy;
    const float f = 3.0f * Cb / rhob;
    const float vhx = gCx - f * (gpx - mub * gCx), vhy = gCy - f * (gpy - mub * gCy);
    const float u_gr = ubx * grx + uby * gry, u_gC = ubx * gCx + uby * gCy, u_vh = ubx * vhx + uby * vhy;
    const float uub15 = 1.5f * (ubx * ubx + uby * uby);
    const float Mlap = c.mobility_f * lapmu;
    // vertex velocity differences to vertex 0
    const float du1x = ux[1] - ux[0], du1y = uy[1] - uy[0], su1x = ux[1] + ux[0], su1y = uy[1] + uy[0];
    const float du2x = ux[2] - ux[0], du2y = uy[2] - uy[0], su2x = ux[2] + ux[0], su2y = uy[2] + uy[0];
    const float uu0 = 1.5f * (ux[0] * ux[0] + uy[0] * uy[0]);
    const float drho1 = drho * dC1, drho2 = drho * dC2;
    // the post-collision deviations of the three vertices, all loaded first
    // (each vertex's row: four 16-byte loads)
    float pg[3][9], ph[3][9];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float4* row = reinterpret_cast<const float4*>(b.dpsi + (size_t)v[k] * 16);
        const float4 a0 = row[0], a1 = row[1], a2 = row[2], a3 = row[3];
        pg[k][1] = a0.x; pg[k][2] = a0.y; pg[k][3] = a0.z; pg[k][4] = a0.w;
        pg[k][5] = a1.x; pg[k][6] = a1.y; pg[k][7] = a1.z; pg[k][8] = a1.w;
        ph[k][1] = a2.x; ph[k][2] = a2.y; ph[k][3] = a2.z; ph[k][4] = a2.w;
        ph[k][5] = a3.x; ph[k][6] = a3.y; ph[k][7] = a3.z; ph[k][8] = a3.w;
    }
    float out[18];
#define FELBM_ELEM32_Q(q)                                                                          \
    {                                                                                              \
        const float w = (float)wq(q);                                                              \
        const float G = gamma32<q>(ubx, uby, uub15);                                               \
        const float phig = third * (G - w) * (edot<q, float>(grx, gry) - u_gr) + mub * G * (edot<q, float>(gCx, gCy) - u_gC); \
        const float phih = ((edot<q, float>(vhx, vhy) - u_vh) + Mlap) * G;                               \
        float dg = 0.0f, dh = 0.0f;                                                                \
        if (q != 0) {                                                                              \
            const float G0 = gamma32<q>(ux[0], uy[0], uu0);                                        \
            const float dG1 = dgamma32<q>(du1x, du1y, su1x, su1y);                                 \
            const float dG2 = dgamma32<q>(du2x, du2y, su2x, su2y);                                 \
            /* differences of the equilibria to vertex 0 */                                       \
            const float dhe1 = (G0 + dG1) * dC1 + C0 * dG1, dhe2 = (G0 + dG2) * dC2 + C0 * dG2;     \
            const float dge1 = w * dp1 + third * (drho1 * (G0 + dG1 - w) + rho0 * dG1);            \
            const float dge2 = w * dp2 + third * (drho2 * (G0 + dG2 - w) + rho0 * dG2);            \
            /* differences of the post-collision deviations */                                     \
            const float g0 = om1[0] * pg[0][q], h0 = om1[0] * ph[0][q];                            \
            const float dgd1 = om1[1] * pg[1][q] - g0;                                             \
            const float dgd2 = om1[2] * pg[2][q] - g0;                                             \
            const float dhd1 = om1[1] * ph[1][q] - h0;                                             \
            const float dhd2 = om1[2] * ph[2][q] - h0;                                             \
            const float eb1 = edot<q, float>(bx[1], by[1]), eb2 = edot<q, float>(bx[2], by[2]);                  \
            dg = (dge1 + dgd1) * eb1 + (dge2 + dgd2) * eb2;                                        \
            dh = (dhe1 + dhd1) * eb1 + (dhe2 + dhd2) * eb2;                                        \
        }                                                                                          \
        out[q] = A * (phig - dg);                                                                  \
        out[9 + q] = A * (phih - dh);                                                              \
    }
    FELBM_ELEM32_Q(0) FELBM_ELEM32_Q(1) FELBM_ELEM32_Q(2) FELBM_ELEM32_Q(3) FELBM_ELEM32_Q(4)
    FELBM_ELEM32_Q(5) FELBM_ELEM32_Q(6) FELBM_ELEM32_Q(7) FELBM_ELEM32_Q(8)
#undef FELBM_ELEM32_Q
    float2* dst = reinterpret_cast<float2*>(b.R32 + (size_t)t * 18);
#pragma unroll
    for (int k = 0; k < 9; ++k) dst[k] = make_float2(out[2 * k], out[2 * k + 1]);
}

// The vertices' 48 deviation values are all loaded (as twelve 16-byte row
// loads) before the per-direction arithmetic, so that they are in flight
// together; 80 registers (6 blocks of 128 per SM).  On the 2.08M-node rough
// wall: 0.229 ms, against 0.300 ms with one array per population and 0.324
// ms with the loads inside the arithmetic at 64 registers.
__global__ void __launch_bounds__(128, 6) k_element32(DevMesh m, Phys c, Bufs b) {
    pdl_release();
    pdl_wait();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m.T) element32_tri(m, c, b, t);
}

// ------------------------------------------ streaming RHS gather (FP32) ----
// As k_rhs; the wall term needs psi_hat_opp - psi_hat at a node, which in the
// split form is  g: -2 w rho (e.u) + (1-omega)(dg_opp - dg),
//                h: -6 w C (e.u)   + (1-omega)(dh_opp - dh).
// kI > 0: the incident triangles from the incidence ELL (padding: the zero
// residual row T), their ids and gradients loaded up front; kI = 0: CSR.
template <int kI = 0, bool kFirst = true>
__device__ __forceinline__ void rhs32_node(const DevMesh& m, const Phys& c, const Bufs& b, int i, float tau0) {
    const int Np = m.Np;
    float acc[18];
#pragma unroll
    for (int q = 0; q < 18; ++q) acc[q] = 0.0f;
    const float c1 = c.dt3_f, c2 = c.dt2h_f;
    constexpr int kIr = kI > 0 ? kI : 1;
    int tt[kIr];
    float bxx[kIr], byy[kIr];
    if constexpr (kI > 0) {
#pragma unroll
        for (int k = 0; k < kI; ++k) {
            tt[k] = m.iell_tri[k * Np + i];
            bxx[k] = m.iell_bx32[k * Np + i];
            byy[k] = m.iell_by32[k * Np + i];
        }
    }
    const int k0 = kI > 0 ? 0 : m.inc_ptr[i], k1 = kI > 0 ? kI : m.inc_ptr[i + 1];
#pragma unroll(kI > 0 ? kIr : 1)
    for (int k = k0; k < k1; ++k) {
        int t;
        float bxi, byi;
        if constexpr (kI > 0) {
            t = tt[k];
            bxi = bxx[k];
            byi = byy[k];
        } else {
            t = m.inc_tri[k];
            bxi = m.inc_bx32[k];
            byi = m.inc_by32[k];
        }
        const float2* src = reinterpret_cast<const float2*>(b.R32 + (size_t)t * 18);
        float r[18];
#pragma unroll
        for (int s = 0; s < 9; ++s) {
            float2 v2 = src[s];
            r[2 * s] = v2.x;
            r[2 * s + 1] = v2.y;
        }
#define FELBM_RHS32_Q(q)                                        \
        {                                                       \
            float w = c1 + c2 * edot<q, float>(bxi, byi);              \
            acc[q] = fmaf(r[q], w, acc[q]);                     \
            acc[9 + q] = fmaf(r[9 + q], w, acc[9 + q]);         \
        }
        FELBM_RHS32_Q(0) FELBM_RHS32_Q(1) FELBM_RHS32_Q(2) FELBM_RHS32_Q(3) FELBM_RHS32_Q(4)
        FELBM_RHS32_Q(5) FELBM_RHS32_Q(6) FELBM_RHS32_Q(7) FELBM_RHS32_Q(8)
#undef FELBM_RHS32_Q
    }
    if (m.winc_ptr[i] < m.winc_ptr[i + 1]) {
        const float drho = c.drho_f;
        for (int k = m.winc_ptr[i]; k < m.winc_ptr[i + 1]; ++k) {
            int e = m.winc_edge[k];
            int o = m.wall_a[e] == i ? m.wall_b[e] : m.wall_a[e];
            float L = (float)m.wall_len[e], nx = (float)m.wall_nx[e], ny = (float)m.wall_ny[e];
            float Ci = (float)b.C[i], Co = (float)b.C[o];
            float rhoi = c.rho_v_f + Ci * drho, rhoo = c.rho_v_f + Co * drho;
            float omi = 1.0f - omega32(Ci, c), omo = 1.0f - omega32(Co, c);
            float uxi = b.ux32[i], uyi = b.uy32[i], uxo = b.ux32[o], uyo = b.uy32[o];
#define FELBM_WALL32_Q(q)                                                                           \
            {                                                                                       \
                float en = edot<q, float>(nx, ny);                                                         \
                if (en < 0.0f) {                                                                    \
                    const float w = (float)wq(q);                                                   \
                    float f = -c.dt_f * en;                                                         \
                    float eui = edot<q, float>(uxi, uyi), euo = edot<q, float>(uxo, uyo);                         \
                    float dgi = -2.0f * w * rhoi * eui + omi * (b.dpsi[dpsi_at(Np, opp(q), i)] - b.dpsi[dpsi_at(Np, q, i)]); \
                    float dgo = -2.0f * w * rhoo * euo + omo * (b.dpsi[dpsi_at(Np, opp(q), o)] - b.dpsi[dpsi_at(Np, q, o)]); \
                    float dhi = -6.0f * w * Ci * eui + omi * (b.dpsi[dpsi_at(Np, (9 + opp(q)), i)] - b.dpsi[dpsi_at(Np, (9 + q), i)]); \
                    float dho = -6.0f * w * Co * euo + omo * (b.dpsi[dpsi_at(Np, (9 + opp(q)), o)] - b.dpsi[dpsi_at(Np, (9 + q), o)]); \
                    acc[q] += f * (L * (1.0f / 3.0f) * dgi + L * (1.0f / 6.0f) * dgo);              \
                    acc[9 + q] += f * (L * (1.0f / 3.0f) * dhi + L * (1.0f / 6.0f) * dho);          \
                }                                                                                   \
            }
            FELBM_WALL32_Q(1) FELBM_WALL32_Q(2) FELBM_WALL32_Q(3) FELBM_WALL32_Q(4)
            FELBM_WALL32_Q(5) FELBM_WALL32_Q(6) FELBM_WALL32_Q(7) FELBM_WALL32_Q(8)
#undef FELBM_WALL32_Q
        }
    }
    float s = m.inv_lumped32[i] * tau0;
#pragma unroll
    for (int q = 0; q < 18; ++q) {
        b.r32[q * Np + i] = acc[q];
        if (kFirst) b.e1[q * Np + i] = acc[q] * s;
    }
}

// at most 64 registers (8 blocks of 128 per SM; 6 % faster than 96 registers)
template <int kI, bool kFirst = true>
__global__ void __launch_bounds__(128, 8) k_rhs32(DevMesh m, Phys c, Bufs b, float tau0) {
    pdl_release();
    pdl_wait();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m.N) rhs32_node<kI, kFirst>(m, c, b, i, tau0);
}

// ---------------------------- update of fields and deviations (node) ------
// With the increment d = psi^{n+1} - psi_hat of all 18 populations at node i:
//   C' = C + sum d_h (FP64), p' = p + sum d_g, rho' u' = rho u + 3 sum e d_g,
//   dpsi' = (1 - omega) dpsi + d + psi^eq(C, p, u) - psi^eq(C', p', u'),
// the equilibrium difference written through dC, dp, du (no cancellation):
//   h: -(Gamma' dC + C (Gamma' - Gamma)),
//   g: -(w dp + cs2 (drho (Gamma' - w) + rho (Gamma' - Gamma))).
__device__ __forceinline__ void dev32_update(const DevMesh& m, const Phys& c, const Bufs& b, int i,
                                             const float (&d)[18]) {
    const int Np = m.Np;
    const double Cd = b.C[i];
    const float C = (float)Cd;
    const float p = b.p32[i], ux = b.ux32[i], uy = b.uy32[i];
    const float om1 = 1.0f - omega32(C, c);
    float dC = 0.0f, dp = 0.0f;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        dC += d[9 + q];
        dp += d[q];
    }
    const float jx = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
    const float jy = (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]);
    const double Cnd = Cd + (double)dC;
    const float drho_c = c.drho_f;
    const float rho = c.rho_v_f + C * drho_c;
    const float rhon = rho + drho_c * dC;
    const float uxn = (rho * ux + 3.0f * jx) / rhon, uyn = (rho * uy + 3.0f * jy) / rhon;
    const float drho = drho_c * dC;
    const float dux = uxn - ux, duy = uyn - uy, sux = uxn + ux, suy = uyn + uy;
    const float uun15 = 1.5f * (uxn * uxn + uyn * uyn);
    const float third = 1.0f / 3.0f;
    // the node's deviations: its 64-byte row (q = 1..8) and the rest populations
    float4* row = reinterpret_cast<float4*>(b.dpsi + (size_t)i * 16);
    const float4 r0 = row[0], r1 = row[1], r2 = row[2], r3 = row[3];
    float dg[9] = {b.dpsi[dpsi_at(Np, 0, i)], r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
    float dh[9] = {b.dpsi[dpsi_at(Np, 9, i)], r2.x, r2.y, r2.z, r2.w, r3.x, r3.y, r3.z, r3.w};
#define FELBM_UPD32_Q(q)                                                                         \
    {                                                                                            \
        const float w = (float)wq(q);                                                            \
        const float Gn = gamma32<q>(uxn, uyn, uun15);                                            \
        const float dG = dgamma32<q>(dux, duy, sux, suy);                                        \
        dg[q] = om1 * dg[q] + d[q] - (w * dp + third * (drho * (Gn - w) + rho * dG));            \
        dh[q] = om1 * dh[q] + d[9 + q] - (Gn * dC + C * dG);                                     \
    }
    FELBM_UPD32_Q(0) FELBM_UPD32_Q(1) FELBM_UPD32_Q(2) FELBM_UPD32_Q(3) FELBM_UPD32_Q(4)
    FELBM_UPD32_Q(5) FELBM_UPD32_Q(6) FELBM_UPD32_Q(7) FELBM_UPD32_Q(8)
#undef FELBM_UPD32_Q
    b.dpsi[dpsi_at(Np, 0, i)] = dg[0];
    b.dpsi[dpsi_at(Np, 9, i)] = dh[0];
    row[0] = make_float4(dg[1], dg[2], dg[3], dg[4]);
    row[1] = make_float4(dg[5], dg[6], dg[7], dg[8]);
    row[2] = make_float4(dh[1], dh[2], dh[3], dh[4]);
    row[3] = make_float4(dh[5], dh[6], dh[7], dh[8]);
    b.C[i] = Cnd;
    b.p32[i] = p + dp;
    b.ux32[i] = uxn;
    b.uy32[i] = uyn;
}

// ------------------------------------ conversions to / from full FP64 ------
// stage [18][N] (caller order) <- psi = psi^eq(C, p, u) + dpsi, in FP64
// (one thread per caller-order node o: the 18 stage streams are written
// coalesced, the node's fields and deviation row read at i = iperm[o])
__global__ void k_dev32_to_full(DevMesh m, Phys c, Bufs b, double* stage) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= m.N) return;
    const int N = m.N, Np = m.Np, i = m.iperm[o];
    double C = b.C[i], p = b.p32[i], ux = b.ux32[i], uy = b.uy32[i];
    double rho = c.rho_v + C * (c.rho_l - c.rho_v);
    double uu15 = 1.5 * (ux * ux + uy * uy);
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        double eu = ex(q) * ux + ey(q) * uy;
        double G = wq(q) * (1.0 + 3.0 * eu + 4.5 * eu * eu - uu15);
        stage[(size_t)q * N + o] = wq(q) * p + rho * (1.0 / 3.0) * (G - wq(q)) + (double)b.dpsi[dpsi_at(Np, q, i)];
        stage[(size_t)(9 + q) * N + o] = G * C + (double)b.dpsi[dpsi_at(Np, (9 + q), i)];
    }
}

// fields and deviations <- psi (stage [18][N], caller order, FP64)
// (one thread per caller-order node o: the 18 stage streams are read
// coalesced, the node's fields and deviation row written at i = iperm[o])
__global__ void k_full_to_dev32(DevMesh m, Phys c, Bufs b, const double* __restrict__ stage) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= m.N) return;
    const int N = m.N, Np = m.Np, i = m.iperm[o];
    double g[9], h[9], C = 0.0, p = 0.0;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        g[q] = stage[(size_t)q * N + o];
        h[q] = stage[(size_t)(9 + q) * N + o];
        C += h[q];
        p += g[q];
    }
    const double jx = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
    const double jy = (g[2] - g[4]) + (g[5] + g[6]) - (g[7] + g[8]);
    const double rho = c.rho_v + C * (c.rho_l - c.rho_v);
    // the stored fields (FP32 p, u; FP64 C); deviations are taken relative to
    // the equilibrium of exactly these values
    const float rhof = (float)rho, Cf = (float)C, pf = (float)p;
    const float uxf = 3.0f * (float)jx / rhof, uyf = 3.0f * (float)jy / rhof;
    const double ps = pf;
    const float uu15 = 1.5f * (uxf * uxf + uyf * uyf);
    const float r3 = rhof * (1.0f / 3.0f);
    // g_q - g_q^eq = (g_q - w p) - (rho/3) w T_q and h_q - h_q^eq = (h_q - w C) - w T_q C,
    // T_q = Gamma_q / w_q - 1 = 3 e.u + 4.5 (e.u)^2 - 1.5 u.u: the large differences in
    // FP64, rounded once to FP32; the velocity terms (O(|u|) of the state) in FP32
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const float wf = (float)wq(q);
        const float eu = (float)ex(q) * uxf + (float)ey(q) * uyf;
        const float T = 3.0f * eu + 4.5f * eu * eu - uu15;
        const float dg0 = (float)(g[q] - wq(q) * ps), dh0 = (float)(h[q] - wq(q) * C);
        b.dpsi[dpsi_at(Np, q, i)] = dg0 - r3 * (wf * T);
        b.dpsi[dpsi_at(Np, (9 + q), i)] = dh0 - (wf * T) * Cf;
    }
    b.C[i] = C;
    b.p32[i] = pf;
    b.ux32[i] = uxf;
    b.uy32[i] = uyf;
}

// Initial state at equilibrium with C0, p0, u0 (the layout of k_init_state):
// the fields are stored and the deviations are zero.
__global__ void k_init_dev32(DevMesh m, Bufs b, const double* __restrict__ stage, int has_p, int has_u) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const int o = m.perm[i], N = m.N;
    const double* u = stage + (has_p ? 2 : 1) * (size_t)N;
    b.C[i] = stage[o];
    b.p32[i] = has_p ? (float)stage[N + o] : 0.0f;
    b.ux32[i] = has_u ? (float)u[o] : 0.0f;
    b.uy32[i] = has_u ? (float)u[N + o] : 0.0f;
#pragma unroll
    for (int q = 0; q < 18; ++q) b.dpsi[dpsi_at(m.Np, q, i)] = 0.0f;
}

__global__ void k_gather_out_f(DevMesh m, const float* __restrict__ src, double* stage) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    stage[m.perm[i]] = (double)src[i];
}
