// FP32 deviation storage of the 3D FE-LBM step (included by felbm3d.cu).
//
// The state is split into the macroscopic fields -- C in FP64, p and u in
// FP32 -- and the FP32 deviations of the distributions from their
// equilibria, dpsi_a = psi_a - psi_a^eq(C, p, u), whose zeroth (and, for g,
// first) moments vanish.  The scheme is that of the FP64 kernels (Sec. II.C
// of arXiv:1708.04678, D3Q19); only storage and arithmetic differ:
//  * collision needs no pass of its own: psi_hat = psi^eq + (1 - omega) dpsi;
//  * gradients and differences of equilibria are formed from differences of
//    the fields (C differences in FP64), so nothing cancels in FP32:
//    h^eq_v - h^eq_0 = Gamma_v (C_v - C_0) + C_0 (Gamma_v - Gamma_0), and
//    Gamma_v - Gamma_0 is a polynomial in u_v - u_0 and u_v + u_0;
//  * the chemical potential (double well and patch Laplacian of C) is FP64;
//  * the mass solve runs in FP32; its last sweep updates the fields (C in
//    FP64) and the deviations in place.
#pragma once

__device__ __forceinline__ float omega32_3(float C, const Phys3& c) {
    float inv_tau = C * c.inv_tau_l_f + (1.0f - C) * c.inv_tau_v_f;
    return 1.0f / (1.0f / inv_tau + 0.5f);
}
__device__ __forceinline__ float gamma32_3(int q, float ux, float uy, float uz, float uu15) {
    float eu = edot3(q, ux, uy, uz);
    return (float)wq3(q) * (1.0f + 3.0f * eu + 4.5f * eu * eu - uu15);
}
// Gamma_q(u1) - Gamma_q(u0) from du = u1 - u0 and su = u1 + u0
__device__ __forceinline__ float dgamma32_3(int q, float dx, float dy, float dz, float sx, float sy, float sz) {
    float edu = edot3(q, dx, dy, dz), esu = edot3(q, sx, sy, sz);
    return (float)wq3(q) * (3.0f * edu + 4.5f * edu * esu - 1.5f * (dx * sx + dy * sy + dz * sz));
}

// ------------------------------------------------- chemical potential ------
__global__ void __launch_bounds__(kBlock) k3_mu32(DevMesh3 m, Phys3 c, Bufs3 b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const double Ci = b.C[i];
    double lap = 0.0;
    for (int k = m.row_ptr[i]; k < m.row_ptr[i + 1]; ++k) lap += m.lval[k] * (b.C[m.col[k]] - Ci);
    double wall = 0.0;
    for (int k = m.winc_ptr[i]; k < m.winc_ptr[i + 1]; ++k) wall += wall_flux3(m, b.C, m.winc_face[k]);
    b.mu32[i] = (float)(2.0 * c.beta * Ci * (Ci - 1.0) * (2.0 * Ci - 1.0) - (c.kappa * lap + wall * m.inv_vol[i]));
}

__global__ void __launch_bounds__(kBlock) k3_gradmu32(DevMesh3 m, Bufs3 b) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m.T) return;
    const int Tp = m.Tp;
    const float mu0 = b.mu32[m.tet[t]];
    float g[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int k = 1; k < 4; ++k) {
        float d = b.mu32[m.tet[k * Tp + t]] - mu0;
#pragma unroll
        for (int a = 0; a < 3; ++a) g[a] = fmaf(d, m.grad32[(3 * k + a) * Tp + t], g[a]);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) b.gmu32[a * Tp + t] = g[a];
}

// ------------------------------- forces and element residual (FP32) ------
__global__ void __launch_bounds__(128) k3_element32(DevMesh3 m, Phys3 c, Bufs3 b) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m.T) return;
    const int Tp = m.Tp, Np = m.Np;
    int v[4];
    float bx[4], by[4], bz[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = m.tet[k * Tp + t];
        bx[k] = m.grad32[(3 * k) * Tp + t];
        by[k] = m.grad32[(3 * k + 1) * Tp + t];
        bz[k] = m.grad32[(3 * k + 2) * Tp + t];
    }
    const float V = m.vol32[t];
    const double C0d = b.C[v[0]];
    const float C0 = (float)C0d;
    float dC[4], p[4], ux[4], uy[4], uz[4], om1[4];
    float mus = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        dC[k] = k == 0 ? 0.0f : (float)(b.C[v[k]] - C0d);
        p[k] = b.p32[v[k]];
        ux[k] = b.ux32[v[k]];
        uy[k] = b.uy32[v[k]];
        uz[k] = b.uz32[v[k]];
        mus += b.mu32[v[k]];
        om1[k] = 1.0f - omega32_3(C0 + dC[k], c);
    }
    const float Cb = C0 + 0.25f * (dC[1] + dC[2] + dC[3]);
    const float ubx = 0.25f * (ux[0] + ux[1] + ux[2] + ux[3]);
    const float uby = 0.25f * (uy[0] + uy[1] + uy[2] + uy[3]);
    const float ubz = 0.25f * (uz[0] + uz[1] + uz[2] + uz[3]);
    const float mub = 0.25f * mus;
    float gC[3] = {0.0f, 0.0f, 0.0f}, gp[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int k = 1; k < 4; ++k) {
        const float dp = p[k] - p[0];
        gC[0] = fmaf(dC[k], bx[k], gC[0]);
        gC[1] = fmaf(dC[k], by[k], gC[1]);
        gC[2] = fmaf(dC[k], bz[k], gC[2]);
        gp[0] = fmaf(dp, bx[k], gp[0]);
        gp[1] = fmaf(dp, by[k], gp[1]);
        gp[2] = fmaf(dp, bz[k], gp[2]);
    }
    const float gm0 = b.gmu32[t], gm1 = b.gmu32[Tp + t], gm2 = b.gmu32[2 * Tp + t];
    float flux = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int nb = m.nbr[k * Tp + t];
        if (nb >= 0)
            flux += (gm0 + b.gmu32[nb]) * bx[k] + (gm1 + b.gmu32[Tp + nb]) * by[k] + (gm2 + b.gmu32[2 * Tp + nb]) * bz[k];
    }
    const float Mlap = c.mobility_f * (-1.5f * flux);
    const float drho = c.drho_f;
    const float rhob = c.rho_v_f + Cb * drho;
    const float rho0 = c.rho_v_f + C0 * drho;
    const float gr[3] = {drho * gC[0], drho * gC[1], drho * gC[2]};
    const float f = 3.0f * Cb / rhob;
    const float vh[3] = {gC[0] - f * (gp[0] - mub * gC[0]), gC[1] - f * (gp[1] - mub * gC[1]),
                         gC[2] - f * (gp[2] - mub * gC[2])};
    const float u_gr = ubx * gr[0] + uby * gr[1] + ubz * gr[2];
    const float u_gC = ubx * gC[0] + uby * gC[1] + ubz * gC[2];
    const float u_vh = ubx * vh[0] + uby * vh[1] + ubz * vh[2];
    const float uub15 = 1.5f * (ubx * ubx + uby * uby + ubz * ubz);
    const float uu0 = 1.5f * (ux[0] * ux[0] + uy[0] * uy[0] + uz[0] * uz[0]);
    float* dst = b.R32 + (size_t)t * kR32;
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        const float w = (float)wq3(q);
        const float G = gamma32_3(q, ubx, uby, ubz, uub15);
        const float phig = (1.0f / 3.0f) * (G - w) * (edot3(q, gr[0], gr[1], gr[2]) - u_gr) +
                           mub * G * (edot3(q, gC[0], gC[1], gC[2]) - u_gC);
        const float phih = ((edot3(q, vh[0], vh[1], vh[2]) - u_vh) + Mlap) * G;
        float dg = 0.0f, dh = 0.0f;
        if (q != 0) {
            const float G0 = gamma32_3(q, ux[0], uy[0], uz[0], uu0);
            const float g0 = om1[0] * b.dpsi[q * Np + v[0]], h0 = om1[0] * b.dpsi[(19 + q) * Np + v[0]];
#pragma unroll
            for (int k = 1; k < 4; ++k) {
                const float dG = dgamma32_3(q, ux[k] - ux[0], uy[k] - uy[0], uz[k] - uz[0], ux[k] + ux[0],
                                            uy[k] + uy[0], uz[k] + uz[0]);
                // differences of the equilibria and of the post-collision deviations to vertex 0
                const float dhe = (G0 + dG) * dC[k] + C0 * dG;
                const float dge = w * (p[k] - p[0]) + (1.0f / 3.0f) * (drho * dC[k] * (G0 + dG - w) + rho0 * dG);
                const float dgd = om1[k] * b.dpsi[q * Np + v[k]] - g0;
                const float dhd = om1[k] * b.dpsi[(19 + q) * Np + v[k]] - h0;
                const float eb = edot3(q, bx[k], by[k], bz[k]);
                dg = fmaf(dge + dgd, eb, dg);
                dh = fmaf(dhe + dhd, eb, dh);
            }
        }
        dst[q] = V * (phig - dg);
        dst[19 + q] = V * (phih - dh);
    }
}

// ------------------------------------------ streaming RHS gather (FP32) ----
// As k3_rhs; the wall term needs psi_hat_opp - psi_hat at a node, which in
// the split form is  g: -2 w rho (e.u) + (1-omega)(dg_opp - dg),
//                    h: -6 w C (e.u)   + (1-omega)(dh_opp - dh).
__device__ __forceinline__ float wall_diff32(const DevMesh3& m, const Phys3& c, const Bufs3& b, int s, int q, int v) {
    const int Np = m.Np;
    const float C = (float)b.C[v];
    const float eu = edot3(q, b.ux32[v], b.uy32[v], b.uz32[v]);
    const float om1 = 1.0f - omega32_3(C, c);
    const float w = (float)wq3(q);
    const float* d = b.dpsi + (size_t)19 * s * Np;
    const float ddev = om1 * (d[opp3(q) * Np + v] - d[q * Np + v]);
    const float eq = s == 0 ? -2.0f * w * (c.rho_v_f + C * c.drho_f) * eu : -6.0f * w * C * eu;
    return eq + ddev;
}

__global__ void __launch_bounds__(kNodeBlock) k3_rhs32(DevMesh3 m, Phys3 c, Bufs3 b, float inv_theta) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const int s = blockIdx.y, Np = m.Np, ninc = m.ninc;
    float acc[19];
#pragma unroll
    for (int q = 0; q < 19; ++q) acc[q] = 0.0f;
    const float c1 = c.dt4_f, c2 = c.dt2h_f;
    for (int k = m.inc_ptr[i]; k < m.inc_ptr[i + 1]; ++k) {
        const float* src = b.R32 + (size_t)m.inc_tet[k] * kR32 + 19 * s;
        const float bxi = m.inc_b32[k], byi = m.inc_b32[ninc + k], bzi = m.inc_b32[2 * ninc + k];
#pragma unroll
        for (int q = 0; q < 19; ++q) acc[q] = fmaf(src[q], c1 + c2 * edot3(q, bxi, byi, bzi), acc[q]);
    }
    const int F = m.F;
    for (int k = m.winc_ptr[i]; k < m.winc_ptr[i + 1]; ++k) {
        const int f = m.winc_face[k];
        int o[2], n = 0;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            int vv = m.wall_v[cc * F + f];
            if (vv != i && n < 2) o[n++] = vv;
        }
        const float A = (float)m.wall_area[f];
        const float nx = (float)m.wall_n[f], ny = (float)m.wall_n[F + f], nz = (float)m.wall_n[2 * F + f];
#pragma unroll
        for (int q = 1; q < 19; ++q) {
            const float en = edot3(q, nx, ny, nz);
            if (en < 0.0f) {
                const float di = wall_diff32(m, c, b, s, q, i);
                const float d1 = wall_diff32(m, c, b, s, q, o[0]);
                const float d2 = wall_diff32(m, c, b, s, q, o[1]);
                acc[q] += -c.dt_f * en * (A * (1.0f / 6.0f) * di + A * (1.0f / 12.0f) * (d1 + d2));
            }
        }
    }
    const float sc = m.inv_lumped32[i] * inv_theta;
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        const size_t r = (size_t)(19 * s + q) * Np + i;
        b.r32[r] = acc[q];
        b.e1[r] = acc[q] * sc;
    }
}

// ------------------------------------------- field and deviation update ----
// psi^{n+1} = psi_hat + d with psi_hat = psi^eq(n) + (1 - omega) dpsi:
//   C' = C + sum d_h (FP64), p' = p + sum d_g, rho' u' = rho u + 3 sum e d_g
//   (the deviations carry no mass or momentum), and
//   dpsi' = (1 - omega) dpsi + d - (psi^eq(n+1) - psi^eq(n)),
//   h^eq' - h^eq = Gamma dC + C' dGamma,
//   g^eq' - g^eq = w dp + (drho dC (Gamma - w) + rho' dGamma) / 3.
__device__ void dev32_update3(const DevMesh3& m, const Phys3& c, const Bufs3& b, int i, const float* d) {
    const int Np = m.Np;
    float sg = 0.0f, sh = 0.0f, mx = 0.0f, my = 0.0f, mz = 0.0f;
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        sg += d[q];
        sh += d[19 + q];
        mx += edot3(q, d[q], 0.0f, 0.0f);
        my += edot3(q, 0.0f, d[q], 0.0f);
        mz += edot3(q, 0.0f, 0.0f, d[q]);
    }
    const double Cd = b.C[i];
    const double Cnd = Cd + (double)sh;
    const float C = (float)Cd, dC = sh;
    const float rho = c.rho_v_f + C * c.drho_f;
    const float rho_n = c.rho_v_f + (float)Cnd * c.drho_f;
    const float ux = b.ux32[i], uy = b.uy32[i], uz = b.uz32[i];
    const float uxn = (rho * ux + 3.0f * mx) / rho_n, uyn = (rho * uy + 3.0f * my) / rho_n,
                uzn = (rho * uz + 3.0f * mz) / rho_n;
    const float om1 = 1.0f - omega32_3(C, c);
    const float uu15 = 1.5f * (ux * ux + uy * uy + uz * uz);
    const float dux = uxn - ux, duy = uyn - uy, duz = uzn - uz, sux = uxn + ux, suy = uyn + uy, suz = uzn + uz;
    const float Cn = (float)Cnd, drho = c.drho_f * dC;
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        const float w = (float)wq3(q);
        const float G = gamma32_3(q, ux, uy, uz, uu15);
        const float dG = dgamma32_3(q, dux, duy, duz, sux, suy, suz);
        const float dgeq = w * sg + (1.0f / 3.0f) * (drho * (G - w) + rho_n * dG);
        const float dheq = G * dC + Cn * dG;
        b.dpsi[q * Np + i] = om1 * b.dpsi[q * Np + i] + d[q] - dgeq;
        b.dpsi[(19 + q) * Np + i] = om1 * b.dpsi[(19 + q) * Np + i] + d[19 + q] - dheq;
    }
    b.C[i] = Cnd;
    b.p32[i] = b.p32[i] + sg;
    b.ux32[i] = uxn;
    b.uy32[i] = uyn;
    b.uz32[i] = uzn;
}

// ---------------------------------------------- conversions (FP64 I/O) ----
// psi = psi^eq(C, p, u) + dpsi, into the caller-order staging rows
__global__ void k3_dev32_to_stage(DevMesh3 m, Phys3 c, Bufs3 b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const size_t N = m.N, o = m.perm[i];
    const double C = b.C[i], p = b.p32[i], ux = b.ux32[i], uy = b.uy32[i], uz = b.uz32[i];
    const double rho = c.rho_v + C * (c.rho_l - c.rho_v);
    const double uu15 = 1.5 * (ux * ux + uy * uy + uz * uz);
    for (int q = 0; q < 19; ++q) {
        double eu = edot3(q, ux, uy, uz);
        double G = wq3(q) * (1.0 + 3.0 * eu + 4.5 * eu * eu - uu15);
        b.stage[(size_t)q * N + o] = wq3(q) * p + rho * (1.0 / 3.0) * (G - wq3(q)) + (double)b.dpsi[q * m.Np + i];
        b.stage[(size_t)(19 + q) * N + o] = G * C + (double)b.dpsi[(19 + q) * m.Np + i];
    }
}

// fields and deviations from full FP64 distributions staged in caller order
__global__ void k3_stage_to_dev32(DevMesh3 m, Phys3 c, Bufs3 b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const size_t N = m.N, o = m.perm[i];
    double C = 0.0, p = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
    for (int q = 0; q < 19; ++q) {
        double g = b.stage[(size_t)q * N + o];
        C += b.stage[(size_t)(19 + q) * N + o];
        p += g;
        mx += edot3(q, g, 0.0, 0.0);
        my += edot3(q, 0.0, g, 0.0);
        mz += edot3(q, 0.0, 0.0, g);
    }
    const double rho = c.rho_v + C * (c.rho_l - c.rho_v);
    const double ux = 3.0 * mx / rho, uy = 3.0 * my / rho, uz = 3.0 * mz / rho;
    const double uu15 = 1.5 * (ux * ux + uy * uy + uz * uz);
    for (int q = 0; q < 19; ++q) {
        double eu = edot3(q, ux, uy, uz);
        double G = wq3(q) * (1.0 + 3.0 * eu + 4.5 * eu * eu - uu15);
        b.dpsi[q * m.Np + i] = (float)(b.stage[(size_t)q * N + o] - (wq3(q) * p + rho * (1.0 / 3.0) * (G - wq3(q))));
        b.dpsi[(19 + q) * m.Np + i] = (float)(b.stage[(size_t)(19 + q) * N + o] - G * C);
    }
    b.C[i] = C;
    b.p32[i] = (float)p;
    b.ux32[i] = (float)ux;
    b.uy32[i] = (float)uy;
    b.uz32[i] = (float)uz;
}

// rest state from C0 staged in caller order: C = C0, p = u = 0, dpsi = 0
__global__ void k3_init_dev32(DevMesh3 m, Bufs3 b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    b.C[i] = b.stage[m.perm[i]];
    b.p32[i] = 0.0f;
    b.ux32[i] = 0.0f;
    b.uy32[i] = 0.0f;
    b.uz32[i] = 0.0f;
    b.mu32[i] = 0.0f;
    for (int q = 0; q < 38; ++q) b.dpsi[q * m.Np + i] = 0.0f;
}
