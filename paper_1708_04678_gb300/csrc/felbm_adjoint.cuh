// Adjoint (reverse mode) of one FP64 time step (included by felbm.cu).
//
// Given lambda = dL/dpsi^{n+1} and the state psi^n, the passes below form
// dL/dpsi^n and add dL/dphi_c (per wall edge).  The step (Sec. II.C of
// arXiv:1708.04678) is   psi^{n+1} = psi_hat + M11^{-1} RHS(psi_hat, Phi),
// psi_hat = collide(psi), Phi = forces(moments, mu, lap mu), so in reverse:
//   lambda_RHS = M11^{-1} lambda                       (M11 symmetric: same solve)
//   A:  per triangle  lambda_R = sum_k w(v_k) lambda_RHS(v_k); the force
//       Jacobian with respect to the nine element scalars (u, C, mu means,
//       grad C, grad p, lap mu) by forward-mode dual numbers, contracted with
//       A lambda_R
//   B:  per triangle  lambda of grad mu (own and the neighbours' lap mu terms)
//   D:  per node      gathers over incident triangles: lambda of psi_hat,
//       mu, C, p, u; transpose of the weak bounce-back wall term
//   E:  per node      transpose of mu (double well, patch Laplacian, wetting
//       flux; per-edge dL/dphi_c), of the collision (dual numbers in C, p,
//       u) and of the moments -> lambda^n.
// Every pass gathers; none scatters, so there are no atomics and the result
// does not depend on scheduling.
#pragma once

// ------------------------------------------------------------ dual numbers
struct Dual {
    double v, d;
};
__device__ __forceinline__ Dual mkd(double v, double d = 0.0) { return Dual{v, d}; }
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator-(Dual a) { return {-a.v, -a.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
    double q = a.v / b.v;
    return {q, (a.d - q * b.d) / b.v};
}
__device__ __forceinline__ Dual operator+(Dual a, double b) { return {a.v + b, a.d}; }
__device__ __forceinline__ Dual operator+(double a, Dual b) { return {a + b.v, b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, double b) { return {a.v - b, a.d}; }
__device__ __forceinline__ Dual operator-(double a, Dual b) { return {a - b.v, -b.d}; }
__device__ __forceinline__ Dual operator*(Dual a, double b) { return {a.v * b, a.d * b}; }
__device__ __forceinline__ Dual operator*(double a, Dual b) { return {a * b.v, a * b.d}; }
__device__ __forceinline__ Dual operator/(Dual a, double b) { return {a.v / b, a.d / b}; }
__device__ __forceinline__ Dual operator/(double a, Dual b) {
    double q = a / b.v;
    return {q, -q * b.d / b.v};
}
__device__ __forceinline__ double val(double x) { return x; }
__device__ __forceinline__ double val(Dual x) { return x.v; }
__device__ __forceinline__ double der(Dual x) { return x.d; }

template <int q>
__device__ __forceinline__ Dual edot(Dual vx, Dual vy) {
    Dual r = mkd(0.0);
    if (ex(q) == 1) r = vx;
    if (ex(q) == -1) r = -vx;
    if (ey(q) == 1) r = r + vy;
    if (ey(q) == -1) r = r - vy;
    return r;
}

// ------------------------------------------ forces as a function of nine
// element scalars: the same expressions as k_element (eq:G, eq:H at the
// barycentre); T = double or Dual.
template <class T>
__device__ __forceinline__ void forces_T(const Phys& c, T ux, T uy, T Cb, T mub, T gCx, T gCy, T gpx, T gpy, T lapmu,
                                         T (&phig)[9], T (&phih)[9]) {
    const double third = 1.0 / 3.0;
    const double drho = c.rho_l - c.rho_v;
    T rhob = c.rho_v + Cb * drho;
    T grx = drho * gCx, gry = drho * gCy;
    T f = 3.0 * Cb / rhob;
    T vhx = gCx - f * (gpx - mub * gCx), vhy = gCy - f * (gpy - mub * gCy);
    T u_gr = ux * grx + uy * gry, u_gC = ux * gCx + uy * gCy, u_vh = ux * vhx + uy * vhy;
    T uu15 = 1.5 * (ux * ux + uy * uy);
    T Mlap = c.mobility * lapmu;
#define FELBM_FT_Q(q)                                                                                  \
    {                                                                                                  \
        T eu = edot<q>(ux, uy);                                                                        \
        T G = wq(q) * (1.0 + 3.0 * eu + 4.5 * eu * eu - uu15);                                          \
        phig[q] = third * (G - wq(q)) * (edot<q>(grx, gry) - u_gr) + mub * G * (edot<q>(gCx, gCy) - u_gC); \
        phih[q] = ((edot<q>(vhx, vhy) - u_vh) + Mlap) * G;                                            \
    }
    FELBM_FT_Q(0) FELBM_FT_Q(1) FELBM_FT_Q(2) FELBM_FT_Q(3) FELBM_FT_Q(4)
    FELBM_FT_Q(5) FELBM_FT_Q(6) FELBM_FT_Q(7) FELBM_FT_Q(8)
#undef FELBM_FT_Q
}

// post-collision populations from the node's populations (fixed) and its
// fields C, p, u (T = Dual to differentiate through the fields only)
template <class T>
__device__ __forceinline__ void collide_T(const Phys& c, const double (&g)[9], const double (&h)[9], T C, T p, T ux,
                                          T uy, T (&gh)[9], T (&hh)[9]) {
    T rho = c.rho_v + C * (c.rho_l - c.rho_v);
    T inv_tau = C * (1.0 / c.tau_l) + (1.0 - C) * (1.0 / c.tau_v);
    T omega = 1.0 / (1.0 / inv_tau + 0.5);
    T uu15 = 1.5 * (ux * ux + uy * uy);
    T rcs2 = rho * (1.0 / 3.0);
#define FELBM_CT_Q(q)                                                  \
    {                                                                  \
        T eu = edot<q>(ux, uy);                                        \
        T G = wq(q) * (1.0 + 3.0 * eu + 4.5 * eu * eu - uu15);         \
        T geq = wq(q) * p + rcs2 * (G - wq(q));                        \
        T heq = G * C;                                                 \
        gh[q] = g[q] - omega * (g[q] - geq);                           \
        hh[q] = h[q] - omega * (h[q] - heq);                           \
    }
    FELBM_CT_Q(0) FELBM_CT_Q(1) FELBM_CT_Q(2) FELBM_CT_Q(3) FELBM_CT_Q(4)
    FELBM_CT_Q(5) FELBM_CT_Q(6) FELBM_CT_Q(7) FELBM_CT_Q(8)
#undef FELBM_CT_Q
}

// ------------------------------------------------------ adjoint buffers
struct AdjBufs {
    double* lam;     // [18][Np] lambda (in: dL/dpsi^{n+1}; out: dL/dpsi^n)
    double* lamhat;  // [18][Np] dL/dpsi_hat
    double* lamR;    // [T][18]  dL/dR
    double* lamE;    // [T][9]   dL/d(C_bar, mu_bar, ux_bar, uy_bar, gCx, gCy, gpx, gpy, lap mu)
    double* lamG;    // [2][Tp]  dL/d(grad mu)
    double* lamMu;   // [Np]
    double* lamC;    // [Np]
    double* lamP;
    double* lamUx;
    double* lamUy;
    double* dphi;    // [E] dL/dphi_c accumulated per wall edge since the seed
    const double* lamRHS;  // [18][Np] M11^{-1} lambda (the solve's output)
    const double* kval;    // [nnz] P1 stiffness entries (symmetric)
};

// A: element residual adjoint and the force Jacobian (9 dual passes)
__global__ void __launch_bounds__(128) k_adj_elem_a(DevMesh m, Phys c, Bufs b, AdjBufs a) {
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
    const double c1 = c.dt * (1.0 / 3.0), c2 = 0.5 * c.dt * c.dt;
    // lambda_R = sum over the vertices of the RHS weights times lambda_RHS
    double lr[18];
#define FELBM_ADJA_Q(q)                                                               \
    {                                                                                 \
        double sg = 0.0, sh = 0.0;                                                    \
        for (int k = 0; k < 3; ++k) {                                                 \
            double w = c1 + c2 * edot<q, double>(bx[k], by[k]);                       \
            sg += w * a.lamRHS[q * Np + v[k]];                                        \
            sh += w * a.lamRHS[(9 + q) * Np + v[k]];                                  \
        }                                                                             \
        lr[q] = sg;                                                                   \
        lr[9 + q] = sh;                                                               \
    }
    FELBM_ADJA_Q(0) FELBM_ADJA_Q(1) FELBM_ADJA_Q(2) FELBM_ADJA_Q(3) FELBM_ADJA_Q(4)
    FELBM_ADJA_Q(5) FELBM_ADJA_Q(6) FELBM_ADJA_Q(7) FELBM_ADJA_Q(8)
#undef FELBM_ADJA_Q
#pragma unroll
    for (int q = 0; q < 18; ++q) a.lamR[(size_t)t * 18 + q] = lr[q];
    // the nine element scalars, as in k_element
    double Cs = 0, uxs = 0, uys = 0, mus = 0, gCx = 0, gCy = 0, gpx = 0, gpy = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double Cv = b.C[v[k]], pv = b.p[v[k]];
        Cs += Cv;
        uxs += b.ux[v[k]];
        uys += b.uy[v[k]];
        mus += b.mu[v[k]];
        gCx += Cv * bx[k];
        gCy += Cv * by[k];
        gpx += pv * bx[k];
        gpy += pv * by[k];
    }
    const double third = 1.0 / 3.0;
    double sv[9] = {uxs * third, uys * third, Cs * third, mus * third, gCx, gCy, gpx, gpy, 0.0};
    {
        double gmx = b.gmu[t], gmy = b.gmu[Tp + t], lapmu = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            int nb = m.nbr[k * Tp + t];
            if (nb >= 0) lapmu -= (gmx + b.gmu[nb]) * bx[k] + (gmy + b.gmu[Tp + nb]) * by[k];
        }
        sv[8] = lapmu;
    }
    // lambda_s[j] = sum_q A lr_q dPhi_q / ds_j
    double ls[9];
    for (int j = 0; j < 9; ++j) {
        Dual s[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) s[k] = mkd(sv[k], k == j ? 1.0 : 0.0);
        Dual pg[9], ph[9];
        forces_T<Dual>(c, s[0], s[1], s[2], s[3], s[4], s[5], s[6], s[7], s[8], pg, ph);
        double acc = 0.0;
#pragma unroll
        for (int q = 0; q < 9; ++q) acc += lr[q] * der(pg[q]) + lr[9 + q] * der(ph[q]);
        ls[j] = A * acc;
    }
    // stored as (C_bar, mu_bar, ux_bar, uy_bar, gCx, gCy, gpx, gpy, lap mu)
    double* dst = a.lamE + (size_t)t * 9;
    dst[0] = ls[2];
    dst[1] = ls[3];
    dst[2] = ls[0];
    dst[3] = ls[1];
    dst[4] = ls[4];
    dst[5] = ls[5];
    dst[6] = ls[6];
    dst[7] = ls[7];
    dst[8] = ls[8];
}

// B: lambda of grad mu_T.  lap mu_T = -sum_k[nb_k] (G_T + G_nb).b_k, so G_T
// receives -lambda_lap(T) b_k(T) from its own edges and -lambda_lap(nb) b_s(nb)
// from each neighbour (s = the shared edge's slot in the neighbour).
__global__ void __launch_bounds__(kBlock) k_adj_elem_b(DevMesh m, AdjBufs a) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m.T) return;
    const int Tp = m.Tp;
    const double lt = a.lamE[(size_t)t * 9 + 8];
    double gx = 0.0, gy = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int nb = m.nbr[k * Tp + t];
        if (nb < 0) continue;
        int sl = m.nbr_slot[k * Tp + t];
        double ln = a.lamE[(size_t)nb * 9 + 8];
        gx -= lt * m.grad[(2 * k) * Tp + t] + ln * m.grad[(2 * sl) * Tp + nb];
        gy -= lt * m.grad[(2 * k + 1) * Tp + t] + ln * m.grad[(2 * sl + 1) * Tp + nb];
    }
    a.lamG[t] = gx;
    a.lamG[Tp + t] = gy;
}

// D: node gathers over the incident triangles and the wall bounce-back term
__global__ void __launch_bounds__(128) k_adj_node_d(DevMesh m, Phys c, AdjBufs a) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const int Np = m.Np;
    double lh[18];
#pragma unroll
    for (int q = 0; q < 18; ++q) lh[q] = a.lam[q * Np + i];
    double lmu = 0.0, lC = 0.0, lp = 0.0, lux = 0.0, luy = 0.0;
    const double third = 1.0 / 3.0;
    for (int k = m.inc_ptr[i]; k < m.inc_ptr[i + 1]; ++k) {
        const int t = m.inc_tri[k];
        const double bxi = m.inc_bx[k], byi = m.inc_by[k];
        const double A = m.area[t];
        const double* lr = a.lamR + (size_t)t * 18;
#define FELBM_ADJD_Q(q)                                          \
        {                                                        \
            double eb = A * edot<q, double>(bxi, byi);           \
            lh[q] -= eb * lr[q];                                 \
            lh[9 + q] -= eb * lr[9 + q];                         \
        }
        FELBM_ADJD_Q(1) FELBM_ADJD_Q(2) FELBM_ADJD_Q(3) FELBM_ADJD_Q(4)
        FELBM_ADJD_Q(5) FELBM_ADJD_Q(6) FELBM_ADJD_Q(7) FELBM_ADJD_Q(8)
#undef FELBM_ADJD_Q
        const double* le = a.lamE + (size_t)t * 9;
        lC += le[0] * third + le[4] * bxi + le[5] * byi;
        lmu += le[1] * third + a.lamG[t] * bxi + a.lamG[m.Tp + t] * byi;
        lux += le[2] * third;
        luy += le[3] * third;
        lp += le[6] * bxi + le[7] * byi;
    }
    // weak bounce-back: RHS_q(i) += f [L/3 (psi_opp - psi_q)(i) + L/6 (psi_opp - psi_q)(o)]
    // for incoming q on each wall edge (i, o); its transpose seen from node i:
    for (int k = m.winc_ptr[i]; k < m.winc_ptr[i + 1]; ++k) {
        const int e = m.winc_edge[k];
        const int o = m.wall_a[e] == i ? m.wall_b[e] : m.wall_a[e];
        const double L = m.wall_len[e], nx = m.wall_nx[e], ny = m.wall_ny[e];
#define FELBM_ADJW_Q(q)                                                                            \
        {                                                                                          \
            double en = edot<q, double>(nx, ny);                                                   \
            if (en < 0.0) {                                                                        \
                double f = -c.dt * en;                                                             \
                double cg = f * (L * (1.0 / 3.0) * a.lamRHS[q * Np + i] + L * (1.0 / 6.0) * a.lamRHS[q * Np + o]); \
                double ch = f * (L * (1.0 / 3.0) * a.lamRHS[(9 + q) * Np + i] +                    \
                                 L * (1.0 / 6.0) * a.lamRHS[(9 + q) * Np + o]);                   \
                lh[opp(q)] += cg;                                                                  \
                lh[q] -= cg;                                                                       \
                lh[9 + opp(q)] += ch;                                                              \
                lh[9 + q] -= ch;                                                                   \
            }                                                                                      \
        }
        FELBM_ADJW_Q(1) FELBM_ADJW_Q(2) FELBM_ADJW_Q(3) FELBM_ADJW_Q(4)
        FELBM_ADJW_Q(5) FELBM_ADJW_Q(6) FELBM_ADJW_Q(7) FELBM_ADJW_Q(8)
#undef FELBM_ADJW_Q
    }
#pragma unroll
    for (int q = 0; q < 18; ++q) a.lamhat[q * Np + i] = lh[q];
    a.lamMu[i] = lmu;
    a.lamC[i] = lC;
    a.lamP[i] = lp;
    a.lamUx[i] = lux;
    a.lamUy[i] = luy;
}

// E: transpose of mu, of the collision and of the moments -> lambda^n.
__global__ void __launch_bounds__(128) k_adj_node_e(DevMesh m, Phys c, Bufs b, AdjBufs a) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const int Np = m.Np;
    const double C = b.C[i], p = b.p[i], ux = b.ux[i], uy = b.uy[i];
    // mu_i = 2 beta C (C-1)(2C-1) - kappa sum_j l_ij C_j + (1/V_i) sum_e phi_e L_e s(C_a, C_b),
    // l_ij = -2 K_ij / V_i with K symmetric
    double lC = a.lamC[i];
    lC += 2.0 * c.beta * (6.0 * C * C - 6.0 * C + 1.0) * a.lamMu[i];
    double kl = 0.0;
    for (int k = m.row_ptr[i]; k < m.row_ptr[i + 1]; ++k) {
        int j = m.col[k];
        kl += a.kval[k] * a.lamMu[j] * m.inv_vol[j];
    }
    lC += 2.0 * c.kappa * kl;
    for (int k = m.winc_ptr[i]; k < m.winc_ptr[i + 1]; ++k) {
        const int e = m.winc_edge[k];
        const int ia = m.wall_a[e], ib = m.wall_b[e];
        const double Ca = b.C[ia], Cb = b.C[ib];
        const double w = a.lamMu[ia] * m.inv_vol[ia] + a.lamMu[ib] * m.inv_vol[ib];
        const double Co = ia == i ? Cb : Ca;
        const double ds = 0.5 - (2.0 * C + Co) * (1.0 / 3.0);   // d s / d C_i
        lC += m.wall_phi[e] * m.wall_len[e] * ds * w;
        if (ia == i) {   // one owner per edge writes its phi_c contribution
            const double sv = 0.5 * (Ca + Cb) - (Ca * Ca + Ca * Cb + Cb * Cb) * (1.0 / 3.0);
            a.dphi[e] += m.wall_len[e] * sv * w;
        }
    }
    // collision: psi_hat = psi - omega(C) (psi - psi_eq(C, p, u)), psi fixed, fields dual
    double g[9], h[9], lh[18];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        g[q] = b.psi[q * Np + i];
        h[q] = b.psi[(9 + q) * Np + i];
        lh[q] = a.lamhat[q * Np + i];
        lh[9 + q] = a.lamhat[(9 + q) * Np + i];
    }
    double lf[4];
    for (int j = 0; j < 4; ++j) {
        Dual gh[9], hh[9];
        collide_T<Dual>(c, g, h, mkd(C, j == 0), mkd(p, j == 1), mkd(ux, j == 2), mkd(uy, j == 3), gh, hh);
        double acc = 0.0;
#pragma unroll
        for (int q = 0; q < 9; ++q) acc += lh[q] * der(gh[q]) + lh[9 + q] * der(hh[q]);
        lf[j] = acc;
    }
    lC += lf[0];
    const double lp = a.lamP[i] + lf[1];
    const double lux = a.lamUx[i] + lf[2], luy = a.lamUy[i] + lf[3];
    // direct dependence of psi_hat on psi: (1 - omega)
    const double inv_tau = C / c.tau_l + (1.0 - C) / c.tau_v;
    const double om1 = 1.0 - 1.0 / (1.0 / inv_tau + 0.5);
    // moments: C = sum h, p = sum g, u = 3 sum e g / rho(C)
    const double rho = c.rho_v + C * (c.rho_l - c.rho_v);
    lC -= (ux * lux + uy * luy) * (c.rho_l - c.rho_v) / rho;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        a.lam[q * Np + i] = om1 * lh[q] + lp + 3.0 * (ex(q) * lux + ey(q) * luy) / rho;
        a.lam[(9 + q) * Np + i] = om1 * lh[9 + q] + lC;
    }
}
