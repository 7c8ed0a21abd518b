// Tiled FP32 solve step: one thread block per (node tile, part of the 18
// right-hand sides).  Included by felbm.cu after the DevMesh/Bufs
// definitions and the programmatic-launch helpers.
//
// The step is the Richardson update of k_sweep32,
//     x_{k+1,i} = x_{k,i} + tau m_i^{-1} (b_i - sum_j M_ij x_{k,j}),
// with the same arithmetic in the same order, so both give the same bits.
// What differs is where x_k comes from.  The nodes of a tile are a
// contiguous range of internal ids (recursive coordinate bisection), so the
// tile's part of each iterate row is one contiguous run of floats: one thread
// issues a 1D TMA bulk copy (cp.async.bulk) per row into shared memory,
// completing on an mbarrier, while the other threads gather the tile's halo
// (the few nodes outside it that its rows reference) from global memory.
// The row products then read shared memory only, through the tile-local
// column indices of the ELL copy (16-bit).  Every global access of the step
// is a coalesced stream (the iterate run, the right-hand side, the matrix
// rows, the new iterate) apart from the halo.

constexpr int kHaloMax = 504;                               // halo capacity of a tile
constexpr int kTileRow = kTileNodes + 8 + kHaloMax;         // floats per staged row (16-byte multiple)
constexpr int kTileThreads = 256;
static_assert(kTileRow % 4 == 0, "staged rows start on 16-byte boundaries");

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of the mbarrier for at most about limit_ns of
// wall time (and a fixed number of polls); false if it did not complete.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
    const uint64_t t0 = global_ns();
    for (int it = 0; it < (1 << 26); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63) == 63 && global_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// 1D TMA: `bytes` (a multiple of 16) from global src to shared dst (both
// 16-byte aligned), completing as transaction bytes on the mbarrier.
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// Error word of the solve kernels: bit 0 = a tiled step gave up waiting for
// its tile copy (the host reports it at the next synchronising call).
constexpr unsigned kErrTileWait = 1u;
constexpr uint64_t kTileWaitNs = 200000000ull;               // 0.2 s

template <int kW, int kParts>
__global__ void __launch_bounds__(kTileThreads) k_sweep_tile32(DevMesh m, Bufs b, const float* __restrict__ cur,
                                                               float* nxt, float tau) {
    pdl_release();
    static_assert(18 % kParts == 0, "parts must divide 18");
    constexpr int NQ = 18 / kParts;
    extern __shared__ __align__(128) float xs[];            // [NQ][kTileRow]
    __shared__ __align__(8) unsigned long long bar;
    const int tile = (int)blockIdx.x / kParts;
    const int q0 = NQ * ((int)blockIdx.x - tile * kParts);
    const int s0 = m.tile_ptr[tile], s1 = m.tile_ptr[tile + 1];
    const int a0 = s0 & ~3, span = ((s1 + 3) & ~3) - a0;    // 16-byte aligned run covering the tile
    const int h0 = m.halo_ptr[tile], nh = m.halo_ptr[tile + 1] - h0;
    const int Np = m.Np;
    const uint32_t bar_s = smem_addr(&bar);
    if (threadIdx.x == 0) mbar_init(bar_s, 1);
    pdl_wait();                                             // x_k is the previous launch's output
    // once a step has failed, later blocks do nothing (so a failure costs one
    // wait limit per resident block, not per block)
    if (__syncthreads_or(threadIdx.x == 0 && *(volatile unsigned*)b.kerr != 0)) return;
    if (threadIdx.x == 0) {
        mbar_expect_tx(bar_s, (uint32_t)(NQ * span * 4));
#pragma unroll 1
        for (int qq = 0; qq < NQ; ++qq)
            bulk_copy_g2s(smem_addr(xs + qq * kTileRow), cur + (size_t)(q0 + qq) * Np + a0, (uint32_t)(span * 4),
                          bar_s);
    }
    for (int hh = threadIdx.x; hh < nh; hh += kTileThreads) {
        const int j = m.halo[h0 + hh];
#pragma unroll
        for (int qq = 0; qq < NQ; ++qq) xs[qq * kTileRow + span + hh] = cur[(size_t)(q0 + qq) * Np + j];
    }
    const bool landed = mbar_wait_bounded(bar_s, 0, kTileWaitNs);
    if (__syncthreads_or(!landed)) {
        // a copy did not complete in time: flag it, and give it as long
        // again to land before the block's shared memory is freed
        if (threadIdx.x == 0) atomicOr(b.kerr, kErrTileWait);
        if (!landed) mbar_wait_bounded(bar_s, 0, kTileWaitNs);
        return;
    }
    for (int l = threadIdx.x; l < s1 - s0; l += kTileThreads) {
        const int i = s0 + l;
        int col[kW];
        float val[kW];
#pragma unroll
        for (int k = 0; k < kW; ++k) {
            col[k] = m.ell_loc[(size_t)k * Np + i];
            val[k] = m.ell_val[(size_t)k * Np + i];
        }
        const float s = tau * m.inv_lumped32[i];
        const int own = i - a0;
#pragma unroll
        for (int qq = 0; qq < NQ; ++qq) {
            const float* row = xs + qq * kTileRow;
            float acc = 0.0f;
#pragma unroll
            for (int k = 0; k < kW; ++k) acc = fmaf(val[k], row[col[k]], acc);
            const size_t r = (size_t)(q0 + qq) * Np + i;
            nxt[r] = fmaf(s, b.r32[r] - acc, row[own]);
        }
    }
}
