// Tiled FP32 solve step: a persistent kernel that walks work items (node
// tile, part of the 18 right-hand sides) through a pipeline of up to four
// shared-memory stages.  Included by felbm.cu after the DevMesh/Bufs definitions and the
// programmatic-launch helpers.
//
// The step is the Richardson update of k_sweep32,
//     x_{k+1,i} = x_{k,i} + tau m_i^{-1} (b_i - sum_j M_ij x_{k,j}),
// with the same arithmetic in the same order, so both give the same bits.
// What differs is how the operands arrive.  The nodes of a tile are a
// contiguous range of internal ids (recursive coordinate bisection), so
// everything a work item reads except the halo is a contiguous run per row:
// the tile's part of each x_k row and of each right-hand-side row, the ELL
// rows (tile-local 16-bit column indices and FP32 mass entries) and the
// inverse lumped mass.  One thread issues a 1D TMA bulk copy (cp.async.bulk)
// per run into one stage of shared memory, completing on that stage's
// mbarrier, and every thread queues cp.async copies of the halo (the nodes
// outside the tile that its rows reference) beside the x_k runs.  While the
// copies of the next items stream into the other stages, the block computes
// item n from its stage, reading shared memory only, and writes x_{k+1}
// with coalesced stores.  Global traffic is therefore the algorithmic streams plus the
// halo, all of it asynchronous.

constexpr int kHaloMax = 504;                               // halo capacity of a tile
constexpr int kTileRow = kTileNodes + 8 + kHaloMax;         // floats per staged x_k row (16-byte multiple)
constexpr int kTileRun = kTileNodes + 16;                   // elements per staged run (aligned tile range)
constexpr int kTileThreads = 512;
constexpr int kTileNPT = kTileNodes / kTileThreads;         // nodes per thread and item
static_assert(kTileRow % 4 == 0 && kTileRun % 8 == 0, "staged rows start on 16-byte boundaries");
static_assert(kTileNodes % kTileThreads == 0, "whole nodes per thread");

// Bytes of one pipeline stage for NQ right-hand sides and ELL width W.
__host__ __device__ constexpr size_t tile_stage_bytes(int nq, int w) {
    return (size_t)nq * kTileRow * 4 + (size_t)nq * kTileRun * 4 + (size_t)w * kTileRun * 4 + (size_t)kTileRun * 4 +
           (size_t)w * kTileRun * 2;
}

// Stages of the pipeline: as many as fit (at most four) in the 227 KB of
// shared memory a block may opt into on this part.
constexpr size_t kTileSmemBudget = 227 * 1024 - 1024;
__host__ __device__ constexpr int tile_stages(int nq, int w) {
    return (int)(kTileSmemBudget / tile_stage_bytes(nq, w)) < 4 ? (int)(kTileSmemBudget / tile_stage_bytes(nq, w))
                                                                : 4;
}

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

// Shared memory read by the generic proxy before a barrier is rewritten by
// the TMA (async proxy) after it.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int kPending>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(kPending) : "memory");
}

// Error word of the solve kernels: bit 0 = a tiled step gave up waiting for
// its copies (the host reports it at the next synchronising call).
constexpr unsigned kErrTileWait = 1u;
constexpr uint64_t kTileWaitNs = 200000000ull;               // 0.2 s

// One work item's runs in a stage: x_k rows (then the halo), right-hand-side
// rows, ELL values, inverse lumped mass, ELL tile-local columns.
template <int NQ, int kW>
struct TileStage {
    float* x;
    float* r;
    float* lv;
    float* il;
    uint16_t* lc;
    __device__ explicit TileStage(unsigned char* base) {
        x = reinterpret_cast<float*>(base);
        r = x + NQ * kTileRow;
        lv = r + NQ * kTileRun;
        il = lv + kW * kTileRun;
        lc = reinterpret_cast<uint16_t*>(il + kTileRun);
    }
};

// Issue the copies of work item w into a stage: the TMA runs from thread 0
// (after the proxy fence: the stage was last read by the generic proxy),
// the halo as cp.async by every thread, committed as one group.
template <int NQ, int kW, int kParts>
__device__ __forceinline__ void tile_issue(const DevMesh& m, const Bufs& b, const float* __restrict__ cur, int w,
                                           const TileStage<NQ, kW>& sg, uint32_t bar) {
    const int tile = w / kParts;
    const int q0 = NQ * (w - tile * kParts);
    const int s0 = m.tile_ptr[tile], s1 = m.tile_ptr[tile + 1];
    const int a0 = s0 & ~3, span = ((s1 + 3) & ~3) - a0;     // float runs: 16-byte aligned
    const int c0 = s0 & ~7, span16 = ((s1 + 7) & ~7) - c0;   // 16-bit runs: 16-byte aligned
    const int Np = m.Np;
    if (threadIdx.x == 0) {
        fence_proxy_async_smem();
        mbar_expect_tx(bar, (uint32_t)((2 * NQ + kW + 1) * span * 4 + kW * span16 * 2));
#pragma unroll 1
        for (int qq = 0; qq < NQ; ++qq) {
            bulk_copy_g2s(smem_addr(sg.x + qq * kTileRow), cur + (size_t)(q0 + qq) * Np + a0, span * 4, bar);
            bulk_copy_g2s(smem_addr(sg.r + qq * kTileRun), b.r32 + (size_t)(q0 + qq) * Np + a0, span * 4, bar);
        }
#pragma unroll 1
        for (int k = 0; k < kW; ++k) {
            bulk_copy_g2s(smem_addr(sg.lv + k * kTileRun), m.ell_val + (size_t)k * Np + a0, span * 4, bar);
            bulk_copy_g2s(smem_addr(sg.lc + k * kTileRun), m.ell_loc + (size_t)k * Np + c0, span16 * 2, bar);
        }
        bulk_copy_g2s(smem_addr(sg.il), m.inv_lumped32 + a0, span * 4, bar);
    }
    const int h0 = m.halo_ptr[tile], nh = m.halo_ptr[tile + 1] - h0;
    for (int hh = threadIdx.x; hh < nh; hh += kTileThreads) {
        const int j = m.halo[h0 + hh];
#pragma unroll
        for (int qq = 0; qq < NQ; ++qq)
            cp_async4(smem_addr(sg.x + qq * kTileRow + span + hh), cur + (size_t)(q0 + qq) * Np + j);
    }
    cp_async_commit();
}

template <int kW, int kParts>
__global__ void __launch_bounds__(kTileThreads, 1) k_sweep_tile32(DevMesh m, Bufs b, const float* __restrict__ cur,
                                                                  float* nxt, float tau) {
    pdl_release();
    static_assert(18 % kParts == 0, "parts must divide 18");
    constexpr int NQ = 18 / kParts;
    constexpr int kS = tile_stages(NQ, kW);
    static_assert(kS >= 2, "at least two stages");
    constexpr size_t kStage = tile_stage_bytes(NQ, kW);
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) unsigned long long bars[4];
    const uint32_t bar0 = smem_addr(&bars[0]);             // stage st's barrier: bar0 + 8 st
    const int n_items = m.n_tiles * kParts;
    const int G = (int)gridDim.x;
    const int Np = m.Np;
    if (threadIdx.x == 0)
        for (int k = 0; k < kS; ++k) mbar_init(bar0 + 8 * k, 1);
    pdl_wait();                                             // x_k is the previous launch's output
    // once a step has failed, later blocks do nothing
    if (__syncthreads_or(threadIdx.x == 0 && *(volatile unsigned*)b.kerr != 0)) return;
    // item it of this block is w = blockIdx.x + it G, in stage it % kS (its
    // (it / kS)-th use, barrier parity (it / kS) & 1); kS - 1 items run ahead,
    // and every iteration commits one cp.async group (empty past the end)
    for (int k = 0; k < kS - 1; ++k) {
        const int w = (int)blockIdx.x + k * G;
        if (w < n_items) tile_issue<NQ, kW, kParts>(m, b, cur, w, TileStage<NQ, kW>(smem + k * kStage), bar0 + 8 * k);
        else cp_async_commit();
    }
    for (int it = 0;; ++it) {
        const int w = (int)blockIdx.x + it * G;
        if (w >= n_items) break;
        const int st = it % kS;
        const int ahead = it + kS - 1, wn = (int)blockIdx.x + ahead * G, sn = ahead % kS;
        if (wn < n_items)
            tile_issue<NQ, kW, kParts>(m, b, cur, wn, TileStage<NQ, kW>(smem + sn * kStage), bar0 + 8 * sn);
        else
            cp_async_commit();
        const bool landed = mbar_wait_bounded(bar0 + 8 * st, (it / kS) & 1, kTileWaitNs);
        cp_async_wait<kS - 1>();                            // this item's halo (groups after it may pend)
        if (__syncthreads_or(!landed)) {
            // a copy did not complete in time: flag it, and give the copies
            // in flight as long again to land before shared memory is freed
            if (threadIdx.x == 0) atomicOr(b.kerr, kErrTileWait);
            for (int k = 0; k < kS; ++k) {
                const int j = it + k;
                if ((int)blockIdx.x + j * G < n_items && (k > 0 || !landed))
                    mbar_wait_bounded(bar0 + 8 * (j % kS), (j / kS) & 1, kTileWaitNs);
            }
            cp_async_wait<0>();
            return;
        }
        const TileStage<NQ, kW> sg(smem + st * kStage);
        const int tile = w / kParts;
        const int q0 = NQ * (w - tile * kParts);
        const int s0 = m.tile_ptr[tile], s1 = m.tile_ptr[tile + 1];
        const int a0 = s0 & ~3, c0 = s0 & ~7;
#pragma unroll
        for (int n = 0; n < kTileNPT; ++n) {
            const int l = (int)threadIdx.x + n * kTileThreads;
            if (l >= s1 - s0) break;
            const int i = s0 + l, o = i - a0;
            int col[kW];
            float val[kW];
#pragma unroll
            for (int k = 0; k < kW; ++k) {
                col[k] = sg.lc[k * kTileRun + (i - c0)];
                val[k] = sg.lv[k * kTileRun + o];
            }
            const float s = tau * sg.il[o];
#pragma unroll
            for (int qq = 0; qq < NQ; ++qq) {
                const float* row = sg.x + qq * kTileRow;
                float acc = 0.0f;
#pragma unroll
                for (int k = 0; k < kW; ++k) acc = fmaf(val[k], row[col[k]], acc);
                nxt[(size_t)(q0 + qq) * Np + i] = fmaf(s, sg.r[qq * kTileRun + o] - acc, row[o]);
            }
        }
        __syncthreads();                                    // this stage is free for item it + kS
    }
}
