// Persistent batched step: many independent lattices of uneven sizes advanced
// together in one launch.  Every lattice is cut into tiles (W columns by a
// strip of rows); the launch's CTAs, all co-resident (cooperative launch), own
// the tiles round-robin and advance each of them step by step.  A tile's step
// reads the post-collision populations of the nodes within two of its own (in
// it or in neighbouring tiles of the same lattice, listed by the host from the
// actual reads, wrap-around included) and overwrites the buffer its readers
// read in the previous step.  So before step t a tile waits until every tile it
// reads or is read by has completed t steps (a per-tile counter, published with
// release semantics after the tile's stores), and there is no grid-wide
// barrier: lattices, and the tiles of one lattice, drift apart by up to one
// step where the work allows.
//
// Progress: every CTA visits its tiles in the same order every step, so the
// CTA that is furthest behind only ever waits for tiles that have already
// finished the steps it needs; with all CTAs resident the launch cannot
// deadlock.  Every wait is nevertheless bounded: after `spin_limit` polls it
// sets a status bit, and every CTA returns at its next tile.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Poll *p until it reaches `want` (counters only grow); false after `limit`
// polls, or as soon as another wait of the launch has given up.
__device__ __forceinline__ bool wait_done(const unsigned* p, unsigned want, long long limit,
                                          const unsigned* status) {
    for (long long it = 0; it < limit; ++it) {
        if ((int)(ld_acquire(p) - want) >= 0) return true;
        if ((it & 63) == 63 && ld_relaxed(status) != 0u) return false;
        __nanosleep(64);
    }
    return false;
}

template <int QS, int NW>
__global__ void __launch_bounds__(32 * NW, 20 / NW) batch_kernel(BatchArgs a) {
    constexpr int W = 32 * NW;
    constexpr int CASE_WORDS = (int)(sizeof(BatchCase) / sizeof(unsigned));
    static_assert(sizeof(BatchCase) % sizeof(unsigned) == 0, "BatchCase is copied as words");
    __shared__ BatchCase sc;
    __shared__ unsigned s_t0;
    __shared__ int s_go;

    // all tiles start a launch with the same count (the previous launch
    // finished every tile's steps); a CTA reads it from its first tile
    if (threadIdx.x == 0) s_t0 = blockIdx.x < a.ntiles ? ld_acquire(a.done + blockIdx.x) : 0u;
    __syncthreads();
    const unsigned t0 = s_t0;

    for (int s = 0; s < a.nsteps; ++s) {
        const unsigned t = t0 + (unsigned)s;  // steps completed before this one
        for (int k = blockIdx.x; k < a.ntiles; k += gridDim.x) {
            if (threadIdx.x == 0) s_go = ld_relaxed(a.status) == 0u;
            __syncthreads();  // also ends the previous tile's use of the shared ring
            if (threadIdx.x < BATCH_NEIGHBOURS) {
                const int nb = a.nbr[BATCH_NEIGHBOURS * k + threadIdx.x];
                if (nb >= 0 && !wait_done(a.done + nb, t, a.spin_limit, a.status)) {
                    atomicOr(a.status, 1u);
                    s_go = 0;
                }
            }
            const BatchTile tl = a.tiles[k];
            const unsigned* src = reinterpret_cast<const unsigned*>(a.cases + tl.c);
            for (int w = threadIdx.x; w < CASE_WORDS; w += W) reinterpret_cast<unsigned*>(&sc)[w] = src[w];
            __syncthreads();
            if (!s_go) return;  // uniform: read after the barrier
            const int par = (int)((sc.cur0 + t) & 1u);
            strip_tile<float, float, QS, false, W, true>(
                static_cast<const float*>(sc.pop[par]), static_cast<float*>(sc.pop[par ^ 1]),
                static_cast<float*>(sc.prev), sc.g, sc.C, sc.flag, 0u, nullptr, 0, tl.x0, tl.ya, tl.yb);
            __syncthreads();
            if (threadIdx.x == 0 && k != a.hold_tile) {
                __threadfence();
                st_release(a.done + k, t + 1u);
            }
        }
    }
}

template <int QS, int NW>
cudaError_t launch_batch_impl(const BatchArgs& a, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)a.grid);
    cfg.blockDim = dim3(32 * NW);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, batch_kernel<QS, NW>, a);
}

template <int QS, int NW>
int batch_blocks_per_sm_impl() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<QS, NW>, 32 * NW, 0) != cudaSuccess)
        return 0;
    return n;
}

}  // namespace lbm
