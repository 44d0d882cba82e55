// Surrogate network convolutions on the 5th-generation tensor cores
// (include/lbm_nn.h: lbm_nn_conv3x3, lbm_nn_conv3x3_wgrad).
//
// GEMM view of a periodic, dilated 3x3 convolution: M = pixels, N = cout,
// K = 9 taps x cin.  A tcgen05.mma (kind::f16: bfloat16 operands, FP32
// accumulation in tensor memory) multiplies 128 pixels of one image row by 16
// input channels.  Operands sit in shared memory in the 32-byte swizzled
// layout, one row (pixel, or weight row) of 16 channels per 32 bytes, so that
// the 128 pixels of a row shifted by a tap (dy, dx) are the same layout at
// another start address: a tap costs a descriptor, not a copy.  Activation
// rows arrive by TMA (cp.async.bulk.tensor) in that layout; the periodic halo
// columns of a unit by cp.async.
//
// Descriptor fields (measured on GB300 with probe kernels against host
// products): for no-swizzle K-major and MN-major operands the leading-byte
// offset steps along K and the stride-byte offset along M/N; for 32-byte
// swizzled MN-major operands the leading-byte offset steps between 16-element
// MN groups and the stride-byte offset between 8-row K groups.  The swizzle
// acts on absolute shared-memory address bits.  With M = 128 row m of the
// accumulator is TMEM lane m; with M = 64, rows 16q .. 16q + 15 are lanes
// 32q .. 32q + 15.  One thread issues a tcgen05.mma only about every 90 cycles,
// so small-N MMAs need more than one issuing warp to keep the tensor cores busy.
//
// Both kernels are persistent (one CTA per SM) over work units of R image rows
// x 128 columns; with dilation d the rows of a unit are d apart, so its input
// is R + 2 rows by 128 + 2d columns.  Warps have fixed roles (TMA issuer, halo
// loaders, MMA issuers, epilogue) and hand off through mbarriers; every wait is
// bounded: one that gives up sets bit 0 of *status and the CTA frees its tensor
// memory and returns.
#include "lbm.h"
#include "lbm_nn.h"
#include "nn_internal.h"

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

namespace {

constexpr int TC_COLS = 128;                    // pixels of one M tile (one image row)
constexpr long long TC_WAIT_LIMIT = 1LL << 24;  // polls of an mbarrier before giving up
constexpr size_t TC_MIN_SMEM = 120 * 1024;      // > half an SM: one CTA per SM (it owns all of TMEM it asks for)

// ------------------------------------------------------------------ PTX --
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor, no swizzle: start, leading-byte offset
// (along K), stride-byte offset (along M/N), all in 16-byte units; bit 46 is
// the descriptor version of sm_100-class tensor cores.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B bfloat16
// (bits 7-9, 10-12 = 1), A / B MN-major (bits 15 / 16), N >> 3 (bits 17-22),
// M >> 4 (bits 24-28).
constexpr uint32_t idesc_bf16(int M, int N, int a_mn, int b_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (long long i = 0; i < TC_WAIT_LIMIT; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// Whole warp: allocate / free `cols` columns of tensor memory (power of 2 >= 32).
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(slot), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(cols) : "memory");
}

// Whole warp: 16 consecutive 32-bit columns of this thread's lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

__host__ __device__ constexpr uint32_t pow2_cols(uint32_t n) {
    return n <= 32 ? 32 : (n <= 64 ? 64 : (n <= 128 ? 128 : (n <= 256 ? 256 : 512)));
}

// A work unit: image n, residue rho of the rows modulo d, row block rb (rows
// rho + (rb R + r) d, r < R), column block cb (columns 128 cb ..).
struct Unit {
    int n, rho, rb, x0;
};
__device__ __forceinline__ Unit unit_of(long long u, int d, int nrb, int ncb) {
    Unit U;
    U.x0 = (int)(u % ncb) * TC_COLS;
    u /= ncb;
    U.rb = (int)(u % nrb);
    u /= nrb;
    U.rho = (int)(u % d);
    U.n = (int)(u / d);
    return U;
}

// ------------------------------------------------------------ forward --
// Operand layout of the forward kernel: 32-byte swizzled, K-major.  A row
// (pixel, or weight row) is 16 channels = 32 bytes; groups of 8 rows are
// 256 bytes apart; the hardware exchanges the two 16-byte halves of rows 4..7
// of every 256-byte group by the absolute shared-memory address (byte-address
// bit 4 ^= bit 7; measured on GB300), so data written with that exchange can be
// read from any 32-byte-aligned start: the tap shift is still a start address.
// The tensor-memory-access unit (TMA) writes the same exchange (SWIZZLE_32B).
__device__ __forceinline__ uint32_t swz32(uint32_t a) { return a ^ (((a >> 7) & 1u) << 4); }

constexpr uint32_t LAYOUT_SW32 = 6;  // descriptor layout type, bits 61-63

__device__ __forceinline__ uint64_t sdesc_sw32(uint32_t saddr) {
    return sdesc(saddr, 16, 256) | ((uint64_t)LAYOUT_SW32 << 61);
}

// Roles of the forward kernel (warp index): 0-7 epilogue (warp w reads TMEM
// lane quarter w % 4, output rows r = w / 4 mod 2), 8 the TMA issuer (lane 0),
// 9-11 halo loaders (warp 9 + h loads the halos of stages q = h mod 3, so three
// stages' halo copies are in flight at once), 12-13 the MMA issuers (lane 0;
// warp 12 + p takes the units j = p mod 2 into accumulator buffer p: one thread
// issues a tcgen05.mma only every ~90 cycles on GB300, two reach the tensor
// cores' rate for these N <= 144 shapes (measured)); warp 12 owns the tensor memory.
constexpr int FW_EPI_WARPS = 8;
constexpr int FW_TMA_WARP = 8, FW_HALO_WARP = 9, FW_HALO_WARPS = 3, FW_MMA_WARP = 12, FW_MMA_WARPS = 2;
constexpr int FW_THREADS = 32 * 14;
// Roles of the weight-gradient kernel: 0-3 epilogue, 4 TMA, 5-7 halo, 8 MMA.
constexpr int WG_TMA_WARP = 4, WG_HALO_WARP = 5, WG_HALO_WARPS = 3, WG_MMA_WARP = 8;
constexpr int WG_THREADS = 32 * 9;
// A row of a stage plane: HALO halo slots, the 128 pixels of the unit, HALO
// halo slots (dilation <= HALO, 4 or 8); the unit's first pixel sits 32 HALO
// bytes into the row (128-byte aligned, as the TMA wants).  The weight-gradient
// kernel uses 8.
constexpr int WG_HALO = 8, WG_PITCH = TC_COLS + 2 * WG_HALO;
// Output staging of the forward kernel: per epilogue warp one row of its 32
// pixels x 48 bfloat16 channels (3 KB), written to global memory by a TMA store.
constexpr uint32_t FW_STG = 32 * 48 * 2;

__device__ __forceinline__ void mbar_init_n(uint32_t mbar, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mbar), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}\n" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}\n" ::"r"(mbar),
                 "r"(bytes)
                 : "memory");
}

// One box of the activation tensor {channel, x, image row} -> shared memory,
// completing `bytes` on the mbarrier.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c, int xx, int row, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c), "r"(xx), "r"(row), "r"(mbar)
        : "memory");
}

// Three 16-column loads of this thread's lane, one wait.
__device__ __forceinline__ void tmem_ld48(uint32_t taddr, float (&v)[48]) {
    uint32_t r[48];
#pragma unroll
    for (int q = 0; q < 3; ++q)
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
            : "=r"(r[16 * q + 0]), "=r"(r[16 * q + 1]), "=r"(r[16 * q + 2]), "=r"(r[16 * q + 3]), "=r"(r[16 * q + 4]),
              "=r"(r[16 * q + 5]), "=r"(r[16 * q + 6]), "=r"(r[16 * q + 7]), "=r"(r[16 * q + 8]),
              "=r"(r[16 * q + 9]), "=r"(r[16 * q + 10]), "=r"(r[16 * q + 11]), "=r"(r[16 * q + 12]),
              "=r"(r[16 * q + 13]), "=r"(r[16 * q + 14]), "=r"(r[16 * q + 15])
            : "r"(taddr + 16u * q));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int j = 0; j < 48; ++j) v[j] = __uint_as_float(r[j]);
}

// Whole warp: zero 16 consecutive 32-bit columns of this thread's lane.
__device__ __forceinline__ void tmem_zero16(uint32_t taddr) {
    const uint32_t z = 0;
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};\n" ::"r"(taddr),
        "r"(z)
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

__device__ __forceinline__ int image_row(const Unit& U, int k, int R, int d, int H) {
    int yy = U.rho + (U.rb * R + k - 1) * d;
    return yy + (yy < 0 ? H : (yy >= H ? -H : 0));
}

// The three row taps (dy) share the A operand: for input row k of a unit, one
// MMA multiplies the shifted row (dx) by the weights of all dy stacked along N
// (rows ordered dy = +1, 0, -1), producing the contributions of that input row
// to output rows k - 2, k - 1, k (those of the unit) in adjacent 48-column
// blocks of tensor memory.  Output row i of a unit owns columns
// [CO i, CO (i + 1)) of its buffer, so the three contributions to one output
// row (from input rows i, i + 1, i + 2) accumulate on the same columns.  Half
// the MMAs of one tap per MMA, each re-reading the 4 KB A tile for only 48 outputs.
// Every MMA accumulates: the epilogue zeroes a buffer after reading it.
template <int CI, int CO, int EPI, int R, int S, int HALO>
__global__ void __launch_bounds__(FW_THREADS, 1)
    conv_tc_kernel(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap ymap,
                   const uint8_t* __restrict__ x,
                   const __nv_bfloat16* __restrict__ w, const float* __restrict__ bias, void* __restrict__ y,
                   const float* __restrict__ res, const uint8_t* __restrict__ mask, int B, int H, int W, int d,
                   int* __restrict__ status) {
    static_assert(CI % 16 == 0 && CO % 16 == 0 && 3 * CO <= 256, "bfloat16 UMMA shapes");
    constexpr int KB = CI / 16;                         // 16-channel planes of the input, K blocks per tap
    constexpr int NC = CI / 8;                          // 16-byte chunks per input pixel
    constexpr uint32_t WBYTES = 9u * CI * CO * 2u;
    constexpr uint32_t ACC = (uint32_t)R * CO;          // TMEM columns of one unit
    constexpr uint32_t TCOLS = pow2_cols(2 * ACC);
    // a pipeline stage holds one 16-channel plane of a unit: (R + 2) rows of
    // PITCH pixel slots, 32 bytes each (a multiple of 256 bytes)
    constexpr int PITCH = TC_COLS + 2 * HALO;
    constexpr uint32_t STAGE = (uint32_t)((R + 2) * PITCH * 32);
    constexpr bool STAGED = CO == 48;                   // bfloat16 output through TMA stores
    constexpr uint32_t STG = STAGED ? FW_EPI_WARPS * FW_STG : 0u;
    constexpr uint32_t TX = (uint32_t)((R + 2) * TC_COLS * 32);  // TMA bytes per stage
    // halo warp h serves the stages s = h mod 3 only, and MMA warp p the stages
    // of the units j = p mod 2, so each waits on every phase of its stages'
    // barriers in order (a parity wait cannot tell phases two apart)
    static_assert(S % FW_HALO_WARPS == 0 && S % (2 * KB) == 0, "stages owned by one halo and one MMA warp");
    extern __shared__ __align__(1024) uint8_t smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // [stages][output staging][weights][bias][barriers: full S, empty S, tfull 2, tempty 2][tmem slot]
    const uint32_t base = smem_u32(smem);
    const uint32_t sin0 = base, sstg = base + S * STAGE, sw0 = sstg + STG;
    float* s_bias = reinterpret_cast<float*>(smem + S * STAGE + STG + WBYTES);
    uint64_t* s_bar = reinterpret_cast<uint64_t*>(s_bias + CO);
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(s_bar + 2 * S + 4);
    auto full = [&](int s) { return smem_u32(&s_bar[s]); };
    auto empty = [&](int s) { return smem_u32(&s_bar[S + s]); };
    auto tfull = [&](int b) { return smem_u32(&s_bar[2 * S + b]); };
    auto tempty = [&](int b) { return smem_u32(&s_bar[2 * S + 2 + b]); };

    // weights [co][t][ci] -> blocks (dx, 16-channel group) of 3 CO rows x 32
    // bytes, swizzled; row bi CO + o of a block holds tap dy = 1 - bi
    for (int i = tid; i < 9 * NC * CO; i += FW_THREADS) {
        const int o = i % CO, rest = i / CO, j = rest % NC, tap = rest / NC;  // tap = 3 bi + dxi
        const int bi = tap / 3, dxi = tap % 3, t = 3 * (2 - bi) + dxi;
        const uint4 v = *reinterpret_cast<const uint4*>(w + ((size_t)o * 9 + t) * CI + 8 * j);
        const uint32_t a = sw0 + (uint32_t)(((dxi * KB + (j >> 1)) * 3 + bi) * CO + o) * 32u + (uint32_t)(j & 1) * 16u;
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(swz32(a)), "r"(v.x), "r"(v.y), "r"(v.z),
                     "r"(v.w)
                     : "memory");
    }
    for (int i = tid; i < CO; i += FW_THREADS) s_bias[i] = (EPI != LBM_NN_MASK && bias) ? bias[i] : 0.0f;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init_n(full(s), 1 + 32);  // the TMA issuer's expect_tx and the 32 lanes of one halo warp
            mbar_init_n(empty(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init_n(tfull(b), 1);
            mbar_init_n(tempty(b), 32 * FW_EPI_WARPS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == FW_MMA_WARP) tmem_alloc(smem_u32(s_tmem), TCOLS);
    fence_proxy_async();  // the weights (generic stores) before the tensor cores read them
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *s_tmem;
    // the accumulators start at zero (every MMA accumulates)
    if (warp < FW_EPI_WARPS) {
        const uint32_t tq = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
        for (int r = warp >> 2; r < R; r += 2)
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int c0 = 0; c0 < CO; c0 += 16) tmem_zero16(tq + (uint32_t)(b * ACC + r * CO + c0));
        tmem_wait_st();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();

    const int nrb = H / d / R, ncb = W / TC_COLS;
    const long long units = (long long)B * d * nrb * ncb;
    const long long mine = units > blockIdx.x ? (units - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    bool ok = true;

    if (warp == FW_TMA_WARP) {
        // ---- TMA issuer: the unit's 128 columns of R + 2 rows, one box per row
        if (lane == 0) {
            for (long long q = 0; q < mine * KB; ++q) {
                const int s = (int)(q % S), kb = (int)(q % KB);
                if (q >= S) ok = mbar_wait(empty(s), (uint32_t)(((q / S) - 1) & 1));
                if (!ok) break;
                const Unit U = unit_of(blockIdx.x + (q / KB) * gridDim.x, d, nrb, ncb);
                mbar_arrive_tx(full(s), TX);
                const uint32_t st = sin0 + (uint32_t)s * STAGE;
#pragma unroll 1
                for (int k = 0; k < R + 2; ++k)
                    tma_load_3d(st + (uint32_t)(k * PITCH + HALO) * 32u, &xmap, 16 * kb, U.x0,
                                U.n * H + image_row(U, k, R, d, H), full(s));
            }
        }
        __syncwarp();
    } else if (warp >= FW_HALO_WARP && warp < FW_HALO_WARP + FW_HALO_WARPS) {
        // ---- halo loaders: d columns on each side, wrapped, 16 bytes per copy
        for (long long q = warp - FW_HALO_WARP; q < mine * KB; q += FW_HALO_WARPS) {
            const int s = (int)(q % S), kb = (int)(q % KB);
            if (q >= S) ok = mbar_wait(empty(s), (uint32_t)(((q / S) - 1) & 1));
            if (!ok) break;
            const Unit U = unit_of(blockIdx.x + (q / KB) * gridDim.x, d, nrb, ncb);
            const uint32_t st = sin0 + (uint32_t)s * STAGE;
            const int per_row = 2 * d * 2;  // 2d columns x two 16-byte halves of the plane
            for (int i = lane; i < (R + 2) * per_row; i += 32) {
                const int k = i / per_row, rem = i % per_row, h = rem & 1, e = rem >> 1;  // e < 2d
                // e < d: left column x0 - 1 - e (slot HALO - 1 - e); else right column x0 + 128 + (e - d)
                int xx = e < d ? U.x0 - 1 - e : U.x0 + TC_COLS + (e - d);
                const int slot = e < d ? HALO - 1 - e : HALO + TC_COLS + (e - d);
                xx += xx < 0 ? W : (xx >= W ? -W : 0);
                const uint8_t* src = x + (((long long)U.n * H + image_row(U, k, R, d, H)) * W + xx) * (16LL * NC) +
                                     32 * kb + 16 * h;
                const uint32_t dst = st + (uint32_t)(k * PITCH + slot) * 32u + (uint32_t)h * 16u;
                cp_async16(swz32(dst), src);
            }
            cp_async_commit();
            cp_async_wait_all();
            fence_proxy_async();
            mbar_arrive(full(s));
        }
    } else if (warp >= FW_MMA_WARP) {
        // ---- MMA issuers: per plane, per input row k, per column tap dx
        if (lane == 0) {
            for (long long j = warp - FW_MMA_WARP; j < mine && ok; j += FW_MMA_WARPS) {
                const int b = (int)(j & 1);
                if (j >= 2) ok = mbar_wait(tempty(b), (uint32_t)(((j >> 1) - 1) & 1));
#pragma unroll 1
                for (int kb = 0; kb < KB && ok; ++kb) {
                    const long long q = j * KB + kb;
                    const int s = (int)(q % S);
                    ok = mbar_wait(full(s), (uint32_t)((q / S) & 1));
                    if (!ok) break;
                    fence_after_sync();
                    const uint32_t sa = sin0 + (uint32_t)s * STAGE;
#pragma unroll 1
                    for (int k = 0; k < R + 2; ++k) {
                        // output rows lo .. hi of the unit receive input row k (dy = k - 1 - i)
                        const int lo = k - 2 > 0 ? k - 2 : 0, hi = k < R - 1 ? k : R - 1;
                        const int n = (hi - lo + 1) * CO, bi = 2 - k + lo;
                        const uint32_t idesc = idesc_bf16(128, n, 0, 0);
                        const uint32_t dcol = tmem + (uint32_t)b * ACC + (uint32_t)(lo * CO);
#pragma unroll
                        for (int dxi = 0; dxi < 3; ++dxi) {
                            const uint32_t aoff = (uint32_t)((k * PITCH + HALO + (dxi - 1) * d) * 32);
                            umma(dcol, sdesc_sw32(sa + aoff),
                                 sdesc_sw32(sw0 + (uint32_t)(((dxi * KB + kb) * 3 + bi) * CO) * 32u), idesc, 1u);
                        }
                    }
                    umma_commit(empty(s));
                }
                if (ok) umma_commit(tfull(b));
            }
        }
        __syncwarp();
    } else {
        // ---- epilogue: TMEM lane quarter warp % 4, pixel x0 + 32 (warp % 4) + lane,
        // output rows r = warp / 4 (mod 2)
        const int quarter = warp & 3;
        const uint32_t stg = sstg + (uint32_t)warp * FW_STG;  // this warp's output staging row
        for (long long j = 0; j < mine; ++j) {
            const int b = (int)(j & 1);
            ok = mbar_wait(tfull(b), (uint32_t)((j >> 1) & 1));
            if (!ok) break;
            fence_after_sync();
            const Unit U = unit_of(blockIdx.x + j * gridDim.x, d, nrb, ncb);
            const uint32_t tb = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)b * ACC;
#pragma unroll 1
            for (int r = warp >> 2; r < R; r += 2) {
                const int yy = U.rho + (U.rb * R + r) * d;
                const long long px = ((long long)U.n * H + yy) * W + U.x0 + 32 * quarter + lane;
                if constexpr (CO == 48) {
                    float v[48];
                    tmem_ld48(tb + (uint32_t)(r * CO), v);
                    uint32_t o[24];
                    if constexpr (EPI == LBM_NN_RELU) {
#pragma unroll
                        for (int q = 0; q < 24; ++q)
                            o[q] = pack_bf16x2(fmaxf(v[2 * q] + s_bias[2 * q], 0.0f),
                                               fmaxf(v[2 * q + 1] + s_bias[2 * q + 1], 0.0f));
                    } else {
                        static_assert(EPI == LBM_NN_MASK || CO != 48, "48-channel epilogues: ReLU or mask");
                        const uint4* mo = reinterpret_cast<const uint4*>(mask + px * CO * 2);
#pragma unroll
                        for (int q4 = 0; q4 < 6; ++q4) {
                            const uint4 m4 = mo[q4];
                            const uint32_t mk[4] = {m4.x, m4.y, m4.z, m4.w};
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const int q = 4 * q4 + e;
                                o[q] = pack_bf16x2(bf16_lo(mk[e]) > 0.0f ? v[2 * q] : 0.0f,
                                                   bf16_hi(mk[e]) > 0.0f ? v[2 * q + 1] : 0.0f);
                            }
                        }
                    }
                    // the previous TMA store from this staging row has read it
                    if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
                    __syncwarp();
#pragma unroll
                    for (int q4 = 0; q4 < 6; ++q4)
                        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(stg + (uint32_t)(lane * 96 + 16 * q4)),
                                     "r"(o[4 * q4]), "r"(o[4 * q4 + 1]), "r"(o[4 * q4 + 2]), "r"(o[4 * q4 + 3])
                                     : "memory");
                    fence_proxy_async();  // the staging row (generic stores) before the TMA reads it
                    __syncwarp();
                    if (lane == 0) {
                        asm volatile(
                            "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];\n" ::"l"(
                                reinterpret_cast<uint64_t>(&ymap)),
                            "r"(0), "r"(U.x0 + 32 * quarter), "r"((int)(U.n * H + yy)), "r"(stg)
                            : "memory");
                        asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
                    }
                } else {
                    static_assert(EPI == LBM_NN_RESIDUAL && CO == 16, "16-channel epilogue: residual");
                    float v[16];
                    tmem_ld16(tb + (uint32_t)(r * CO), v);
                    const float4* ro = reinterpret_cast<const float4*>(res + px * CO);
                    float4* yo = reinterpret_cast<float4*>(static_cast<float*>(y) + px * CO);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 a = ro[q];
                        yo[q] = make_float4(a.x + v[4 * q] + s_bias[4 * q], a.y + v[4 * q + 1] + s_bias[4 * q + 1],
                                            a.z + v[4 * q + 2] + s_bias[4 * q + 2], a.w + v[4 * q + 3] + s_bias[4 * q + 3]);
                    }
                }
#pragma unroll
                for (int c0 = 0; c0 < CO; c0 += 16) tmem_zero16(tb + (uint32_t)(r * CO + c0));
            }
            tmem_wait_st();
            fence_before_sync();
            mbar_arrive(tempty(b));
        }
        // every TMA store of this warp complete before the CTA (and its staging) goes away
        if (STAGED && lane == 0) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
    }
    if (!ok) atomicOr(status, 1);
    cp_async_wait_all();
    fence_before_sync();
    __syncthreads();
    if (warp == FW_MMA_WARP) {
        fence_after_sync();
        tmem_free(tmem, TCOLS);
    }
}

template <int CI, int CO, int R, int S, int HALO>
constexpr size_t conv_tc_smem() {
    return (size_t)S * ((R + 2) * (TC_COLS + 2 * HALO) * 32) + (CO == 48 ? FW_EPI_WARPS * FW_STG : 0) +
           9u * CI * CO * 2u + CO * 4 + (2 * S + 4) * 8 + 16;
}

// Tensor map of an NHWC bfloat16 activation: {channel, x, image row}, boxes of
// 16 channels x 128 pixels x 1 row, 32-byte swizzle.
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

bool activation_map(CUtensorMap* map, const void* x, int C, int B, int H, int W) {
    const EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)B * H};
    const cuuint64_t strides[2] = {(cuuint64_t)C * 2, (cuuint64_t)W * C * 2};
    const cuuint32_t box[3] = {16, (cuuint32_t)TC_COLS, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(x), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor map of a 48-channel NHWC bfloat16 output: boxes of all 48 channels x
// 32 pixels x 1 row (one epilogue warp's staging row), no swizzle.
bool output_map(CUtensorMap* map, void* y, int B, int H, int W) {
    const EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const cuuint64_t dims[3] = {48, (cuuint64_t)W, (cuuint64_t)B * H};
    const cuuint64_t strides[2] = {96, (cuuint64_t)W * 96};
    const cuuint32_t box[3] = {48, 32, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, y, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

template <int CI, int CO, int EPI, int R, int S, int HALO>
int conv_tc_launch(const void* x, const void* w, const float* bias, void* y, const float* res, const void* mask, int B,
                   int H, int W, int d, int* status, cudaStream_t s) {
    auto k = conv_tc_kernel<CI, CO, EPI, R, S, HALO>;
    const size_t smem = std::max(conv_tc_smem<CI, CO, R, S, HALO>(), TC_MIN_SMEM);
    static_assert(conv_tc_smem<CI, CO, R, S, HALO>() <= 227 * 1024, "shared memory");
    CUtensorMap map, ymap;
    if (!activation_map(&map, x, CI, B, H, W)) return LBM_ERR_CUDA;
    if (CO == 48 ? !output_map(&ymap, y, B, H, W) : !activation_map(&ymap, x, CI, B, H, W)) return LBM_ERR_CUDA;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return LBM_ERR_CUDA;
    const long long units = (long long)B * d * (H / d / R) * (W / TC_COLS);
    const int grid = (int)std::min<long long>(units, (long long)nn_sm_count());
    k<<<grid, FW_THREADS, smem, s>>>(map, ymap, static_cast<const uint8_t*>(x), static_cast<const __nv_bfloat16*>(w),
                                     bias, y, res, static_cast<const uint8_t*>(mask), B, H, W, d, status);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

// Rows per unit, stages (one 16-channel plane of a unit each) and halo slots:
// 4 rows, 6 stages, 4 halo slots for dilations up to 4 where the rows divide by
// 4; else 2 rows, 6 stages, 8 slots where they divide by 2; else 1 row.
template <int CI, int CO, int EPI>
int conv_tc_dispatch(const void* x, const void* w, const float* bias, void* y, const float* res, const void* mask,
                     int B, int H, int W, int d, int* status, cudaStream_t s) {
    if ((H / d) % 4 == 0 && d <= 4)
        return conv_tc_launch<CI, CO, EPI, 4, 6, 4>(x, w, bias, y, res, mask, B, H, W, d, status, s);
    if ((H / d) % 2 == 0) return conv_tc_launch<CI, CO, EPI, 2, 6, 8>(x, w, bias, y, res, mask, B, H, W, d, status, s);
    return conv_tc_launch<CI, CO, EPI, 1, 6, 8>(x, w, bias, y, res, mask, B, H, W, d, status, s);
}

// ------------------------------------------------------ weight gradient --
// dw[o][t][c] = sum_p dy[p][o] x[p + d off_t][c].  Per tap t one accumulator
// D_t (M = 64 rows, N columns) in tensor memory, K = pixels, 16 per MMA.  The
// larger of (cin, cout) is the M side (rows beyond it are computed from
// whatever follows in shared memory and never read).  Both operands are the
// activations' 32-byte swizzled planes read MN-major: channels are the
// contiguous (MN) direction, pixels the K direction; for MN-major swizzled
// operands the leading-byte offset steps between 16-channel planes and the
// stride-byte offset between groups of 8 pixels (256 bytes; measured on
// GB300).  The shifted operand is x (with its halo), dy is read at the unit's
// own pixels.  Roles as in the forward kernel: epilogue warps 0-3 (write the
// CTA's partial at the end), TMA issuer, three halo loaders, MMA issuer.  Each
// CTA accumulates over its units and writes one partial per tap; a second
// kernel adds the partials in a fixed order: deterministic.
// Bytes the M = 64 side reads past the end of a stage: its fourth plane (rows 48..63
// of M: read by the tensor cores, never used).
__host__ __device__ constexpr uint32_t wgrad_slack(int CI, int CO, int R) {
    const uint32_t psx = (uint32_t)((R + 2) * WG_PITCH * 32), psd = (uint32_t)(R * TC_COLS * 32);
    const uint32_t stage = (uint32_t)(CI / 16) * psx + (uint32_t)(CO / 16) * psd;
    const uint32_t a_end = CI >= CO ? 4 * psx : (uint32_t)(CI / 16) * psx + 4 * psd;
    return a_end > stage ? a_end - stage : 0u;
}

template <int CI, int CO, int R, int S>
__global__ void __launch_bounds__(WG_THREADS, 1)
    wgrad_tc_kernel(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap dmap,
                    const uint8_t* __restrict__ x, float* __restrict__ partials, int B, int H, int W, int d,
                    int* __restrict__ status) {
    constexpr bool A_IS_X = CI >= CO;
    constexpr int KX = CI / 16, KD = CO / 16;          // 16-channel planes of x and dy
    constexpr int NCX = CI / 8;                        // 16-byte chunks per x pixel
    constexpr int N = A_IS_X ? CO : CI;                // accumulator columns per tap
    constexpr int MREAL = A_IS_X ? CI : CO;            // real rows of M = 64
    constexpr uint32_t TCOLS = pow2_cols(9 * N);
    constexpr uint32_t IDESC = idesc_bf16(64, N, 1, 1);
    constexpr uint32_t PSX = (uint32_t)((R + 2) * WG_PITCH * 32);  // x plane: R + 2 rows with halo slots
    constexpr uint32_t PSD = (uint32_t)(R * TC_COLS * 32);         // dy plane: R rows of 128 pixels
    constexpr uint32_t STAGE = KX * PSX + KD * PSD;
    constexpr uint32_t TX = (uint32_t)((R + 2) * KX + R * KD) * TC_COLS * 32;
    constexpr int HW = S;  // halo warps in use: one per stage
    static_assert(MREAL <= 64 && N % 16 == 0, "M = 64 UMMA shapes");
    static_assert(S <= WG_HALO_WARPS, "one halo warp per stage");
    extern __shared__ __align__(1024) uint8_t smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sin0 = smem_u32(smem);
    // after the stages: room for the A side's fourth plane (read, never used), then barriers
    constexpr uint32_t SLACK = wgrad_slack(CI, CO, R);
    uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem + S * STAGE + SLACK);
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(s_bar + 2 * S + 1);
    auto full = [&](int s) { return smem_u32(&s_bar[s]); };
    auto empty = [&](int s) { return smem_u32(&s_bar[S + s]); };
    const uint32_t done = smem_u32(&s_bar[2 * S]);
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init_n(full(s), 1 + 32);
            mbar_init_n(empty(s), 1);
        }
        mbar_init_n(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == WG_MMA_WARP) tmem_alloc(smem_u32(s_tmem), TCOLS);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *s_tmem;
    const int nrb = H / d / R, ncb = W / TC_COLS;
    const long long units = (long long)B * d * nrb * ncb;
    const long long mine = units > blockIdx.x ? (units - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    bool ok = true;

    if (warp == WG_TMA_WARP) {
        if (lane == 0) {
            for (long long j = 0; j < mine; ++j) {
                const int s = (int)(j % S);
                if (j >= S) ok = mbar_wait(empty(s), (uint32_t)(((j / S) - 1) & 1));
                if (!ok) break;
                const Unit U = unit_of(blockIdx.x + j * gridDim.x, d, nrb, ncb);
                mbar_arrive_tx(full(s), TX);
                const uint32_t st = sin0 + (uint32_t)s * STAGE;
#pragma unroll 1
                for (int k = 0; k < R + 2; ++k) {
                    const int row = U.n * H + image_row(U, k, R, d, H);
#pragma unroll
                    for (int kb = 0; kb < KX; ++kb)
                        tma_load_3d(st + (uint32_t)kb * PSX + (uint32_t)(k * WG_PITCH + WG_HALO) * 32u, &xmap, 16 * kb,
                                    U.x0, row, full(s));
                    if (k >= 1 && k <= R) {
#pragma unroll
                        for (int kb = 0; kb < KD; ++kb)
                            tma_load_3d(st + KX * PSX + (uint32_t)kb * PSD + (uint32_t)((k - 1) * TC_COLS) * 32u, &dmap,
                                        16 * kb, U.x0, row, full(s));
                    }
                }
            }
        }
        __syncwarp();
    } else if (warp >= WG_HALO_WARP && warp < WG_HALO_WARP + HW) {
        // halo warp h serves stage h only, so it waits on every phase of that
        // stage's barrier in order (a parity wait cannot tell phases two apart)
        for (long long j = warp - WG_HALO_WARP; j < mine; j += HW) {
            const int s = (int)(j % S);
            if (j >= S) ok = mbar_wait(empty(s), (uint32_t)(((j / S) - 1) & 1));
            if (!ok) break;
            const Unit U = unit_of(blockIdx.x + j * gridDim.x, d, nrb, ncb);
            const uint32_t st = sin0 + (uint32_t)s * STAGE;
            const int per_row = 2 * d * NCX;
            for (int i = lane; i < (R + 2) * per_row; i += 32) {
                const int k = i / per_row, rem = i % per_row, jc = rem % NCX, e = rem / NCX;
                int xx = e < d ? U.x0 - 1 - e : U.x0 + TC_COLS + (e - d);
                const int slot = e < d ? WG_HALO - 1 - e : WG_HALO + TC_COLS + (e - d);
                xx += xx < 0 ? W : (xx >= W ? -W : 0);
                const uint8_t* src = x + (((long long)U.n * H + image_row(U, k, R, d, H)) * W + xx) * (16LL * NCX) + 16 * jc;
                const uint32_t dst = st + (uint32_t)(jc >> 1) * PSX + (uint32_t)(k * WG_PITCH + slot) * 32u +
                                     (uint32_t)(jc & 1) * 16u;
                cp_async16(swz32(dst), src);
            }
            cp_async_commit();
            cp_async_wait_all();
            fence_proxy_async();
            mbar_arrive(full(s));
        }
    } else if (warp == WG_MMA_WARP) {
        if (lane == 0) {
            for (long long j = 0; j < mine; ++j) {
                const int s = (int)(j % S);
                ok = mbar_wait(full(s), (uint32_t)((j / S) & 1));
                if (!ok) break;
                fence_after_sync();
                const uint32_t sx = sin0 + (uint32_t)s * STAGE, sd = sx + KX * PSX;
#pragma unroll 1
                for (int r = 0; r < R; ++r) {
#pragma unroll 1
                    for (int p0 = 0; p0 < TC_COLS; p0 += 16) {
                        const uint64_t dd = sdesc(sd + (uint32_t)(r * TC_COLS + p0) * 32u, PSD, 256) |
                                            ((uint64_t)LAYOUT_SW32 << 61);
#pragma unroll
                        for (int t = 0; t < 9; ++t) {
                            const int dy = t / 3 - 1, dx = t % 3 - 1;
                            const uint64_t xd =
                                sdesc(sx + (uint32_t)((r + 1 + dy) * WG_PITCH + WG_HALO + dx * d + p0) * 32u, PSX, 256) |
                                ((uint64_t)LAYOUT_SW32 << 61);
                            const uint32_t first = (j == 0 && r == 0 && p0 == 0);
                            umma(tmem + (uint32_t)(t * N), A_IS_X ? xd : dd, A_IS_X ? dd : xd, IDESC, !first);
                        }
                    }
                }
                umma_commit(empty(s));
            }
            umma_commit(done);
        }
        __syncwarp();
    } else {
        // ---- epilogue: D_t row m (m < 64) lives in lane 32 (m / 16) + m % 16
        if (mine > 0) ok = mbar_wait(done, 0);
        fence_after_sync();
        float* out = partials + (size_t)blockIdx.x * 9 * CI * CO;
        const int m = 16 * warp + lane;  // valid for lane < 16
#pragma unroll 1
        for (int t = 0; t < 9; ++t) {
#pragma unroll
            for (int c0 = 0; c0 < N; c0 += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(t * N + c0), v);
                if (lane < 16 && m < MREAL) {
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const int nn = c0 + e;
                        const float val = (mine > 0 && ok) ? v[e] : 0.0f;
                        if (A_IS_X) out[((size_t)t * CO + nn) * CI + m] = val;  // m = ci, nn = co
                        else out[((size_t)t * CO + m) * CI + nn] = val;         // m = co, nn = ci
                    }
                }
            }
        }
    }
    if (!ok) atomicOr(status, 1);
    cp_async_wait_all();
    fence_before_sync();
    __syncthreads();
    if (warp == WG_MMA_WARP) {
        fence_after_sync();
        tmem_free(tmem, TCOLS);
    }
}

// dw[o][t][c] = sum_b partials[b][t][o][c], fixed order
__global__ void wgrad_tc_reduce(const float* __restrict__ partials, int nb, int CO, int CI, float* __restrict__ dw) {
    const int n = 9 * CO * CI;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int c = i % CI, o = (i / CI) % CO, t = i / (CI * CO);
        float s = 0.0f;
        for (int b = 0; b < nb; ++b) s += partials[((size_t)b * 9 + t) * CO * CI + (size_t)o * CI + c];
        dw[((size_t)o * 9 + t) * CI + c] = s;
    }
}

template <int CI, int CO, int R, int S>
constexpr size_t wgrad_tc_smem() {
    return (size_t)S * ((CI / 16) * (R + 2) * WG_PITCH * 32 + (CO / 16) * R * TC_COLS * 32) +
           wgrad_slack(CI, CO, R) + (2 * S + 1) * 8 + 16;
}

long long wgrad_units(int B, int H, int W, int d, int R) { return (long long)B * d * (H / d / R) * (W / TC_COLS); }

// two rows per unit and two stages (both fit in shared memory), else one row
int wgrad_rows(int H, int d) { return (H / d) % 2 == 0 ? 2 : 1; }

template <int CI, int CO, int R, int S>
int wgrad_tc_launch(const void* x, const void* dy, float* dw, float* part, int B, int H, int W, int d, int* status,
                    cudaStream_t s) {
    auto k = wgrad_tc_kernel<CI, CO, R, S>;
    static_assert(wgrad_tc_smem<CI, CO, R, S>() <= 227 * 1024, "shared memory");
    const size_t smem = std::max(wgrad_tc_smem<CI, CO, R, S>(), TC_MIN_SMEM);
    CUtensorMap xmap, dmap;
    if (!activation_map(&xmap, x, CI, B, H, W) || !activation_map(&dmap, dy, CO, B, H, W)) return LBM_ERR_CUDA;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return LBM_ERR_CUDA;
    const int grid = (int)std::min<long long>(wgrad_units(B, H, W, d, R), (long long)nn_sm_count());
    k<<<grid, WG_THREADS, smem, s>>>(xmap, dmap, static_cast<const uint8_t*>(x), part, B, H, W, d, status);
    wgrad_tc_reduce<<<64, 256, 0, s>>>(part, grid, CO, CI, dw);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

template <int CI, int CO>
int wgrad_tc_dispatch(const void* x, const void* dy, float* dw, float* part, int B, int H, int W, int d, int* status,
                      cudaStream_t s) {
    if (wgrad_rows(H, d) == 2) return wgrad_tc_launch<CI, CO, 2, 2>(x, dy, dw, part, B, H, W, d, status, s);
    return wgrad_tc_launch<CI, CO, 1, 3>(x, dy, dw, part, B, H, W, d, status, s);
}

bool conv_shape_ok(int B, int H, int W, int d) {
    return B >= 1 && d >= 1 && d <= 8 && H >= d && H % d == 0 && W >= TC_COLS && W % TC_COLS == 0 &&
           (long long)B * H * W < (1LL << 40);
}

}  // namespace

extern "C" {

int lbm_nn_conv3x3(const void* x, int32_t cin, const void* weights, const float* bias, int32_t cout, int32_t epilogue,
                   const float* residual, const void* mask, void* y, int32_t batch, int32_t h, int32_t w,
                   int32_t dilation, int32_t* status, void* stream) {
    if (!x || !weights || !y || !status || !conv_shape_ok(batch, h, w, dilation)) return LBM_ERR_ARG;
    if (((uintptr_t)x | (uintptr_t)weights | (uintptr_t)y | (uintptr_t)residual | (uintptr_t)mask) % 16 != 0)
        return LBM_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int d = dilation;
    if (epilogue == LBM_NN_RELU) {
        if (cin == 16 && cout == 48)
            return conv_tc_dispatch<16, 48, LBM_NN_RELU>(x, weights, bias, y, nullptr, nullptr, batch, h, w, d, status, s);
        if (cin == 48 && cout == 48)
            return conv_tc_dispatch<48, 48, LBM_NN_RELU>(x, weights, bias, y, nullptr, nullptr, batch, h, w, d, status, s);
    } else if (epilogue == LBM_NN_RESIDUAL) {
        if (!residual) return LBM_ERR_ARG;
        if (cin == 48 && cout == 16)
            return conv_tc_dispatch<48, 16, LBM_NN_RESIDUAL>(x, weights, bias, y, residual, nullptr, batch, h, w, d,
                                                             status, s);
    } else if (epilogue == LBM_NN_MASK) {
        if (!mask) return LBM_ERR_ARG;
        if (cin == 48 && cout == 48)
            return conv_tc_dispatch<48, 48, LBM_NN_MASK>(x, weights, nullptr, y, nullptr, mask, batch, h, w, d, status, s);
        if (cin == 16 && cout == 48)
            return conv_tc_dispatch<16, 48, LBM_NN_MASK>(x, weights, nullptr, y, nullptr, mask, batch, h, w, d, status, s);
    }
    return LBM_ERR_ARG;
}

size_t lbm_nn_wgrad_partial_bytes(int32_t cin, int32_t cout, int32_t batch, int32_t h, int32_t w, int32_t dilation) {
    if (!conv_shape_ok(batch, h, w, dilation) || cin < 1 || cout < 1) return 0;
    const long long units = wgrad_units(batch, h, w, dilation, wgrad_rows(h, dilation));
    return (size_t)std::min<long long>(units, (long long)nn_sm_count()) * 9 * cin * cout * sizeof(float);
}

int lbm_nn_conv3x3_wgrad(const void* x, int32_t cin, const void* dy, int32_t cout, float* dw, void* partials,
                         size_t partial_bytes, int32_t batch, int32_t h, int32_t w, int32_t dilation, int32_t* status,
                         void* stream) {
    if (!x || !dy || !dw || !partials || !status || !conv_shape_ok(batch, h, w, dilation)) return LBM_ERR_ARG;
    if (((uintptr_t)x | (uintptr_t)dy) % 16 != 0) return LBM_ERR_ARG;
    if (partial_bytes < lbm_nn_wgrad_partial_bytes(cin, cout, batch, h, w, dilation)) return LBM_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float* part = static_cast<float*>(partials);
    const int d = dilation;
    if (cin == 16 && cout == 48) return wgrad_tc_dispatch<16, 48>(x, dy, dw, part, batch, h, w, d, status, s);
    if (cin == 48 && cout == 48) return wgrad_tc_dispatch<48, 48>(x, dy, dw, part, batch, h, w, d, status, s);
    if (cin == 48 && cout == 16) return wgrad_tc_dispatch<48, 16>(x, dy, dw, part, batch, h, w, d, status, s);
    return LBM_ERR_ARG;
}

}  // extern "C"
