// Device code of the fused phase-field / flow / two-scalar LB step.
//
// Step kernel ("strip" design).  A CTA of 4 warps owns 128 consecutive columns
// and marches up a strip of rows, one thread per column.  For row y it
//   a. pulls g and reads the previous-step macros of its node (row y), and
//      pulls f, h1, h2 of row y+1: streaming happens on the read (pull scheme),
//      half-way bounce-back where the upstream node is behind a wall;
//   b. forms the zeroth moments of row y+1: phi = sum f (Eq. 26) and the
//      implicit c1, c2 of Eq. (37), solved exactly as a 2x2 system, into a
//      4-row ring in shared memory (lanes 0 and 127 also cover the two halo
//      columns);
//   c. after one barrier, evaluates the D2Q9 isotropic stencils of Eqs. (41)-(42)
//      for grad phi, lap phi, grad c1, grad c2 at row y from rows y-1..y+1;
//   d. forms mu_phi (Eqs. 4-5), the force, u and p (Eq. 32), the viscosity and
//      tau_g (Eq. 33 with Eq. 7, Eq. 48 or the exponential law) and the
//      backward differences d/dt(chi u);
//   e. collides f (Eqs. 23-25), g (Eqs. 28-31), h1 and h2 (Eqs. 34-36) in
//      registers, with f, h1, h2 of row y kept from the previous iteration,
//      and stores the post-collision populations at the node itself.
// Each node's f, h1, h2 are read from DRAM once per step; only the two halo
// rows and columns of a strip are pulled twice (L2 hits).
//
// The collisions are written in factored form, w_i [a + c_i . b + ...], and
// the rest populations of f, h1, h2 take the exact post-collision sums minus
// the moving populations, so rounding of the lattice weights cannot bias the
// conserved totals.  Laplacians are formed from differences to the centre
// node.
//
// Readings of points the paper leaves open (shared with the CPU oracle only
// through their written statement): d/dt(chi u) = (chi u)^n - (chi u)^{n-1};
// n = grad phi / (|grad phi| + 1e-4); mirror ghosts at walls for the stencils;
// rho and mu use phi clipped to [0, 1]; D_m = 0 where its denominator <= 0.
#pragma once

#include "lbm_internal.h"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

namespace lbm {

// ---- lattice: D2Q9 order rest, +x, +y, -x, -y, (+,+), (-,+), (-,-), (+,-) ----
__host__ __device__ constexpr int cx(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cy(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
// opposite direction: 1<->3, 2<->4, 5<->7, 6<->8
__host__ __device__ constexpr int opp(int i) {
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5);
}
template <typename R>
__host__ __device__ constexpr R w9(int i) {
    return i == 0 ? R(4) / R(9) : (i <= 4 ? R(1) / R(9) : R(1) / R(36));
}
// D2Q5 keeps cs^2 = 1/3 with w0 = 1/3, w1..4 = 1/6
template <typename R, int Q>
__host__ __device__ constexpr R wq(int i) {
    return Q == 5 ? (i == 0 ? R(1) / R(3) : R(1) / R(6)) : w9<R>(i);
}

// w_i * s with the weight rounding removed.  In FP32 the weights 4/9, 1/9, 1/36
// all round up by the same 7.45e-9 relative; multiplying by them directly would
// scale the collided momentum by (1 + 7.45e-9 w_g) every step.  Splitting
// w_i = hi + lo and fusing s*hi + (s*lo) rounds s*w_i once, without the bias.
__device__ __forceinline__ float w9_times(int i, float s) {
    const float hi = w9<float>(i);
    const float lo = (float)(w9<double>(i) - (double)hi);
    return __fmaf_rn(s, hi, s * lo);
}
__device__ __forceinline__ double w9_times(int i, double s) { return w9<double>(i) * s; }
// (3/5) * s, rounded once: the pressure of Eq. (32b) feeds the next equilibrium,
// so a biased 3/5 would compound by ~4e-8 per step in FP32
__device__ __forceinline__ float three_fifths(float s) {
    return __fmaf_rn(s, 0.6f, s * (float)(0.6 - (double)0.6f));
}
__device__ __forceinline__ double three_fifths(double s) { return 0.6 * s; }

#if LBM_DEBUG
// Debug build: the range a CTA's accesses must fall in (set by dbg_begin) and
// the status word a failed check reports to: a device global of this
// translation unit (always a valid address, whatever the CTA's range holds),
// read and cleared by the host through debug_status_take.
__shared__ const char* dbg_lo;
__shared__ const char* dbg_hi;
static __device__ unsigned dbg_status;
namespace {
unsigned dbg_status_take_here() {
    unsigned v = 0;
    const unsigned zero = 0;
    if (cudaMemcpyFromSymbol(&v, dbg_status, sizeof v) != cudaSuccess) v = FLAG_BOUNDS;
    cudaMemcpyToSymbol(dbg_status, &zero, sizeof zero);
    return v;
}
const bool dbg_registered = (register_debug_status(dbg_status_take_here), true);
}  // namespace
#endif
// Whole CTA, at the start of a kernel that loads through ld / stores through
// st_chk and stcs: its range of device memory (a no-op in a release build).
__device__ __forceinline__ void dbg_begin(const char* lo, const char* hi) {
#if LBM_DEBUG
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        dbg_lo = lo;
        dbg_hi = hi;
    }
    __syncthreads();
#endif
}
// Whether an access of n bytes at p is inside the CTA's range (always in a
// release build); outside, FLAG_BOUNDS is reported and the caller skips it.
__device__ __forceinline__ bool dbg_in(const void* p, size_t n) {
#if LBM_DEBUG
    const char* c = static_cast<const char*>(p);
    if (c >= dbg_lo && c + n <= dbg_hi) return true;
    atomicOr(&dbg_status, FLAG_BOUNDS);
    return false;
#else
    (void)p;
    (void)n;
    return true;
#endif
}
// Population / macro loads of the step: through the read-only path when the
// buffer is constant for the kernel's lifetime (one step per launch), or cached
// in L2 only (CG) when other CTAs of the same launch rewrite it between steps
// (the persistent batched kernel), so that no stale L1 line is read.
template <bool CG, typename T>
__device__ __forceinline__ T ld(const T* p) {
    if (!dbg_in(p, sizeof(T))) return T{};
    if constexpr (CG) return __ldcg(p);
    else return __ldg(p);
}
// a plain load and a plain store of the workspace, checked in a debug build
// (for data the kernel itself rewrites, which the read-only path may not cache)
template <typename T>
__device__ __forceinline__ T ld_plain(const T* p) {
    if (!dbg_in(p, sizeof(T))) return T{};
    return *p;
}
template <typename T>
__device__ __forceinline__ void st_chk(T* p, T v) {
    if (dbg_in(p, sizeof(T))) *p = v;
}
template <typename T>
__device__ __forceinline__ void stcs(T* p, T v) {
    if (dbg_in(p, sizeof(T))) __stcs(p, v);
}
__device__ __forceinline__ void stcs(__half* p, __half v) {
    if (dbg_in(p, sizeof v)) __stcs(reinterpret_cast<unsigned short*>(p), __half_as_ushort(v));
}
__device__ __forceinline__ void stcs(__nv_bfloat16* p, __nv_bfloat16 v) {
    if (dbg_in(p, sizeof v)) __stcs(reinterpret_cast<unsigned short*>(p), __bfloat16_as_ushort(v));
}

// Storage <-> arithmetic conversions (16-bit storage rounds to nearest even).
template <typename T>
struct IsHalf { static constexpr bool value = false; };
template <>
struct IsHalf<__half> { static constexpr bool value = true; };
template <>
struct IsHalf<__nv_bfloat16> { static constexpr bool value = true; };
template <typename R>
__device__ __forceinline__ R to_r(int v) { return R(v); }
template <typename R>
__device__ __forceinline__ R to_r(float v) { return R(v); }
template <typename R>
__device__ __forceinline__ R to_r(double v) { return R(v); }
template <typename R>
__device__ __forceinline__ R to_r(__half v) { return R(__half2float(v)); }
template <typename R>
__device__ __forceinline__ R to_r(__nv_bfloat16 v) { return R(__bfloat162float(v)); }
template <typename T, typename R>
__device__ __forceinline__ T from_r(R v) {
    if constexpr (std::is_same<T, __half>::value) return __float2half_rn(float(v));
    else if constexpr (std::is_same<T, __nv_bfloat16>::value) return __float2bfloat16_rn(float(v));
    else return T(v);
}

// 16-bit storage pairs two populations pulled from the same upstream node in
// one 32-bit word: (f_i, g_i) for each D2Q9 direction i and (h1_i, h2_i) for
// each scalar direction, so that a warp's load is 128 contiguous bytes as in
// FP32.  lo16 / hi16 give the low / high value of a word in FP32.
template <typename T>
__device__ __forceinline__ float lo16(uint32_t w) {
    if constexpr (std::is_same<T, __half>::value) return __half2float(__ushort_as_half((unsigned short)(w & 0xffffu)));
    else return __uint_as_float(w << 16);
}
template <typename T>
__device__ __forceinline__ float hi16(uint32_t w) {
    if constexpr (std::is_same<T, __half>::value) return __half2float(__ushort_as_half((unsigned short)(w >> 16)));
    else return __uint_as_float(w & 0xffff0000u);
}

// IEEE half storage keeps g_i * 2^10: the flow populations are of the order of
// the pressure (1e-6 .. 1e-2 in lattice units), much of which lies below half's
// smallest normal number (6.1e-5), while |g_i| 2^10 stays far below its largest
// (65504) for any state with |u| < 1.  Scaling by a power of two is exact.
template <typename T>
struct GScale { static constexpr float up = 1.0f, down = 1.0f; };
template <>
struct GScale<__half> { static constexpr float up = 1024.0f, down = 1.0f / 1024.0f; };
template <typename T, typename R>
__device__ __forceinline__ R g_value(R stored) {
    if constexpr (std::is_same<T, __half>::value) return stored * R(GScale<T>::down);
    else return stored;
}
template <typename T, typename R>
__device__ __forceinline__ R g_stored(R v) {
    if constexpr (std::is_same<T, __half>::value) return v * R(GScale<T>::up);
    else return v;
}

// Stochastic rounding to 16 bits (Croci & Giles 2020; Connolly, Higham & Mary
// 2021): a value between two neighbours of the 16-bit grid is rounded up with
// probability equal to its distance from the lower one, in ulps.  The stored
// value is then exact on average, and increments smaller than half an ulp -- the
// slow diffusive and sharpening updates of the populations -- are not rounded
// away every step as they are under round-to-nearest.
//
// The two populations of a stored word are rounded and packed by one hardware
// conversion with stochastic rounding (cvt.rs.{bf16x2,f16x2}.f32, Blackwell):
// for bfloat16 it adds the random bits r & 0xffff (low value) and r >> 16 (high
// value) to the float encodings and truncates; for half, bits 0-12 and 16-28 of
// r round the 13 dropped significand bits (subnormals at their own spacing).
//
// Random bits: a seed per node and step (the 32-bit finalizer of MurmurHash3
// applied to the node's coordinates and the bits of its new macros) is xored
// with the bits of the word's low value and multiplied by an odd constant per
// word (a multiplicative hash, Knuth's Fibonacci hashing).  For a uniform seed
// the product's low and high halves are uniform and independent of the value,
// so the rounding stays unbiased, and a run is deterministic: graph and plain
// launches, and a restart from a checkpoint, give the same bits.
__device__ __forceinline__ uint32_t mix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}
// random word for stored word j (0 .. 17) of a node with seed h, low value lo
__device__ __forceinline__ uint32_t sr_word(uint32_t h, float lo, int j) {
    return (h ^ __float_as_uint(lo)) * (0x9e3779b9u + (uint32_t)j * 0x3c6ef372u);
}
// lo and hi rounded stochastically to T with the random word r, packed as one
// stored word (lo in the low half); lo16 / hi16 read the rounded values back
template <typename T>
__device__ __forceinline__ uint32_t round_pair(float lo, float hi, uint32_t r) {
    uint32_t w;
    if constexpr (std::is_same<T, __half>::value)
        asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(w) : "f"(hi), "f"(lo), "r"(r));
    else
        asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(w) : "f"(hi), "f"(lo), "r"(r));
    return w;
}
// A value of the arithmetic type R as stored in T (FP32 / FP64 storage: exact).
template <typename T, typename R>
__device__ __forceinline__ T store_value(R v) {
    static_assert(!IsHalf<T>::value, "16-bit storage rounds word pairs (round_pair)");
    return T(v);
}

// Node coordinate seen by a stencil: periodic wrap, or the mirror ghost of
// a half-way wall (the ghost takes the value of the adjacent fluid node).
__device__ __forceinline__ int resolve(int v, int n, int wall) {
    if (wall) return v < 0 ? 0 : (v >= n ? n - 1 : v);
    v %= n;
    return v < 0 ? v + n : v;
}

// Element offset of value q = 0 of node (x, y) in a buffer with NQ values per node.
template <int NQ>
__device__ __forceinline__ long long node_off(const Geometry& g, int x, int y) {
    return ((long long)y * g.nxb + (x >> 5)) * (NQ * 32) + (x & 31);
}

// Populations per node: 9 f, 9 g, QS h1, QS h2.
__host__ __device__ constexpr int nq_of(int qs) { return 18 + 2 * qs; }

// Population i of the lattice whose first plane is `plane0`, pulled into node
// (x, y): the post-collision value of the upstream node x - c_i, or -- if that
// node is behind a wall -- the node's own value in the opposite direction
// (half-way bounce-back).  Any node; used off the fast path.
template <int NQ>
__device__ __forceinline__ long long pull_off(const Geometry& g, int x, int y, int plane0, int i) {
    int sx = x - cx(i), sy = y - cy(i);
    const bool ox = sx < 0 || sx >= g.nx, oy = sy < 0 || sy >= g.ny;
    if ((ox && g.wall_x) || (oy && g.wall_y)) return node_off<NQ>(g, x, y) + (plane0 + opp(i)) * 32;
    if (ox) sx = sx < 0 ? sx + g.nx : sx - g.nx;
    if (oy) sy = sy < 0 ? sy + g.ny : sy - g.ny;
    return node_off<NQ>(g, sx, sy) + (plane0 + i) * 32;
}
// Element offset of population plane q (f: 0-8, g: 9-17, h1: 18.., h2: 18+QS..)
// of node (x, y).  FP32/FP64: plane q of the node's 32-node block.  16-bit: the
// node's word j of the block (j = i for f_i, g_i; 9 + i for h1_i, h2_i), low
// half for f and h1, high half for g and h2.
template <typename T, int NQ>
__device__ __forceinline__ long long pop_off(const Geometry& g, int x, int y, int q) {
    if constexpr (IsHalf<T>::value) {
        constexpr int QS = (NQ - 18) / 2;
        const int j = q < 9 ? q : (q < 18 ? q - 9 : (q < 18 + QS ? q - 9 : q - 9 - QS));
        const int hi = (q >= 9 && q < 18) || q >= 18 + QS;
        return 2 * (node_off<NQ / 2>(g, x, y) + j * 32) + hi;
    } else {
        return node_off<NQ>(g, x, y) + q * 32;
    }
}
// pull_off in element units of a population buffer of storage type T
template <typename T, int NQ>
__device__ __forceinline__ long long pop_pull_off(const Geometry& g, int x, int y, int plane0, int i) {
    if constexpr (IsHalf<T>::value) {
        int sx = x - cx(i), sy = y - cy(i);
        const bool ox = sx < 0 || sx >= g.nx, oy = sy < 0 || sy >= g.ny;
        if ((ox && g.wall_x) || (oy && g.wall_y)) return pop_off<T, NQ>(g, x, y, plane0 + opp(i));
        if (ox) sx = sx < 0 ? sx + g.nx : sx - g.nx;
        if (oy) sy = sy < 0 ? sy + g.ny : sy - g.ny;
        return pop_off<T, NQ>(g, sx, sy, plane0 + i);
    } else {
        return pull_off<NQ>(g, x, y, plane0, i);
    }
}
template <int NQ, typename T, typename R, bool CG = false>
__device__ __forceinline__ R pull_any(const T* __restrict__ src, const Geometry& g, int x, int y,
                                      int plane0, int i) {
    if constexpr (IsHalf<T>::value) return to_r<R>(ld<CG>(src + pop_pull_off<T, NQ>(g, x, y, plane0, i)));
    int sx = x - cx(i), sy = y - cy(i);
    const bool ox = sx < 0 || sx >= g.nx, oy = sy < 0 || sy >= g.ny;
    if ((ox && g.wall_x) || (oy && g.wall_y))
        return to_r<R>(ld<CG>(src + node_off<NQ>(g, x, y) + (plane0 + opp(i)) * 32));
    if (ox) sx += sx < 0 ? g.nx : -g.nx;
    if (oy) sy += sy < 0 ? g.ny : -g.ny;
    return to_r<R>(ld<CG>(src + node_off<NQ>(g, sx, sy) + (plane0 + i) * 32));
}

// Node (sx, sy) that population i pulled into (x, y) comes from: the upstream
// node x - c_i (periodic image), or the node itself behind a wall (half-way
// bounce-back returns its own population of the opposite direction).
__device__ __forceinline__ void pull_src(const Geometry& g, int x, int y, int i, int& sx, int& sy) {
    sx = x - cx(i);
    sy = y - cy(i);
    const bool ox = sx < 0 || sx >= g.nx, oy = sy < 0 || sy >= g.ny;
    if ((ox && g.wall_x) || (oy && g.wall_y)) {
        sx = x;
        sy = y;
        return;
    }
    if (ox) sx += sx < 0 ? g.nx : -g.nx;
    if (oy) sy += sy < 0 ? g.ny : -g.ny;
}

// 16-bit storage keeps the flow populations as g_i - b_i(p), p the pressure of
// the node that wrote them: b_i(p) = 3 bw_i p for i > 0 and 3 (bw_0 - 1) p for
// i = 0, the pressure part of g_i^eq (Eqs. 29-30) up to the base weights bw_i
// below.  In a light phase the
// pressure part dominates g_i (p ~ 1e-4 against rho u ~ 1e-6 in the gas of a
// density-ratio-1000 bubble), so 8 significant bits of g_i carry almost nothing
// of the momentum; the difference is of the order of rho u and the
// non-equilibrium part.  The reader adds b_i back with the writer's FP32 p.
//
// Base weights b_i of these offsets: the D2Q9 weights rounded to multiples of
// 2^-20 (116508 / 2^20 = 1/9 - 4e-7, a quarter of that for the diagonals, and
// the rest weight 466036 / 2^20 = 4/9 + 2e-6), so that they sum to exactly 1
// and each is exact in FP32.  With the FP32-rounded weights (their sum is
// 1 + 7.5e-9) every node would gain 7.5e-9 phi per step: the gas of a bubble
// lost 3.5 nodes of area over 4000 steps on 256 x 512.
template <typename R>
__host__ __device__ constexpr R bw9(int i) {
    return i == 0 ? R(466036.0 / 1048576.0) : (i <= 4 ? R(116508.0 / 1048576.0) : R(29127.0 / 1048576.0));
}
// ... and of the scalar populations, stored as h_k,i - bq_i c_k,w with c_k,w the
// writer's FP32 c_k: the D2Q5 weights rounded the same way (174763 / 2^20 =
// 1/6 + 3e-7 on the axes, the rest 349524 / 2^20), the D2Q9 ones for scalar_q = 9.
template <typename R, int QS>
__host__ __device__ constexpr R bwq(int i) {
    return QS == 5 ? (i == 0 ? R(349524.0 / 1048576.0) : R(174763.0 / 1048576.0)) : bw9<R>(i);
}
template <typename R>
__device__ __forceinline__ R p_base(int i, R p) {
    return i == 0 ? (R(3) * (bw9<R>(0) - R(1))) * p : (R(3) * bw9<R>(i)) * p;
}
// ... and the phase-field populations as f_i - bw_i phi_w, phi_w the phase field
// of the node that wrote them (the equilibrium of Eq. 24 at rest, up to the
// base weights).  Stored
// whole (or as f_i - w_i / 2), their 8-bit rounding put noise of ~1e-3 into phi
// in the bulk phases, and the surface-tension force of that noise, divided by
// the gas density, drove the gas velocity; the remainder is of the order of
// w_i phi c_i.u and the non-equilibrium part.  One fused multiply-add decodes
// it, the same one wherever a population is read.
__device__ __forceinline__ float f_dec(float stored, int i, float phw) { return fmaf(bw9<float>(i), phw, stored); }

// Writers' bases (16-bit storage), per node at index k = y * nxb * 32 + x:
// the FP32 pair (p, phi) at floats 2k, 2k + 1 of Geometry::pb_in / pb_out, and
// (c1, c2) as two IEEE halves in word k of the plane that follows (from float
// 2 N on, N = ny * nxb * 32); then the step counter (word 3 N).  The writer
// stores its populations as offsets from these values and the reader adds the
// same values back: rounding c1, c2 to half only leaves a slightly larger
// remainder of h to store (half's 11 bits keep it far below the remainder of
// the equilibrium).  phi and p stay FP32: the decoded f are summed into phi
// every step, and the FP32 rounding of b_i phi_w + stored, with phi_w on the
// coarse half grid, repeats the same way every step of a steady state and
// drifts the phase field.
__device__ __forceinline__ float half_lo(uint32_t w) { return lo16<__half>(w); }
__device__ __forceinline__ float half_hi(uint32_t w) { return hi16<__half>(w); }
__device__ __forceinline__ uint32_t half_pair(float lo, float hi) {
    const __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
}
// The column of a thread, for the index of the node that population i pulled
// into (x, y) comes from (pull_src) without the general wrap and wall tests in
// rows 1 .. ny - 2.
struct PbCol {
    int x, xm, xp;  // the column and its periodic x neighbours
    bool bl, br;    // behind a left / right x wall
};
__device__ __forceinline__ PbCol pb_col(const Geometry& g, int x) {
    PbCol c;
    c.x = x;
    c.xm = x == 0 ? g.nx - 1 : x - 1;
    c.xp = x == g.nx - 1 ? 0 : x + 1;
    c.bl = g.wall_x && x == 0;
    c.br = g.wall_x && x == g.nx - 1;
    return c;
}
__device__ __forceinline__ long long pb_src(const Geometry& g, const PbCol& c, int y, int i, bool inner) {
    int sx, sy;
    if (inner) {
        const bool bb = (cx(i) == 1 && c.bl) || (cx(i) == -1 && c.br);
        sx = bb ? c.x : (cx(i) == 1 ? c.xm : (cx(i) == -1 ? c.xp : c.x));
        sy = bb ? y : y - cy(i);
    } else {
        pull_src(g, c.x, y, i, sx, sy);
    }
    return (long long)sy * (g.nxb * 32) + sx;
}

// omp = 1 - phi, passed separately so that it keeps full precision near phi = 1
// FP32 uses the hardware-approximation intrinsics (a few ulp; the parity budget
// is 1e-5), FP64 the IEEE operations.
__device__ __forceinline__ float exp_r(float v) { return __expf(v); }
__device__ __forceinline__ double exp_r(double v) { return exp(v); }
__device__ __forceinline__ float div_r(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double div_r(double a, double b) { return a / b; }
// |(x, y)|
__device__ __forceinline__ float norm_r(float x, float y) {
    const float s = x * x + y * y;
    return s > 0.0f ? s * rsqrtf(s) : 0.0f;
}
__device__ __forceinline__ double norm_r(double x, double y) { return sqrt(x * x + y * y); }

template <typename R>
__device__ __forceinline__ R mixed_diffusivity(const Coeffs<R>& C, R phi, R omp) {
    const R den = C.KD1 * omp + C.D2 * phi;  // Eq. (18)
    return den > R(0) ? div_r(C.D1D2, den) : R(0);
}

// Eq. (37): c1 = P1 + (A D_m / 2)[K c2 phi - c1 (1 - phi)], c2 symmetric.
// With a = A D_m / 2, a1 = a (1 - phi), a2 = a K phi and P = P1 + P2:
//   c1 = (P1 + a2 P) / (1 + a1 + a2),  c2 = (P2 + a1 P) / (1 + a1 + a2).
template <typename R>
__device__ __forceinline__ void solve_scalars(const Coeffs<R>& C, R phi, R omp, R P1, R P2, R& c1,
                                              R& c2) {
    const R a = C.halfA * mixed_diffusivity(C, phi, omp);
    const R a1 = a * omp, a2 = a * C.K * phi;
    const R P = P1 + P2;
    const R inv = div_r(R(1), R(1) + a1 + a2);
    c1 = (P1 + a2 * P) * inv;
    c2 = (P2 + a1 * P) * inv;
}

template <typename R>
__device__ __forceinline__ R clip01(R v) { return v < R(0) ? R(0) : (v > R(1) ? R(1) : v); }

template <typename R>
__device__ __forceinline__ R viscosity(const Coeffs<R>& C, R phi, R c1, R c2) {
    const R mu_lin = C.mu2 + C.dmu * clip01(phi);
    if (C.visc_model == 1) return exp_r(c1 * C.log_mu1 + c2 * C.log_mu2);    // Eq. (48)
    if (C.visc_model == 2) return mu_lin * exp_r(-C.visc_beta * (c1 + c2));
    return mu_lin;                                                          // Eq. (7)
}

template <typename R>
__device__ __forceinline__ bool finite5(R a, R b, R c, R d, R e) {
    return isfinite(a) && isfinite(b) && isfinite(c) && isfinite(d) && isfinite(e);
}

// Phase-field storage.  FP32 runs keep the f populations as int32 fixed point,
// F_i = (f_i - w_i / 2) * 2^31, so that their sum is Phi = (phi - 1/2) * 2^31
// (phi in (-1/2, 3/2)): phi = sum f and the stencils of phi are then exact
// integer sums, the collision only rounds the small change f* - f (to 2^-31),
// and sum(phi) is conserved bit for bit.  FP64 runs store f as double.
template <typename T>
struct PhaseFix { static constexpr bool on = false; using S = T; };
template <>
struct PhaseFix<float> { static constexpr bool on = true; using S = int; };
// 16-bit storage: f is stored as f_i - bw_i phi_w (f_dec) and handled in FP32
// once loaded
template <>
struct PhaseFix<__half> { static constexpr bool on = false; using S = float; };
template <>
struct PhaseFix<__nv_bfloat16> { static constexpr bool on = false; using S = float; };

// f_i at element offset `off` of a population buffer, in its arithmetic form
template <typename T, bool CG = false>
__device__ __forceinline__ typename PhaseFix<T>::S load_f(const T* __restrict__ src, long long off, int i) {
    if constexpr (PhaseFix<T>::on) return ld<CG>(reinterpret_cast<const int*>(src) + off);
    else if constexpr (IsHalf<T>::value) return to_r<float>(ld<CG>(src + off));  // f_i - bw_i phi_w (see f_dec)
    else return ld<CG>(src + off);
}
constexpr float FIX_ONE = 2147483648.0f;                 // 2^31
constexpr float FIX_EPS = 4.656612873077392578125e-10f;  // 2^-31
constexpr double FIX_EPS_D = 4.656612873077392578125e-10;

// Pulled f, h1, h2 of one node (f in its storage form).
__device__ __forceinline__ uint32_t word_of(int v) { return (uint32_t)v; }
__device__ __forceinline__ uint32_t word_of(float v) { return __float_as_uint(v); }
__device__ __forceinline__ void word_to(uint32_t w, int& v) { v = (int)w; }
__device__ __forceinline__ void word_to(uint32_t w, float& v) { v = __uint_as_float(w); }
template <typename T, typename R, int QS, bool PAIRED = IsHalf<T>::value>
struct NodeFH {
    typename PhaseFix<T>::S f[9];
    R h1[QS], h2[QS];
    __device__ __forceinline__ typename PhaseFix<T>::S F(int i) const { return f[i]; }
    __device__ __forceinline__ R H1(int i) const { return h1[i]; }
    __device__ __forceinline__ R H2(int i) const { return h2[i]; }
    // 32-bit words per node, and their copy to / from word k * stride of p
    // (4-byte arithmetic types only)
    static constexpr int NW = 9 + 2 * QS;
    __device__ __forceinline__ void save(uint32_t* p, int stride) const {
#pragma unroll
        for (int i = 0; i < 9; ++i) p[i * stride] = word_of(f[i]);
#pragma unroll
        for (int i = 0; i < QS; ++i) {
            p[(9 + i) * stride] = word_of(h1[i]);
            p[(9 + QS + i) * stride] = word_of(h2[i]);
        }
    }
    __device__ __forceinline__ void load(const uint32_t* p, int stride) {
#pragma unroll
        for (int i = 0; i < 9; ++i) word_to(p[i * stride], f[i]);
#pragma unroll
        for (int i = 0; i < QS; ++i) {
            word_to(p[(9 + i) * stride], h1[i]);
            word_to(p[(9 + QS + i) * stride], h2[i]);
        }
    }
};
// 16-bit storage: the pulled words as loaded, converted where used; the g
// halves ride along with f and are used one row later
template <typename T, typename R, int QS>
struct NodeFH<T, R, QS, true> {
    uint32_t fg[9];   // (f_i - bw_i phi_w, g_i - b_i(p_w)): see f_dec, p_base
    uint32_t hh[QS];  // (h1_i, h2_i)
    __device__ __forceinline__ float F(int i) const { return lo16<T>(fg[i]); }
    __device__ __forceinline__ float G(int i) const { return hi16<T>(fg[i]); }
    __device__ __forceinline__ float H1(int i) const { return lo16<T>(hh[i]); }
    __device__ __forceinline__ float H2(int i) const { return hi16<T>(hh[i]); }
    static constexpr int NW = 9 + QS;
    __device__ __forceinline__ void save(uint32_t* p, int stride) const {
#pragma unroll
        for (int i = 0; i < 9; ++i) p[i * stride] = fg[i];
#pragma unroll
        for (int i = 0; i < QS; ++i) p[(9 + i) * stride] = hh[i];
    }
    __device__ __forceinline__ void load(const uint32_t* p, int stride) {
#pragma unroll
        for (int i = 0; i < 9; ++i) fg[i] = p[i * stride];
#pragma unroll
        for (int i = 0; i < QS; ++i) hh[i] = p[(9 + i) * stride];
    }
};

// Fast pull: interior node at element offset `nd`, upstream offsets `doff`.
// ONE: one-scalar model, the h1 planes hold h3 and the h2 planes are unused.
template <int QS, typename T, typename R, bool CG = false, bool ONE = false>
__device__ __forceinline__ void pull_fh_fast(const T* __restrict__ src, long long nd,
                                             const int (&doff)[9], NodeFH<T, R, QS>& P) {
    if constexpr (IsHalf<T>::value) {
        // nd, doff in 32-bit words
        const uint32_t* sw = reinterpret_cast<const uint32_t*>(src);
#pragma unroll
        for (int i = 0; i < 9; ++i) P.fg[i] = ld<CG>(sw + nd + doff[i] + i * 32);
#pragma unroll
        for (int i = 0; i < QS; ++i) P.hh[i] = ld<CG>(sw + nd + doff[i] + (9 + i) * 32);
        return;
    } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) P.f[i] = load_f<T, CG>(src, nd + doff[i] + i * 32, i);
#pragma unroll
    for (int i = 0; i < QS; ++i) {
        P.h1[i] = to_r<R>(ld<CG>(src + nd + doff[i] + (18 + i) * 32));
        P.h2[i] = ONE ? R(0) : to_r<R>(ld<CG>(src + nd + doff[i] + (18 + QS + i) * 32));
    }
    }
}

template <int QS, typename T, typename R, bool CG = false, bool ONE = false>
__device__ __forceinline__ void pull_fh_any(const T* __restrict__ src, const Geometry& g, int x,
                                            int y, NodeFH<T, R, QS>& P) {
    constexpr int NQ = nq_of(QS);
    if constexpr (IsHalf<T>::value) {
        // whole words: bounce-back takes f and g (h1 and h2) of the same
        // opposite direction, which share a word
        const uint32_t* sw = reinterpret_cast<const uint32_t*>(src);
#pragma unroll
        for (int i = 0; i < 9; ++i) P.fg[i] = ld<CG>(sw + pull_off<NQ / 2>(g, x, y, 0, i));
#pragma unroll
        for (int i = 0; i < QS; ++i) P.hh[i] = ld<CG>(sw + pull_off<NQ / 2>(g, x, y, 9, i));
        return;
    } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        if constexpr (PhaseFix<T>::on)
            P.f[i] = pull_any<NQ, int, int, CG>(reinterpret_cast<const int*>(src), g, x, y, 0, i);
        else
            P.f[i] = load_f<T, CG>(src, pull_off<NQ>(g, x, y, 0, i), i);
    }
#pragma unroll
    for (int i = 0; i < QS; ++i) {
        P.h1[i] = pull_any<NQ, T, R, CG>(src, g, x, y, 18, i);
        P.h2[i] = ONE ? R(0) : pull_any<NQ, T, R, CG>(src, g, x, y, 18 + QS, i);
    }
    }
}

// phi in storage form (exact integer sum for fixed point) and as a number
template <typename T, typename R, int QS>
__device__ __forceinline__ typename PhaseFix<T>::S phase_sum(const NodeFH<T, R, QS>& P) {
    return ((P.F(0) + (P.F(1) + P.F(3))) + (P.F(2) + P.F(4))) + ((P.F(5) + P.F(7)) + (P.F(6) + P.F(8)));
}
// phi and 1 - phi from the stored form; in fixed point each is formed as an
// exact integer before the conversion, so phi is exact to float precision
// near 0 and 1 - phi near 1
// (32-bit integer work only: phi * 2^31 = Phi + 2^30 fits an int32 while phi < 1,
// and (1 - phi) * 2^31 = 2^30 - Phi while phi > 0; beyond those ends the other
// form is used, which is exact enough there.)
template <typename T, typename R>
__device__ __forceinline__ R phase_value(typename PhaseFix<T>::S v) {
    if constexpr (PhaseFix<T>::on)
        return v < (1 << 30) ? R(v + (1 << 30)) * R(FIX_EPS) : R(v) * R(FIX_EPS) + R(0.5);
    else return R(v);
}
template <typename T, typename R>
__device__ __forceinline__ R phase_omp(typename PhaseFix<T>::S v) {
    if constexpr (PhaseFix<T>::on)
        return v > -(1 << 30) ? R((1 << 30) - v) * R(FIX_EPS) : R(0.5) - R(v) * R(FIX_EPS);
    else return R(1) - R(v);
}
template <typename T>
__device__ __forceinline__ double phase_value_d(typename PhaseFix<T>::S v) {
    if constexpr (PhaseFix<T>::on) return double(v) * FIX_EPS_D + 0.5;
    else return double(v);
}

// One-scalar model (Eq. 31 and the relations after it), phi clipped to [0, 1]:
// K_eff = K phi + (1 - phi); c split between the phases at the Henry
// equilibrium, c1 = K phi c / K_eff, c2 = (1 - phi) c / K_eff.
template <typename R>
__device__ __forceinline__ void henry_split(const Coeffs<R>& C, R phi, R c, R& c1, R& c2) {
    const R ph = phi < R(0) ? R(0) : (phi > R(1) ? R(1) : phi);
    const R inv = div_r(c, C.K * ph + (R(1) - ph));
    c1 = C.K * ph * inv;
    c2 = (R(1) - ph) * inv;
}

template <typename T, typename R, int QS, bool ONE = false>
__device__ __forceinline__ void zeroth(const Coeffs<R>& C, const NodeFH<T, R, QS>& P,
                                       typename PhaseFix<T>::S& phis, R& phi, R& c1, R& c2) {
    phis = phase_sum<T, R, QS>(P);
    phi = phase_value<T, R>(phis);
    const R omp = phase_omp<T, R>(phis);
    R P1 = R(0), P2 = R(0);
#pragma unroll
    for (int i = 0; i < QS; ++i) {
        P1 += P.H1(i);
        P2 += P.H2(i);
    }
    if constexpr (ONE) henry_split(C, phi, P1, c1, c2);  // c = sum_i h3_i
    else solve_scalars(C, phi, omp, P1, P2, c1, c2);
}

// The same for 16-bit storage, the stored f decoded with the phase fields phs
// of the nodes they were pulled from (f_dec), summed in phase_sum's order; the
// stored h decoded by adding cb1 = sum_i bq_i c1_w,i and cb2 (the writers' c).
template <typename T, typename R, int QS, bool ONE = false>
__device__ __forceinline__ void zeroth_b(const Coeffs<R>& C, const NodeFH<T, R, QS>& P, const float (&phs)[9],
                                         float cb1, float cb2, float& phis, R& phi, R& c1, R& c2) {
    float f[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = f_dec(P.F(i), i, phs[i]);
    phis = ((f[0] + (f[1] + f[3])) + (f[2] + f[4])) + ((f[5] + f[7]) + (f[6] + f[8]));
    phi = R(phis);
    const R omp = R(1) - R(phis);
    R P1 = R(0), P2 = R(0);
#pragma unroll
    for (int i = 0; i < QS; ++i) {
        P1 += P.H1(i);
        P2 += P.H2(i);
    }
    P1 += R(cb1);
    P2 += R(cb2);
    if constexpr (ONE) henry_split(C, phi, P1, c1, c2);
    else solve_scalars(C, phi, omp, P1, P2, c1, c2);
}

// D2Q9 stencils of phi at the ring centre column X (Eqs. 41-42).  Fixed-point
// phi: the differences and the Laplacian's sums are exact integers, converted
// once; the cubic of Eq. (4) gets the low bits of phi through its derivative.
template <typename T, typename R>
struct PhiStencil {
    R phi, omp, dx, dy, lap, bulk;  // omp = 1 - phi, bulk = phi (phi - 1)(phi - 1/2)
};

template <typename T, typename R, int W2>
__device__ __forceinline__ PhiStencil<T, R> phi_stencil(const typename PhaseFix<T>::S (*rs),
                                                        const typename PhaseFix<T>::S (*r0),
                                                        const typename PhaseFix<T>::S (*rn), int X) {
    PhiStencil<T, R> o;
    if constexpr (PhaseFix<T>::on) {
        const int c = r0[X];
        const int e = r0[X + 1] - c, w = r0[X - 1] - c, n = rn[X] - c, s = rs[X] - c;
        const int ne = rn[X + 1] - c, nw = rn[X - 1] - c, sw = rs[X - 1] - c, se = rs[X + 1] - c;
        o.dx = R(e - w) * R(FIX_EPS / 3.0f) + R((ne - nw) + (se - sw)) * R(FIX_EPS / 12.0f);
        o.dy = R(n - s) * R(FIX_EPS / 3.0f) + R((ne - se) + (nw - sw)) * R(FIX_EPS / 12.0f);
        // second differences: exact in int32 for any state whose node-to-node
        // change of phi is below 1/4 (a tanh profile of width W = 4 stays below 1/4)
        const int ax = (e + w) + (n + s), dg = (ne + nw) + (sw + se);
        o.lap = R(ax) * R(FIX_EPS * (2.0f / 3.0f)) + R(dg) * R(FIX_EPS / 6.0f);
        // phi, 1 - phi and phi - 1/2 = c 2^-31 are each exact to float precision
        // where they are small, so the cubic as their product has no cancellation
        o.phi = phase_value<T, R>(c);
        o.omp = phase_omp<T, R>(c);
        o.bulk = -(o.phi * o.omp) * (R(c) * R(FIX_EPS));
    } else {
        const R c = r0[X];
        const R e = r0[X + 1] - c, w = r0[X - 1] - c, n = rn[X] - c, s = rs[X] - c;
        const R ne = rn[X + 1] - c, nw = rn[X - 1] - c, sw = rs[X - 1] - c, se = rs[X + 1] - c;
        o.dx = (e - w) * R(1.0 / 3.0) + ((ne - nw) + (se - sw)) * R(1.0 / 12.0);
        o.dy = (n - s) * R(1.0 / 3.0) + ((ne - se) + (nw - sw)) * R(1.0 / 12.0);
        o.lap = ((e + w) + (n + s)) * R(2.0 / 3.0) + ((ne + nw) + (sw + se)) * R(1.0 / 6.0);
        o.phi = c;
        o.omp = R(1) - c;
        o.bulk = c * (c - R(1)) * (c - R(0.5));
    }
    return o;
}

// Post-collision f of one node: f*_i = (1 - w_f) f_i + w_i (w_f phi + c_i . B)
// (Eqs. 23-25 with f^eq and F_i gathered).  The rest population takes
// phi - sum_{i>0} f*_i, so sum f* = phi exactly.
template <typename T, typename R>
__device__ __forceinline__ void collide_f(T* __restrict__ o, const typename PhaseFix<T>::S (&f)[9],
                                          typename PhaseFix<T>::S phis, R phi, R omega, R Bx, R By) {
    if constexpr (PhaseFix<T>::on) {
        // f*_i - f_i = w_f (w_i phi - f_i) + w_i c_i . B.  In the offset encoding
        // w_i phi - f_i = w_i Phi - F_i (the w_i / 2 offsets cancel); Phi - 9 F_i
        // (or Phi - 36 F_i) is the small non-equilibrium part, exact in int32,
        // and is divided by 9 (36) only after the conversion
        int* oi = reinterpret_cast<int*>(o);
        const R sc9 = omega * R(FIX_EPS / 9.0f), sc36 = omega * R(FIX_EPS / 36.0f);
        int sum = 0;
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const R neq = i <= 4 ? sc9 * R(phis - 9 * f[i]) : sc36 * R(phis - 36 * f[i]);
            const R cB = (cx(i) ? R(cx(i)) * Bx : R(0)) + (cy(i) ? R(cy(i)) * By : R(0));
            const R d = neq + w9<R>(i) * cB;
            const int v = f[i] + __float2int_rn(d * R(FIX_ONE));
            sum += v;
            stcs(oi + i * 32, v);
        }
        stcs(oi, phis - sum);
    } else {
        const R a0 = omega * phi, keep = R(1) - omega;
        R sum = R(0);
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const R cB = (cx(i) ? R(cx(i)) * Bx : R(0)) + (cy(i) ? R(cy(i)) * By : R(0));
            const T vs = keep * R(f[i]) + w9<R>(i) * (a0 + cB);
            sum += vs;
            stcs(o + i * 32, vs);
        }
        stcs(o, phi - sum);
    }
}
// The same for 16-bit storage: fd are the pulled f decoded with their writers'
// phase fields (f_dec); the forms to store, f*_i - bw_i phi (phi: this node's,
// written beside them), go to fv[1..8] unrounded: each is rounded
// stochastically together with g*_i, the other half of its word.  With
// f*_i - bw_i phi = (1 - w_f)(f_i - bw_i phi) + w_f (w_i - bw_i) phi + w_i c_i.B,
// and the rest population taking what the moving ones leave of phi, its stored
// form is minus the sum of the rounded moving ones (the bw_i sum to 1).
template <typename R>
__device__ __forceinline__ void collide_f16(float (&fv)[9], const float (&fd)[9], R phi, R omega, R Bx, R By) {
    const R keep = R(1) - omega;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const R cB = (cx(i) ? R(cx(i)) * Bx : R(0)) + (cy(i) ? R(cy(i)) * By : R(0));
        const R d = R(fd[i]) - bw9<R>(i) * phi;
        const R dw = R(w9<double>(i) - bw9<double>(i));  // folded: i is unrolled
        fv[i] = float(keep * d + w9<R>(i) * cB + (dw * omega) * phi);
    }
}

// One tile of the fused step (FIELDS = false) or of the macroscopic-field
// evaluation of the current state (FIELDS = true): the W columns x0 .. x0+W-1
// (one thread each) of rows ya .. yb-1, marched upwards.  CG selects the load
// path (see ld).  The caller's block has exactly W threads.
// VAR: model variant, bit 0 = one-scalar model, bits 1-2 = gradient scheme
// (0: stencils of Eq. 41; 1: local grad c1, grad c2 of Eq. 39; 2: also the local
// grad phi).  VAR = 0 is the paper's default configuration.
template <typename T, typename R, int QS, bool FIELDS, int W, bool CG, int VAR = 0>
__device__ __forceinline__ void strip_tile(const T* __restrict__ src, T* __restrict__ dst,
                                           R* __restrict__ prev, const Geometry& g, const Coeffs<R>& C,
                                           unsigned* __restrict__ flag, uint32_t mask,
                                           void* __restrict__ out, int out_f64, int x0, int ya,
                                           int yb) {
    constexpr int NQ = nq_of(QS);
    // 16-bit storage is addressed in 32-bit words (two populations each)
    constexpr bool PAIRED = IsHalf<T>::value;
    constexpr int NQL = PAIRED ? NQ / 2 : NQ;
    constexpr int W2 = W + 2;
    constexpr bool ONE = (VAR & 1) != 0;
    constexpr int GS = VAR >> 1;
    using PS = typename PhaseFix<T>::S;
    __shared__ PS s_phi[4][W2];
    __shared__ R s_c[4][2][W2];
    // With 4-byte arithmetic the pulled f, h (and g) of a row wait for their
    // collision, one row later, in shared memory rather than in registers: the
    // row of look-ahead would otherwise hold them live through the next row's
    // loads and push the kernel into spilling, and spilled values, in local
    // memory, are evicted from L1 by the streaming loads.  Each thread reads
    // back only its own words.
    constexpr bool CUR_SMEM = sizeof(R) == 4;
    constexpr int NWC = CUR_SMEM ? NodeFH<T, R, QS>::NW : 1;
    __shared__ uint32_t s_cur[2][NWC * W];

    dbg_begin(g.ws_lo, g.ws_hi);  // debug build: the range every global access is checked against
    const int tid = threadIdx.x, lane = tid & 31;
    const int x = x0 + tid;
    const bool col_in = x < g.nx;
    const int rx = col_in ? x : resolve(x, g.nx, g.wall_x);
    // Halo columns: lane 0 (tid 0) takes the right one, x0 + W, and lane 31
    // (tid W - 1) the left one, x0 - 1 (resolved: periodic image or wall ghost).
    const bool halo = tid == 0 || tid == W - 1;
    const int hx = resolve(tid == 0 ? x0 + W : x0 - 1, g.nx, g.wall_x);
    const int hcol = tid == 0 ? W + 1 : 0;

    // Upstream offsets (element or word units, relative to the node) of the
    // nodes of column cxn in rows 1 .. ny-2, the periodic image folded into the
    // x neighbours; behind an x wall (bl: left, br: right) the node's own
    // population of the opposite direction (half-way bounce-back).  The x
    // boundary columns then take the same branch-free pull as the interior, and
    // only rows 0 and ny-1 need pull_fh_any.
    const int row = g.nxb * NQL * 32;
    auto column_offsets = [&](int cxn, int (&d)[9]) {
        const int xmn = cxn == 0 ? g.nx - 1 : cxn - 1, xpn = cxn == g.nx - 1 ? 0 : cxn + 1;
        const int xm = ((xmn >> 5) - (cxn >> 5)) * (NQL * 32) + ((xmn & 31) - (cxn & 31));
        const int xp = ((xpn >> 5) - (cxn >> 5)) * (NQL * 32) + ((xpn & 31) - (cxn & 31));
        const bool bl = g.wall_x && cxn == 0, br = g.wall_x && cxn == g.nx - 1;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int std = -cy(i) * row + (cx(i) == 1 ? xm : (cx(i) == -1 ? xp : 0));
            const bool bb = (cx(i) == 1 && bl) || (cx(i) == -1 && br);
            d[i] = bb ? (opp(i) - i) * 32 : std;
        }
    };
    int doff[9];
    column_offsets(rx, doff);
    const int pb_row = g.nxb * 32;  // nodes per row of the writers' bases planes
    // 16-bit storage: the (c1, c2) half pairs of the writers' bases
    const uint32_t* pb_c = PAIRED ? reinterpret_cast<const uint32_t*>(g.pb_in + 2LL * g.ny * pb_row) : nullptr;
    // 16-bit storage: the step counter kept after the last node of the bases
    // plane (read from the input plane, written incremented to the output one
    // by the first CTA of a step launch); it seeds the stochastic rounding, so
    // that a value that stays the same from step to step is not rounded the
    // same way every step
    uint32_t tstep = 0;
    if constexpr (PAIRED) {
        const long long cnt = 3LL * g.ny * pb_row;  // in 4-byte words
        tstep = ld<CG>(reinterpret_cast<const uint32_t*>(g.pb_in) + cnt);
        if (!FIELDS && x0 == 0 && ya == 0 && tid == 0) st_chk(reinterpret_cast<uint32_t*>(g.pb_out) + cnt, tstep + 1u);
    }
    __shared__ int s_hoff[2][9];  // the halo nodes' offsets
    if (halo) {
        int hd[9];
        column_offsets(hx, hd);
#pragma unroll
        for (int i = 0; i < 9; ++i) s_hoff[tid == 0 ? 0 : 1][i] = hd[i];
    }
    // Halo nodes with at least two warps: the warp of each halo thread (the
    // first warp: right halo; the last: left halo) loads the halo node's words
    // one per lane, beside the lanes' own loads, and the halo thread sums them
    // from shared memory in the same order as any node's; it then waits for one
    // memory round trip per row instead of two.  16-bit storage adds the halo
    // node's writers' bases (9 phase fields, QS (c1, c2) words): 28 words with
    // the D2Q5 scalars, one per lane.
    constexpr int NHW = PAIRED ? NWC + 9 + QS : NWC;  // words loaded for a halo node
    constexpr bool HALO_SPLIT = CUR_SMEM && W >= 64 && NHW <= 32;
    const int wid = tid >> 5;
    const bool hwarp = wid == 0 || wid == W / 32 - 1;
    const int hkw = wid == 0 ? 0 : 1;
    const int hxw = resolve(wid == 0 ? x0 + W : x0 - 1, g.nx, g.wall_x);
    __shared__ uint32_t s_hpop[2][HALO_SPLIT ? NHW : 1];
    int hoffk = 0;       // this lane's word of the halo node, relative to the node
    bool hload = false;  // whether this lane loads one
    if constexpr (HALO_SPLIT) {
        __syncthreads();  // s_hoff
        const int k = lane;
        if (hwarp && k < NWC) {
            int dir, plane;
            if constexpr (PAIRED) {
                dir = k < 9 ? k : k - 9;
                plane = k;
            } else {
                dir = k < 9 ? k : (k < 9 + QS ? k - 9 : k - 9 - QS);
                plane = k < 9 ? k : (k < 9 + QS ? 18 + (k - 9) : 18 + QS + (k - 9 - QS));
            }
            hoffk = s_hoff[hkw][dir] + plane * 32;
            hload = !(ONE && !PAIRED && k >= 9 + QS);  // one-scalar model: no h2
        }
        if (PAIRED && hwarp && k >= NWC && k < NHW) {
            // a base of the writer of direction i of the halo node: its index in
            // the bases planes relative to the row's first node (rows 1 .. ny - 2)
            const int i = k < NWC + 9 ? k - NWC : k - NWC - 9;
            hoffk = (int)pb_src(g, pb_col(g, hxw), 0, i, true);
            hload = true;
        }
    }

    // 16-bit storage: the writers' bases of the pulled populations: phase fields
    // phs of the writers of f, and sum_i bq_i c_k,w,i of the writers of h.  Off
    // the x boundary columns and the first and last rows the writers are the
    // 3 x 3 neighbourhood: one row pointer and constant offsets.
    auto writer_bases = [&](const PbCol& pc, int ry, bool y_in, float (&phs)[9], float& cb1, float& cb2) {
        cb1 = 0.0f;
        cb2 = 0.0f;
        auto take = [&](int i, long long k) {
            phs[i] = ld<CG>(g.pb_in + 2 * k + 1);
            if (i < QS) {
                const uint32_t cw = ld<CG>(pb_c + k);
                cb1 = fmaf(bwq<float, QS>(i), half_lo(cw), cb1);
                cb2 = fmaf(bwq<float, QS>(i), half_hi(cw), cb2);
            }
        };
        if (y_in && pc.x >= 1 && pc.x <= g.nx - 2) {
            const long long c = (long long)ry * pb_row + pc.x;
#pragma unroll
            for (int i = 0; i < 9; ++i) take(i, c + (-cy(i) * pb_row - cx(i)));
        } else {
#pragma unroll
            for (int i = 0; i < 9; ++i) take(i, pb_src(g, pc, ry, i, y_in));
        }
    };
    const PbCol pcol = pb_col(g, rx);
    const PbCol hcolp = pb_col(g, hx);

    // zeroth moments of row yy into ring slot yy & 3; the pulled pops go to P
    auto moments_row = [&](int yy, NodeFH<T, R, QS>& P) {
        const int ry = resolve(yy, g.ny, g.wall_y);
        const bool y_in = ry >= 1 && ry <= g.ny - 2;
        PS phis;
        R phi, c1, c2;
        uint32_t hv = 0;
        float phs[9], cb1, cb2;
        if (y_in) {
            pull_fh_fast<QS, T, R, CG, ONE>(src, node_off<NQL>(g, rx, ry), doff, P);
            if constexpr (HALO_SPLIT) {
                if (hload) {
                    if (lane < NWC) {
                        hv = ld<CG>(reinterpret_cast<const uint32_t*>(src) + node_off<NQL>(g, hxw, ry) + hoffk);
                    } else if constexpr (PAIRED) {
                        // writer of direction i of the halo node: its phase field, then its (c1, c2)
                        const long long k = (long long)ry * pb_row + hoffk;
                        hv = lane < NWC + 9 ? __float_as_uint(ld<CG>(g.pb_in + 2 * k + 1)) : ld<CG>(pb_c + k);
                    }
                }
            }
        } else {
            pull_fh_any<QS, T, R, CG, ONE>(src, g, rx, ry, P);
        }
        if constexpr (PAIRED) {
            writer_bases(pcol, ry, y_in, phs, cb1, cb2);
            zeroth_b<T, R, QS, ONE>(C, P, phs, cb1, cb2, phis, phi, c1, c2);
        } else {
            zeroth<T, R, QS, ONE>(C, P, phis, phi, c1, c2);
        }
        if constexpr (CUR_SMEM) P.save(&s_cur[yy & 1][tid], W);
        s_phi[yy & 3][tid + 1] = phis;
        s_c[yy & 3][0][tid + 1] = c1;
        s_c[yy & 3][1][tid + 1] = c2;
        if constexpr (HALO_SPLIT) {
            if (hwarp && y_in) {
                __syncwarp();  // the halo thread has read the previous row's words
                if (lane < NHW) s_hpop[hkw][lane] = hv;
                __syncwarp();
                if (halo) {
                    NodeFH<T, R, QS> hp;
                    hp.load(s_hpop[hkw], 1);
                    PS hs;
                    R a, b, c;
                    if constexpr (PAIRED) {
                        // the bases in writer_bases' order
                        float hphs[9], hc1 = 0.0f, hc2 = 0.0f;
#pragma unroll
                        for (int i = 0; i < 9; ++i) hphs[i] = __uint_as_float(s_hpop[hkw][NWC + i]);
#pragma unroll
                        for (int i = 0; i < QS; ++i) {
                            const uint32_t cw = s_hpop[hkw][NWC + 9 + i];
                            hc1 = fmaf(bwq<float, QS>(i), half_lo(cw), hc1);
                            hc2 = fmaf(bwq<float, QS>(i), half_hi(cw), hc2);
                        }
                        zeroth_b<T, R, QS, ONE>(C, hp, hphs, hc1, hc2, hs, a, b, c);
                    } else {
                        zeroth<T, R, QS, ONE>(C, hp, hs, a, b, c);
                    }
                    s_phi[yy & 3][hcol] = hs;
                    s_c[yy & 3][0][hcol] = b;
                    s_c[yy & 3][1][hcol] = c;
                }
                return;
            }
        }
        if (halo) {
            NodeFH<T, R, QS> hp;
            PS hs;
            R a, b, c;
            if (y_in)
                pull_fh_fast<QS, T, R, CG, ONE>(src, node_off<NQL>(g, hx, ry), s_hoff[tid == 0 ? 0 : 1], hp);
            else
                pull_fh_any<QS, T, R, CG, ONE>(src, g, hx, ry, hp);
            if constexpr (PAIRED) {
                writer_bases(hcolp, ry, y_in, phs, cb1, cb2);
                zeroth_b<T, R, QS, ONE>(C, hp, phs, cb1, cb2, hs, a, b, c);
            } else {
                zeroth<T, R, QS, ONE>(C, hp, hs, a, b, c);
            }
            s_phi[yy & 3][hcol] = hs;
            s_c[yy & 3][0][hcol] = b;
            s_c[yy & 3][1][hcol] = c;
        }
    };

    NodeFH<T, R, QS> cur;
    moments_row(ya - 1, cur);
    moments_row(ya, cur);

    for (int y = ya; y < yb; ++y) {
        const bool inner = y >= 1 && y <= g.ny - 2;
        const long long nd = node_off<NQL>(g, x, y);
        // ---- a. loads of row y: g (pulled) and the previous-step macros ----
        R gp[9], pv[5];
        // 16-bit storage: the pulled f and h, decoded with their writers' bases
        float fd[PAIRED ? 9 : 1], h1d[PAIRED ? QS : 1], h2d[PAIRED ? QS : 1];
        if (col_in) {
            if constexpr (PAIRED) {
                // decoded after the row barrier below: held from here through the
                // look-ahead row they pushed the kernel into spilling
            } else if (inner) {
#pragma unroll
                for (int i = 0; i < 9; ++i) gp[i] = g_value<T>(to_r<R>(ld<CG>(src + nd + doff[i] + (9 + i) * 32)));
            } else {
#pragma unroll
                for (int i = 0; i < 9; ++i) gp[i] = g_value<T>(pull_any<NQ, T, R, CG>(src, g, x, y, 9, i));
            }
            if constexpr (!FIELDS || GS == 2) {
                const R* pp = prev + node_off<5>(g, x, y);
#pragma unroll
                for (int k = 0; k < 5; ++k) pv[k] = CG ? ld<true>(pp + k * 32) : ld_plain(pp + k * 32);
            }
        }
        // ---- b. zeroth moments of row y+1 (f, h1, h2 pulled once per node) ----
        NodeFH<T, R, QS> nxt;
        moments_row(y + 1, nxt);
        __syncthreads();
        if constexpr (CUR_SMEM) cur.load(&s_cur[y & 1][tid], W);

        if (col_in) {
            if constexpr (PAIRED) {
                // g pulled with f one row ago (this thread's words of the shared
                // slot, which the look-ahead row does not touch), stored relative
                // to the writer's pressure part (p_base), added back here with the
                // writer's p; the writer's phi decodes f in the collision
                // (and h stored relative to the writer's c1, c2, decoded here)
                const float2* pb2 = reinterpret_cast<const float2*>(g.pb_in);
                auto take = [&](int i, long long k) {
                    const float2 w = ld<CG>(pb2 + k);
                    if (i < QS) {
                        const uint32_t cw = ld<CG>(pb_c + k);
                        h1d[i] = fmaf(bwq<float, QS>(i), half_lo(cw), cur.H1(i));
                        h2d[i] = fmaf(bwq<float, QS>(i), half_hi(cw), cur.H2(i));
                    }
                    fd[i] = f_dec(cur.F(i), i, w.y);
                    gp[i] = g_value<T>(R(cur.G(i))) + p_base<R>(i, R(w.x));
                };
                if (inner && x >= 1 && x <= g.nx - 2) {
                    const long long c = (long long)y * pb_row + x;
#pragma unroll
                    for (int i = 0; i < 9; ++i) take(i, c + (-cy(i) * pb_row - cx(i)));
                } else {
#pragma unroll
                    for (int i = 0; i < 9; ++i) take(i, pb_src(g, pcol, y, i, inner));
                }
            }
            // ---- c. stencils (Eqs. 41-42, D2Q9 weights) from the shared ring ----
            const int X = tid + 1;
            const PhiStencil<T, R> st = phi_stencil<T, R, W2>(s_phi[(y - 1) & 3], s_phi[y & 3],
                                                              s_phi[(y + 1) & 3], X);
            const R phi = st.phi, omp = st.omp, lap = st.lap;
            R dphix = st.dx, dphiy = st.dy;
            if constexpr (GS == 2) {
                // local grad phi (the scheme after Eq. 39): C = sum_i c_i f_i - (phi +
                // phi_prev) u_prev / 2 (the previous step's velocity: u needs the
                // surface force, which needs grad phi), B = 4 M phi (1 - phi) / W,
                // grad phi = -C (|C| + B) / (tau_f cs^2 |C|) = -3 w_f C (|C| + B) / |C|
                R mx, my;
                if constexpr (PhaseFix<T>::on) {
                    // fixed point: the w_i / 2 offsets cancel in the first moment
                    const int ix = (cur.f[1] - cur.f[3]) + ((cur.f[5] - cur.f[7]) + (cur.f[8] - cur.f[6]));
                    const int iy = (cur.f[2] - cur.f[4]) + ((cur.f[5] - cur.f[7]) + (cur.f[6] - cur.f[8]));
                    mx = R(ix) * R(FIX_EPS);
                    my = R(iy) * R(FIX_EPS);
                } else {
                    mx = (R(cur.f[1]) - R(cur.f[3])) + ((R(cur.f[5]) - R(cur.f[7])) + (R(cur.f[8]) - R(cur.f[6])));
                    my = (R(cur.f[2]) - R(cur.f[4])) + ((R(cur.f[5]) - R(cur.f[7])) + (R(cur.f[6]) - R(cur.f[8])));
                }
                const R hp = R(0.5) * (phi + pv[0]);
                const R Cx = mx - hp * pv[1], Cy = my - hp * pv[2];
                const R Cn = norm_r(Cx, Cy);
                const R B = C.M * C.four_over_W * phi * omp;
                const R a = Cn > R(0) ? -R(3) * C.omega_f * div_r(Cn + B, Cn) : R(0);
                dphix = a * Cx;
                dphiy = a * Cy;
            }
            const R(*rs)[W2] = s_c[(y - 1) & 3];
            const R(*r0)[W2] = s_c[y & 3];
            const R(*rn)[W2] = s_c[(y + 1) & 3];
            const R c1 = r0[0][X], c2 = r0[1][X];
            R dc1x, dc1y, dc2x, dc2y;
            {
                const R e = r0[0][X + 1], w = r0[0][X - 1], n = rn[0][X], s = rs[0][X];
                const R ne = rn[0][X + 1], nw = rn[0][X - 1], sw = rs[0][X - 1], se = rs[0][X + 1];
                dc1x = (e - w) * R(1.0 / 3.0) + ((ne - nw) + (se - sw)) * R(1.0 / 12.0);
                dc1y = (n - s) * R(1.0 / 3.0) + ((ne - se) + (nw - sw)) * R(1.0 / 12.0);
            }
            {
                const R e = r0[1][X + 1], w = r0[1][X - 1], n = rn[1][X], s = rs[1][X];
                const R ne = rn[1][X + 1], nw = rn[1][X - 1], sw = rs[1][X - 1], se = rs[1][X + 1];
                dc2x = (e - w) * R(1.0 / 3.0) + ((ne - nw) + (se - sw)) * R(1.0 / 12.0);
                dc2y = (n - s) * R(1.0 / 3.0) + ((ne - se) + (nw - sw)) * R(1.0 / 12.0);
            }

            // ---- d. flow macros ----
            const R phic = clip01(phi);
            const R rho = C.rho2 + C.drho * phic;                                   // Eq. (6)
            const R mu_phi = C.beta4 * st.bulk - C.kappa * lap;                     // Eq. (4)
            const R Fx = mu_phi * dphix + ((rho - C.g_rho_ref) * C.gx + C.Fx);     // F_s + G
            const R Fy = mu_phi * dphiy + ((rho - C.g_rho_ref) * C.gy + C.Fy);
            const R jx = (gp[1] - gp[3]) + ((gp[5] - gp[7]) + (gp[8] - gp[6]));
            const R jy = (gp[2] - gp[4]) + ((gp[5] - gp[7]) + (gp[6] - gp[8]));
            const R gs = ((gp[1] + gp[3]) + (gp[2] + gp[4])) + ((gp[5] + gp[7]) + (gp[6] + gp[8]));
            const R inv_rho = div_r(R(1), rho);
            const R ux = (jx + R(0.5) * Fx) * inv_rho;                              // Eq. (32a)
            const R uy = (jy + R(0.5) * Fy) * inv_rho;
            const R uu = ux * ux + uy * uy;
            // Eq. (32b): cs^2/(1-w0) = 3/5, s_0(u) = -w0 u.u/(2 cs^2) = -(2/3) u.u
            const R p = three_fifths(gs + R(0.5) * C.drho * (ux * dphix + uy * dphiy) - R(2.0 / 3.0) * rho * uu);
            const R mu = viscosity<R>(C, phi, c1, c2);

            if constexpr (FIELDS) {
                const size_t o = (size_t)y * g.nx + x, nn = (size_t)g.nx * g.ny;
                const R vals[8] = {phi, ux, uy, p, c1, c2, rho, mu};
                int j = 0;
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    if (mask & (1u << b)) {
                        if (b == 0) {  // phi exactly as stored
                            const double v = phase_value_d<T>(s_phi[y & 3][X]);
                            if (out_f64) static_cast<double*>(out)[j * nn + o] = v;
                            else static_cast<float*>(out)[j * nn + o] = float(v);
                        } else if (out_f64) {
                            static_cast<double*>(out)[j * nn + o] = double(vals[b]);
                        } else {
                            static_cast<float*>(out)[j * nn + o] = float(vals[b]);
                        }
                        ++j;
                    }
                }
            } else {
                const R omega_g = div_r(R(1), R(3) * mu * inv_rho + R(0.5));  // Eq. (33): 1/tau_g
                const R force_g = R(1) - R(0.5) * omega_g;

                // backward differences against the previous step's macros
                const R dpux = phi * ux - pv[0] * pv[1], dpuy = phi * uy - pv[0] * pv[2];
                const R d1ux = c1 * ux - pv[3] * pv[1], d1uy = c1 * uy - pv[3] * pv[2];
                const R d2ux = c2 * ux - pv[4] * pv[1], d2uy = c2 * uy - pv[4] * pv[2];
                {
                    // one-scalar model: the c1 slot holds c = c1 + c2, the c2 slot 0
                    R* pp = prev + node_off<5>(g, x, y);
                    st_chk(pp, phi);
                    st_chk(pp + 32, ux);
                    st_chk(pp + 64, uy);
                    st_chk(pp + 96, ONE ? c1 + c2 : c1);
                    st_chk(pp + 128, ONE ? R(0) : c2);
                }
                // non-finite values, or phi outside the fixed-point range
                // (16-bit storage also checks p: rounding a NaN population can lose
                // it, and g_0 reaches no other macro)
                if (!finite5(phi, ux, uy, c1, c2) || !(phi > R(-1.5) && phi < R(1.5)) ||
                    (IsHalf<T>::value && !isfinite(p)))
                    atomicOr(flag, 1u);

                // unit normal (Eq. 1), regularised
                const R inv_norm = div_r(R(1), norm_r(dphix, dphiy) + R(1e-4));
                const R nxv = dphix * inv_norm, nyv = dphiy * inv_norm;
                T* o = dst + nd;
                uint32_t* ow = reinterpret_cast<uint32_t*>(dst) + nd;  // 16-bit storage
                // stochastic-rounding seed of this node and step (16-bit storage only)
                const uint32_t key =
                    IsHalf<T>::value ? mix32(((uint32_t)y * 0x01000193u + (uint32_t)x) ^ __float_as_uint(float(p)) ^
                                             (__float_as_uint(float(ux)) * 0x2545f491u) ^ (tstep * 0x9e3779b1u))
                                     : 0u;

                // ---- e1. f (Eqs. 23-25) ----
                // 16-bit storage: this node's bases, written beside its populations,
                // which are stored relative to them: p, phi in FP32, c1, c2 rounded
                // to half
                uint32_t cbase = 0u;
                R c1r = R(0), c2r = R(0);
                if constexpr (PAIRED) {
                    cbase = half_pair(float(c1), float(c2));
                    c1r = R(half_lo(cbase));
                    c2r = R(half_hi(cbase));
                }
                float fv[9];  // 16-bit storage: f* to store, rounded with g*
                {
                    const R sharp = C.force_f * C.four_over_W * phi * omp;
                    const R Bx = (R(3) * (C.omega_f * phi * ux + C.force_f * dpux) + sharp * nxv);
                    const R By = (R(3) * (C.omega_f * phi * uy + C.force_f * dpuy) + sharp * nyv);
                    if constexpr (PAIRED) collide_f16<R>(fv, fd, phi, C.omega_f, Bx, By);
                    else collide_f<T, R>(o, cur.f, s_phi[y & 3][X], phi, C.omega_f, Bx, By);
                }
                // ---- e2. g (Eqs. 28-31) ----
                {
                    const R alpha = omega_g * (R(3) * p - R(1.5) * rho * uu);
                    const R Vx = R(3) * (omega_g * rho * ux + force_g * Fx);
                    const R Vy = R(3) * (omega_g * rho * uy + force_g * Fy);
                    const R gam = R(4.5) * omega_g * rho;
                    const R del = R(3) * force_g * C.drho;
                    const R keep = R(1) - omega_g;
                    float fsum = 0.0f;  // 16-bit storage: the rounded stored f*_1..8
                    // moving populations first: with 16-bit storage the rest f* is
                    // minus the sum of the rounded moving ones
#pragma unroll
                    for (int k = 0; k < 9; ++k) {
                        const int i = PAIRED ? (k + 1) % 9 : k;
                        const R cu = (cx(i) ? R(cx(i)) * ux : R(0)) + (cy(i) ? R(cy(i)) * uy : R(0));
                        const R cg = (cx(i) ? R(cx(i)) * dphix : R(0)) + (cy(i) ? R(cy(i)) * dphiy : R(0));
                        const R cV = (cx(i) ? R(cx(i)) * Vx : R(0)) + (cy(i) ? R(cy(i)) * Vy : R(0));
                        R v = keep * gp[i] + w9_times(i, alpha + cV + cu * (gam * cu + del * cg));
                        if (i == 0) v -= R(3) * omega_g * p;
                        if constexpr (PAIRED) {
                            v -= p_base<R>(i, p);
                            const float fo = i == 0 ? -fsum : fv[i];
                            const uint32_t wv = round_pair<T>(fo, float(g_stored<T>(v)), sr_word(key, fo, i));
                            if (i != 0) fsum += lo16<T>(wv);
                            stcs(ow + i * 32, wv);
                        } else {
                            stcs(o + (9 + i) * 32, store_value<T>(v));
                        }
                    }
                }
                if constexpr (PAIRED) {
                    const long long k = (long long)y * pb_row + x;
                    st_chk(reinterpret_cast<float2*>(g.pb_out) + k, make_float2(float(p), float(phi)));
                    st_chk(reinterpret_cast<uint32_t*>(g.pb_out + 2LL * g.ny * pb_row) + k, cbase);
                }
                // ---- e3. h1, h2 (Eqs. 34-36) ----
                if constexpr (ONE) {
                    // ---- e3'. h3: one-scalar model (Sec. III D) ----
                    // h3*_i = h3_i - w3 (h3_i - h3_i^eq) + (1 - w3/2) H3_i with
                    // tau_h3 = D_eff / cs^2 + 1/2 per node; the rest population takes
                    // what the moving ones leave of c = sum_i h3_i (exact conservation)
                    R P1 = R(0), s1 = R(0);
#pragma unroll
                    for (int i = 0; i < QS; ++i) P1 += cur.H1(i);
                    const R ph = phi < R(0) ? R(0) : (phi > R(1) ? R(1) : phi);
                    const R omp_c = R(1) - ph;
                    const R w3 = div_r(R(1), R(3) * (C.KD1 * ph + C.D2 * omp_c) + R(0.5));
                    const R f3 = R(1) - R(0.5) * w3;
                    const R a3 = w3 * div_r(P1, C.K * ph + omp_c);
                    const R dcux = P1 * ux - pv[3] * pv[1], dcuy = P1 * uy - pv[3] * pv[2];
                    const R B3x = R(3) * (w3 * P1 * ux + f3 * dcux), B3y = R(3) * (w3 * P1 * uy + f3 * dcuy);
                    const R k3 = R(1) - w3;
#pragma unroll
                    for (int i = 1; i < QS; ++i) {
                        const R w = wq<R, QS>(i);
                        const R cB = (cx(i) ? R(cx(i)) * B3x : R(0)) + (cy(i) ? R(cy(i)) * B3y : R(0));
                        const T v = store_value<T>(k3 * cur.H1(i) + w * (a3 + cB));
                        s1 += to_r<R>(v);
                        stcs(o + (18 + i) * 32, v);
                    }
                    stcs(o + 18 * 32, store_value<T>(P1 - s1));
                } else {
                    if constexpr (GS >= 1) {
                        // local grad c1, grad c2 (Eq. 39) from the first moments of h1, h2
                        R m1x = R(0), m1y = R(0), m2x = R(0), m2y = R(0);
#pragma unroll
                        for (int i = 1; i < QS; ++i) {
                            if (cx(i)) { m1x += R(cx(i)) * cur.H1(i); m2x += R(cx(i)) * cur.H2(i); }
                            if (cy(i)) { m1y += R(cy(i)) * cur.H1(i); m2y += R(cy(i)) * cur.H2(i); }
                        }
                        const R s1n = C.D1 * C.four_over_W * omp * c1, s2n = C.D2 * C.four_over_W * phi * c2;
                        const R k1 = R(3) * C.omega_h1, k2 = R(3) * C.omega_h2;  // 1 / (tau cs^2)
                        dc1x = k1 * (-m1x + c1 * ux - R(0.5) * d1ux + s1n * nxv);
                        dc1y = k1 * (-m1y + c1 * uy - R(0.5) * d1uy + s1n * nyv);
                        dc2x = k2 * (-m2x + c2 * ux - R(0.5) * d2ux - s2n * nxv);
                        dc2y = k2 * (-m2y + c2 * uy - R(0.5) * d2uy - s2n * nyv);
                    }
                    const R Dm = mixed_diffusivity(C, phi, omp);
                    const R S1 = C.A * Dm * (C.K * c2 * phi - c1 * omp);
                    const R Ht = Dm * (dphix * (dc1x + C.K * dc2x) + dphiy * (dc1y + C.K * dc2y));
                    const R t1 = C.force_h1 * C.four_over_W * omp * c1;
                    const R t2 = C.force_h2 * C.four_over_W * phi * c2;
                    const R a1 = C.omega_h1 * c1 + C.force_h1 * S1 - Ht;
                    const R a2 = C.omega_h2 * c2 - C.force_h2 * S1 + Ht;
                    const R B1x = (R(3) * (C.omega_h1 * c1 * ux + C.force_h1 * d1ux) + t1 * nxv);
                    const R B1y = (R(3) * (C.omega_h1 * c1 * uy + C.force_h1 * d1uy) + t1 * nyv);
                    const R B2x = (R(3) * (C.omega_h2 * c2 * ux + C.force_h2 * d2ux) - t2 * nxv);
                    const R B2y = (R(3) * (C.omega_h2 * c2 * uy + C.force_h2 * d2uy) - t2 * nyv);
                    const R k1 = R(1) - C.omega_h1, k2 = R(1) - C.omega_h2;
                    // the pulled h (16-bit storage: decoded with the writers' c)
                    auto h1 = [&](int i) -> R {
                        if constexpr (PAIRED) return R(h1d[i]);
                        else return cur.H1(i);
                    };
                    auto h2 = [&](int i) -> R {
                        if constexpr (PAIRED) return R(h2d[i]);
                        else return cur.H2(i);
                    };
                    R P1 = R(0), P2 = R(0), s1 = R(0), s2 = R(0);
#pragma unroll
                    for (int i = 0; i < QS; ++i) {
                        P1 += h1(i);
                        P2 += h2(i);
                    }
#pragma unroll
                    for (int i = 1; i < QS; ++i) {
                        const R w = wq<R, QS>(i);
                        const R c1B = (cx(i) ? R(cx(i)) * B1x : R(0)) + (cy(i) ? R(cy(i)) * B1y : R(0));
                        const R c2B = (cx(i) ? R(cx(i)) * B2x : R(0)) + (cy(i) ? R(cy(i)) * B2y : R(0));
                        const R v1 = k1 * h1(i) + w * (a1 + c1B);
                        const R v2 = k2 * h2(i) + w * (a2 + c2B);
                        if constexpr (PAIRED) {
                            // stored relative to this node's c1, c2 bases
                            const float e1 = float(v1) - bwq<float, QS>(i) * float(c1r);
                            const float e2 = float(v2) - bwq<float, QS>(i) * float(c2r);
                            const uint32_t wv = round_pair<T>(e1, e2, sr_word(key, e1, 9 + i));
                            s1 += lo16<T>(wv);
                            s2 += hi16<T>(wv);
                            stcs(ow + (9 + i) * 32, wv);
                        } else {
                            const T t1 = store_value<T>(v1), t2 = store_value<T>(v2);
                            s1 += to_r<R>(t1);
                            s2 += to_r<R>(t2);
                            stcs(o + (18 + i) * 32, t1);
                            stcs(o + (18 + QS + i) * 32, t2);
                        }
                    }
                    // post-collision sums: with c1 = P1 + S1/2 (Eq. 37) the BGK update gives
                    // sum h1* = P1 + S1 - Ht and sum h2* = P2 - S1 + Ht exactly; written
                    // without c1 they cannot inherit its rounding, and P1 + P2 is kept
                    // (16-bit storage: s1, s2 sum the stored remainders, whose bases
                    // bq_i c1r, bq_i c2r sum to the bases c1r, c2r)
                    if constexpr (PAIRED) {
                        const float r1 = float(((P1 - c1r) + (S1 - Ht)) - s1);
                        const float r2 = float(((P2 - c2r) - (S1 - Ht)) - s2);
                        stcs(ow + 9 * 32, round_pair<T>(r1, r2, sr_word(key, r1, 9)));
                    } else {
                        const R r1 = (P1 + (S1 - Ht)) - s1, r2 = (P2 - (S1 - Ht)) - s2;
                        stcs(o + 18 * 32, store_value<T>(r1));
                        stcs(o + (18 + QS) * 32, store_value<T>(r2));
                    }
                }
            }
        }
        if constexpr (!CUR_SMEM) cur = nxt;
    }
}

// One launch = one step (or one field evaluation) of a single lattice: CTA
// (bx, by) owns columns bx*STRIP_W .. +STRIP_W-1 of rows by*strip_h .. +strip_h-1.
template <typename T, typename R, int QS, bool FIELDS, int VAR = 0>
__global__ void __launch_bounds__(STRIP_W, IsHalf<T>::value ? STRIP_MIN_BLOCKS_16
                                           : (sizeof(R) == 8 ? STRIP_MIN_BLOCKS_64 : STRIP_MIN_BLOCKS))
    strip_kernel(const T* __restrict__ src, T* __restrict__ dst, R* __restrict__ prev, Geometry g,
                 Coeffs<R> C, unsigned* __restrict__ flag, uint32_t mask, void* __restrict__ out,
                 int out_f64) {
    const int ya = blockIdx.y * g.strip_h;
    strip_tile<T, R, QS, FIELDS, STRIP_W, false, VAR>(src, dst, prev, g, C, flag, mask, out, out_f64,
                                                      blockIdx.x * STRIP_W, ya, min(ya + g.strip_h, g.ny));
}

// Initial state: populations at the (source-shifted) equilibria of the given
// fields, written at the upstream node they will be pulled from, so that the
// first step's read returns f_i = f_i^eq (Eq. 24), g_i = g_i^eq (Eqs. 29-30) and
// h_k,i = h_k,i^eq (Eq. 35) -/+ w_i S/2, so that Eq. (37) gives back c_k.
// With u = 0, p = 0: f_i = w_i phi, g_i = 0, h_k,i = w_i (c_k -/+ S/2).
// 16-bit storage: the (c1, c2) half pair that node (x, y) writes among the
// bases of its initial populations (as the step kernel would)
__device__ __forceinline__ uint32_t init_cbase(const InitFields& in, const Geometry& g, int x, int y) {
    const size_t k = (size_t)y * g.nx + x;
    return half_pair(float(in.c1[k]), float(in.c2[k]));
}
template <typename T, typename R, int QS>
__global__ void init_kernel(InitFields in, T* __restrict__ pop, R* __restrict__ prev, Geometry g,
                            Coeffs<R> C) {
    constexpr int NQ = nq_of(QS);
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= g.nx || y >= g.ny) return;
    const size_t k = (size_t)y * g.nx + x;
    const double phi_d = in.phi[k];
    const R phi = R(phi_d), c1 = R(in.c1[k]), c2 = R(in.c2[k]);
    const R ux = in.ux ? R(in.ux[k]) : R(0), uy = in.uy ? R(in.uy[k]) : R(0), p = in.p ? R(in.p[k]) : R(0);
    const R S1 = C.A * mixed_diffusivity(C, phi, R(1) - phi) * (C.K * c2 * phi - c1 * (R(1) - phi));
    const R phic = phi < R(0) ? R(0) : (phi > R(1) ? R(1) : phi);
    const R rho = C.rho2 + C.drho * phic, uu = ux * ux + uy * uy;
    // populations are written pre-streamed: direction i of node (x, y) goes where
    // the next step pulls it from
    auto put = [&](int plane0, int i, R v) {
        pop[pop_pull_off<T, NQ>(g, x, y, plane0, i)] = from_r<T>(v);
    };
    auto cu_of = [&](int i) { return R(cx(i)) * ux + R(cy(i)) * uy; };
    for (int i = 0; i < 9; ++i) {
        const R w = w9<R>(i), cu = cu_of(i);
        const R s = w * (R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu);
        R v = (i == 0 ? R(3) * p * (w - R(1)) : R(3) * p * w) + rho * s;
        if constexpr (IsHalf<T>::value) {
            // relative to the pressure base of the node this slot is pulled from
            int sx, sy;
            pull_src(g, x, y, i, sx, sy);
            v -= p_base<R>(i, in.p ? R(in.p[(size_t)sy * g.nx + sx]) : R(0));
        }
        put(9, i, g_stored<T>(v));
    }
    if constexpr (IsHalf<T>::value) {
        const size_t kb = (size_t)y * g.nxb * 32 + x, N = (size_t)g.ny * g.nxb * 32;
        reinterpret_cast<float2*>(g.pb_out)[kb] = make_float2(float(p), float(phi));
        reinterpret_cast<uint32_t*>(g.pb_out + 2 * N)[kb] = init_cbase(in, g, x, y);
        if (x == 0 && y == 0) reinterpret_cast<uint32_t*>(g.pb_out)[3 * N] = 0u;  // step counter
    }
    if constexpr (PhaseFix<T>::on) {
        // the collision's rest-population rule: sum_i F_i = round((phi - 1/2) 2^31),
        // taken from the input in double so that the phase field's total is exact
        int* fp = reinterpret_cast<int*>(pop);
        const long long Phi = llrint((phi_d - 0.5) * 2147483648.0);
        long long rest = Phi;
        for (int i = 1; i < 9; ++i) {
            const R w = w9<R>(i);
            // the FP32 value times 2^31 (exact) rounded to the nearest integer, ties
            // to even: the integer a double llrint gives, without FP64 arithmetic
            // (the values stay below 1 in magnitude for |u| below the lattice speed)
            const int Fi = __float2int_rn((w * phi * (R(1) + R(3) * cu_of(i)) - R(0.5) * w) * 2147483648.0f);
            rest -= Fi;
            fp[pull_off<NQ>(g, x, y, 0, i)] = Fi;
        }
        fp[pull_off<NQ>(g, x, y, 0, 0)] = (int)rest;
    } else if constexpr (IsHalf<T>::value) {
        // stored as f_i - w_i phi_w, phi_w the phase field of the node the slot
        // is pulled from (f_dec); the rest population, pulled from the node
        // itself, takes what the rounded moving ones leave of phi
        R sum = R(0);
        for (int i = 1; i < 9; ++i) {
            const R w = w9<R>(i);
            int sx, sy;
            pull_src(g, x, y, i, sx, sy);
            const R phs = R(float(in.phi[(size_t)sy * g.nx + sx]));
            const T v = from_r<T>(w * phi * (R(1) + R(3) * cu_of(i)) - bw9<R>(i) * phs);
            sum += to_r<R>(v) + bw9<R>(i) * phs;
            pop[pop_pull_off<T, NQ>(g, x, y, 0, i)] = v;
        }
        put(0, 0, (phi - sum) - bw9<R>(0) * phi);
    } else {
        for (int i = 0; i < 9; ++i) put(0, i, w9<R>(i) * phi * (R(1) + R(3) * cu_of(i)));
    }
    R* pp = prev + node_off<5>(g, x, y);
    pp[0] = phi;
    pp[32] = ux;
    pp[64] = uy;
    if (g.one_scalar) {
        // h3 at the equilibrium of Sec. III D for c = c1 + c2; the h2 planes stay 0
        const R c = c1 + c2, ke = C.K * phic + (R(1) - phic);
        for (int i = 0; i < QS; ++i) {
            const R w = wq<R, QS>(i);
            put(18, i, (i == 0 ? c + (w - R(1)) * c / ke : w * c / ke) + R(3) * w * cu_of(i) * c);
            put(18 + QS, i, R(0));
        }
        pp[96] = c;
        pp[128] = R(0);
        return;
    }
    for (int i = 0; i < QS; ++i) {
        const R w = wq<R, QS>(i), e = R(1) + R(3) * cu_of(i);
        R v1 = w * (c1 * e - R(0.5) * S1), v2 = w * (c2 * e + R(0.5) * S1);
        if constexpr (IsHalf<T>::value) {
            // relative to the c1, c2 bases of the node this slot is pulled from
            int sx, sy;
            pull_src(g, x, y, i, sx, sy);
            const uint32_t cw = init_cbase(in, g, sx, sy);
            v1 -= bwq<R, QS>(i) * R(half_lo(cw));
            v2 -= bwq<R, QS>(i) * R(half_hi(cw));
        }
        put(18, i, v1);
        put(18 + QS, i, v2);
    }
    pp[96] = c1;
    pp[128] = c2;
}

// Block partials of {sum phi, sum(c1 + c2)}; c1 + c2 = sum h1 + sum h2 exactly
// (the two interfacial exchange terms of Eq. 37 cancel).
template <typename T, int QS>
__global__ void __launch_bounds__(RED_THREADS)
    conserved_partials(const T* __restrict__ pop, Geometry g, double* __restrict__ partials) {
    dbg_begin(g.ws_lo, g.ws_hi);
    constexpr int NQ = nq_of(QS);
    // fixed point: sum of the integers Phi (exact); otherwise sum of phi
    long long ai = 0;
    double a = 0.0, b = 0.0;
    const long long n = (long long)g.nx * g.ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / g.nx), x = (int)(k - (long long)y * g.nx);
        if constexpr (PhaseFix<T>::on) {
            long long s = 0;
            for (int i = 0; i < 9; ++i) s += load_f<T>(pop, pull_off<NQ>(g, x, y, 0, i), i);
            ai += s;
        } else {
            for (int i = 0; i < 9; ++i) a += double(load_f<T>(pop, pop_pull_off<T, NQ>(g, x, y, 0, i), i));
            // 16-bit storage: every node's phi_w is the base of the nine slots its
            // populations went to, with weights summing to 1
            if constexpr (IsHalf<T>::value) a += double(g.pb_in[2 * ((long long)y * g.nxb * 32 + x) + 1]);
        }
        double c = 0.0;
        for (int i = 0; i < QS; ++i)
            c += pull_any<NQ, T, double>(pop, g, x, y, 18, i) +
                 (g.one_scalar ? 0.0 : pull_any<NQ, T, double>(pop, g, x, y, 18 + QS, i));
        // ... and its c1_w, c2_w of the slots of its h
        if constexpr (IsHalf<T>::value) {
            const long long N = (long long)g.ny * g.nxb * 32;
            const uint32_t cw = reinterpret_cast<const uint32_t*>(g.pb_in + 2 * N)[(long long)y * g.nxb * 32 + x];
            c += double(half_lo(cw)) + double(half_hi(cw));
        }
        b += c;
    }
    __shared__ double sa[RED_THREADS / 32], sb[RED_THREADS / 32];
    __shared__ long long si[RED_THREADS / 32];
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, off);
        b += __shfl_down_sync(0xffffffffu, b, off);
        ai += __shfl_down_sync(0xffffffffu, ai, off);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sa[wid] = a; sb[wid] = b; si[wid] = ai; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double A = 0.0, B = 0.0;
        long long AI = 0;
        for (int w = 0; w < RED_THREADS / 32; ++w) { A += sa[w]; B += sb[w]; AI += si[w]; }
        partials[2 * blockIdx.x] = PhaseFix<T>::on ? __longlong_as_double(AI) : A;
        partials[2 * blockIdx.x + 1] = B;
    }
}

// Final pass over the block partials in a fixed order (deterministic).  For the
// fixed-point phase field the integer total is exact and converted once:
// sum phi = (sum Phi) 2^-31 + n / 2.
template <typename T>
__global__ void __launch_bounds__(RED_THREADS)
    conserved_final(const double* __restrict__ partials, int nblocks, long long nodes,
                    double* __restrict__ out) {
    __shared__ double sa[RED_THREADS], sb[RED_THREADS];
    __shared__ long long si[RED_THREADS];
    double a = 0.0, b = 0.0;
    long long ai = 0;
    for (int k = threadIdx.x; k < nblocks; k += blockDim.x) {
        if (PhaseFix<T>::on) ai += __double_as_longlong(partials[2 * k]);
        else a += partials[2 * k];
        b += partials[2 * k + 1];
    }
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    si[threadIdx.x] = ai;
    __syncthreads();
    for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sa[threadIdx.x] += sa[threadIdx.x + s];
            sb[threadIdx.x] += sb[threadIdx.x + s];
            si[threadIdx.x] += si[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = PhaseFix<T>::on ? double(si[0]) * FIX_EPS_D + 0.5 * double(nodes) : sa[0];
        out[1] = sb[0];
    }
}

// ---- launchers ----
inline dim3 strip_grid(const Geometry& g) {
    return dim3((g.nx + STRIP_W - 1) / STRIP_W, (g.ny + g.strip_h - 1) / g.strip_h);
}

template <typename T, typename R>
cudaError_t launch_step_impl(const void* src, void* dst, void* prev, const Geometry& g,
                             const Coeffs<R>& C, int q, unsigned* flag, cudaStream_t s) {
    if constexpr (!IsHalf<T>::value) {
        if (variant_of(g)) return launch_variant<T, R>(src, dst, prev, g, C, q, flag, 0u, nullptr, 0, false, s);
    }
    if (q == 5)
        strip_kernel<T, R, 5, false><<<strip_grid(g), STRIP_W, 0, s>>>(
            (const T*)src, (T*)dst, (R*)prev, g, C, flag, 0u, nullptr, 0);
    else
        strip_kernel<T, R, 9, false><<<strip_grid(g), STRIP_W, 0, s>>>(
            (const T*)src, (T*)dst, (R*)prev, g, C, flag, 0u, nullptr, 0);
    return cudaGetLastError();
}

template <typename T, typename R>
cudaError_t launch_fields_impl(const void* src, const void* prev, const Geometry& g, const Coeffs<R>& C,
                               int q, uint32_t mask, void* out, int out_f64, cudaStream_t s) {
    if constexpr (!IsHalf<T>::value) {
        if (variant_of(g))
            return launch_variant<T, R>(src, nullptr, const_cast<void*>(prev), g, C, q, nullptr, mask, out,
                                        out_f64, true, s);
    }
    if (q == 5)
        strip_kernel<T, R, 5, true><<<strip_grid(g), STRIP_W, 0, s>>>(
            (const T*)src, nullptr, nullptr, g, C, nullptr, mask, out, out_f64);
    else
        strip_kernel<T, R, 9, true><<<strip_grid(g), STRIP_W, 0, s>>>(
            (const T*)src, nullptr, nullptr, g, C, nullptr, mask, out, out_f64);
    return cudaGetLastError();
}

// Launch of a model variant (one-scalar model and/or local gradients), for the
// step (FIELDS = false) or the field evaluation; compiled in its own units.
template <typename T, typename R, int VAR>
cudaError_t launch_variant_impl(const void* src, void* dst, void* prev, const Geometry& g, const Coeffs<R>& C,
                                int q, unsigned* flag, uint32_t mask, void* out, int out_f64, bool fields,
                                cudaStream_t s) {
    if (fields) {
        if (q == 5)
            strip_kernel<T, R, 5, true, VAR><<<strip_grid(g), STRIP_W, 0, s>>>(
                (const T*)src, nullptr, (R*)prev, g, C, nullptr, mask, out, out_f64);
        else
            strip_kernel<T, R, 9, true, VAR><<<strip_grid(g), STRIP_W, 0, s>>>(
                (const T*)src, nullptr, (R*)prev, g, C, nullptr, mask, out, out_f64);
    } else {
        if (q == 5)
            strip_kernel<T, R, 5, false, VAR><<<strip_grid(g), STRIP_W, 0, s>>>(
                (const T*)src, (T*)dst, (R*)prev, g, C, flag, 0u, nullptr, 0);
        else
            strip_kernel<T, R, 9, false, VAR><<<strip_grid(g), STRIP_W, 0, s>>>(
                (const T*)src, (T*)dst, (R*)prev, g, C, flag, 0u, nullptr, 0);
    }
    return cudaGetLastError();
}

template <typename T, typename R>
cudaError_t launch_init_impl(const InitFields& in, void* pop, void* prev, const Geometry& g,
                             const Coeffs<R>& C, int q, cudaStream_t s) {
    dim3 block(32, 8), grid((g.nx + 31) / 32, (g.ny + 7) / 8);
    if (q == 5)
        init_kernel<T, R, 5><<<grid, block, 0, s>>>(in, (T*)pop, (R*)prev, g, C);
    else
        init_kernel<T, R, 9><<<grid, block, 0, s>>>(in, (T*)pop, (R*)prev, g, C);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_conserved_impl(const void* pop, const Geometry& g, int q, double* partials,
                                  double* out, cudaStream_t s) {
    if (q == 5)
        conserved_partials<T, 5><<<RED_BLOCKS, RED_THREADS, 0, s>>>((const T*)pop, g, partials);
    else
        conserved_partials<T, 9><<<RED_BLOCKS, RED_THREADS, 0, s>>>((const T*)pop, g, partials);
    conserved_final<T><<<1, RED_THREADS, 0, s>>>(partials, RED_BLOCKS, (long long)g.nx * g.ny, out);
    return cudaGetLastError();
}

template <typename T, typename R>
int step_blocks_per_sm_impl(int q) {
    int n = 0;
    if (q == 5)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, strip_kernel<T, R, 5, false>, STRIP_W, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, strip_kernel<T, R, 9, false>, STRIP_W, 0);
    return n;
}

}  // namespace lbm
