// Internal host/device interface of liblbm: storage layout, run constants and
// the kernel launchers that the C ABI (lbm_api.cu) dispatches to.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "lbm.h"

#include <nvtx3/nvToolsExt.h>

namespace lbm {

// Host-side NVTX range around a library call (a profiler shows the calls'
// extents on the timeline; without a tool attached it costs a few nanoseconds).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Step kernel: a CTA of STRIP_WARPS warps owns STRIP_W consecutive columns and
// marches up a strip of `strip_h` rows, one thread per column.
#ifndef LBM_STRIP_WARPS
#define LBM_STRIP_WARPS 4
#endif
#ifndef LBM_STRIP_MIN_BLOCKS
#define LBM_STRIP_MIN_BLOCKS 6
#endif
constexpr int STRIP_WARPS = LBM_STRIP_WARPS;
constexpr int STRIP_W = 32 * STRIP_WARPS;
constexpr int STRIP_MIN_BLOCKS = LBM_STRIP_MIN_BLOCKS;  // occupancy target (register cap)
// (6 CTAs = 24 warps per SM, 80 registers; FP32 fits it because the pulled
// populations of the look-ahead row wait in shared memory.)  16-bit storage
// has its own cap, measured separately: 5 CTAs per SM, 96 registers without
// spills (6 CTAs at 80 registers spill 54 bytes and ran 2 % slower).
#ifndef LBM_STRIP_MIN_BLOCKS_16
#define LBM_STRIP_MIN_BLOCKS_16 5
#endif
constexpr int STRIP_MIN_BLOCKS_16 = LBM_STRIP_MIN_BLOCKS_16;
// FP64 arithmetic: 3 CTAs per SM (168 registers) keep it free of spills; its
// speed is set by the FP64 pipe, not by memory
constexpr int STRIP_MIN_BLOCKS_64 = 3;
// Blocks of the conserved-sum reduction (fixed, so the summation order is fixed).
constexpr int RED_BLOCKS = 304;
constexpr int RED_THREADS = 256;

// Storage layout (array of structures of arrays, 32-node blocks).  Rows are cut
// into blocks of 32 consecutive nodes; a block stores its NQ populations as NQ
// runs of 32 values.  Value q of node (x, y) lives at element
//     ((y * nxb + x / 32) * NQ + q) * 32 + x % 32,      nxb = ceil(nx / 32).
// The population planes are f_0..f_8 -> q = 0..8, g_0..g_8 -> 9..17,
// h1_0..h1_{Q-1} -> 18..17+Q, h2_0..h2_{Q-1} -> 18+Q..17+2Q.  A warp touches
// 128 contiguous bytes per population (FP32), and every population of a node
// sits at a compile-time offset from the node's first value.  The five
// previous-step macros (phi, ux, uy, c1, c2) use the same layout with NQ = 5.
struct Geometry {
    int nx, ny, nxb;
    int wall_x, wall_y;
    int strip_h;     // rows per CTA of the step kernel
    int one_scalar;  // one-scalar model: h1 planes hold h3, h2 planes unused
    int grad_scheme; // 0: stencils (Eq. 41); 1: local grad c (Eq. 39); 2: also local grad phi
    // 16-bit storage only (else NULL): the bases of the node that wrote each
    // stored population, (p, phi) in FP32 then (c1, c2) in halves, per node
    // at y * nxb * 32 + x, read for the populations a launch pulls (pb_in) and
    // written beside the ones it stores (pb_out).  Set per launch: the two
    // planes alternate with the population buffers.
    const float* pb_in;
    float* pb_out;
    // The device memory the step may touch: the handle's workspace (or the
    // state given to lbm_conserved_noalloc).  Read only by an LBM_DEBUG build,
    // whose step kernel checks every global access against it.
    const char* ws_lo;
    const char* ws_hi;
};

// Debug build (compiled with -DLBM_DEBUG=1): the step kernel checks every
// global load and store of the workspace against Geometry::ws_lo .. ws_hi; an
// access outside sets FLAG_BOUNDS in a device status word and is skipped (a
// load returns zero), so a bad index is reported and never faults.
#ifndef LBM_DEBUG
#define LBM_DEBUG 0
#endif
constexpr unsigned FLAG_BOUNDS = 2u;
// Debug build: the OR of FLAG_BOUNDS of every checked kernel since the last
// read; cleared by the read (0 in a release build).  Each translation unit
// with checked kernels registers the reader of its own status word.
unsigned debug_status_take();
void register_debug_status(unsigned (*take)());

// Model variant of the step kernel: bit 0 one-scalar, bits 1-2 gradient scheme.
inline int variant_of(const Geometry& g) { return (g.one_scalar ? 1 : 0) | (g.grad_scheme << 1); }

// Per-run constants, derived once on the host in double and cast to the
// compute type R (float or double).
template <typename R>
struct Coeffs {
    R omega_f, force_f;      // 1/tau_f, 1 - 1/(2 tau_f)
    R omega_h1, force_h1;    // 1/tau_h1, 1 - 1/(2 tau_h1)
    R omega_h2, force_h2;
    R beta4, kappa;          // 4 beta = 48 sigma / W,  k = 3 sigma W / 2
    R rho1, rho2, drho;      // drho = rho1 - rho2
    R mu2, dmu;              // linear viscosity mu2 + dmu * phi
    R log_mu1, log_mu2, visc_beta;
    R D1D2, KD1, D2, K;      // D_m = D1 D2 / (K D1 (1 - phi) + D2 phi)
    R D1, M;                 // diffusivity of scalar 1, mobility (local gradient schemes)
    R halfA, A;
    R four_over_W;
    R gx, gy, g_rho_ref, Fx, Fy;
    int visc_model;
};

inline size_t lattice_elems(const Geometry& g, int nq) { return (size_t)g.ny * g.nxb * nq * 32; }

// Storage precisions: the type T a population is stored in and the type R the
// collision computes in.  by_storage calls fn(T{}, R{}) for a precision code.
//   LBM_FP64 -> (double, double)         LBM_FP32 -> (float, float)
//   LBM_FP32_BF16STORE -> (bf16, float)  LBM_FP32_FP16STORE -> (half, float)
template <typename Fn>
auto by_storage(int precision, Fn&& fn) {
    switch (precision) {
        case LBM_FP64: return fn(double{}, double{});
        case LBM_FP32_BF16STORE: return fn(__nv_bfloat16{}, float{});
        case LBM_FP32_FP16STORE: return fn(__half{}, float{});
        default: return fn(float{}, float{});
    }
}

// Launchers (one instantiation per storage type, defined in lbm_step_f64.cu,
// lbm_step_f32.cu, lbm_step_bf16.cu and lbm_step_f16.cu).  `src` holds the post-collision populations of the last
// step (pull scheme: streaming happens on the read), `dst` receives the new
// ones; `prev` holds phi, ux, uy, c1, c2 of the last step (updated in place).
template <typename T, typename R>
cudaError_t launch_step(const void* src, void* dst, void* prev, const Geometry& geo,
                        const Coeffs<R>& C, int scalar_q, unsigned* flag, cudaStream_t s);

// Macroscopic fields of the state in `src` (no collision), written as dense
// nx*ny arrays in mask-bit order (double or float); `prev` (the previous-step
// macros) is read by the local grad phi scheme only.
template <typename T, typename R>
cudaError_t launch_fields(const void* src, const void* prev, const Geometry& geo, const Coeffs<R>& C,
                          int scalar_q, uint32_t mask, void* out, int out_f64, cudaStream_t s);

// The step or field evaluation of a model variant (variant_of(geo) != 0), FP32
// and FP64 only (lbm_step_var_f32.cu, lbm_step_var_f64.cu).
template <typename T, typename R>
cudaError_t launch_variant(const void* src, void* dst, void* prev, const Geometry& geo, const Coeffs<R>& C,
                           int scalar_q, unsigned* flag, uint32_t mask, void* out, int out_f64, bool fields,
                           cudaStream_t s);

// Macroscopic fields of an initial state: dense nx*ny double arrays; ux, uy, p
// may be NULL (zero).
struct InitFields {
    const double *phi, *ux, *uy, *p, *c1, *c2;
};

// Initial populations at the equilibria of the given fields, written
// pre-streamed so the first pulled read returns them (arithmetic in R).
template <typename T, typename R>
cudaError_t launch_init(const InitFields& in, void* pop, void* prev, const Geometry& geo,
                        const Coeffs<R>& C, int scalar_q, cudaStream_t s);

// phi = 1/2 + 1/2 tanh(2 l / W) (Eq. 2), c1 = c1t phi, c2 = c2t (1 - phi), into
// three dense staging arrays (sdf may alias phi).
cudaError_t launch_sdf_to_fields(const double* sdf, double* phi, double* c1, double* c2, size_t n,
                                 double W, double c1t, double c2t, cudaStream_t s);

// {sum phi, sum(c1 + c2)} of the current state: block partials + a fixed-order final pass.
template <typename T>
cudaError_t launch_conserved(const void* pop, const Geometry& geo, int scalar_q,
                             double* partials, double* out, cudaStream_t s);

// CTAs of the step kernel that fit on one SM (for the strip-height choice).
template <typename T, typename R>
int step_blocks_per_sm(int scalar_q);

// ---- batched runner: many independent FP32 lattices in one persistent launch ----
// One lattice of a batch, as the persistent kernel sees it.
struct BatchCase {
    Geometry g;          // strip_h unused
    Coeffs<float> C;
    void* pop[2];        // population buffers
    void* prev;          // previous-step macros
    unsigned* flag;      // non-finite flag of the lattice
    int cur0;            // buffer that held the state when the step counters were reset
};
// A tile: columns x0 .. x0+W-1 (clipped to nx) of rows ya .. yb-1 of lattice c.
struct BatchTile {
    int c, x0, ya, yb;
};
// Tiles a tile waits for before each step (-1 = none): those whose nodes its step
// reads and those that read its nodes.  Usually the 8 around it; a tail tile one
// row or column wide lets the reads of its neighbours wrap past it, so the list
// is computed from the actual reads and may be longer.
constexpr int BATCH_NEIGHBOURS = 32;

struct BatchArgs {
    const BatchCase* cases;
    const BatchTile* tiles;
    const int* nbr;           // BATCH_NEIGHBOURS per tile
    unsigned* done;           // steps completed, per tile
    unsigned* status;         // bit 0: a wait gave up
    int ntiles;
    int nsteps;               // steps every tile advances in this launch
    long long spin_limit;     // polls before a wait gives up
    int hold_tile;            // fault injection: this tile never reports done (-1: none)
    int grid;                 // CTAs (all co-resident: cooperative launch)
};

// Tile widths of the batched kernel: 32 * NW columns, NW in {1, 2, 4}.
template <int QS, int NW>
cudaError_t launch_batch(const BatchArgs& a, cudaStream_t s);
template <int QS, int NW>
int batch_blocks_per_sm();

}  // namespace lbm
