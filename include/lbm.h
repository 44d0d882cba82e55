/*
 * liblbm -- GB300-native phase-field lattice Boltzmann solver for two-phase
 * flow with interfacial mass/heat transfer (Chen, Zhan, Chai & Shi,
 * arXiv 2402.15752).  C ABI: plain pointers and sizes, no C++ or torch types.
 *
 * One time step (lbm_step) is the paper's coupled collide-and-stream over four
 * lattices, in lattice units (dx = dt = 1, cs^2 = 1/3):
 *   f  (D2Q9)  conservative Allen-Cahn phase field          Sec. III A, Eqs. (23)-(27)
 *   g  (D2Q9)  pressure-based incompressible two-phase flow Sec. III B, Eqs. (28)-(33)
 *              with the surface-tension force mu_phi grad(phi), Eqs. (4)-(5)
 *   h1, h2     two-scalar mass/heat transfer with the auxiliary interfacial
 *   (D2Q5|Q9)  source H~, Sec. III C, Eqs. (34)-(38)
 * gradients and the Laplacian use the isotropic central stencils of
 * Eqs. (41)-(42); viscosity is linear in phi (Eq. 7), follows Eq. (48), or
 * mu = mu_lin(phi) * exp(-visc_beta * (c1 + c2)).
 *
 * Ownership.  The caller owns the device workspace, the CUDA stream and every
 * input/output buffer.  The library allocates no device memory; it owns only
 * the small host-side handle (plus 16 bytes of pinned host memory for the
 * asynchronous status word).  Every call is asynchronous on the handle's
 * stream unless its comment says it synchronises.
 *
 * Errors.  Every int-returning call returns LBM_OK (0) or a negative LBM_ERR_*
 * code; lbm_last_error() gives a message.  No C++ exception crosses the ABI
 * and no kernel traps or asserts.
 *
 * Field layout.  Every host or device field is row-major, index = y*nx + x,
 * node coordinates x = 0..nx-1, y = 0..ny-1.
 */
#ifndef PFLBM_LBM_H
#define PFLBM_LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ---- */
#define LBM_OK                0
#define LBM_ERR_ARG          (-1) /* bad pointer, size, enum or physical parameter   */
#define LBM_ERR_UNSTABLE_TAU (-2) /* a relaxation time would be <= 1/2                */
#define LBM_ERR_WORKSPACE    (-3) /* workspace too small or misaligned                */
#define LBM_ERR_CUDA         (-4) /* a CUDA runtime call failed                       */
#define LBM_ERR_NONFINITE    (-5) /* a NaN/Inf macro value was produced by a step     */
#define LBM_ERR_TIMEOUT      (-6) /* a bounded device wait gave up (batched runner)   */
#define LBM_ERR_BOUNDS       (-7) /* debug build only: an access fell outside the
                                     workspace (it was skipped, see lbm_debug_build) */

/* ---- enums ---- */
#define LBM_BC_PERIODIC 0
#define LBM_BC_WALL     1 /* half-way bounce-back (Sec. IV): no-slip, no-flux */

#define LBM_FP64           0 /* FP64 storage and arithmetic                      */
#define LBM_FP32           1 /* FP32 storage and arithmetic                      */
/* 16-bit population storage, FP32 arithmetic: each population is read, converted
 * and collided in FP32 and rounded stochastically on the store (the random bits
 * are a hash seeded per node and step from the node's coordinates, its new
 * macros and a step counter kept in the state: deterministic, so runs and
 * restarts are reproducible).  Each node also writes its pressure and phase
 * field (FP32) and its scalars (rounded to IEEE half) beside its populations,
 * which are stored as offsets from their writer's: f_i - b_i phi_w,
 * g_i - 3 b_i p_w (g_0 - 3 (b_0 - 1) p_w) and h_k,i - bq_i c_k,w, with b_i and
 * bq_i the D2Q9 and scalar-lattice weights rounded to multiples of 2^-20 so that
 * they sum to exactly 1; g in half is scaled by 2^10; the five previous-step
 * macros stay FP32; c1 and c2 must stay below 65504 in magnitude (their bases
 * are halves).  Not in the paper: 56 population bytes per node instead of 112
 * (scalar_q = 5), plus 12 bytes of (p, phi, c1, c2), at a field error of
 * 1e-4..1e-3 (half) and 1e-3..1e-2 (bfloat16), the density-ratio-1000 bubble
 * included.  A step of a 16-bit run also reports a non-finite pressure. */
#define LBM_FP32_BF16STORE 2 /* bfloat16 storage (8-bit significand, FP32 range)  */
#define LBM_FP32_FP16STORE 3 /* IEEE half storage (11-bit significand, |x| < 65504;
                                values below 6.1e-5 lose bits as subnormals)        */

#define LBM_VISC_LINEAR 0 /* mu = phi (mu1 - mu2) + mu2                 Eq. (7)  */
#define LBM_VISC_LOG_C  1 /* log mu = c1 log mu1 + c2 log mu2          Eq. (48) */
#define LBM_VISC_EXP_T  2 /* mu = [phi (mu1 - mu2) + mu2] exp(-visc_beta (c1 + c2)) */

/* Scalar transport.  TWO: the two-scalar lattices h1, h2 with the auxiliary
 * interfacial source (Sec. III C, Eqs. 34-38).  ONE: the one-scalar lattice h3 for
 * the total c = c1 + c2 (Sec. III D): h3_0^eq = c + (w_0 - 1) c / K_eff,
 * h3_i^eq = w_i c / K_eff + w_i c_i.(c u) / cs^2, source w_i c_i.d_t(c u) / cs^2,
 * tau_h3 = D_eff / cs^2 + 1/2 per node, with K_eff = K phi + (1 - phi) and
 * D_eff = D1 K phi + D2 (1 - phi) (Eq. 31, phi clipped to [0, 1]); c1 and c2 are then
 * the Henry split c1 = K phi c / K_eff, c2 = (1 - phi) c / K_eff (fields, viscosity).
 * ONE runs in LBM_FP64 and LBM_FP32, on single lattices (not in a batch). */
#define LBM_SCALAR_TWO 0
#define LBM_SCALAR_ONE 1

/* Gradients.  STENCIL: grad phi, grad c1, grad c2 by the isotropic stencil of
 * Eq. (41).  LOCAL_C: grad c1, grad c2 by the local scheme of Eq. (39) (first
 * moments of h1, h2, with u, d_t(c_k u) and the normal of the step).  LOCAL_ALL:
 * also grad phi and |grad phi| by the local scheme given after Eq. (39) (first
 * moment of f), with the previous step's velocity in its C term (the velocity of
 * the step needs the surface force, which needs grad phi).  The Laplacian is
 * Eq. (42) in every scheme.  LOCAL_* run in LBM_FP64 and LBM_FP32, single lattices. */
#define LBM_GRAD_STENCIL   0
#define LBM_GRAD_LOCAL_C   1
#define LBM_GRAD_LOCAL_ALL 2

/* field mask bits for lbm_get_fields; fields are written in this order */
#define LBM_FIELD_PHI (1u << 0)
#define LBM_FIELD_UX  (1u << 1)
#define LBM_FIELD_UY  (1u << 2)
#define LBM_FIELD_P   (1u << 3)
#define LBM_FIELD_C1  (1u << 4)
#define LBM_FIELD_C2  (1u << 5)
#define LBM_FIELD_RHO (1u << 6)
#define LBM_FIELD_MU  (1u << 7)
#define LBM_FIELD_ALL 0xffu

#define LBM_OUT_F64 0
#define LBM_OUT_F32 1

/*
 * Problem parameters, in lattice units, as the paper states the problem:
 * Eqs. (4)-(7) and (17)-(18) for the physics, Eqs. (27), (33), (38) for the
 * relaxation times derived from M, mu/rho and D_k.  Phase 1 is phi = 1.
 */
typedef struct {
    int32_t nx, ny;        /* grid nodes, each >= 1                                  */
    int32_t bc_x, bc_y;    /* LBM_BC_PERIODIC or LBM_BC_WALL                         */
    int32_t scalar_q;      /* 5 (D2Q5) or 9 (D2Q9) for h1, h2                        */
    int32_t precision;     /* LBM_FP64, LBM_FP32, LBM_FP32_BF16STORE or LBM_FP32_FP16STORE */
    double W, M, sigma;    /* interface width, mobility, surface tension (> 0, > 0, >= 0) */
    double rho1, rho2;     /* densities (> 0)                                        */
    double mu1, mu2;       /* dynamic viscosities (> 0)                              */
    double D1, D2;         /* scalar diffusivities (> 0)                             */
    double Keq, A;         /* equilibrium jump K_eq (> 0), inverse time scale A (>= 0) */
    double gx, gy;         /* body force G = (rho - g_rho_ref) (gx, gy) + (Fx, Fy)   */
    double g_rho_ref;
    double Fx, Fy;
    int32_t visc_model;    /* LBM_VISC_*                                             */
    double visc_beta;      /* exponent of LBM_VISC_EXP_T                             */
    int32_t scalar_model;  /* LBM_SCALAR_TWO or LBM_SCALAR_ONE                       */
    int32_t grad_scheme;   /* LBM_GRAD_STENCIL, LBM_GRAD_LOCAL_C or LBM_GRAD_LOCAL_ALL */
} lbm_params;

typedef struct lbm_handle lbm_handle;

/* Bytes of device workspace the parameters need (0 if the parameters are invalid).
 * Layout per node: two population buffers (28 values for scalar_q = 5, 36 for 9, of
 * 8, 4 or 2 bytes), five previous-step macros (8 bytes for LBM_FP64, else 4), with
 * 16-bit storage two sets of the writers' (p, phi, c1, c2) bases (12 bytes per node each),
 * plus a few KB of reduction partials and flags. */
size_t lbm_workspace_bytes(const lbm_params* params);

/* Validate parameters (Sec. III relaxation-time relations: every tau > 1/2),
 * carve the caller's device workspace (256-byte aligned, >= lbm_workspace_bytes)
 * and bind the CUDA stream (a cudaStream_t; NULL = legacy default stream).
 * Host only: no kernel runs.  On success *out is a new handle. */
int lbm_create(const lbm_params* params, void* d_workspace, size_t workspace_bytes,
               void* cuda_stream, lbm_handle** out);

/* Initial state from a signed-distance field l(x) (nx*ny doubles, host or device):
 * phi = 1/2 + 1/2 tanh(2 l / W) (Eq. 2), c1 = c1_tilde * phi, c2 = c2_tilde * (1 - phi),
 * u = 0, p = 0.  Populations start at their equilibria (f_i = w_i phi, g_i = 0) and
 * h_k,i = w_i (c_k -/+ S/2) so that Eq. (37) returns the given c_k; the time counter
 * restarts at 0.  A host sdf is read on the stream: page-locked (mapped) memory in
 * place by the GPU, so keep it unchanged until the stream has passed this call;
 * pageable memory through a copy that completes before the call returns. */
int lbm_init(lbm_handle* h, const double* sdf, int32_t sdf_on_device,
             double c1_tilde, double c2_tilde);

/* Same, from explicit phi, c1, c2 fields (nx*ny doubles each, host or device). */
int lbm_init_fields(lbm_handle* h, const double* phi, const double* c1, const double* c2,
                    int32_t on_device);

/* Same, from all six macroscopic fields (nx*ny doubles each, host or device):
 * populations at the equilibria of Eqs. (24), (29)-(30) and (35) for phi, u, p, c1,
 * c2 (h shifted by -/+ w_i S/2 as above), previous-step macros phi, u, c1, c2.  A
 * restart from macroscopic fields (the non-equilibrium parts start at zero); the
 * surrogate network's judge uses it.  Not in the paper. */
int lbm_init_macros(lbm_handle* h, const double* phi, const double* ux, const double* uy,
                    const double* p, const double* c1, const double* c2, int32_t on_device);

/* Advance nsteps >= 0 time steps (asynchronous).  Returns LBM_ERR_NONFINITE if an
 * earlier call's steps, already finished on the GPU, produced a NaN/Inf.  Steps
 * are replayed from captured CUDA graphs of 32, 16, .., 2 steps (the binary
 * digits of nsteps), an odd last step is one plain launch; the first call with
 * nsteps >= 2 captures them (call it before any stream capture of your own). */
int lbm_step(lbm_handle* h, int64_t nsteps);

/* Macroscopic fields of the current state (the zeroth/first moments of the current
 * populations, Eqs. (26), (32), (37), with the stencils of Eqs. (41)-(42)).
 * out receives popcount(mask) consecutive fields of nx*ny values, in mask-bit order,
 * as doubles (LBM_OUT_F64) or floats (LBM_OUT_F32).  out_on_device = 0: out is host
 * memory (page-locked, mapped memory is written in place by the GPU, other memory
 * through device staging and a copy) and the call synchronises the stream before
 * returning. */
int lbm_get_fields(lbm_handle* h, uint32_t mask, void* out, int32_t out_on_device,
                   int32_t out_dtype);

/* {sum phi, sum (c1 + c2)} over all nodes of the current state, reduced on the GPU in
 * FP64 in a fixed order (deterministic).  Synchronises; also reports a pending
 * non-finite flag as LBM_ERR_NONFINITE. */
int lbm_conserved(lbm_handle* h, double out[2]);

/* Synchronise the stream and report LBM_ERR_NONFINITE if any finished step
 * produced a NaN/Inf; clears nothing.  A debug build first reports
 * LBM_ERR_BOUNDS if a checked access failed since the last lbm_sync of any
 * handle (that check is cleared by the report). */
int lbm_sync(lbm_handle* h);

/* 1 if this library is the debug build (compiled with LBM_DEBUG=1), else 0.
 * In the debug build the step, field and reduction kernels check every global
 * load and store of the workspace against the handle's workspace range (the
 * state's range for lbm_conserved_noalloc); an access outside it is skipped (a
 * load reads zero), recorded, and reported by lbm_sync as LBM_ERR_BOUNDS.
 * Nothing faults or traps.  A development aid, not in the paper. */
int lbm_debug_build(void);

/* Debug build only (LBM_ERR_ARG otherwise): check the handle's kernels against
 * the first `bytes` of its workspace instead of all of it (bytes <= the
 * workspace size), so that a test can show an access beyond the range being
 * skipped and reported.  Synchronises the stream and drops the captured graphs. */
int lbm_debug_limit_workspace(lbm_handle* h, size_t bytes);

/* Checkpoint: the populations and previous-step macros of the current state,
 * and with 16-bit storage the (p, phi) FP32 and (c1, c2) half bases of every node that the stored
 * populations are offsets from and the step counter of the rounding (in that order:
 * populations, macros, bases, counter).
 * lbm_state_bytes gives the size; get/set copy to/from caller memory: a host
 * buffer synchronises the stream, a device buffer (on_device != 0) is copied
 * asynchronously on the handle's stream.  Restoring then stepping is
 * bit-identical to never having stopped. */
size_t lbm_state_bytes(const lbm_handle* h);
int lbm_get_state(lbm_handle* h, void* buf, size_t bytes, int32_t on_device);
int lbm_set_state(lbm_handle* h, const void* buf, size_t bytes, int32_t on_device);

/* Steps taken since the last init or set_state. */
int64_t lbm_time(const lbm_handle* h);

/* Conserved sums {sum phi, sum (c1 + c2)} of a solver state that lives in device
 * memory (the bytes lbm_get_state writes, on the device), without a handle and
 * without allocating anything.  The paper has no counterpart: this is a service of
 * the library.
 * Who needs it: code that must not touch the device allocator -- a monitor or
 * checkpoint validator running inside a host application whose GPU memory is owned
 * by another allocator or fully reserved, a process that has run out of device
 * memory and still has to verify a saved state, or code issued between stream
 * captures that must not change the memory footprint.  lbm_conserved needs a handle,
 * and a handle needs a caller workspace; this call needs neither.
 * Scratch: a fixed array of 131,088 bytes in the library's device data (held by each
 * GPU that loads the library until the process exits) holds one partial per chunk of
 * 8192 nodes; grids above 67,108,864 nodes (8192 x 8192) are rejected with
 * LBM_ERR_ARG.  No cudaMalloc, cudaFree or allocating library routine is called.
 * The first call on a device looks up the array's device address (once per device,
 * under a lock); make that first call before any stream capture on that device.
 * All calls on a device share the array, so calls whose work overlaps on the GPU
 * (different streams, or different host threads) race: serialise them.  Every slot a
 * call reads is written by the same call first.
 * params: the parameters the state was created with; only the layout fields are read
 * (nx, ny, bc_x, bc_y, scalar_q, precision, scalar_model), the physical ones are
 * ignored, and an invalid layout field returns LBM_ERR_ARG.  d_state: device pointer,
 * 16-byte aligned (LBM_ERR_ARG otherwise), state_bytes >= its population part
 * (FP64, FP32) or >= lbm_state_bytes (16-bit storage, whose stored f and h are
 * offsets from the writers' phi, c1 and c2 in the state's last part).  cuda_stream: stream to run on (NULL = legacy default).  out: 2 doubles,
 * host (the call synchronises the stream) or device (out_on_device != 0, asynchronous).
 * err: optional buffer of err_len bytes for an error message (may be NULL). */
int lbm_conserved_noalloc(const lbm_params* params, const void* d_state, size_t state_bytes,
                          void* cuda_stream, double* out, int32_t out_on_device, char* err,
                          size_t err_len);

/* Release the handle (and its CUDA graphs/events); the workspace stays the caller's. */
void lbm_destroy(lbm_handle* h);

/*
 * Batched runner.  Many independent lattices of uneven sizes (each an lbm_handle
 * with its own parameters and workspace) advanced together by one persistent
 * kernel: each lattice is cut into tiles of tile_w x tile_h nodes, the launch's
 * CTAs (all co-resident: a cooperative launch) own the tiles round-robin, and a
 * tile waits only for the tiles of the same lattice whose nodes it reads or that
 * read its nodes (usually the 8 around it) to finish the previous step (per-tile
 * step counters), never for the whole grid.  Full runs of
 * 32 steps are replayed from a captured CUDA graph.  Every node evaluates the
 * expressions of lbm_step in the same order; the batched kernel is compiled
 * separately (and once per tile width), so the compiler may fuse a different set
 * of multiply-adds and results agree with lbm_step to FP32 rounding.  Any two
 * tile heights of one tile width give identical bits, and runs are deterministic.
 * The paper runs one case at a time; batching is a service of the library.
 * Requirements: every case LBM_FP32, one scalar_q, one device and one stream
 * (the batch runs on it).  The cases stay usable through their own calls
 * (init, get_fields, conserved, state); if one of them is stepped, initialised or
 * restored on its own the batch notices and restarts its counters.  Destroy the
 * batch before its cases.
 * Waits are bounded: a wait that gives up (spin_limit polls) sets a status bit,
 * every CTA returns, and lbm_batch_sync reports LBM_ERR_TIMEOUT; the lattices are
 * then out of step until they are re-initialised and lbm_batch_set_tiling is
 * called. */
typedef struct lbm_batch lbm_batch;

/* Bytes of device workspace for the batch's tables (case descriptors, tiles,
 * neighbour lists, step counters); 0 if the cases do not qualify. */
size_t lbm_batch_workspace_bytes(lbm_handle* const* cases, int32_t ncases);

/* Build a batch over ncases handles (the array is copied; the handles stay the
 * caller's) with a caller-owned, 256-byte aligned device workspace.  The initial
 * tiling is 128 x 16.  Synchronises the stream. */
int lbm_batch_create(lbm_handle* const* cases, int32_t ncases, void* d_workspace,
                     size_t workspace_bytes, lbm_batch** out);

/* Tile shape: tile_w in {32, 64, 128} columns, tile_h >= 4 rows.  Rebuilds the
 * tile tables and restarts the step counters; synchronises. */
int lbm_batch_set_tiling(lbm_batch* b, int32_t tile_w, int32_t tile_h);

/* Current tile shape, tile count and CTAs per launch (any pointer may be NULL). */
int lbm_batch_tiling(const lbm_batch* b, int32_t* tile_w, int32_t* tile_h, int32_t* ntiles,
                     int32_t* grid);

/* Advance every case by nsteps >= 0 time steps (asynchronous on the stream). */
int lbm_batch_step(lbm_batch* b, int64_t nsteps);

/* Synchronise; LBM_ERR_TIMEOUT if a wait gave up, else the first case's
 * LBM_ERR_NONFINITE, else LBM_OK. */
int lbm_batch_sync(lbm_batch* b);

/* Time every candidate tiling (tile_w 32, 64, 128 x tile_h 8, 16, 32, 64) over
 * steps_per_trial steps (after 2 untimed ones) and keep the fastest.  The trial
 * steps are real steps of every case (every tiling computes the same update), so
 * the cases advance by 12 * (steps_per_trial + 2) steps.  table (optional) receives
 * up to table_rows rows of {tile_w, tile_h, ms per step, tiles, CTAs}. */
int lbm_batch_autotune(lbm_batch* b, int32_t steps_per_trial, double* table, int32_t table_rows,
                       int32_t* rows_written);

/* Fault injection for tests of the bounded waits: polls per wait before it gives
 * up (default 2^21, about a second) and a tile whose completion is never
 * published (-1: none). */
int lbm_batch_set_wait_limit(lbm_batch* b, int64_t spin_limit, int32_t hold_tile);

/* Restart every case at the equilibria of its six macroscopic fields, as
 * lbm_init_macros does case by case.  macros: the cases' fields concatenated in
 * the batch's case order, each case as six (ny, nx) row-major FP64 arrays
 * {phi, ux, uy, p, c1, c2} (6 * nx * ny doubles per case), on the host or, with
 * on_device != 0, in device memory (asynchronous on the stream).  The batch
 * notices the restart at its next step.  An error names the failing case; the
 * cases before it have been restarted. */
int lbm_batch_init_macros(lbm_batch* b, const double* macros, int32_t on_device);

/* lbm_get_fields of every case into one buffer: case by case, in the batch's
 * order, the selected fields (k of them, in LBM_FIELD bit order) as k (ny, nx)
 * row-major arrays of out_dtype.  Device output is asynchronous on the stream;
 * host output synchronises. */
int lbm_batch_get_fields(lbm_batch* b, uint32_t mask, void* out, int32_t out_on_device,
                         int32_t out_dtype);

/* Checkpoint of every case: lbm_get_state / lbm_set_state of each case into or
 * out of consecutive slices of one buffer of lbm_batch_state_bytes bytes
 * (case i's slice starts at the sum of the earlier cases' lbm_state_bytes).  A
 * device buffer is copied asynchronously on the stream; a host buffer
 * synchronises.  After set_state every case's step count restarts at 0. */
size_t lbm_batch_state_bytes(const lbm_batch* b);
int lbm_batch_get_state(lbm_batch* b, void* buf, size_t bytes, int32_t on_device);
int lbm_batch_set_state(lbm_batch* b, const void* buf, size_t bytes, int32_t on_device);

/* Release the batch (and its graph); workspace and cases stay the caller's. */
void lbm_batch_destroy(lbm_batch* b);

/* Message of the batch's last error; with b == NULL, the calling thread's last
 * lbm_batch_create/lbm_batch_workspace_bytes error. */
const char* lbm_batch_last_error(const lbm_batch* b);

/* Message of the last error on this handle; with h == NULL, the calling thread's
 * last lbm_create/lbm_workspace_bytes error. */
const char* lbm_last_error(const lbm_handle* h);

#ifdef __cplusplus
}
#endif
#endif
