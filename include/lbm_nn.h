/*
 * liblbm -- surrogate network kernels.  Not in the paper (arXiv 2402.15752 has
 * no learned component): a residual CNN of 3x3 convolutions that maps the
 * macroscopic fields (phi, ux, uy, p, c1 + c2) of a lattice to the same fields
 * 16 time steps later, trained on trajectories of the solver itself, which
 * stays the fallback and the judge of the network's error.
 *
 * Tensors (device memory, caller-owned, row-major, 16-byte aligned):
 *   activation  NHWC bfloat16 [batch][h][w][C], C = 16 or 48 channels
 *   state       NHWC float    [batch][h][w][16] (channels 0..4 used, rest zero)
 *   weights     bfloat16 [cout][9][cin], tap t = 3 (dy + 1) + (dx + 1)
 *   bias        float [cout]
 * A 3x3 convolution with dilation d is periodic in both directions (the
 * lattices are periodic):
 *   y[n, i, j, o] = b[o] + sum_{t, c} w[o, t, c] x[n, (i + d dy_t) mod h, (j + d dx_t) mod w, c].
 * Products are formed from bfloat16 operands and accumulated in FP32 on the
 * 5th-generation tensor cores (tcgen05.mma, accumulators in tensor memory).
 * Shapes: w a multiple of 128, 1 <= d <= 8, h a multiple of d, (cin, cout) in
 * {(16, 48), (48, 48), (48, 16)}.  status: a device int32 that the kernels OR
 * bit 0 into if one of their bounded waits on the tensor cores gives up (the
 * result is then incomplete); the caller clears and reads it.  Every call is
 * asynchronous on `stream` (a cudaStream_t, NULL = legacy default) and returns
 * LBM_OK (0), LBM_ERR_ARG (-1) for a bad shape, pointer or alignment, or
 * LBM_ERR_CUDA (-4) if a launch failed.
 */
#ifndef PFLBM_LBM_NN_H
#define PFLBM_LBM_NN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_NN_RELU     0 /* y = max(conv + b, 0), bfloat16 activation                */
#define LBM_NN_RESIDUAL 1 /* y = residual + conv + b, float state (cout = 16)          */
#define LBM_NN_MASK     2 /* y = conv * (mask > 0), bfloat16 (backward through a ReLU) */

/* 3x3 periodic convolution with dilation `dilation` and a fused epilogue (see
 * LBM_NN_*).  residual: float state for LBM_NN_RESIDUAL; mask: bfloat16 activation
 * with cout channels for LBM_NN_MASK (the forward output of the ReLU the gradient
 * flows back through); bias may be NULL for LBM_NN_MASK. */
int lbm_nn_conv3x3(const void* x, int32_t cin, const void* weights, const float* bias,
                   int32_t cout, int32_t epilogue, const float* residual, const void* mask,
                   void* y, int32_t batch, int32_t h, int32_t w, int32_t dilation,
                   int32_t* status, void* stream);

/* Weights of the adjoint convolution: wt[c][t][o] = w[o][8 - t][c], so that the
 * gradient with respect to a convolution's input is lbm_nn_conv3x3 of the
 * output gradient with wt (cin and cout swapped, the same dilation). */
int lbm_nn_flip_weights(const void* w, int32_t cin, int32_t cout, void* wt, void* stream);

/* Weight gradient dw[o][t][c] = sum_{n,i,j} dy[n,i,j,o] x[n,(i+d dy_t),(j+d dx_t),c]
 * (float, overwritten), one partial per CTA reduced in a fixed order through
 * `partials` (lbm_nn_wgrad_partial_bytes bytes of device scratch, which depends
 * on the current device's SM count): deterministic. */
size_t lbm_nn_wgrad_partial_bytes(int32_t cin, int32_t cout, int32_t batch, int32_t h, int32_t w,
                                  int32_t dilation);
int lbm_nn_conv3x3_wgrad(const void* x, int32_t cin, const void* dy, int32_t cout, float* dw,
                         void* partials, size_t partial_bytes, int32_t batch, int32_t h,
                         int32_t w, int32_t dilation, int32_t* status, void* stream);

/* Bias gradient db[o] = sum over pixels of dy[., o] (float, overwritten), fixed
 * order through `partials` (>= 1024 * cout floats). */
int lbm_nn_bias_grad(const void* dy, int32_t cout, int64_t pixels, float* db, float* partials,
                     void* stream);

/* Mean squared error over the first `used` channels of two float states and its
 * gradient with respect to `pred`, as a bfloat16 activation of 16 channels
 * (zero beyond `used`): dpred = 2 (pred - target) / (pixels * used).
 * loss_partials: >= 1024 doubles of scratch; *loss (device double) receives the
 * mean.  dpred may be NULL (loss only). */
int lbm_nn_mse(const float* pred, const float* target, int32_t used, int64_t pixels, void* dpred,
               double* loss_partials, double* loss, void* stream);

/* One Adam step (Kingma & Ba 2015) on n float parameters with float moments m, v:
 * step number t >= 1, bias-corrected.  Entries whose mask byte is 0 stay zero
 * (channel padding).  If wbf16 is not NULL it receives the updated parameters
 * rounded to bfloat16 (the copy the convolutions read). */
int lbm_nn_adam(float* param, const float* grad, float* m, float* v, const uint8_t* mask,
                void* wbf16, int64_t n, float lr, float beta1, float beta2, float eps,
                int32_t t, void* stream);

/* Fields -> network state: from `fields`, six float planes [6][h][w] per sample
 * (phi, ux, uy, p, c1, c2, as lbm_get_fields writes them), batch samples back to
 * back, to a float state of the five network channels (phi, ux, uy, p, C = c1 + c2)
 * s = (f - shift) * scale (per channel; channels 5..15 zero) and, if act is not
 * NULL, its bfloat16 copy with 16 channels. */
int lbm_nn_pack(const float* fields, int32_t batch, int32_t h, int32_t w, const float* shift,
                const float* scale, float* state, void* act, void* stream);

/* Network state -> fields: f = s / scale + shift, five float planes per sample. */
int lbm_nn_unpack(const float* state, int32_t batch, int32_t h, int32_t w, const float* shift,
                  const float* scale, float* fields, void* stream);

/* Network state -> the six fields of a solver restart (lbm_init_macros), double
 * planes [6][h][w] per sample: phi, ux, uy, p, and C split between the phases at
 * the Henry equilibrium c1 / phi = K c2 / (1 - phi) with the sample's keq[n]. */
int lbm_nn_unpack_macros(const float* state, int32_t batch, int32_t h, int32_t w, const float* shift,
                         const float* scale, const float* keq, double* macros, void* stream);

/* Distance between two float states, per sample n and channel c < 5:
 * out[2 (5 n + c)] = max over pixels |a - b|, out[2 (5 n + c) + 1] = RMS of a - b
 * (pixels per sample; partials: >= 640 * batch floats of scratch). */
int lbm_nn_state_diff(const float* a, const float* b, int32_t batch, int64_t pixels, float* partials,
                      float* out, void* stream);

/* Add independent Gaussian noise of standard deviation sigma to the first `used`
 * channels of a float state of `pixels` pixels (training-time input corruption);
 * the draws are a deterministic function of (seed, element). */
int lbm_nn_add_noise(float* state, int64_t pixels, int32_t used, float sigma, uint32_t seed,
                     void* stream);

/* Float state -> bfloat16 activation of 16 channels. */
int lbm_nn_to_bf16(const float* state, int64_t values, void* act, void* stream);

/* bfloat16 values -> float (e.g. a loss gradient joining a float residual path). */
int lbm_nn_to_f32(const void* act, int64_t values, float* state, void* stream);

/* y += a x over n floats (gradient accumulation across unrolled hops). */
int lbm_nn_axpy(float* y, const float* x, float a, int64_t n, void* stream);

#ifdef __cplusplus
}
#endif
#endif
