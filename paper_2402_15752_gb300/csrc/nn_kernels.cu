// Surrogate network kernels (include/lbm_nn.h) other than the convolutions
// (nn_conv.cu): weight flipping, bias gradient, the MSE loss, Adam, and the
// packing between solver fields and network states.
#include "lbm.h"
#include "lbm_nn.h"
#include "nn_internal.h"

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

namespace {

// ---------------------------------------------------------------- helpers --
int launch_status() {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

// -------------------------------------------------------- small kernels --
__global__ void flip_kernel(const __nv_bfloat16* __restrict__ w, int CI, int CO, __nv_bfloat16* __restrict__ wt) {
    const int n = 9 * CI * CO;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int o = i % CO, t = (i / CO) % 9, c = i / (9 * CO);  // wt[c][t][o]
        wt[i] = w[((size_t)o * 9 + (8 - t)) * CI + c];
    }
}

constexpr int RED_BLOCKS = 1024;

__global__ void bias_grad_partials(const __nv_bfloat16* __restrict__ dy, int CO, long long P, float* __restrict__ part) {
    __shared__ float s[256];
    // thread i takes channel i % CO of pixels i / CO, i / CO + rows, ...
    const int rows = blockDim.x / CO;
    float a = 0.0f;
    const int o = threadIdx.x % CO, r = threadIdx.x / CO;
    if (r < rows)
        for (long long p = (long long)blockIdx.x * rows + r; p < P; p += (long long)gridDim.x * rows)
            a += __bfloat162float(dy[p * CO + o]);
    s[threadIdx.x] = r < rows ? a : 0.0f;
    __syncthreads();
    if (threadIdx.x < CO) {
        float t = 0.0f;
        for (int k = 0; k < rows; ++k) t += s[k * CO + threadIdx.x];
        part[(size_t)blockIdx.x * CO + threadIdx.x] = t;
    }
}

__global__ void sum_partials(const float* __restrict__ part, int nb, int CO, float* __restrict__ out) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= CO) return;
    float t = 0.0f;
    for (int b = 0; b < nb; ++b) t += part[(size_t)b * CO + o];
    out[o] = t;
}

__global__ void mse_partials(const float* __restrict__ pred, const float* __restrict__ target, int U, long long P,
                             __nv_bfloat16* __restrict__ dpred, double* __restrict__ part) {
    __shared__ double s[256];
    const double inv = 1.0 / ((double)P * U);
    double a = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P * 16; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % 16);
        const double d = c < U ? (double)pred[i] - (double)target[i] : 0.0;
        a += d * d;
        if (dpred) dpred[i] = __float2bfloat16_rn((float)(2.0 * inv * d));
    }
    s[threadIdx.x] = a;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0] * inv;
}

__global__ void mse_final(const double* __restrict__ part, int nb, double* __restrict__ loss) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < nb; ++b) t += part[b];
        *loss = t;
    }
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                            const uint8_t* __restrict__ mask, __nv_bfloat16* __restrict__ wb, long long n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float val = 0.0f;
        if (!mask || mask[i]) {
            const float gi = g[i];
            const float mi = b1 * m[i] + (1.0f - b1) * gi;
            const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
            m[i] = mi;
            v[i] = vi;
            val = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        }
        p[i] = val;
        if (wb) wb[i] = __float2bfloat16_rn(val);
    }
}

__global__ void pack_kernel(const float* __restrict__ fields, int B, int H, int W, const float* __restrict__ shift,
                            const float* __restrict__ scale, float* __restrict__ state, __nv_bfloat16* __restrict__ act) {
    const long long HW = (long long)H * W, P = B * HW;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P * 16; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % 16);
        const long long p = i / 16, n = p / HW, q = p % HW;
        const float* f = fields + n * 6 * HW + q;  // phi, ux, uy, p, c1, c2
        float v = 0.0f;
        if (c < 4) v = (f[c * HW] - shift[c]) * scale[c];
        else if (c == 4) v = ((f[4 * HW] + f[5 * HW]) - shift[4]) * scale[4];
        state[i] = v;
        if (act) act[i] = __float2bfloat16_rn(v);
    }
}

// State -> the six fields of a solver restart, in double: phi, u, p as they
// are, and c1 + c2 = C split between the phases at the Henry equilibrium
// c1 / phi = K c2 / (1 - phi) (phi clipped to [0, 1]).
__global__ void unpack_macros_kernel(const float* __restrict__ state, int B, int H, int W,
                                     const float* __restrict__ shift, const float* __restrict__ scale,
                                     const float* __restrict__ keq, double* __restrict__ out) {
    const long long HW = (long long)H * W, P = B * HW;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (long long)gridDim.x * blockDim.x) {
        const long long n = i / HW, q = i % HW;
        const float* s = state + i * 16;
        double f[5];
        for (int c = 0; c < 5; ++c) f[c] = (double)(s[c] / scale[c] + shift[c]);
        const double ph = f[0] < 0.0 ? 0.0 : (f[0] > 1.0 ? 1.0 : f[0]);
        const double K = keq[n], den = K * ph + (1.0 - ph);
        double* o = out + n * 6 * HW + q;
        o[0] = f[0];
        o[HW] = f[1];
        o[2 * HW] = f[2];
        o[3 * HW] = f[3];
        o[4 * HW] = f[4] * K * ph / den;
        o[5 * HW] = f[4] * (1.0 - ph) / den;
    }
}

__global__ void unpack_kernel(const float* __restrict__ state, int B, int H, int W, const float* __restrict__ shift,
                              const float* __restrict__ scale, float* __restrict__ fields) {
    const long long HW = (long long)H * W, P = B * HW;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P * 5; i += (long long)gridDim.x * blockDim.x) {
        const long long q = i % HW, c = (i / HW) % 5, n = i / (5 * HW);
        fields[i] = state[(n * HW + q) * 16 + c] / scale[c] + shift[c];
    }
}

// Per sample and channel (first 5): max |a - b| and sum (a - b)^2 over pixels.
__global__ void state_diff_kernel(const float* __restrict__ a, const float* __restrict__ b, long long HW,
                                  float* __restrict__ out) {
    __shared__ float smax[5][256];
    __shared__ double ssum[5][256];
    const int n = blockIdx.y;
    float mx[5] = {0, 0, 0, 0, 0};
    double sm[5] = {0, 0, 0, 0, 0};
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < HW; q += (long long)gridDim.x * blockDim.x) {
        const long long i = ((long long)n * HW + q) * 16;
        for (int c = 0; c < 5; ++c) {
            const float d = a[i + c] - b[i + c];
            mx[c] = fmaxf(mx[c], fabsf(d));
            sm[c] += (double)d * d;
        }
    }
    for (int c = 0; c < 5; ++c) { smax[c][threadIdx.x] = mx[c]; ssum[c][threadIdx.x] = sm[c]; }
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k)
            for (int c = 0; c < 5; ++c) {
                smax[c][threadIdx.x] = fmaxf(smax[c][threadIdx.x], smax[c][threadIdx.x + k]);
                ssum[c][threadIdx.x] += ssum[c][threadIdx.x + k];
            }
        __syncthreads();
    }
    if (threadIdx.x < 5) {
        // one block column per sample: partials [n][block][c][2]
        float* o = out + (((size_t)n * gridDim.x + blockIdx.x) * 5 + threadIdx.x) * 2;
        o[0] = smax[threadIdx.x][0];
        o[1] = (float)ssum[threadIdx.x][0];
    }
}

__global__ void state_diff_final(const float* __restrict__ part, int nblk, long long HW, float* __restrict__ out) {
    const int n = blockIdx.x, c = threadIdx.x;
    if (c >= 5) return;
    float mx = 0.0f;
    double sm = 0.0;
    for (int b = 0; b < nblk; ++b) {
        const float* o = part + (((size_t)n * nblk + b) * 5 + c) * 2;
        mx = fmaxf(mx, o[0]);
        sm += o[1];
    }
    out[((size_t)n * 5 + c) * 2] = mx;
    out[((size_t)n * 5 + c) * 2 + 1] = (float)sqrt(sm / (double)HW);
}

// Gaussian noise on the first `used` channels of a float state: Box-Muller
// (1958) on two uniforms from a counter-based hash (the MurmurHash3 32-bit
// finalizer) of (seed, element index): reproducible for a given seed.
__device__ __forceinline__ uint32_t nn_mix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

__global__ void add_noise_kernel(float* __restrict__ s, long long P, int used, float sigma, uint32_t seed) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P * used;
         i += (long long)gridDim.x * blockDim.x) {
        const long long p = i / used;
        const int c = (int)(i % used);
        const uint32_t k = nn_mix32(seed ^ nn_mix32((uint32_t)i ^ (uint32_t)(i >> 32) * 0x9e3779b9u));
        const float u1 = ((float)(k >> 8) + 1.0f) * 0x1p-24f;  // (0, 1]
        const float u2 = (float)(nn_mix32(k + 0x68e31da4u) >> 8) * 0x1p-24f;
        s[p * 16 + c] += sigma * sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
    }
}

__global__ void to_f32_kernel(const __nv_bfloat16* __restrict__ a, long long n, float* __restrict__ s) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s[i] = __bfloat162float(a[i]);
}

__global__ void axpy_kernel(float* __restrict__ y, const float* __restrict__ x, float a, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] += a * x[i];
}

__global__ void to_bf16_kernel(const float* __restrict__ s, long long n, __nv_bfloat16* __restrict__ a) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a[i] = __float2bfloat16_rn(s[i]);
}

int grid_for(long long n, int threads) { return (int)std::max<long long>(1, std::min<long long>((n + threads - 1) / threads, 152LL * 16)); }

}  // namespace

extern "C" {

int lbm_nn_flip_weights(const void* w, int32_t cin, int32_t cout, void* wt, void* stream) {
    if (!w || !wt || cin < 1 || cout < 1) return LBM_ERR_ARG;
    const int n = 9 * cin * cout;
    flip_kernel<<<grid_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const __nv_bfloat16*>(w), cin, cout, static_cast<__nv_bfloat16*>(wt));
    return launch_status();
}

int lbm_nn_bias_grad(const void* dy, int32_t cout, int64_t pixels, float* db, float* partials, void* stream) {
    if (!dy || !db || !partials || (cout != 16 && cout != 48) || pixels < 1) return LBM_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int threads = cout == 16 ? 256 : 240;  // a whole number of pixels per pass
    bias_grad_partials<<<RED_BLOCKS, threads, 0, s>>>(static_cast<const __nv_bfloat16*>(dy), cout, pixels, partials);
    sum_partials<<<1, 64, 0, s>>>(partials, RED_BLOCKS, cout, db);
    return launch_status();
}

int lbm_nn_mse(const float* pred, const float* target, int32_t used, int64_t pixels, void* dpred, double* loss_partials,
               double* loss, void* stream) {
    if (!pred || !target || !loss_partials || !loss || used < 1 || used > 16 || pixels < 1) return LBM_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    mse_partials<<<RED_BLOCKS, 256, 0, s>>>(pred, target, used, pixels, static_cast<__nv_bfloat16*>(dpred), loss_partials);
    mse_final<<<1, 32, 0, s>>>(loss_partials, RED_BLOCKS, loss);
    return launch_status();
}

int lbm_nn_adam(float* param, const float* grad, float* m, float* v, const uint8_t* mask, void* wbf16, int64_t n,
                float lr, float beta1, float beta2, float eps, int32_t t, void* stream) {
    if (!param || !grad || !m || !v || n < 1 || t < 1) return LBM_ERR_ARG;
    const float c1 = 1.0f - powf(beta1, (float)t), c2 = 1.0f - powf(beta2, (float)t);
    adam_kernel<<<grid_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        param, grad, m, v, mask, static_cast<__nv_bfloat16*>(wbf16), n, lr, beta1, beta2, eps, c1, c2);
    return launch_status();
}

int lbm_nn_pack(const float* fields, int32_t batch, int32_t h, int32_t w, const float* shift, const float* scale,
                float* state, void* act, void* stream) {
    if (!fields || !shift || !scale || !state || batch < 1 || h < 1 || w < 1) return LBM_ERR_ARG;
    const long long n = (long long)batch * h * w * 16;
    pack_kernel<<<grid_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        fields, batch, h, w, shift, scale, state, static_cast<__nv_bfloat16*>(act));
    return launch_status();
}

int lbm_nn_unpack(const float* state, int32_t batch, int32_t h, int32_t w, const float* shift, const float* scale,
                  float* fields, void* stream) {
    if (!state || !shift || !scale || !fields || batch < 1 || h < 1 || w < 1) return LBM_ERR_ARG;
    const long long n = (long long)batch * h * w * 5;
    unpack_kernel<<<grid_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(state, batch, h, w, shift, scale, fields);
    return launch_status();
}

int lbm_nn_unpack_macros(const float* state, int32_t batch, int32_t h, int32_t w, const float* shift,
                         const float* scale, const float* keq, double* macros, void* stream) {
    if (!state || !shift || !scale || !keq || !macros || batch < 1 || h < 1 || w < 1) return LBM_ERR_ARG;
    const long long n = (long long)batch * h * w;
    unpack_macros_kernel<<<grid_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        state, batch, h, w, shift, scale, keq, macros);
    return launch_status();
}

int lbm_nn_state_diff(const float* a, const float* b, int32_t batch, int64_t pixels, float* partials, float* out,
                      void* stream) {
    if (!a || !b || !partials || !out || batch < 1 || pixels < 1) return LBM_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    constexpr int NBLK = 64;
    state_diff_kernel<<<dim3(NBLK, batch), 256, 0, s>>>(a, b, pixels, partials);
    state_diff_final<<<batch, 32, 0, s>>>(partials, NBLK, pixels, out);
    return launch_status();
}

int lbm_nn_add_noise(float* state, int64_t pixels, int32_t used, float sigma, uint32_t seed, void* stream) {
    if (!state || pixels < 1 || used < 1 || used > 16) return LBM_ERR_ARG;
    const long long n = (long long)pixels * used;
    add_noise_kernel<<<grid_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(state, pixels, used, sigma, seed);
    return launch_status();
}

int lbm_nn_to_bf16(const float* state, int64_t values, void* act, void* stream) {
    if (!state || !act || values < 1) return LBM_ERR_ARG;
    to_bf16_kernel<<<grid_for(values, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        state, values, static_cast<__nv_bfloat16*>(act));
    return launch_status();
}

int lbm_nn_to_f32(const void* act, int64_t values, float* state, void* stream) {
    if (!state || !act || values < 1) return LBM_ERR_ARG;
    to_f32_kernel<<<grid_for(values, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const __nv_bfloat16*>(act), values, state);
    return launch_status();
}

int lbm_nn_axpy(float* y, const float* x, float a, int64_t n, void* stream) {
    if (!y || !x || n < 1) return LBM_ERR_ARG;
    axpy_kernel<<<grid_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(y, x, a, n);
    return launch_status();
}

}  // extern "C"
