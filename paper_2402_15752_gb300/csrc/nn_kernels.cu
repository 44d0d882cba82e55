// Surrogate network kernels (include/lbm_nn.h): periodic 3x3 convolutions on
// NHWC bfloat16 activations with FP32 accumulation on the tensor cores
// (mma.sync m16n8k16), their weight and bias gradients, the MSE loss, Adam, and
// the packing between solver fields and network states.
#include "lbm.h"
#include "lbm_nn.h"

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

namespace {

// ---------------------------------------------------------------- helpers --
__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Four 8x8 bfloat16 matrices from shared memory, one row address per lane
// (lanes 8m .. 8m+7 give the rows of matrix m): thread t receives row t/4,
// columns 2(t%4) and 2(t%4)+1 of each matrix -- the mma.m16n8k16 fragment layout.
__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], const uint32_t* row_addr) {
    const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(row_addr));
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x = lo -> low 16 bits
    return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
    return sms;
}

int launch_status() {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

// ---------------------------------------------------- forward convolution --
// A CTA of 4 warps computes an 8-row x 16-pixel output tile of one sample for
// all cout channels; warp w owns rows 2w and 2w+1 (two m16 tiles sharing every
// weight fragment).  GEMM view: M = pixels, N = cout, K = 9 taps x cin.  The
// weights (all of them) and the tile's input with a one-pixel periodic halo are
// staged in shared memory; rows are padded by 4 words so that the fragment loads
// are free of bank conflicts.  Persistent CTAs loop over the tiles; the input of
// the next tile is copied asynchronously (cp.async, two buffers) while the
// current one is computed, so that the tensor cores do not wait for it.
constexpr int CONV_THREADS = 128;
constexpr int TROWS = 8, TCOLS = 16;

template <int CI>
constexpr int in_words() { return CI / 2 + 4; }
template <int CI>
constexpr int w_words() { return 9 * CI / 2 + 4; }
template <int CI>
constexpr int tile_words() { return (TROWS + 2) * (TCOLS + 2) * in_words<CI>(); }
template <int CI, int CO>
constexpr size_t conv_smem() {
    return sizeof(uint32_t) * ((size_t)CO * w_words<CI>() + 2 * (size_t)tile_words<CI>());
}

__device__ __forceinline__ void cp_async16(uint32_t* dst, const uint32_t* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(
                     static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <int CI, int CO, int EPI>
__global__ void __launch_bounds__(CONV_THREADS)
    conv3x3_kernel(const uint32_t* __restrict__ x, const uint32_t* __restrict__ w, const float* __restrict__ bias,
                   void* __restrict__ y, const float* __restrict__ res, const uint32_t* __restrict__ mask,
                   int B, int H, int W) {
    extern __shared__ __align__(16) uint32_t smem[];
    static_assert(CI % 16 == 0 && CO % 16 == 0, "k steps of 16 and pairs of n tiles");
    constexpr int IW = in_words<CI>(), WW = w_words<CI>(), CW = CI / 2, KW = 9 * CI / 2;
    constexpr int TW = tile_words<CI>(), CH = CW / 4;  // 16-byte chunks per pixel
    static_assert(CW % 4 == 0 && IW % 4 == 0, "16-byte pixel rows");
    uint32_t* s_w = smem;
    for (int i = threadIdx.x; i < CO * KW; i += CONV_THREADS) s_w[(i / KW) * WW + (i % KW)] = w[i];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tig = lane & 3;
    const int tiles_y = H / TROWS, tiles_x = W / TCOLS;
    const long long ntiles = (long long)B * tiles_y * tiles_x;
    // the input of a tile (with its periodic halo) into buffer b, asynchronously
    auto load_tile = [&](long long tile, int b) {
        const int tx = (int)(tile % tiles_x);
        const long long r = tile / tiles_x;
        const int ty = (int)(r % tiles_y), n = (int)(r / tiles_y);
        const int y0 = ty * TROWS, x0 = tx * TCOLS;
        uint32_t* dst = smem + CO * WW + b * TW;
        for (int i = threadIdx.x; i < (TROWS + 2) * (TCOLS + 2) * CH; i += CONV_THREADS) {
            const int c = i % CH, p = i / CH, col = p % (TCOLS + 2), row = p / (TCOLS + 2);
            const int yy = wrap(y0 - 1 + row, H), xx = wrap(x0 - 1 + col, W);
            cp_async16(dst + p * IW + 4 * c, x + (((long long)n * H + yy) * W + xx) * CW + 4 * c);
        }
        cp_async_commit();
    };
    if (blockIdx.x < ntiles) load_tile(blockIdx.x, 0);
    int buf = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, buf ^= 1) {
        const int tx = (int)(tile % tiles_x);
        const long long r = tile / tiles_x;
        const int ty = (int)(r % tiles_y), n = (int)(r / tiles_y);
        const int y0 = ty * TROWS, x0 = tx * TCOLS;
        // the other buffer was last read in the previous iteration, which every
        // thread has finished (barrier at its end): start the next tile's copy
        if (tile + gridDim.x < ntiles) {
            load_tile(tile + gridDim.x, buf ^ 1);
            cp_async_wait<1>();  // this tile's copy (all but the newest group)
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();  // this tile's input (and, the first time, the weights) visible
        const uint32_t* s_in = smem + CO * WW + buf * TW;

        float acc[2][CO / 8][4];
#pragma unroll
        for (int m = 0; m < 2; ++m)
#pragma unroll
            for (int j = 0; j < CO / 8; ++j)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[m][j][q] = 0.0f;

        // ldmatrix row addresses: lane l serves matrix l / 8, row l % 8.
        //   A (pixels x channels): matrix m covers pixels 8 (m & 1) .. +7 and
        //   channels 8 (m >> 1) .. +7 of the k16 step;
        //   B (couts x k, k contiguous): matrices 2q, 2q+1 cover couts
        //   8 (j + q) .. +7 with k 0..7 and 8..15, for n tiles j, j + 1.
        const int lm = lane >> 3, lr = lane & 7;
        const int a_pix = lr + 8 * (lm & 1), a_kw = 4 * (lm >> 1);
        const int b_n = lr + 8 * (lm >> 1), b_kw = 4 * (lm & 1);
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int dy = t / 3 - 1, dx = t % 3 - 1;
#pragma unroll
            for (int c0 = 0; c0 < CI; c0 += 16) {
                uint32_t a[2][4];
#pragma unroll
                for (int m = 0; m < 2; ++m)
                    ldmatrix_x4(a[m], s_in + ((2 * warp + m + dy + 1) * (TCOLS + 2) + a_pix + dx + 1) * IW +
                                          c0 / 2 + a_kw);
                const int kw = (t * CI + c0) / 2;
#pragma unroll
                for (int j = 0; j < CO / 8; j += 2) {
                    uint32_t bq[4];
                    ldmatrix_x4(bq, s_w + (j * 8 + b_n) * WW + kw + b_kw);
                    const uint32_t b0[2] = {bq[0], bq[1]}, b1[2] = {bq[2], bq[3]};
                    mma_bf16_16816(acc[0][j], a[0], b0);
                    mma_bf16_16816(acc[1][j], a[1], b0);
                    mma_bf16_16816(acc[0][j + 1], a[0], b1);
                    mma_bf16_16816(acc[1][j + 1], a[1], b1);
                }
            }
        }

#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const long long pa = ((long long)n * H + y0 + 2 * warp + m) * W + x0 + g;  // rows g, g + 8
#pragma unroll
            for (int j = 0; j < CO / 8; ++j) {
                const int ch = j * 8 + 2 * tig;
                const float b0 = (EPI != LBM_NN_MASK && bias) ? bias[ch] : 0.0f;
                const float b1 = (EPI != LBM_NN_MASK && bias) ? bias[ch + 1] : 0.0f;
#pragma unroll
                for (int h2 = 0; h2 < 2; ++h2) {
                    const long long p = pa + 8 * h2;
                    float v0 = acc[m][j][2 * h2] + b0, v1 = acc[m][j][2 * h2 + 1] + b1;
                    if constexpr (EPI == LBM_NN_RELU) {
                        static_cast<uint32_t*>(y)[(p * CO + ch) / 2] = pack_bf16x2(fmaxf(v0, 0.0f), fmaxf(v1, 0.0f));
                    } else if constexpr (EPI == LBM_NN_RESIDUAL) {
                        float* yo = static_cast<float*>(y) + p * CO + ch;
                        const float* ro = res + p * CO + ch;
                        yo[0] = ro[0] + v0;
                        yo[1] = ro[1] + v1;
                    } else {
                        const uint32_t mk = mask[(p * CO + ch) / 2];
                        v0 = bf16_lo(mk) > 0.0f ? v0 : 0.0f;
                        v1 = bf16_hi(mk) > 0.0f ? v1 : 0.0f;
                        static_cast<uint32_t*>(y)[(p * CO + ch) / 2] = pack_bf16x2(v0, v1);
                    }
                }
            }
        }
        __syncthreads();  // every warp is done with buffer `buf` before it is refilled
    }
}

template <int CI, int CO, int EPI>
int conv_launch(const void* x, const void* w, const float* bias, void* y, const float* res, const void* mask,
                int B, int H, int W, cudaStream_t s) {
    auto k = conv3x3_kernel<CI, CO, EPI>;
    constexpr size_t smem = conv_smem<CI, CO>();
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return LBM_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, CONV_THREADS, smem) != cudaSuccess || per_sm < 1)
        return LBM_ERR_CUDA;
    const long long tiles = (long long)B * (H / TROWS) * (W / TCOLS);
    const int grid = (int)std::min<long long>(tiles, (long long)per_sm * sm_count());
    k<<<grid, CONV_THREADS, smem, s>>>(static_cast<const uint32_t*>(x), static_cast<const uint32_t*>(w), bias, y,
                                       res, static_cast<const uint32_t*>(mask), B, H, W);
    return launch_status();
}

// ------------------------------------------------------- weight gradient --
// dw[o][t][c] = sum_p dy[p][o] x[p + off_t][c].  GEMM view per tap t:
// M = cout, N = cin, K = pixels.  blockIdx.y = tap; blockIdx.x strides over
// chunks of 64 pixels; the 4 warps take 16 pixels each.  Both operands are
// staged as pixel pairs (two consecutive pixels of one channel per word), the
// K-pair layout of the mma fragments.  The warps' sums are added in a fixed
// order, and every CTA writes its own partial (no atomics): deterministic.
constexpr int WG_THREADS = 128;
constexpr int WG_CHUNK = 64;

template <int CI, int CO>
__global__ void __launch_bounds__(WG_THREADS)
    wgrad_kernel(const uint32_t* __restrict__ x, const uint32_t* __restrict__ dy, float* __restrict__ partials,
                 int B, int H, int W) {
    constexpr int DW = CO + 8, XW = CI + 8;
    __shared__ uint32_t s_dy[WG_CHUNK / 2][DW];
    __shared__ uint32_t s_x[WG_CHUNK / 2][XW];
    __shared__ float s_red[CO][CI];
    const int t = blockIdx.y, oy = t / 3 - 1, ox = t % 3 - 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tig = lane & 3;
    const long long P = (long long)B * H * W, nchunks = P / WG_CHUNK;

    float acc[CO / 16][CI / 8][4];
#pragma unroll
    for (int mi = 0; mi < CO / 16; ++mi)
#pragma unroll
        for (int nj = 0; nj < CI / 8; ++nj)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[mi][nj][q] = 0.0f;

    for (long long chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
        const long long p0 = chunk * WG_CHUNK;
        __syncthreads();
        for (int i = threadIdx.x; i < (WG_CHUNK / 2) * (CO / 2); i += WG_THREADS) {
            const int q = i / (CO / 2), cp = i % (CO / 2);
            const uint32_t we = dy[(p0 + 2 * q) * (CO / 2) + cp], wo = dy[(p0 + 2 * q + 1) * (CO / 2) + cp];
            s_dy[q][2 * cp] = __byte_perm(we, wo, 0x5410);
            s_dy[q][2 * cp + 1] = __byte_perm(we, wo, 0x7632);
        }
        for (int i = threadIdx.x; i < (WG_CHUNK / 2) * (CI / 2); i += WG_THREADS) {
            const int q = i / (CI / 2), cp = i % (CI / 2);
            uint32_t wv[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const long long p = p0 + 2 * q + e;
                const int xx = (int)(p % W);
                const long long rr = p / W;
                const int yy = (int)(rr % H), n = (int)(rr / H);
                const long long src = ((long long)n * H + wrap(yy + oy, H)) * W + wrap(xx + ox, W);
                wv[e] = x[src * (CI / 2) + cp];
            }
            s_x[q][2 * cp] = __byte_perm(wv[0], wv[1], 0x5410);
            s_x[q][2 * cp + 1] = __byte_perm(wv[0], wv[1], 0x7632);
        }
        __syncthreads();
        const int qa = 8 * warp + tig, qb = 8 * warp + 4 + tig;  // pixel pairs of this warp's k16 step
#pragma unroll
        for (int mi = 0; mi < CO / 16; ++mi) {
            const uint32_t a[4] = {s_dy[qa][mi * 16 + g], s_dy[qa][mi * 16 + g + 8], s_dy[qb][mi * 16 + g],
                                   s_dy[qb][mi * 16 + g + 8]};
#pragma unroll
            for (int nj = 0; nj < CI / 8; ++nj) {
                const uint32_t b[2] = {s_x[qa][nj * 8 + g], s_x[qb][nj * 8 + g]};
                mma_bf16_16816(acc[mi][nj], a, b);
            }
        }
    }
    // fixed-order sum of the 4 warps, then one partial per CTA and tap
    for (int i = threadIdx.x; i < CO * CI; i += WG_THREADS) (&s_red[0][0])[i] = 0.0f;
    for (int wv = 0; wv < WG_THREADS / 32; ++wv) {
        __syncthreads();
        if (warp == wv) {
#pragma unroll
            for (int mi = 0; mi < CO / 16; ++mi)
#pragma unroll
                for (int nj = 0; nj < CI / 8; ++nj) {
                    const int o = mi * 16 + g, c = nj * 8 + 2 * tig;
                    s_red[o][c] += acc[mi][nj][0];
                    s_red[o][c + 1] += acc[mi][nj][1];
                    s_red[o + 8][c] += acc[mi][nj][2];
                    s_red[o + 8][c + 1] += acc[mi][nj][3];
                }
        }
    }
    __syncthreads();
    float* out = partials + ((size_t)blockIdx.x * 9 + t) * CO * CI;
    for (int i = threadIdx.x; i < CO * CI; i += WG_THREADS) out[i] = (&s_red[0][0])[i];
}

// dw[o][t][c] = sum_b partials[b][t][o][c]
__global__ void wgrad_reduce_kernel(const float* __restrict__ partials, int nb, int CO, int CI, float* __restrict__ dw) {
    const int n = 9 * CO * CI;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int c = i % CI, o = (i / CI) % CO, t = i / (CI * CO);
        float s = 0.0f;
        for (int b = 0; b < nb; ++b) s += partials[((size_t)b * 9 + t) * CO * CI + (size_t)o * CI + c];
        dw[((size_t)o * 9 + t) * CI + c] = s;
    }
}

constexpr int WG_GRID_X = 64;

template <int CI, int CO>
int wgrad_launch(const void* x, const void* dy, float* dw, float* part, int B, int H, int W, cudaStream_t s) {
    const long long nchunks = (long long)B * H * W / WG_CHUNK;
    const int gx = (int)std::min<long long>(WG_GRID_X, nchunks);
    wgrad_kernel<CI, CO><<<dim3(gx, 9), WG_THREADS, 0, s>>>(static_cast<const uint32_t*>(x),
                                                             static_cast<const uint32_t*>(dy), part, B, H, W);
    wgrad_reduce_kernel<<<64, 256, 0, s>>>(part, gx, CO, CI, dw);
    return launch_status();
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

__global__ void to_bf16_kernel(const float* __restrict__ s, long long n, __nv_bfloat16* __restrict__ a) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a[i] = __float2bfloat16_rn(s[i]);
}

bool conv_shape_ok(int B, int H, int W) { return B >= 1 && H >= TROWS && W >= TCOLS && H % TROWS == 0 && W % TCOLS == 0; }

int grid_for(long long n, int threads) { return (int)std::max<long long>(1, std::min<long long>((n + threads - 1) / threads, 152LL * 16)); }

}  // namespace

extern "C" {

int lbm_nn_conv3x3(const void* x, int32_t cin, const void* weights, const float* bias, int32_t cout, int32_t epilogue,
                   const float* residual, const void* mask, void* y, int32_t batch, int32_t h, int32_t w, void* stream) {
    if (!x || !weights || !y || !conv_shape_ok(batch, h, w)) return LBM_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (epilogue == LBM_NN_RELU) {
        if (cin == 16 && cout == 48) return conv_launch<16, 48, LBM_NN_RELU>(x, weights, bias, y, nullptr, nullptr, batch, h, w, s);
        if (cin == 48 && cout == 48) return conv_launch<48, 48, LBM_NN_RELU>(x, weights, bias, y, nullptr, nullptr, batch, h, w, s);
    } else if (epilogue == LBM_NN_RESIDUAL) {
        if (!residual) return LBM_ERR_ARG;
        if (cin == 48 && cout == 16) return conv_launch<48, 16, LBM_NN_RESIDUAL>(x, weights, bias, y, residual, nullptr, batch, h, w, s);
    } else if (epilogue == LBM_NN_MASK) {
        if (!mask) return LBM_ERR_ARG;
        if (cin == 48 && cout == 48) return conv_launch<48, 48, LBM_NN_MASK>(x, weights, nullptr, y, nullptr, mask, batch, h, w, s);
        if (cin == 16 && cout == 48) return conv_launch<16, 48, LBM_NN_MASK>(x, weights, nullptr, y, nullptr, mask, batch, h, w, s);
    }
    return LBM_ERR_ARG;
}

int lbm_nn_flip_weights(const void* w, int32_t cin, int32_t cout, void* wt, void* stream) {
    if (!w || !wt || cin < 1 || cout < 1) return LBM_ERR_ARG;
    const int n = 9 * cin * cout;
    flip_kernel<<<grid_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const __nv_bfloat16*>(w), cin, cout, static_cast<__nv_bfloat16*>(wt));
    return launch_status();
}

size_t lbm_nn_wgrad_partial_bytes(int32_t cin, int32_t cout, int32_t batch, int32_t h, int32_t w) {
    if (!conv_shape_ok(batch, h, w) || cin < 1 || cout < 1) return 0;
    const long long nchunks = (long long)batch * h * w / WG_CHUNK;
    return (size_t)std::min<long long>(WG_GRID_X, nchunks) * 9 * cin * cout * sizeof(float);
}

int lbm_nn_conv3x3_wgrad(const void* x, int32_t cin, const void* dy, int32_t cout, float* dw, void* partials,
                         size_t partial_bytes, int32_t batch, int32_t h, int32_t w, void* stream) {
    if (!x || !dy || !dw || !partials || !conv_shape_ok(batch, h, w)) return LBM_ERR_ARG;
    if (partial_bytes < lbm_nn_wgrad_partial_bytes(cin, cout, batch, h, w)) return LBM_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float* part = static_cast<float*>(partials);
    if (cin == 16 && cout == 48) return wgrad_launch<16, 48>(x, dy, dw, part, batch, h, w, s);
    if (cin == 48 && cout == 48) return wgrad_launch<48, 48>(x, dy, dw, part, batch, h, w, s);
    if (cin == 48 && cout == 16) return wgrad_launch<48, 16>(x, dy, dw, part, batch, h, w, s);
    return LBM_ERR_ARG;
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

}  // extern "C"
