// lbm_conserved_noalloc: conserved sums of a device-resident state with no
// allocation at all.  The reduction's scratch (one partial per chunk of nodes
// plus the two totals) lives in a file-scope __device__ array instead of a
// caller workspace, so a caller that cannot allocate device memory can still
// check what the solver conserves.
#include "lbm.h"
#include "lbm_kernels.cuh"

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <mutex>

namespace {

constexpr int NA_THREADS = 256;
constexpr long long NA_CHUNK = 8192;   // nodes per partial
constexpr int NA_MAX_CHUNKS = 8192;    // => at most 8192 * 8192 = 67,108,864 nodes
constexpr int NA_MAX_DEVICES = 64;
constexpr uintptr_t NA_STATE_ALIGN = 16;

// Scratch shared by every call on a device: partials then the two totals.
// 2 * 8192 + 2 doubles = 131,088 bytes, held by each GPU that loads the library
// until the process exits.
static __device__ __align__(256) double na_scratch[2 * NA_MAX_CHUNKS + 2];

std::mutex na_mutex;
double* na_addr[NA_MAX_DEVICES] = {};  // device address of na_scratch, per device

// One block per chunk of NA_CHUNK consecutive nodes (row-major node index);
// every partial slot in use is overwritten, nothing relies on earlier contents.
template <typename T, int QS>
__global__ void __launch_bounds__(NA_THREADS)
    na_chunk_partials(const T* __restrict__ pop, lbm::Geometry g, double* __restrict__ part) {
    lbm::dbg_begin(g.ws_lo, g.ws_hi);  // debug build: the caller's state is the whole range
    constexpr int NQ = lbm::nq_of(QS);
    const long long n = (long long)g.nx * g.ny;
    const long long k0 = blockIdx.x * NA_CHUNK, k1 = min(k0 + NA_CHUNK, n);
    long long ai = 0;
    double a = 0.0, b = 0.0;
    for (long long k = k0 + threadIdx.x; k < k1; k += NA_THREADS) {
        const int y = (int)(k / g.nx), x = (int)(k - (long long)y * g.nx);
        if constexpr (lbm::PhaseFix<T>::on) {
            long long s = 0;
            for (int i = 0; i < 9; ++i) s += lbm::load_f<T>(pop, lbm::pull_off<NQ>(g, x, y, 0, i), i);
            ai += s;
        } else {
            for (int i = 0; i < 9; ++i) a += double(lbm::load_f<T>(pop, lbm::pop_pull_off<T, NQ>(g, x, y, 0, i), i));
            // 16-bit storage: plus the writers' phase fields (the base of the stored f)
            if constexpr (lbm::IsHalf<T>::value) a += double(g.pb_in[2 * ((long long)y * g.nxb * 32 + x) + 1]);
        }
        for (int i = 0; i < QS; ++i)
            b += lbm::pull_any<NQ, T, double>(pop, g, x, y, 18, i) +
                 (g.one_scalar ? 0.0 : lbm::pull_any<NQ, T, double>(pop, g, x, y, 18 + QS, i));
        // ... and their c1, c2 (the bases of the stored h)
        if constexpr (lbm::IsHalf<T>::value) {
            const long long N = (long long)g.ny * g.nxb * 32;
            const uint32_t cw = reinterpret_cast<const uint32_t*>(g.pb_in + 2 * N)[(long long)y * g.nxb * 32 + x];
            b += double(lbm::half_lo(cw)) + double(lbm::half_hi(cw));
        }
    }
    __shared__ double sa[NA_THREADS], sb[NA_THREADS];
    __shared__ long long si[NA_THREADS];
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    si[threadIdx.x] = ai;
    __syncthreads();
    for (int s = NA_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sa[threadIdx.x] += sa[threadIdx.x + s];
            sb[threadIdx.x] += sb[threadIdx.x + s];
            si[threadIdx.x] += si[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = lbm::PhaseFix<T>::on ? __longlong_as_double(si[0]) : sa[0];
        part[2 * blockIdx.x + 1] = sb[0];
    }
}

// Fixed-order sum of the chunk partials into part[2 * NA_MAX_CHUNKS + {0, 1}].
template <typename T>
__global__ void __launch_bounds__(NA_THREADS)
    na_final(double* __restrict__ part, int nchunks, long long nodes) {
    __shared__ double sa[NA_THREADS], sb[NA_THREADS];
    __shared__ long long si[NA_THREADS];
    double a = 0.0, b = 0.0;
    long long ai = 0;
    for (int k = threadIdx.x; k < nchunks; k += NA_THREADS) {
        if (lbm::PhaseFix<T>::on) ai += __double_as_longlong(part[2 * k]);
        else a += part[2 * k];
        b += part[2 * k + 1];
    }
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    si[threadIdx.x] = ai;
    __syncthreads();
    for (int s = NA_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sa[threadIdx.x] += sa[threadIdx.x + s];
            sb[threadIdx.x] += sb[threadIdx.x + s];
            si[threadIdx.x] += si[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * NA_MAX_CHUNKS] =
            lbm::PhaseFix<T>::on ? double(si[0]) * lbm::FIX_EPS_D + 0.5 * double(nodes) : sa[0];
        part[2 * NA_MAX_CHUNKS + 1] = sb[0];
    }
}

template <typename T>
cudaError_t na_launch(const void* pop, const lbm::Geometry& g, int q, double* scratch, int nchunks,
                      cudaStream_t s) {
    if (q == 5)
        na_chunk_partials<T, 5><<<nchunks, NA_THREADS, 0, s>>>((const T*)pop, g, scratch);
    else
        na_chunk_partials<T, 9><<<nchunks, NA_THREADS, 0, s>>>((const T*)pop, g, scratch);
    na_final<T><<<1, NA_THREADS, 0, s>>>(scratch, nchunks, (long long)g.nx * g.ny);
    return cudaGetLastError();
}

// error message into the caller's buffer, if it gave one
int na_fail(char* err, size_t err_len, int code, const char* msg) {
    if (err && err_len) snprintf(err, err_len, "%s", msg);
    return code;
}

}  // namespace

extern "C" int lbm_conserved_noalloc(const lbm_params* params, const void* d_state, size_t state_bytes,
                                     void* cuda_stream, double* out, int32_t out_on_device, char* err,
                                     size_t err_len) {
    if (err && err_len) err[0] = '\0';
    if (!params || !d_state || !out)
        return na_fail(err, err_len, LBM_ERR_ARG, "params, state and out must be non-NULL");
    // Only the layout fields are read; the physical parameters do not enter a sum.
    const lbm_params* p = params;
    if (p->nx < 1 || p->ny < 1 || p->nx > (1 << 28) || p->ny > (1 << 28))
        return na_fail(err, err_len, LBM_ERR_ARG, "nx and ny must be in [1, 2^28]");
    if ((p->bc_x != LBM_BC_PERIODIC && p->bc_x != LBM_BC_WALL) || (p->bc_y != LBM_BC_PERIODIC && p->bc_y != LBM_BC_WALL))
        return na_fail(err, err_len, LBM_ERR_ARG, "bc_x/bc_y must be LBM_BC_PERIODIC or LBM_BC_WALL");
    if (p->scalar_q != 5 && p->scalar_q != 9) return na_fail(err, err_len, LBM_ERR_ARG, "scalar_q must be 5 or 9");
    if (p->precision < LBM_FP64 || p->precision > LBM_FP32_FP16STORE)
        return na_fail(err, err_len, LBM_ERR_ARG, "unknown precision");
    if (p->scalar_model != LBM_SCALAR_TWO && p->scalar_model != LBM_SCALAR_ONE)
        return na_fail(err, err_len, LBM_ERR_ARG, "unknown scalar_model");
    if (p->scalar_model == LBM_SCALAR_ONE && p->precision != LBM_FP64 && p->precision != LBM_FP32)
        return na_fail(err, err_len, LBM_ERR_ARG, "the one-scalar model runs in LBM_FP64 or LBM_FP32");
    // the kernels load 4- and 8-byte words: a misaligned state would fault the context
    if (reinterpret_cast<uintptr_t>(d_state) % NA_STATE_ALIGN != 0)
        return na_fail(err, err_len, LBM_ERR_ARG, "state must be 16-byte aligned");
    const long long nodes = (long long)params->nx * params->ny;
    const long long nchunks = (nodes + NA_CHUNK - 1) / NA_CHUNK;
    if (nchunks > NA_MAX_CHUNKS) {
        char msg[200];
        snprintf(msg, sizeof(msg), "grid of %lld nodes exceeds the %lld-node limit of lbm_conserved_noalloc",
                 nodes, (long long)NA_MAX_CHUNKS * NA_CHUNK);
        return na_fail(err, err_len, LBM_ERR_ARG, msg);
    }
    const int qs = params->scalar_q;
    const int nxb = (params->nx + 31) / 32;
    const size_t elem = params->precision == LBM_FP64 ? 8 : (params->precision == LBM_FP32 ? 4 : 2);
    const size_t pop_bytes = (size_t)params->ny * nxb * lbm::nq_of(qs) * 32 * elem;
    if (state_bytes < pop_bytes) return na_fail(err, err_len, LBM_ERR_ARG, "state smaller than the populations of these parameters");
    // 16-bit storage: the writers' bases ((p, phi) FP32 pairs, then (c1, c2)
    // half pairs) follow the populations and the previous-step macros
    // (lbm_get_state's layout); phi, c1 and c2 are part of the stored f and h
    const size_t pb_off = pop_bytes + (size_t)params->ny * nxb * 5 * 32 * sizeof(float);
    const size_t pb_bytes = elem == 2 ? (size_t)params->ny * nxb * 32 * 12 + 8 : 0;  // bases, step counter
    if (elem == 2 && state_bytes < pb_off + pb_bytes)
        return na_fail(err, err_len, LBM_ERR_ARG, "16-bit state smaller than lbm_state_bytes() of these parameters");

    int dev = 0;
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, d_state) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return na_fail(err, err_len, LBM_ERR_ARG, "state is not device memory");
    }
    dev = attr.device;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return na_fail(err, err_len, LBM_ERR_ARG, "device index out of range");
    int prev_dev = -1;
    cudaGetDevice(&prev_dev);
    if (prev_dev != dev) cudaSetDevice(dev);

    // set-up, once per device, with that device current
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(na_mutex);
        if (!na_addr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, na_scratch);
            if (e != cudaSuccess) {
                if (prev_dev >= 0 && prev_dev != dev) cudaSetDevice(prev_dev);
                char msg[200];
                snprintf(msg, sizeof(msg), "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
                return na_fail(err, err_len, LBM_ERR_CUDA, msg);
            }
            na_addr[dev] = static_cast<double*>(p);
        }
        scratch = na_addr[dev];
    }

    lbm::Geometry g;
    g.nx = params->nx;
    g.ny = params->ny;
    g.nxb = nxb;
    g.wall_x = params->bc_x == LBM_BC_WALL;
    g.wall_y = params->bc_y == LBM_BC_WALL;
    g.strip_h = params->ny;
    g.one_scalar = params->scalar_model == LBM_SCALAR_ONE;
    g.grad_scheme = params->grad_scheme;
    g.pb_in = elem == 2 ? reinterpret_cast<const float*>(static_cast<const uint8_t*>(d_state) + pb_off) : nullptr;
    g.pb_out = nullptr;
    g.ws_lo = static_cast<const char*>(d_state);
    g.ws_hi = g.ws_lo + state_bytes;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = lbm::by_storage(params->precision, [&](auto t, auto) {
        return na_launch<decltype(t)>(d_state, g, qs, scratch, (int)nchunks, s);
    });
    if (e == cudaSuccess) {
        if (out_on_device) {
            e = cudaMemcpyAsync(out, scratch + 2 * NA_MAX_CHUNKS, 2 * sizeof(double), cudaMemcpyDeviceToDevice, s);
        } else {
            e = cudaMemcpyAsync(out, scratch + 2 * NA_MAX_CHUNKS, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        }
    }
    if (prev_dev >= 0 && prev_dev != dev) cudaSetDevice(prev_dev);
    if (e != cudaSuccess) {
        char msg[200];
        snprintf(msg, sizeof(msg), "lbm_conserved_noalloc: %s", cudaGetErrorString(e));
        return na_fail(err, err_len, LBM_ERR_CUDA, msg);
    }
    return LBM_OK;
}
