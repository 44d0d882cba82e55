// Internal: the solver handle behind the C ABI's lbm_handle, shared by the
// single-lattice API (lbm_api.cu) and the batched runner (lbm_batch.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <type_traits>

#include "lbm.h"
#include "lbm_internal.h"

namespace lbm {
namespace detail {

// Captured step sequences: level k replays 2^(k+1) steps (2, 4, .., 32), one
// graph per starting buffer.  Even lengths keep the state in its buffer.
constexpr int GRAPH_LEVELS = 5;
constexpr int GRAPH_STEPS = 2 << (GRAPH_LEVELS - 1);  // the longest: 32 steps

struct Layout {
    int nq;             // populations per node
    size_t elem, relem; // bytes of a stored population / of a previous-step macro
    int nxb;            // 32-node blocks per row
    size_t pop_elems, prev_elems;
    size_t pb_elems;    // 16-bit storage: 4-byte words per plane of the writers' bases (else 0)
    size_t pop_bytes, prev_bytes, pb_bytes, part_bytes, misc_bytes;
    size_t off_pop[2], off_prev, off_pb, off_part, off_misc, total;
};

// Makes the handle's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1, want;
    explicit DeviceGuard(int dev) : want(dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != want) cudaSetDevice(want);
    }
    ~DeviceGuard() { if (prev >= 0 && prev != want) cudaSetDevice(prev); }
};

}  // namespace detail
}  // namespace lbm

struct lbm_handle {
    lbm_params p;
    lbm::detail::Layout L;
    lbm::Geometry geo;
    lbm::Coeffs<float> cf;
    lbm::Coeffs<double> cd;
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t capture = nullptr;
    uint8_t* ws = nullptr;
    int cur = 0;
    int64_t t = 0;
    cudaGraphExec_t graph[2][lbm::detail::GRAPH_LEVELS] = {};  // [starting buffer][level]
    unsigned* h_status = nullptr;
    cudaEvent_t status_ev = nullptr;
    bool status_pending = false;
    bool nonfinite = false;  // sticky until the next init / set_state
    char err[512] = "";

    void* pop(int k) const { return ws + L.off_pop[k]; }
    void* prev() const { return ws + L.off_prev; }
    // plane of the writers' bases that goes with population buffer k (16-bit storage)
    float* pb(int k) const { return L.pb_elems ? reinterpret_cast<float*>(ws + L.off_pb + k * L.pb_bytes) : nullptr; }
    // the geometry of a launch that reads population buffer `from`
    lbm::Geometry geo_from(int from) const {
        lbm::Geometry g = geo;
        g.pb_in = pb(from);
        g.pb_out = pb(from ^ 1);
        return g;
    }
    double* partials() const { return reinterpret_cast<double*>(ws + L.off_part); }
    unsigned* flag() const { return reinterpret_cast<unsigned*>(ws + L.off_misc); }
    double* sums() const { return reinterpret_cast<double*>(ws + L.off_misc + 16); }

    int fail(int code, const char* what, cudaError_t e = cudaSuccess) {
        if (e != cudaSuccess) snprintf(err, sizeof(err), "%s: %s", what, cudaGetErrorString(e));
        else snprintf(err, sizeof(err), "%s", what);
        return code;
    }

    template <typename R>
    const lbm::Coeffs<R>& coeffs() const {
        if constexpr (std::is_same<R, double>::value) return cd;
        else return cf;
    }

    cudaError_t step_once(int from, cudaStream_t s) {
        return lbm::by_storage(p.precision, [&](auto t, auto r) {
            using T = decltype(t);
            using R = decltype(r);
            return lbm::launch_step<T, R>(pop(from), pop(from ^ 1), prev(), geo_from(from), coeffs<R>(), p.scalar_q,
                                          flag(), s);
        });
    }

    cudaError_t fields(int from, uint32_t mask, void* out, int out_f64, cudaStream_t s) {
        return lbm::by_storage(p.precision, [&](auto t, auto r) {
            using T = decltype(t);
            using R = decltype(r);
            return lbm::launch_fields<T, R>(pop(from), prev(), geo_from(from), coeffs<R>(), p.scalar_q, mask, out,
                                            out_f64, s);
        });
    }

    // Populations at the equilibria of `in` (buffer 0) and a cleared status
    // word, on stream s; restarted() then resets the host-side counters.
    cudaError_t init_on(const lbm::InitFields& in, cudaStream_t s) {
        cudaError_t e = lbm::by_storage(p.precision, [&](auto t, auto r) {
            using T = decltype(t);
            using R = decltype(r);
            lbm::Geometry gi = geo;
            gi.pb_in = nullptr;
            gi.pb_out = pb(0);  // the first step reads buffer 0
            return lbm::launch_init<T, R>(in, pop(0), prev(), gi, coeffs<R>(), p.scalar_q, s);
        });
        if (e == cudaSuccess) e = cudaMemsetAsync(flag(), 0, 16, s);
        return e;
    }

    void restarted() {
        cur = 0;
        t = 0;
        status_pending = false;
        nonfinite = false;
        *h_status = 0u;
    }

    size_t state_bytes() const { return L.pop_elems * L.elem + L.prev_elems * L.relem + L.pb_elems * sizeof(float); }

    // Checkpoint copies on stream s: the current populations and the previous-step
    // macros out of (get) or into (set, then buffer 0 and a cleared status word)
    // the caller's buffer.  After a set the caller calls restarted().
    cudaError_t copy_state(void* buf, bool get, bool on_device, cudaStream_t s) {
        const size_t a = L.pop_elems * L.elem, b = L.prev_elems * L.relem, c = L.pb_elems * sizeof(float);
        uint8_t* u = static_cast<uint8_t*>(buf);
        cudaError_t e;
        if (get) {
            const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
            e = cudaMemcpyAsync(u, pop(cur), a, k, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(u + a, prev(), b, k, s);
            if (e == cudaSuccess && c) e = cudaMemcpyAsync(u + a + b, pb(cur), c, k, s);
        } else {
            const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
            e = cudaMemcpyAsync(pop(0), u, a, k, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(prev(), u + a, b, k, s);
            if (e == cudaSuccess && c) e = cudaMemcpyAsync(pb(0), u + a + b, c, k, s);
            if (e == cudaSuccess) e = cudaMemsetAsync(flag(), 0, 16, s);
        }
        return e;
    }

    cudaError_t build_graph(int parity, int level) {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(capture, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        int c = parity;
        cudaError_t le = cudaSuccess;
        for (int k = 0; k < (2 << level) && le == cudaSuccess; ++k, c ^= 1) le = step_once(c, capture);
        e = cudaStreamEndCapture(capture, &g);
        if (le != cudaSuccess) { if (g) cudaGraphDestroy(g); return le; }
        if (e != cudaSuccess) return e;
        e = cudaGraphInstantiate(&graph[parity][level], g, 0);
        cudaGraphDestroy(g);
        // upload now rather than at the first launch, which may be inside a
        // caller's timed region
        if (e == cudaSuccess) e = cudaGraphUpload(graph[parity][level], stream);
        return e;
    }
    void drop_graphs() {
        for (auto& row : graph)
            for (auto& g : row)
                if (g) {
                    cudaGraphExecDestroy(g);
                    g = nullptr;
                }
    }
    // Every level for both starting buffers, on the first call that steps at
    // least twice, so that later calls of any length launch no capture.
    cudaError_t build_graphs() {
        cudaError_t e = cudaSuccess;
        for (int parity = 0; parity < 2; ++parity)
            for (int level = 0; level < lbm::detail::GRAPH_LEVELS && e == cudaSuccess; ++level)
                if (!graph[parity][level]) e = build_graph(parity, level);
        return e;
    }

    // Non-blocking look at the status word copied back after the last lbm_step.
    bool nonfinite_seen() {
        if (status_pending && cudaEventQuery(status_ev) == cudaSuccess) {
            status_pending = false;
            if (*h_status != 0u) nonfinite = true;
        }
        return nonfinite;
    }
};

