// C ABI of liblbm (declared in include/lbm.h): parameter validation, workspace
// carving, stepping with CUDA graphs, field read-back, conserved sums,
// checkpoints and error reporting.  Host code plus the small init kernel that
// turns a signed-distance field into phi, c1, c2.
#include "lbm.h"
#include "lbm_handle.h"
#include "lbm_internal.h"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <type_traits>
#include <vector>

using lbm::detail::DeviceGuard;
using lbm::detail::Layout;

namespace {

constexpr double CS2 = 1.0 / 3.0;
constexpr size_t ALIGN = 256;

thread_local char g_thread_error[512] = "";

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

// Returns LBM_OK or an error code with a message in `err`.
int validate(const lbm_params* p, char* err, size_t n) {
    if (!p) { snprintf(err, n, "params is NULL"); return LBM_ERR_ARG; }
    if (p->nx < 1 || p->ny < 1) { snprintf(err, n, "nx and ny must be >= 1 (got %d x %d)", p->nx, p->ny); return LBM_ERR_ARG; }
    if (p->nx > (1 << 28) || p->ny > (1 << 28) || (double)p->nx * p->ny > 4e9) { snprintf(err, n, "grid %d x %d too large", p->nx, p->ny); return LBM_ERR_ARG; }
    if ((p->bc_x != LBM_BC_PERIODIC && p->bc_x != LBM_BC_WALL) || (p->bc_y != LBM_BC_PERIODIC && p->bc_y != LBM_BC_WALL)) {
        snprintf(err, n, "bc_x/bc_y must be LBM_BC_PERIODIC or LBM_BC_WALL"); return LBM_ERR_ARG;
    }
    if (p->scalar_q != 5 && p->scalar_q != 9) { snprintf(err, n, "scalar_q must be 5 or 9 (got %d)", p->scalar_q); return LBM_ERR_ARG; }
    if (p->precision < LBM_FP64 || p->precision > LBM_FP32_FP16STORE) { snprintf(err, n, "unknown precision %d", p->precision); return LBM_ERR_ARG; }
    if (p->visc_model < LBM_VISC_LINEAR || p->visc_model > LBM_VISC_EXP_T) { snprintf(err, n, "unknown visc_model %d", p->visc_model); return LBM_ERR_ARG; }
    if (p->scalar_model != LBM_SCALAR_TWO && p->scalar_model != LBM_SCALAR_ONE) { snprintf(err, n, "unknown scalar_model %d", p->scalar_model); return LBM_ERR_ARG; }
    if (p->grad_scheme < LBM_GRAD_STENCIL || p->grad_scheme > LBM_GRAD_LOCAL_ALL) { snprintf(err, n, "unknown grad_scheme %d", p->grad_scheme); return LBM_ERR_ARG; }
    if ((p->scalar_model != LBM_SCALAR_TWO || p->grad_scheme != LBM_GRAD_STENCIL) && p->precision != LBM_FP64 &&
        p->precision != LBM_FP32) {
        snprintf(err, n, "the one-scalar model and the local gradient schemes run in LBM_FP64 or LBM_FP32"); return LBM_ERR_ARG;
    }
    if (!finite_pos(p->W)) { snprintf(err, n, "W must be > 0"); return LBM_ERR_ARG; }
    if (!finite_pos(p->rho1) || !finite_pos(p->rho2)) { snprintf(err, n, "rho1, rho2 must be > 0"); return LBM_ERR_ARG; }
    if (!finite_pos(p->Keq)) { snprintf(err, n, "Keq must be > 0"); return LBM_ERR_ARG; }
    if (!std::isfinite(p->sigma) || p->sigma < 0 || !std::isfinite(p->A) || p->A < 0) { snprintf(err, n, "sigma and A must be finite and >= 0"); return LBM_ERR_ARG; }
    const double fin[] = {p->gx, p->gy, p->g_rho_ref, p->Fx, p->Fy, p->visc_beta, p->M, p->D1, p->D2, p->mu1, p->mu2};
    for (double v : fin) if (!std::isfinite(v)) { snprintf(err, n, "parameters must be finite"); return LBM_ERR_ARG; }
    // Eqs. (27), (33), (38): every relaxation time must exceed 1/2
    if (!(p->M > 0)) { snprintf(err, n, "tau_f = M/cs^2 + 1/2 <= 1/2 (M = %g)", p->M); return LBM_ERR_UNSTABLE_TAU; }
    if (!(p->D1 > 0) || !(p->D2 > 0)) { snprintf(err, n, "tau_h = D/cs^2 + 1/2 <= 1/2 (D1 = %g, D2 = %g)", p->D1, p->D2); return LBM_ERR_UNSTABLE_TAU; }
    if (!(p->mu1 > 0) || !(p->mu2 > 0)) { snprintf(err, n, "tau_g = mu/(rho cs^2) + 1/2 <= 1/2 (mu1 = %g, mu2 = %g)", p->mu1, p->mu2); return LBM_ERR_UNSTABLE_TAU; }
    return LBM_OK;
}

Layout layout_of(const lbm_params* p) {
    Layout L;
    L.nq = 18 + 2 * p->scalar_q;  // f, g, h1, h2
    L.elem = p->precision == LBM_FP64 ? 8 : (p->precision == LBM_FP32 ? 4 : 2);
    L.relem = p->precision == LBM_FP64 ? 8 : 4;  // previous-step macros: arithmetic type
    L.nxb = (p->nx + 31) / 32;
    L.pop_elems = (size_t)p->ny * L.nxb * L.nq * 32;
    L.prev_elems = (size_t)p->ny * L.nxb * 5 * 32;
    // per node (p, phi) in FP32 and (c1, c2) in halves, then the step counter
    // (and a pad word)
    L.pb_elems = L.elem == 2 ? (size_t)p->ny * L.nxb * 32 * 3 + 2 : 0;
    L.pop_bytes = align_up(L.pop_elems * L.elem, ALIGN);
    L.prev_bytes = align_up(L.prev_elems * L.relem, ALIGN);
    L.pb_bytes = align_up(L.pb_elems * sizeof(float), ALIGN);
    L.part_bytes = align_up((size_t)lbm::RED_BLOCKS * 2 * sizeof(double), ALIGN);
    L.misc_bytes = ALIGN;
    L.off_pop[0] = 0;
    L.off_pop[1] = L.pop_bytes;
    L.off_prev = 2 * L.pop_bytes;
    L.off_pb = L.off_prev + L.prev_bytes;
    L.off_part = L.off_pb + 2 * L.pb_bytes;
    L.off_misc = L.off_part + L.part_bytes;
    L.total = L.off_misc + L.misc_bytes;
    return L;
}

template <typename R>
lbm::Coeffs<R> coeffs_of(const lbm_params* p) {
    lbm::Coeffs<R> C;
    const double tf = p->M / CS2 + 0.5, t1 = p->D1 / CS2 + 0.5, t2 = p->D2 / CS2 + 0.5;
    C.omega_f = R(1.0 / tf);  C.force_f = R(1.0 - 0.5 / tf);
    C.omega_h1 = R(1.0 / t1); C.force_h1 = R(1.0 - 0.5 / t1);
    C.omega_h2 = R(1.0 / t2); C.force_h2 = R(1.0 - 0.5 / t2);
    C.beta4 = R(4.0 * 12.0 * p->sigma / p->W);
    C.kappa = R(1.5 * p->sigma * p->W);
    C.rho1 = R(p->rho1); C.rho2 = R(p->rho2); C.drho = R(p->rho1 - p->rho2);
    C.mu2 = R(p->mu2); C.dmu = R(p->mu1 - p->mu2);
    C.log_mu1 = R(std::log(p->mu1)); C.log_mu2 = R(std::log(p->mu2));
    C.visc_beta = R(p->visc_beta);
    C.D1D2 = R(p->D1 * p->D2); C.KD1 = R(p->Keq * p->D1); C.D2 = R(p->D2); C.K = R(p->Keq);
    C.D1 = R(p->D1); C.M = R(p->M);
    C.halfA = R(0.5 * p->A); C.A = R(p->A);
    C.four_over_W = R(4.0 / p->W);
    C.gx = R(p->gx); C.gy = R(p->gy); C.g_rho_ref = R(p->g_rho_ref);
    C.Fx = R(p->Fx); C.Fy = R(p->Fy);
    C.visc_model = p->visc_model;
    return C;
}

// two_over_W = 2 / W, taken once on the host: an FP64 division per node would
// cost more than the kernel's memory traffic
__global__ void sdf_to_fields_kernel(const double* __restrict__ sdf, double* phi, double* c1, double* c2,
                                     size_t n, double two_over_W, double c1t, double c2t) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const double a = sdf[k] * two_over_W;
        // Eq. (2).  tanh saturates: for |a| >= 20, 1 - |tanh a| < 1e-17, below half
        // the spacing of doubles under 1, so the rounded profile is exactly 0 or 1
        // there, and only the interface band pays for the FP64 tanh
        const double ph = fabs(a) >= 20.0 ? (a > 0.0 ? 1.0 : 0.0) : 0.5 + 0.5 * tanh(a);
        phi[k] = ph;
        c1[k] = c1t * ph;
        c2[k] = c2t * (1.0 - ph);
    }
}

}  // namespace

namespace lbm {
cudaError_t launch_sdf_to_fields(const double* sdf, double* phi, double* c1, double* c2, size_t n,
                                 double W, double c1t, double c2t, cudaStream_t s) {
    const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 152 * 16);
    sdf_to_fields_kernel<<<blocks, 256, 0, s>>>(sdf, phi, c1, c2, n, 2.0 / W, c1t, c2t);
    return cudaGetLastError();
}
}  // namespace lbm

// Rows per CTA of the step kernel: the strip height that fills the SMs in whole
// waves with the least idle capacity, counting the two halo rows each strip
// evaluates twice.
static int choose_strip_height(const lbm_handle* h) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess || sms <= 0) sms = 1;
    int per_sm = lbm::by_storage(h->p.precision, [&](auto t, auto r) {
        return lbm::step_blocks_per_sm<decltype(t), decltype(r)>(h->p.scalar_q);
    });
    cudaGetLastError();
    if (per_sm <= 0) per_sm = 1;
    const long long slots = (long long)sms * per_sm;
    const int ny = h->p.ny;
    const long long cx = (h->p.nx + lbm::STRIP_W - 1) / lbm::STRIP_W;
    int best_h = ny;
    double best = -1.0;
    for (int waves = 1; waves <= 16; ++waves) {
        long long cy = std::max<long long>(1, waves * slots / cx);
        int H = (int)std::max<long long>(1, (ny + cy - 1) / cy);
        if (H < 4 && ny >= 4) H = 4;
        H = std::max(H, (ny + 65534) / 65535);  // grid.y <= 65535
        const long long ctas = cx * ((ny + H - 1) / H);
        const long long used_waves = (ctas + slots - 1) / slots;
        const double fill = (double)ctas / (double)(used_waves * slots);
        const double eff = fill * (double)H / (double)(H + 2) * (double)ny / (double)(((ny + H - 1) / H) * H);
        if (eff > best + 1e-9) { best = eff; best_h = H; }
    }
    return best_h;
}

// Debug build: the readers of the status words of every translation unit with
// checked kernels (registered during static initialisation).
namespace lbm {
namespace {
std::vector<unsigned (*)()>& debug_readers() {
    static std::vector<unsigned (*)()> readers;
    return readers;
}
}  // namespace
void register_debug_status(unsigned (*take)()) { debug_readers().push_back(take); }
unsigned debug_status_take() {
    unsigned v = 0;
    for (auto take : debug_readers()) v |= take();
    return v;
}
}  // namespace lbm

extern "C" {

size_t lbm_workspace_bytes(const lbm_params* params) {
    if (validate(params, g_thread_error, sizeof(g_thread_error)) != LBM_OK) return 0;
    return layout_of(params).total;
}

int lbm_create(const lbm_params* params, void* d_workspace, size_t workspace_bytes, void* cuda_stream,
               lbm_handle** out) {
    if (!out) { snprintf(g_thread_error, sizeof(g_thread_error), "out is NULL"); return LBM_ERR_ARG; }
    *out = nullptr;
    int rc = validate(params, g_thread_error, sizeof(g_thread_error));
    if (rc != LBM_OK) return rc;
    const Layout L = layout_of(params);
    if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) % ALIGN) != 0) {
        snprintf(g_thread_error, sizeof(g_thread_error), "workspace must be a non-NULL %zu-byte aligned device pointer", ALIGN);
        return LBM_ERR_WORKSPACE;
    }
    if (workspace_bytes < L.total) {
        snprintf(g_thread_error, sizeof(g_thread_error), "workspace too small: %zu bytes given, %zu needed", workspace_bytes, L.total);
        return LBM_ERR_WORKSPACE;
    }
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, d_workspace) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        snprintf(g_thread_error, sizeof(g_thread_error), "workspace is not device memory");
        return LBM_ERR_WORKSPACE;
    }
    lbm_handle* h = new (std::nothrow) lbm_handle();
    if (!h) { snprintf(g_thread_error, sizeof(g_thread_error), "out of host memory"); return LBM_ERR_ARG; }
    h->p = *params;
    h->L = L;
    h->geo.nx = params->nx; h->geo.ny = params->ny; h->geo.nxb = L.nxb;
    h->geo.wall_x = params->bc_x == LBM_BC_WALL; h->geo.wall_y = params->bc_y == LBM_BC_WALL;
    h->geo.strip_h = params->ny;
    h->geo.one_scalar = params->scalar_model == LBM_SCALAR_ONE;
    h->geo.grad_scheme = params->grad_scheme;
    h->geo.pb_in = nullptr;
    h->geo.pb_out = nullptr;
    h->cf = coeffs_of<float>(params);
    h->cd = coeffs_of<double>(params);
    h->device = attr.device;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->ws = static_cast<uint8_t*>(d_workspace);
    h->geo.ws_lo = reinterpret_cast<const char*>(h->ws);
    h->geo.ws_hi = h->geo.ws_lo + L.total;
    DeviceGuard dg(h->device);
    cudaError_t e = cudaStreamCreateWithFlags(&h->capture, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->status_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&h->h_status), 16);
    if (e != cudaSuccess) {
        snprintf(g_thread_error, sizeof(g_thread_error), "CUDA setup failed: %s", cudaGetErrorString(e));
        lbm_destroy(h);
        return LBM_ERR_CUDA;
    }
    *h->h_status = 0u;
    h->geo.strip_h = choose_strip_height(h);
    *out = h;
    return LBM_OK;
}

static int init_common(lbm_handle* h, const double* phi, const double* c1, const double* c2,
                       const double* ux = nullptr, const double* uy = nullptr, const double* p = nullptr) {
    const lbm::InitFields in{phi, ux, uy, p, c1, c2};
    const cudaError_t e = h->init_on(in, h->stream);
    if (e != cudaSuccess) return h->fail(LBM_ERR_CUDA, "init kernel", e);
    h->restarted();
    return LBM_OK;
}

// Device address of a host buffer that the GPU can read and write in place
// (page-locked memory mapped into the current device's address space; on a
// Grace-Blackwell node over NVLink-C2C, faster than a copy-engine transfer of
// the same bytes), or nullptr: then the call stages through device memory.
static void* mapped_host(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

int lbm_init(lbm_handle* h, const double* sdf, int32_t sdf_on_device, double c1_tilde, double c2_tilde) {
    if (!h) return LBM_ERR_ARG;
    if (!sdf) return h->fail(LBM_ERR_ARG, "sdf is NULL");
    if (!std::isfinite(c1_tilde) || !std::isfinite(c2_tilde)) return h->fail(LBM_ERR_ARG, "c1_tilde/c2_tilde must be finite");
    DeviceGuard dg(h->device);
    const size_t n = (size_t)h->p.nx * h->p.ny;
    double* st = static_cast<double*>(h->pop(1));  // staging: the population buffer the first step writes
    double *phi = st, *c1 = st + n, *c2 = st + 2 * n;
    cudaError_t e = cudaSuccess;
    const double* src = sdf;
    if (!sdf_on_device) {
        // mapped host memory is read in place by the kernel, else copied first
        src = static_cast<const double*>(mapped_host(sdf));
        if (!src) {
            e = cudaMemcpyAsync(phi, sdf, n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
            src = phi;
        }
    }
    if (e == cudaSuccess) e = lbm::launch_sdf_to_fields(src, phi, c1, c2, n, h->p.W, c1_tilde, c2_tilde, h->stream);
    if (e != cudaSuccess) return h->fail(LBM_ERR_CUDA, "lbm_init", e);
    return init_common(h, phi, c1, c2);
}

int lbm_init_fields(lbm_handle* h, const double* phi, const double* c1, const double* c2, int32_t on_device) {
    if (!h) return LBM_ERR_ARG;
    if (!phi || !c1 || !c2) return h->fail(LBM_ERR_ARG, "phi, c1, c2 must be non-NULL");
    DeviceGuard dg(h->device);
    if (on_device) return init_common(h, phi, c1, c2);
    const size_t n = (size_t)h->p.nx * h->p.ny;
    double* st = static_cast<double*>(h->pop(1));
    cudaError_t e = cudaMemcpyAsync(st, phi, n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(st + n, c1, n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(st + 2 * n, c2, n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return h->fail(LBM_ERR_CUDA, "lbm_init_fields copy", e);
    return init_common(h, st, st + n, st + 2 * n);
}

int lbm_init_macros(lbm_handle* h, const double* phi, const double* ux, const double* uy, const double* p,
                    const double* c1, const double* c2, int32_t on_device) {
    if (!h) return LBM_ERR_ARG;
    if (!phi || !ux || !uy || !p || !c1 || !c2) return h->fail(LBM_ERR_ARG, "all six fields must be non-NULL");
    DeviceGuard dg(h->device);
    if (on_device) return init_common(h, phi, c1, c2, ux, uy, p);
    const size_t n = (size_t)h->p.nx * h->p.ny;
    double* st = static_cast<double*>(h->pop(1));  // 48 B per node: fits every population buffer
    const double* src[6] = {phi, ux, uy, p, c1, c2};
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 6 && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(st + k * n, src[k], n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return h->fail(LBM_ERR_CUDA, "lbm_init_macros copy", e);
    return init_common(h, st, st + 4 * n, st + 5 * n, st + n, st + 2 * n, st + 3 * n);
}

int lbm_step(lbm_handle* h, int64_t nsteps) {
    const lbm::NvtxRange range("lbm_step");
    if (!h) return LBM_ERR_ARG;
    if (nsteps < 0) return h->fail(LBM_ERR_ARG, "nsteps must be >= 0");
    if (h->nonfinite_seen()) return h->fail(LBM_ERR_NONFINITE, "a previous step produced a non-finite macro value");
    if (nsteps == 0) return LBM_OK;
    DeviceGuard dg(h->device);
    int64_t left = nsteps;
    cudaError_t e = cudaSuccess;
    // n = 32 a + the binary digits of the rest: captured sequences of 32, 16,
    // .., 2 steps (even: the state stays in buffer cur), then at most one
    // plain launch
    if (left >= 2) {
        using lbm::detail::GRAPH_LEVELS;
        e = h->build_graphs();
        while (e == cudaSuccess && left >= lbm::detail::GRAPH_STEPS) {
            e = cudaGraphLaunch(h->graph[h->cur][GRAPH_LEVELS - 1], h->stream);
            left -= lbm::detail::GRAPH_STEPS;
        }
        for (int lv = GRAPH_LEVELS - 2; lv >= 0 && e == cudaSuccess; --lv) {
            if (left >= (2 << lv)) {
                e = cudaGraphLaunch(h->graph[h->cur][lv], h->stream);
                left -= 2 << lv;
            }
        }
    }
    while (e == cudaSuccess && left > 0) {
        e = h->step_once(h->cur, h->stream);
        h->cur ^= 1;
        --left;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->h_status, h->flag(), sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(h->status_ev, h->stream);
    if (e != cudaSuccess) return h->fail(LBM_ERR_CUDA, "lbm_step", e);
    h->status_pending = true;
    h->t += nsteps - left;
    return LBM_OK;
}

int lbm_get_fields(lbm_handle* h, uint32_t mask, void* out, int32_t out_on_device, int32_t out_dtype) {
    const lbm::NvtxRange range("lbm_get_fields");
    if (!h) return LBM_ERR_ARG;
    mask &= LBM_FIELD_ALL;
    if (!mask || !out) return h->fail(LBM_ERR_ARG, "empty field mask or NULL output");
    if (out_dtype != LBM_OUT_F64 && out_dtype != LBM_OUT_F32) return h->fail(LBM_ERR_ARG, "out_dtype must be LBM_OUT_F64 or LBM_OUT_F32");
    DeviceGuard dg(h->device);
    const int f64 = out_dtype == LBM_OUT_F64;
    cudaError_t e = cudaSuccess;
    if (out_on_device) {
        e = h->fields(h->cur, mask, out, f64, h->stream);
        if (e != cudaSuccess) return h->fail(LBM_ERR_CUDA, "lbm_get_fields", e);
        return LBM_OK;
    }
    // host output the GPU can write in place (mapped page-locked memory): one
    // evaluation straight into it
    if (void* mapped = mapped_host(out)) {
        e = h->fields(h->cur, mask, mapped, f64, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return h->fail(LBM_ERR_CUDA, "lbm_get_fields", e);
        return LBM_OK;
    }
    // other host output: evaluate into the idle population buffer, in batches
    // that fit, and copy
    const size_t per_field = (size_t)h->p.nx * h->p.ny * (f64 ? 8 : 4);
    const size_t batch = h->L.pop_bytes / per_field;
    uint8_t* dst = static_cast<uint8_t*>(out);
    void* staging = h->pop(h->cur ^ 1);
    uint32_t rest = mask;
    while (rest && e == cudaSuccess) {
        uint32_t sub = 0;
        size_t k = 0;
        for (int b = 0; b < 8 && k < batch; ++b)
            if (rest & (1u << b)) { sub |= 1u << b; ++k; }
        rest &= ~sub;
        e = h->fields(h->cur, sub, staging, f64, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, staging, k * per_field, cudaMemcpyDeviceToHost, h->stream);
        dst += k * per_field;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return h->fail(LBM_ERR_CUDA, "lbm_get_fields", e);
    return LBM_OK;
}

int lbm_debug_build(void) { return LBM_DEBUG; }

int lbm_debug_limit_workspace(lbm_handle* h, size_t bytes) {
    if (!h) return LBM_ERR_ARG;
    if (!LBM_DEBUG) return h->fail(LBM_ERR_ARG, "lbm_debug_limit_workspace needs the debug build");
    if (bytes > h->L.total) return h->fail(LBM_ERR_ARG, "the checked range cannot exceed the workspace");
    DeviceGuard dg(h->device);
    const cudaError_t e = cudaStreamSynchronize(h->stream);  // no launch in flight uses the old range
    if (e != cudaSuccess) return h->fail(LBM_ERR_CUDA, "lbm_debug_limit_workspace", e);
    h->geo.ws_hi = h->geo.ws_lo + bytes;
    h->drop_graphs();  // they were captured with the old range
    return LBM_OK;
}

int lbm_sync(lbm_handle* h) {
    if (!h) return LBM_ERR_ARG;
    DeviceGuard dg(h->device);
    cudaError_t e = cudaMemcpyAsync(h->h_status, h->flag(), sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return h->fail(LBM_ERR_CUDA, "lbm_sync", e);
    if (LBM_DEBUG && lbm::debug_status_take() != 0u)
        return h->fail(LBM_ERR_BOUNDS, "debug build: a kernel access fell outside the workspace (skipped)");
    h->status_pending = false;
    if (*h->h_status) h->nonfinite = true;
    if (h->nonfinite) return h->fail(LBM_ERR_NONFINITE, "a step produced a non-finite macro value");
    return LBM_OK;
}

int lbm_conserved(lbm_handle* h, double out[2]) {
    const lbm::NvtxRange range("lbm_conserved");
    if (!h) return LBM_ERR_ARG;
    if (!out) return h->fail(LBM_ERR_ARG, "out is NULL");
    DeviceGuard dg(h->device);
    cudaError_t e = lbm::by_storage(h->p.precision, [&](auto t, auto) {
        return lbm::launch_conserved<decltype(t)>(h->pop(h->cur), h->geo_from(h->cur), h->p.scalar_q, h->partials(), h->sums(),
                                                  h->stream);
    });
    double tmp[2] = {0.0, 0.0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, h->sums(), 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return h->fail(LBM_ERR_CUDA, "lbm_conserved", e);
    const int rc = lbm_sync(h);
    out[0] = tmp[0];
    out[1] = tmp[1];
    return rc;
}

size_t lbm_state_bytes(const lbm_handle* h) {
    if (!h) return 0;
    return h->state_bytes();
}

int lbm_get_state(lbm_handle* h, void* buf, size_t bytes, int32_t on_device) {
    if (!h) return LBM_ERR_ARG;
    if (!buf || bytes < h->state_bytes()) return h->fail(LBM_ERR_ARG, "state buffer NULL or smaller than lbm_state_bytes()");
    DeviceGuard dg(h->device);
    cudaError_t e = h->copy_state(buf, true, on_device != 0, h->stream);
    if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return h->fail(LBM_ERR_CUDA, "lbm_get_state", e);
    return LBM_OK;
}

int lbm_set_state(lbm_handle* h, const void* buf, size_t bytes, int32_t on_device) {
    if (!h) return LBM_ERR_ARG;
    if (!buf || bytes < h->state_bytes()) return h->fail(LBM_ERR_ARG, "state buffer NULL or smaller than lbm_state_bytes()");
    DeviceGuard dg(h->device);
    cudaError_t e = h->copy_state(const_cast<void*>(buf), false, on_device != 0, h->stream);
    if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return h->fail(LBM_ERR_CUDA, "lbm_set_state", e);
    h->restarted();
    return LBM_OK;
}

int64_t lbm_time(const lbm_handle* h) { return h ? h->t : -1; }

void lbm_destroy(lbm_handle* h) {
    if (!h) return;
    {
        DeviceGuard dg(h->device);
        if (h->stream || h->capture) cudaStreamSynchronize(h->stream);
        h->drop_graphs();
        if (h->status_ev) cudaEventDestroy(h->status_ev);
        if (h->capture) cudaStreamDestroy(h->capture);
        if (h->h_status) cudaFreeHost(h->h_status);
    }
    delete h;
}

const char* lbm_last_error(const lbm_handle* h) { return h ? h->err : g_thread_error; }

}  // extern "C"
