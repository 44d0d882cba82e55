// Instantiations of the fused step, field, init and reduction kernels for
// bfloat16 storage with float arithmetic.
#include "lbm_kernels.cuh"

namespace lbm {

template <>
cudaError_t launch_step<__nv_bfloat16, float>(const void* src, void* dst, void* prev, const Geometry& g,
                                const Coeffs<float>& C, int q, unsigned* flag, cudaStream_t s) {
    return launch_step_impl<__nv_bfloat16, float>(src, dst, prev, g, C, q, flag, s);
}

template <>
cudaError_t launch_fields<__nv_bfloat16, float>(const void* src, const void* prev, const Geometry& g, const Coeffs<float>& C,
                                  int q, uint32_t mask, void* out, int out_f64, cudaStream_t s) {
    return launch_fields_impl<__nv_bfloat16, float>(src, prev, g, C, q, mask, out, out_f64, s);
}

template <>
cudaError_t launch_init<__nv_bfloat16, float>(const InitFields& in, void* pop, void* prev, const Geometry& g,
                                const Coeffs<float>& C, int q, cudaStream_t s) {
    return launch_init_impl<__nv_bfloat16, float>(in, pop, prev, g, C, q, s);
}

template <>
cudaError_t launch_conserved<__nv_bfloat16>(const void* pop, const Geometry& g, int q, double* partials,
                                 double* out, cudaStream_t s) {
    return launch_conserved_impl<__nv_bfloat16>(pop, g, q, partials, out, s);
}

template <>
int step_blocks_per_sm<__nv_bfloat16, float>(int q) {
    return step_blocks_per_sm_impl<__nv_bfloat16, float>(q);
}

}  // namespace lbm
