// Instantiations of the fused step, field, init and reduction kernels for
// float storage with float arithmetic.
#include "lbm_kernels.cuh"

namespace lbm {

template <>
cudaError_t launch_step<float, float>(const void* src, void* dst, void* prev, const Geometry& g,
                                const Coeffs<float>& C, int q, unsigned* flag, cudaStream_t s) {
    return launch_step_impl<float, float>(src, dst, prev, g, C, q, flag, s);
}

template <>
cudaError_t launch_fields<float, float>(const void* src, const void* prev, const Geometry& g, const Coeffs<float>& C,
                                  int q, uint32_t mask, void* out, int out_f64, cudaStream_t s) {
    return launch_fields_impl<float, float>(src, prev, g, C, q, mask, out, out_f64, s);
}

template <>
cudaError_t launch_init<float, float>(const InitFields& in, void* pop, void* prev, const Geometry& g,
                                const Coeffs<float>& C, int q, cudaStream_t s) {
    return launch_init_impl<float, float>(in, pop, prev, g, C, q, s);
}

template <>
cudaError_t launch_conserved<float>(const void* pop, const Geometry& g, int q, double* partials,
                                 double* out, cudaStream_t s) {
    return launch_conserved_impl<float>(pop, g, q, partials, out, s);
}

template <>
int step_blocks_per_sm<float, float>(int q) {
    return step_blocks_per_sm_impl<float, float>(q);
}

}  // namespace lbm
