// Instantiations of the fused step, field, init and reduction kernels for
// double storage with double arithmetic.
#include "lbm_kernels.cuh"

namespace lbm {

template <>
cudaError_t launch_step<double, double>(const void* src, void* dst, void* prev, const Geometry& g,
                                const Coeffs<double>& C, int q, unsigned* flag, cudaStream_t s) {
    return launch_step_impl<double, double>(src, dst, prev, g, C, q, flag, s);
}

template <>
cudaError_t launch_fields<double, double>(const void* src, const void* prev, const Geometry& g, const Coeffs<double>& C,
                                  int q, uint32_t mask, void* out, int out_f64, cudaStream_t s) {
    return launch_fields_impl<double, double>(src, prev, g, C, q, mask, out, out_f64, s);
}

template <>
cudaError_t launch_init<double, double>(const InitFields& in, void* pop, void* prev, const Geometry& g,
                                const Coeffs<double>& C, int q, cudaStream_t s) {
    return launch_init_impl<double, double>(in, pop, prev, g, C, q, s);
}

template <>
cudaError_t launch_conserved<double>(const void* pop, const Geometry& g, int q, double* partials,
                                 double* out, cudaStream_t s) {
    return launch_conserved_impl<double>(pop, g, q, partials, out, s);
}

template <>
int step_blocks_per_sm<double, double>(int q) {
    return step_blocks_per_sm_impl<double, double>(q);
}

}  // namespace lbm
