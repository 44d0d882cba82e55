// Model variants of the fused step for float storage and arithmetic: the
// one-scalar model (Sec. III D) and the local gradient schemes (Eq. 39 and the
// local grad phi), alone and combined.
#include "lbm_kernels.cuh"

namespace lbm {

template <>
cudaError_t launch_variant<float, float>(const void* src, void* dst, void* prev, const Geometry& g,
                                  const Coeffs<float>& C, int q, unsigned* flag, uint32_t mask, void* out,
                                  int out_f64, bool fields, cudaStream_t s) {
    switch (variant_of(g)) {
        case 1:  // one-scalar
        case 3:  // one-scalar + local grad c (no grad c in the one-scalar model)
            return launch_variant_impl<float, float, 1>(src, dst, prev, g, C, q, flag, mask, out, out_f64, fields, s);
        case 2:  // local grad c
            return launch_variant_impl<float, float, 2>(src, dst, prev, g, C, q, flag, mask, out, out_f64, fields, s);
        case 4:  // local grad c and grad phi
            return launch_variant_impl<float, float, 4>(src, dst, prev, g, C, q, flag, mask, out, out_f64, fields, s);
        case 5:  // one-scalar + local grad phi
            return launch_variant_impl<float, float, 5>(src, dst, prev, g, C, q, flag, mask, out, out_f64, fields, s);
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace lbm
