// Instantiations of the persistent batched step for D2Q5 scalar lattices,
// tile widths of 32, 64 and 128 columns.
#include "lbm_batch_kernels.cuh"

namespace lbm {

#define LBM_BATCH_INSTANCE(NW)                                                   \
    template <>                                                                  \
    cudaError_t launch_batch<5, NW>(const BatchArgs& a, cudaStream_t s) {       \
        return launch_batch_impl<5, NW>(a, s);                                  \
    }                                                                            \
    template <>                                                                  \
    int batch_blocks_per_sm<5, NW>() {                                          \
        return batch_blocks_per_sm_impl<5, NW>();                               \
    }

LBM_BATCH_INSTANCE(1)
LBM_BATCH_INSTANCE(2)
LBM_BATCH_INSTANCE(4)

#undef LBM_BATCH_INSTANCE

}  // namespace lbm
