// Internal helpers shared by the surrogate network's translation units.
#pragma once

#include <cuda_runtime.h>

// Streaming multiprocessors of the current device (>= 1).
inline int nn_sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
    return sms;
}
