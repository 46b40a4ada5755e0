// Facts about the current CUDA device used to size grids (internal header).
#pragma once
#include <cuda_runtime.h>

namespace fps {

// Streaming multiprocessors of the current device (1 if the query fails).
inline int current_sm_count()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return 1;
    return sms;
}

}  // namespace fps
