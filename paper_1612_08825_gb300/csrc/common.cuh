// Shared host/device helpers of the fastttc CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "fastttc.h"

namespace ft {

// Records the text of a CUDA error for ft_last_cuda_error() (thread-local).
void set_cuda_error(cudaError_t e);

// the byte count TMA-fed kernels add to their barriers' expected bytes (test switch)
void set_tma_extra_tx(unsigned v);

// FT_OK if the last launch on this thread succeeded, else FT_ERR_CUDA.
inline ft_status check_launch()
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return FT_ERR_CUDA;
    }
    return FT_OK;
}

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// A named NVTX range around one C-ABI call, for timeline profilers (a push and a pop
// that cost a branch each when no tool is attached).
struct ApiRange {
    explicit ApiRange(const char *name) { nvtxRangePushA(name); }
    ~ApiRange() { nvtxRangePop(); }
    ApiRange(const ApiRange &) = delete;
    ApiRange &operator=(const ApiRange &) = delete;
};

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace ft

// the range of the enclosing C-ABI function, named after it
#define FT_API_RANGE ft::ApiRange ft_api_range_(__func__)

