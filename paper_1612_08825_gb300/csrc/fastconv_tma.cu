// FastConv TMA-fed kernel for FP32 inputs, the FastConv status word and fastconv_check.
#include <mutex>

#include "conv_tma.cuh"

// set to 1 when a wait of a TMA-fed FastConv kernel gave up (read by fastconv_check)
__device__ int g_fastconv_status;

namespace ft_conv {

int *fastconv_status_word()
{
    void *st = nullptr;
    if (cudaGetSymbolAddress(&st, g_fastconv_status) != cudaSuccess) return nullptr;
    return static_cast<int *>(st);
}

ft_status launch_conv_tma(const ConvParams &p, int64_t planes, cudaStream_t s, bool *used)
{
    return launch_conv_tma_t<float>(p, planes, s, used);
}

}  // namespace ft_conv

extern "C" ft_status fastconv_check(void *stream)
{
    int v = 0;
    const int zero = 0;
    cudaError_t e = cudaStreamSynchronize(ft::as_stream(stream));
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&v, g_fastconv_status, sizeof(int));
    if (e == cudaSuccess && v) e = cudaMemcpyToSymbol(g_fastconv_status, &zero, sizeof(int));
    if (e != cudaSuccess) {
        ft::set_cuda_error(e);
        return FT_ERR_CUDA;
    }
    return v ? FT_ERR_TIMEOUT : FT_OK;
}
