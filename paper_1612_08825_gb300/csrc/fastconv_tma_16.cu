// FastConv TMA-fed kernel for 16-bit inputs: the dispatcher over int16, float16 and
// bfloat16 (each instantiated in its own unit: fastconv_tma_i16.cu, _f16.cu, _bf16.cu).
#include "conv.cuh"

namespace ft_conv {

ft_status launch_conv_tma_i16(const ConvParams &p, int64_t planes, cudaStream_t s, bool *used);
ft_status launch_conv_tma_f16(const ConvParams &p, int64_t planes, cudaStream_t s, bool *used);
ft_status launch_conv_tma_bf16(const ConvParams &p, int64_t planes, cudaStream_t s, bool *used);

ft_status launch_conv_tma_16(const ConvParams &p, int64_t planes, cudaStream_t s, bool *used)
{
    switch (p.in_dtype) {
    case FT_I16: return launch_conv_tma_i16(p, planes, s, used);
    case FT_F16: return launch_conv_tma_f16(p, planes, s, used);
    case FT_BF16: return launch_conv_tma_bf16(p, planes, s, used);
    default: *used = false; return FT_OK;
    }
}

}  // namespace ft_conv
