// FastConv TMA-fed kernel for float16 inputs (staged in their own type, widened to
// FP32 exactly).
#include "conv_tma.cuh"

namespace ft_conv {

ft_status launch_conv_tma_f16(const ConvParams &p, int64_t planes, cudaStream_t s, bool *used)
{
    return launch_conv_tma_t<__half>(p, planes, s, used);
}

}  // namespace ft_conv
