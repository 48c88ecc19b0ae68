// FastConv TMA-fed kernel for int16 inputs (staged in their own type, widened to
// FP32 exactly).
#include "conv_tma.cuh"

namespace ft_conv {

ft_status launch_conv_tma_i16(const ConvParams &p, int64_t planes, cudaStream_t s, bool *used)
{
    return launch_conv_tma_t<short>(p, planes, s, used);
}

}  // namespace ft_conv
