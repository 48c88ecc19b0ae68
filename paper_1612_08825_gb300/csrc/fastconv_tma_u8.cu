// FastConv TMA-fed kernel for uint8 inputs (staged as bytes, widened to FP32 exactly).
#include "conv_tma.cuh"

namespace ft_conv {

ft_status launch_conv_tma_u8(const ConvParams &p, int64_t planes, cudaStream_t s, bool *used)
{
    return launch_conv_tma_t<unsigned char>(p, planes, s, used);
}

}  // namespace ft_conv
