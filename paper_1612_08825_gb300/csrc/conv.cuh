// Shared declarations of the FastConv translation units (not part of the C ABI).
#pragma once

#include "common.cuh"

namespace ft_conv {

constexpr int kThreads = 256;

struct ConvParams {
    const float *in;
    const float *ker;
    float *out;
    int nlead;                           // number of leading dimensions (rank - 2, or 0)
    int64_t in_lead[FT_MAX_NDIM];        // leading input extents
    int64_t k_lead[FT_MAX_NDIM];         // leading kernel extents
    int64_t out_lead[FT_MAX_NDIM];       // leading output extents
    int64_t k_lead_total;                // prod(k_lead)
    int64_t Nr, Nc, Kr, Kc, Mr, Mc;      // plane extents: input, kernel, output
    int64_t tiles_x, tiles_per_plane;
    int vec_in;                          // 1: input rows allow 16-byte loads
    int vec_out;                         // 1: output rows allow 16-byte stores
    const void *in_t;                    // input of another element type (FT_U8, FT_I16, FT_F16, FT_BF16)
    int in_dtype;                        // element type of in_t
};

// input plane feeding output plane `plane` through leading kernel index R, or -1 when
// it lies outside the input (ranks <= 3 need no division)
__device__ __forceinline__ int64_t lead_plane(const ConvParams &p, int64_t plane, int64_t R)
{
    if (p.nlead == 0) return 0;
    if (p.nlead == 1) {
        const int64_t q = plane - R;
        return (q >= 0 && q < p.in_lead[0]) ? q : -1;
    }
    int64_t q = 0, stride = 1, rp = plane, rr = R;
    for (int d = p.nlead - 1; d >= 0; --d) {
        const int64_t pd = rp % p.out_lead[d], rd = rr % p.k_lead[d];
        rp /= p.out_lead[d];
        rr /= p.k_lead[d];
        const int64_t qd = pd - rd;
        if (qd < 0 || qd >= p.in_lead[d]) return -1;
        q += qd * stride;
        stride *= p.in_lead[d];
    }
    return q;
}

// the NTAP taps of one kernel row (float4 groups in shared memory) applied to one
// output row's four columns from the thread's window: acc[c] += k[b] * in[c - b]
template <int NTAP, int PADC>
__device__ __forceinline__ void fma_row(float (&acc)[4], const float (&win)[PADC + 4], const float4 *krow)
{
#pragma unroll
    for (int g = 0; g < (NTAP + 3) / 4; ++g) {
        const float4 k4 = krow[g];
        const float kv[4] = {k4.x, k4.y, k4.z, k4.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int b = 4 * g + j;
            if (b < NTAP) {
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[c] = fmaf(kv[j], win[c - b + PADC], acc[c]);
            }
        }
    }
}

template <int PADC>
__device__ __forceinline__ void load_window(float (&win)[PADC + 4], const float *row)
{
    const float4 *r4 = reinterpret_cast<const float4 *>(row);
#pragma unroll
    for (int v = 0; v < (PADC + 4) / 4; ++v) {
        const float4 f = r4[v];
        win[4 * v + 0] = f.x;
        win[4 * v + 1] = f.y;
        win[4 * v + 2] = f.z;
        win[4 * v + 3] = f.w;
    }
}

// the persistent TMA-fed kernel for kernels of at most 17 columns when the input rows
// meet the copy engine's rules; *used = false otherwise.  launch_conv_tma reads p.in
// (FP32); the typed launchers read p.in_t (their element type).
ft_status launch_conv_tma(const ConvParams &p, int64_t planes, cudaStream_t s, bool *used);
ft_status launch_conv_tma_u8(const ConvParams &p, int64_t planes, cudaStream_t s, bool *used);
ft_status launch_conv_tma_16(const ConvParams &p, int64_t planes, cudaStream_t s, bool *used);

// device address of the FastConv status word (set when a bounded wait gives up)
int *fastconv_status_word();

}  // namespace ft_conv
