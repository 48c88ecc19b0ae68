// FastConv: direct n-dimensional full convolution on sm_103a (Sec. IV-C, Eq. conv2).
//
// out[p] = sum_r k[r] * in[p - r] over every kernel index r with p - r inside the
// input; out extent N_d + K_d - 1.  The paper's rank-generic code generation
// (Sec. IV-C, steps 1-3) becomes one tiled 2-D plane kernel plus a loop over the
// leading (rank - 2) dimensions: output plane P receives, for every leading kernel
// index R with P - R inside the input, the 2-D convolution of input plane P - R with
// kernel slice R.  Rank 1 is a plane with one row.
//
// Tile kernel: a CTA of 256 threads owns an output tile of TH x TW.  It stages the
// zero-padded input tile ((TH + Kr - 1) x (TW + PADC) floats) and the kernel slice in
// shared memory with coalesced 16-byte loads, then every thread computes OY rows x 4
// consecutive columns from a register window of PADC + 4 floats per input row
// (float4 shared loads, conflict-free).  The output tile goes back through shared
// memory so that global stores are fully coalesced 128-byte rows whatever the
// alignment of the output row length.  Accumulation is FP32 FMA in a fixed order.
#include <cstdio>

#include "common.cuh"

namespace {

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
};

// TW = 128 * WX columns, TH = OY * (8 / WX) rows; PADC >= Kc - 1, multiple of 4.
template <int PADC, int OY, int WX>
__global__ void __launch_bounds__(kThreads)
conv_tile_kernel(const ConvParams p)
{
    constexpr int TW = 128 * WX;
    constexpr int TH = OY * (8 / WX);
    constexpr int SW = TW + PADC;        // shared row width, floats (multiple of 4)
    constexpr int SW4 = SW / 4;
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);

    const int Kr = (int)p.Kr, Kc = (int)p.Kc;
    const int SH = TH + Kr - 1;
    float *ks = sm + SH * SW;            // kernel slice, Kr * Kc floats

    const int tid = threadIdx.x;
    const int64_t bid = blockIdx.x;
    const int64_t plane = bid / p.tiles_per_plane;
    const int64_t t = bid - plane * p.tiles_per_plane;
    const int64_t ty = t / p.tiles_x;
    const int64_t tx = t - ty * p.tiles_x;
    const int64_t oy0 = ty * TH, ox0 = tx * TW;

    int64_t pm[FT_MAX_NDIM];
    {
        int64_t r = plane;
        for (int d = p.nlead - 1; d >= 0; --d) {
            pm[d] = r % p.out_lead[d];
            r /= p.out_lead[d];
        }
    }

    const int c0 = 4 * (tid % (32 * WX));
    const int r0 = OY * (tid / (32 * WX));

    float acc[OY][4];
#pragma unroll
    for (int y = 0; y < OY; ++y)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[y][c] = 0.f;

    bool first = true;
    for (int64_t R = 0; R < p.k_lead_total; ++R) {
        // input plane Q = P - R (leading dims), skipped when outside the input
        int64_t q = 0, rr = R, stride = 1;
        bool inside = true;
        for (int d = p.nlead - 1; d >= 0; --d) {
            int64_t rd = rr % p.k_lead[d];
            rr /= p.k_lead[d];
            int64_t qd = pm[d] - rd;
            if (qd < 0 || qd >= p.in_lead[d]) inside = false;
            q += qd * stride;
            stride *= p.in_lead[d];
        }
        if (!inside) continue;           // uniform over the CTA
        if (!first) __syncthreads();
        first = false;

        const float *src = p.in + q * p.Nr * p.Nc;
        const float *kk = p.ker + R * p.Kr * p.Kc;
        for (int i = tid; i < Kr * Kc; i += kThreads) ks[i] = __ldg(kk + i);

        const int64_t iy0 = oy0 - (Kr - 1), ix0 = ox0 - PADC;
        if (p.vec_in) {
            for (int i = tid; i < SH * SW4; i += kThreads) {
                const int r = i / SW4, c4 = i - r * SW4;
                const int64_t gy = iy0 + r, gx = ix0 + 4 * c4;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (gy >= 0 && gy < p.Nr && gx >= 0 && gx < p.Nc)
                    v = __ldg(reinterpret_cast<const float4 *>(src + gy * p.Nc + gx));
                smem4[i] = v;
            }
        } else {
            for (int i = tid; i < SH * SW; i += kThreads) {
                const int r = i / SW, c = i - r * SW;
                const int64_t gy = iy0 + r, gx = ix0 + c;
                float v = 0.f;
                if (gy >= 0 && gy < p.Nr && gx >= 0 && gx < p.Nc) v = __ldg(src + gy * p.Nc + gx);
                sm[i] = v;
            }
        }
        __syncthreads();

        // shared row r0 + ir holds input row oy0 + r0 + ir - (Kr - 1); it feeds output
        // rows y = ir - (Kr - 1) + a for kernel rows a.
        for (int ir = 0; ir < OY + Kr - 1; ++ir) {
            float win[PADC + 4];
            const float4 *rowp = reinterpret_cast<const float4 *>(sm + (r0 + ir) * SW + c0);
#pragma unroll
            for (int v = 0; v < (PADC + 4) / 4; ++v) {
                const float4 f = rowp[v];
                win[4 * v + 0] = f.x;
                win[4 * v + 1] = f.y;
                win[4 * v + 2] = f.z;
                win[4 * v + 3] = f.w;
            }
#pragma unroll
            for (int y = 0; y < OY; ++y) {
                const int a = y + Kr - 1 - ir;
                if (a < 0 || a >= Kr) continue;
                const float *krow = ks + a * Kc;
#pragma unroll
                for (int b = 0; b <= PADC; ++b) {
                    if (b >= Kc) break;
                    const float kv = krow[b];
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[y][c] = fmaf(kv, win[c - b + PADC], acc[y][c]);
                }
            }
        }
    }

    // stage the output tile in shared memory, then store coalesced rows
    __syncthreads();
#pragma unroll
    for (int y = 0; y < OY; ++y)
        *reinterpret_cast<float4 *>(sm + (r0 + y) * TW + c0) =
            make_float4(acc[y][0], acc[y][1], acc[y][2], acc[y][3]);
    __syncthreads();
    float *dst = p.out + plane * p.Mr * p.Mc;
    const int64_t rows = p.Mr - oy0 < TH ? p.Mr - oy0 : TH;
    const int64_t cols = p.Mc - ox0 < TW ? p.Mc - ox0 : TW;
    for (int i = tid; i < TH * TW; i += kThreads) {
        const int r = i / TW, c = i - r * TW;
        if (r < rows && c < cols) dst[(oy0 + r) * p.Mc + ox0 + c] = sm[i];
    }
}

// Fallback for kernels too large for the tiled path: one thread per output element.
__global__ void __launch_bounds__(kThreads)
conv_direct_kernel(const ConvParams p, int64_t total)
{
    const int64_t o = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (o >= total) return;
    const int64_t plane_size = p.Mr * p.Mc;
    const int64_t plane = o / plane_size;
    const int64_t rem = o - plane * plane_size;
    const int64_t oy = rem / p.Mc, ox = rem - oy * p.Mc;
    int64_t pm[FT_MAX_NDIM];
    {
        int64_t r = plane;
        for (int d = p.nlead - 1; d >= 0; --d) {
            pm[d] = r % p.out_lead[d];
            r /= p.out_lead[d];
        }
    }
    float acc = 0.f;
    for (int64_t R = 0; R < p.k_lead_total; ++R) {
        int64_t q = 0, rr = R, stride = 1;
        bool inside = true;
        for (int d = p.nlead - 1; d >= 0; --d) {
            int64_t rd = rr % p.k_lead[d];
            rr /= p.k_lead[d];
            int64_t qd = pm[d] - rd;
            if (qd < 0 || qd >= p.in_lead[d]) inside = false;
            q += qd * stride;
            stride *= p.in_lead[d];
        }
        if (!inside) continue;
        const float *src = p.in + q * p.Nr * p.Nc;
        const float *kk = p.ker + R * p.Kr * p.Kc;
        const int64_t a_lo = oy - (p.Nr - 1) > 0 ? oy - (p.Nr - 1) : 0;
        const int64_t a_hi = oy < p.Kr - 1 ? oy : p.Kr - 1;
        const int64_t b_lo = ox - (p.Nc - 1) > 0 ? ox - (p.Nc - 1) : 0;
        const int64_t b_hi = ox < p.Kc - 1 ? ox : p.Kc - 1;
        for (int64_t a = a_lo; a <= a_hi; ++a)
            for (int64_t b = b_lo; b <= b_hi; ++b)
                acc = fmaf(__ldg(kk + a * p.Kc + b), __ldg(src + (oy - a) * p.Nc + (ox - b)), acc);
    }
    p.out[o] = acc;
}

template <int PADC, int OY, int WX>
ft_status launch_tile(const ConvParams &p0, int64_t planes, cudaStream_t s)
{
    constexpr int TW = 128 * WX;
    constexpr int TH = OY * (8 / WX);
    ConvParams p = p0;
    const int64_t tiles_y = ft::ceil_div(p.Mr, TH);
    p.tiles_x = ft::ceil_div(p.Mc, TW);
    p.tiles_per_plane = tiles_y * p.tiles_x;
    const int64_t blocks = planes * p.tiles_per_plane;
    if (blocks > 0x7fffffffLL) return FT_ERR_UNSUPPORTED;
    const size_t smem = sizeof(float) * ((size_t)(TH + p.Kr - 1) * (TW + PADC) + (size_t)(p.Kr * p.Kc));
    if (smem > 48 * 1024) {              // opt-in above 48 KB (current device)
        cudaError_t e = cudaFuncSetAttribute(conv_tile_kernel<PADC, OY, WX>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) {
            ft::set_cuda_error(e);
            return FT_ERR_CUDA;
        }
    }
    conv_tile_kernel<PADC, OY, WX><<<(unsigned)blocks, kThreads, smem, s>>>(p);
    return ft::check_launch();
}

template <int OY, int WX>
ft_status launch_by_pad(const ConvParams &p, int64_t planes, cudaStream_t s)
{
    const int64_t need = p.Kc - 1;
    if (need <= 4) return launch_tile<4, OY, WX>(p, planes, s);
    if (need <= 8) return launch_tile<8, OY, WX>(p, planes, s);
    if (need <= 16) return launch_tile<16, OY, WX>(p, planes, s);
    if (need <= 32) return launch_tile<32, OY, WX>(p, planes, s);
    return launch_tile<64, OY, WX>(p, planes, s);
}

}  // namespace

extern "C" ft_status fastconv_out_dims(int nd, const int64_t *dims, const int64_t *kdims,
                                       int64_t *out_dims)
{
    if (!dims || !kdims || !out_dims) return FT_ERR_INVALID_ARG;
    if (nd < 1 || nd > FT_MAX_NDIM) return FT_ERR_SHAPE;
    for (int d = 0; d < nd; ++d)
        if (dims[d] < 1 || kdims[d] < 1) return FT_ERR_SHAPE;
    for (int d = 0; d < nd; ++d) out_dims[d] = dims[d] + kdims[d] - 1;
    return FT_OK;
}

extern "C" ft_status fastconv_nd(const float *input, const int64_t *dims, int nd,
                                 const float *kernel, const int64_t *kdims, float *out,
                                 void *stream)
{
    if (!input || !dims || !kernel || !kdims || !out) return FT_ERR_INVALID_ARG;
    int64_t odims[FT_MAX_NDIM];
    ft_status st = fastconv_out_dims(nd, dims, kdims, odims);
    if (st != FT_OK) return st;
    // overflow guard: every size must stay below 2^62
    const int64_t lim = (int64_t)1 << 62;
    int64_t tot_in = 1, tot_k = 1, tot_out = 1;
    for (int d = 0; d < nd; ++d) {
        if (odims[d] > lim / tot_out || dims[d] > lim / tot_in || kdims[d] > lim / tot_k)
            return FT_ERR_UNSUPPORTED;
        tot_in *= dims[d];
        tot_k *= kdims[d];
        tot_out *= odims[d];
    }

    ConvParams p{};
    p.in = input;
    p.ker = kernel;
    p.out = out;
    p.nlead = nd >= 2 ? nd - 2 : 0;
    p.k_lead_total = 1;
    int64_t planes = 1;
    for (int d = 0; d < p.nlead; ++d) {
        p.in_lead[d] = dims[d];
        p.k_lead[d] = kdims[d];
        p.out_lead[d] = odims[d];
        p.k_lead_total *= kdims[d];
        planes *= odims[d];
    }
    p.Nr = nd >= 2 ? dims[nd - 2] : 1;
    p.Kr = nd >= 2 ? kdims[nd - 2] : 1;
    p.Mr = nd >= 2 ? odims[nd - 2] : 1;
    p.Nc = dims[nd - 1];
    p.Kc = kdims[nd - 1];
    p.Mc = odims[nd - 1];
    p.vec_in = ((reinterpret_cast<uintptr_t>(input) & 15) == 0 && (p.Nc & 3) == 0) ? 1 : 0;

    cudaStream_t s = ft::as_stream(stream);
    const bool tiled = p.Kc <= 65 && p.Kr <= 129;
    if (!tiled) {
        if (tot_out / 256 + 1 > 0x7fffffffLL) return FT_ERR_UNSUPPORTED;
        const unsigned blocks = (unsigned)ft::ceil_div(tot_out, kThreads);
        conv_direct_kernel<<<blocks, kThreads, 0, s>>>(p, tot_out);
        return ft::check_launch();
    }
    if (p.Mr == 1) return launch_by_pad<1, 8>(p, planes, s);          // rank 1 (one row)
    if (p.Kr * p.Kc <= 16) return launch_by_pad<4, 1>(p, planes, s);  // small, memory-bound
    return launch_by_pad<8, 1>(p, planes, s);                           // FMA-bound
}
