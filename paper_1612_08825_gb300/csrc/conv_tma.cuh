// FastConv: the persistent FMA-bound kernel fed by the Tensor Memory Accelerator
// (Sec. IV-C, Eq. conv2 read as the full linear convolution), as a template over the
// input element type; instantiated by fastconv_tma*.cu.
#pragma once

#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "conv.cuh"
#include "tma.cuh"

namespace ft_conv {

namespace conv_tma {

constexpr int OY = 4, TH = 8 * OY, TW = 128;

// Staged element types: the copy engine moves the input in its own type (a box row is a
// whole number of 16-byte units, so the box starts PADT >= PADC columns left of the
// tile), and the window loads widen four elements at a time to FP32, exactly.
template <typename T> struct Elem;
template <> struct Elem<float> {
    static constexpr CUtensorMapDataType map = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    __device__ static void load4(const float *p, float *w)
    {
        const float4 f = *reinterpret_cast<const float4 *>(p);
        w[0] = f.x; w[1] = f.y; w[2] = f.z; w[3] = f.w;
    }
};
template <> struct Elem<unsigned char> {
    static constexpr CUtensorMapDataType map = CU_TENSOR_MAP_DATA_TYPE_UINT8;
    __device__ static void load4(const unsigned char *p, float *w)
    {
        // 2^23 + v assembled in the mantissa, minus 2^23: exact
        const uint32_t x = *reinterpret_cast<const uint32_t *>(p);
        w[0] = __uint_as_float(__byte_perm(x, 0x4B000000u, 0x7440)) - 8388608.f;
        w[1] = __uint_as_float(__byte_perm(x, 0x4B000000u, 0x7441)) - 8388608.f;
        w[2] = __uint_as_float(__byte_perm(x, 0x4B000000u, 0x7442)) - 8388608.f;
        w[3] = __uint_as_float(__byte_perm(x, 0x4B000000u, 0x7443)) - 8388608.f;
    }
};
template <> struct Elem<short> {
    // the copy moves the bits as they are (zero fill is the value 0)
    static constexpr CUtensorMapDataType map = CU_TENSOR_MAP_DATA_TYPE_UINT16;
    __device__ static void load4(const short *p, float *w)
    {
        // v + 2^15 (sign bit flipped) assembled as 2^23 + (v + 2^15), minus 2^23 + 2^15: exact
        const uint2 x = *reinterpret_cast<const uint2 *>(p);
        const uint32_t a = x.x ^ 0x80008000u, b = x.y ^ 0x80008000u;
        w[0] = __uint_as_float(__byte_perm(a, 0x4B000000u, 0x7410)) - 8421376.f;
        w[1] = __uint_as_float(__byte_perm(a, 0x4B000000u, 0x7432)) - 8421376.f;
        w[2] = __uint_as_float(__byte_perm(b, 0x4B000000u, 0x7410)) - 8421376.f;
        w[3] = __uint_as_float(__byte_perm(b, 0x4B000000u, 0x7432)) - 8421376.f;
    }
};
template <> struct Elem<__half> {
    static constexpr CUtensorMapDataType map = CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    __device__ static void load4(const __half *p, float *w)
    {
        const uint2 x = *reinterpret_cast<const uint2 *>(p);
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&x.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&x.y));
        w[0] = a.x; w[1] = a.y; w[2] = b.x; w[3] = b.y;
    }
};
template <> struct Elem<__nv_bfloat16> {
    static constexpr CUtensorMapDataType map = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    __device__ static void load4(const __nv_bfloat16 *p, float *w)
    {
        // a bfloat16 is the upper half of the float with the same value
        const uint2 x = *reinterpret_cast<const uint2 *>(p);
        w[0] = __uint_as_float(x.x << 16); w[1] = __uint_as_float(x.x & 0xffff0000u);
        w[2] = __uint_as_float(x.y << 16); w[3] = __uint_as_float(x.y & 0xffff0000u);
    }
};

// columns a box is widened by on the left: PADC rounded up to whole 16-byte units of T
template <typename T, int PADC>
__host__ __device__ constexpr int padt() { return (PADC * (int)sizeof(T) + 15) / 16 * 16 / (int)sizeof(T); }

template <typename T, int PADC>
__device__ __forceinline__ void load_window_t(float (&win)[PADC + 4], const T *row)
{
#pragma unroll
    for (int v = 0; v < (PADC + 4) / 4; ++v) Elem<T>::load4(row + 4 * v, win + 4 * v);
}

struct Params {
    ConvParams p;
    int planes;                  // output planes
    int tiles_x, tiles_per_plane;
    int SH;                      // staged rows per tile: TH + Kr - 1
    int buf_bytes;               // bytes per staging buffer (whole 128-byte units)
    int store_tma;               // 1: output tiles leave by TMA store, 0: by plain stores
    int *status;                 // set to 1 when a wait gives up
    unsigned extra_tx;           // added to the expected bytes (0; tests of the timeout path)
};

// work items: (plane, tile, R) with tile t of output plane `plane` (the CTA's tiles are
// blockIdx.x, + gridDim.x, ... over all planes) and leading kernel index R whose input
// plane q exists
struct Item {
    int plane, tile;
    int64_t R, q;
};

// the first item at or after `it` (R included)
__device__ __forceinline__ bool advance(const Params &cp, Item &it)
{
    while (it.plane < cp.planes) {
        for (; it.R < cp.p.k_lead_total; ++it.R) {
            it.q = lead_plane(cp.p, it.plane, it.R);
            if (it.q >= 0) return true;
        }
        it.R = 0;
        it.tile += gridDim.x;
        while (it.tile >= cp.tiles_per_plane && it.plane < cp.planes) {
            it.tile -= cp.tiles_per_plane;
            ++it.plane;
        }
    }
    return false;
}

// elected thread: the staged box of item (t, q) into `buf` (rows oy0 - (Kr - 1) ..,
// columns ox0 - PADC ..; the copy engine zero-fills outside the input)
template <typename T, int PADT>
__device__ __forceinline__ void issue(const CUtensorMap *m, const Params &cp, const Item &it, unsigned char *buf,
                                      uint64_t *bar)
{
    const int ty = it.tile / cp.tiles_x, tx = it.tile - ty * cp.tiles_x;
    ft_tma::fence_proxy_async();
    ft_tma::mbar_expect_tx(bar, (uint32_t)(cp.SH * (TW + PADT) * (int)sizeof(T)) + cp.extra_tx);
    ft_tma::tma_load_3d(buf, m, tx * TW - PADT, ty * TH - ((int)cp.p.Kr - 1), (int)it.q, bar);
}

// A CTA walks tiles blockIdx.x, + gridDim.x, ... and, for each, the leading kernel
// indices whose input plane exists (one work item each).  One elected thread brings the
// next item's box into the other of two staging buffers while the CTA computes the
// current one (completion tracked by an mbarrier with the box's byte count), so the
// copies overlap the FMAs.  The arithmetic per item is that of conv_fma_kernel (three
// branch-free phases of staged rows, OY rows x 4 columns per thread, kernel taps four
// at a time from shared memory); all kernel slices are staged once.  Finished tiles go
// out through a shared-memory staging tile, by TMA store when the output rows allow it.
// Every wait is bounded: on expiry the CTA sets the status word, waits a bounded time
// for its copy in flight, and returns.
template <typename T, int NTAP, bool SMALLR>
__global__ void __launch_bounds__(kThreads, NTAP <= 9 ? 3 : 2)
conv_tma_kernel(const __grid_constant__ CUtensorMap in_map, const __grid_constant__ CUtensorMap out_map,
                const Params cp)
{
    constexpr int PADC = (NTAP - 1 + 3) & ~3;
    constexpr int PADT = padt<T, PADC>();
    constexpr int BW = TW + PADT;        // staged row, elements of T
    constexpr int KS = (NTAP + 3) & ~3;
    extern __shared__ __align__(128) unsigned char smb[];
    const ConvParams &p = cp.p;
    const int tid = threadIdx.x;
    const int Kr = (int)p.Kr, Kc = (int)p.Kc;
    unsigned char *buf0 = smb, *buf1 = smb + cp.buf_bytes;
    float *so = reinterpret_cast<float *>(smb + 2 * cp.buf_bytes);
    float *ks = so + TH * TW;
    const int nk = (int)p.k_lead_total * Kr * KS;
    uint64_t *bar = reinterpret_cast<uint64_t *>(ks + ((nk + 3) & ~3));
    // the copy engine writes 128-byte aligned boxes; refuse (and report) otherwise
    if (ft_tma::smem_addr(smb) & 127) {
        if (tid == 0) atomicExch(cp.status, 2);
        return;
    }
    for (int i = tid; i < nk; i += kThreads) {
        const int row = i / KS, b = i - row * KS;      // row = R * Kr + a
        ks[i] = b < Kc ? __ldg(p.ker + (int64_t)row * Kc + b) : 0.f;
    }
    if (tid == 0) {
        ft_tma::mbar_init(&bar[0], 1);
        ft_tma::mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    Item it{0, (int)blockIdx.x, 0, 0};
    while (it.tile >= cp.tiles_per_plane && it.plane < cp.planes) {
        it.tile -= cp.tiles_per_plane;
        ++it.plane;
    }
    bool have = advance(cp, it);
    if (tid == 0 && have) issue<T, PADT>(&in_map, cp, it, buf0, &bar[0]);

    const int c0 = 4 * (tid & 31);
    const int r0 = OY * (tid >> 5);
    float acc[OY][4];
#pragma unroll
    for (int y = 0; y < OY; ++y)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[y][c] = 0.f;

    for (int k = 0; have; ++k) {
        Item nx = it;
        ++nx.R;
        const bool hn = advance(cp, nx);
        const T *cur = reinterpret_cast<const T *>((k & 1) ? buf1 : buf0);
        // the other buffer was released by the barrier that ended the previous item
        if (tid == 0 && hn) issue<T, PADT>(&in_map, cp, nx, (k & 1) ? buf0 : buf1, &bar[(k + 1) & 1]);
        const bool ok = ft_tma::mbar_wait(&bar[k & 1], (k >> 1) & 1);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(cp.status, 1);
                if (hn) ft_tma::mbar_wait(&bar[(k + 1) & 1], ((k + 1) >> 1) & 1);
                if (cp.store_tma) ft_tma::bulk_wait();
            }
            __syncthreads();
            return;
        }

        const float4 *ks4 = reinterpret_cast<const float4 *>(ks + (int64_t)it.R * Kr * KS);
        const T *base = cur + r0 * BW + c0 + (PADT - PADC);
        float win[PADC + 4];
        if constexpr (SMALLR) {
            // kernels of fewer rows than OY (Kr <= 3): each of the OY + Kr - 1 staged rows
            // is loaded once and applied to every output row it reaches (kernel row
            // a = y + Kr - 1 - ir); rows are taken last to first, so that each output
            // row sees its kernel rows in increasing order
#pragma unroll
            for (int ir = OY + 1; ir >= 0; --ir) {
                if (ir < OY + Kr - 1) {
                    load_window_t<T, PADC>(win, base + ir * BW);
#pragma unroll
                    for (int y = 0; y < OY; ++y) {
                        const int a = y + Kr - 1 - ir;
                        if (a >= 0 && a < Kr) fma_row<NTAP, PADC>(acc[y], win, ks4 + a * (KS / 4));
                    }
                }
            }
        } else {
#pragma unroll
        for (int ir = 0; ir < OY - 1; ++ir) {
            load_window_t<T, PADC>(win, base + ir * BW);
#pragma unroll
            for (int y = 0; y <= ir; ++y) fma_row<NTAP, PADC>(acc[y], win, ks4 + (y + Kr - 1 - ir) * (KS / 4));
        }
        for (int ir = OY - 1; ir < Kr; ++ir) {
            load_window_t<T, PADC>(win, base + ir * BW);
            const float4 *kb = ks4 + (Kr - 1 - ir) * (KS / 4);
#pragma unroll
            for (int y = 0; y < OY; ++y) fma_row<NTAP, PADC>(acc[y], win, kb + y * (KS / 4));
        }
#pragma unroll
        for (int t3 = 1; t3 < OY; ++t3) {
            load_window_t<T, PADC>(win, base + (Kr - 1 + t3) * BW);
#pragma unroll
            for (int y = t3; y < OY; ++y) fma_row<NTAP, PADC>(acc[y], win, ks4 + (y - t3) * (KS / 4));
        }
        }
        __syncthreads();          // buffer `cur` is free for the copy issued next

        if (!hn || nx.tile != it.tile || nx.plane != it.plane) {
            // the tile is complete: out through the staging tile
            const int plane = it.plane;
            const int ty = it.tile / cp.tiles_x, tx = it.tile - ty * cp.tiles_x;
            if (cp.store_tma && tid == 0) ft_tma::bulk_wait_read();   // the previous store has read `so`
            __syncthreads();
#pragma unroll
            for (int y = 0; y < OY; ++y)
                *reinterpret_cast<float4 *>(so + (r0 + y) * TW + c0) =
                    make_float4(acc[y][0], acc[y][1], acc[y][2], acc[y][3]);
            if (cp.store_tma) ft_tma::fence_proxy_async();
            __syncthreads();
            if (cp.store_tma) {
                if (tid == 0) {
                    ft_tma::tma_store_3d(&out_map, so, tx * TW, ty * TH, plane);
                    ft_tma::bulk_commit();
                }
            } else {
                // plain stores: a thread keeps one column (pair) and walks rows
                const int64_t oy0 = (int64_t)ty * TH, ox0 = (int64_t)tx * TW;
                const int rows = p.Mr - oy0 < TH ? (int)(p.Mr - oy0) : TH;
                const int cols = p.Mc - ox0 < TW ? (int)(p.Mc - ox0) : TW;
                float *dst = p.out + ((int64_t)plane * p.Mr + oy0) * p.Mc + ox0;
                if (cp.store_tma == 0 && (p.Mc & 1) == 0 && (reinterpret_cast<uintptr_t>(p.out) & 7) == 0) {
                    const int c = 2 * (tid & (TW / 2 - 1));
                    if (c < cols) {
                        for (int r = tid / (TW / 2); r < rows; r += kThreads / (TW / 2)) {
                            const float2 v = *reinterpret_cast<const float2 *>(so + r * TW + c);
                            if (c + 1 < cols) *reinterpret_cast<float2 *>(dst + r * p.Mc + c) = v;
                            else dst[r * p.Mc + c] = v.x;
                        }
                    }
                } else {
                    const int c = tid & (TW - 1);
                    if (c < cols)
                        for (int r = tid / TW; r < rows; r += kThreads / TW) dst[r * p.Mc + c] = so[r * TW + c];
                }
            }
#pragma unroll
            for (int y = 0; y < OY; ++y)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[y][c] = 0.f;
        }
        it = nx;
        have = hn;
    }
    if (cp.store_tma && tid == 0) ft_tma::bulk_wait();
}

}  // namespace conv_tma

// 3-D map over `planes` planes of rows x cols elements (row-major, contiguous), box
// bw x bh x 1
inline bool plane_map(CUtensorMap *m, CUtensorMapDataType type, int es, const void *base, int64_t cols,
                      int64_t rows, int64_t planes, int bw, int bh)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = ft::tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)(cols * es), (cuuint64_t)(cols * rows * es)};
    const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, type, 3, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// the persistent TMA kernel when the input rows meet the copy engine's rules (16-byte
// aligned base, row length a multiple of 4 floats) and the staging fits; *used = false
// otherwise (the caller then takes conv_fma_kernel)
template <typename T, int NTAP, bool SMALLR>
ft_status launch_tma(const ConvParams &p, int64_t planes, cudaStream_t s, bool *used)
{
    using namespace conv_tma;
    constexpr int PADC = (NTAP - 1 + 3) & ~3;
    constexpr int PADT = padt<T, PADC>();
    constexpr int BW = TW + PADT;
    constexpr int KS = (NTAP + 3) & ~3;
    constexpr bool F32 = sizeof(T) == 4;
    *used = false;
    const void *in = F32 ? static_cast<const void *>(p.in) : p.in_t;
    // the copy engine needs a 16-byte aligned base and rows of whole 16-byte units
    if (!in || (reinterpret_cast<uintptr_t>(in) & 15) || ((p.Nc * (int64_t)sizeof(T)) & 15)) return FT_OK;
    if (p.Kr + TH - 1 > 256) return FT_OK;
    int64_t in_planes = 1;
    for (int d = 0; d < p.nlead; ++d) in_planes *= p.in_lead[d];
    const int64_t tiles_y = ft::ceil_div(p.Mr, TH), tiles_x = ft::ceil_div(p.Mc, TW);
    if (tiles_y * tiles_x * planes > 0x7fffffffLL) return FT_OK;
    Params cp{};
    cp.p = p;
    cp.planes = (int)planes;
    cp.tiles_x = (int)tiles_x;
    cp.tiles_per_plane = (int)(tiles_x * tiles_y);
    const int64_t total_tiles = planes * cp.tiles_per_plane;
    cp.SH = TH + (int)p.Kr - 1;
    cp.buf_bytes = (cp.SH * BW * (int)sizeof(T) + 127) / 128 * 128;
    const int64_t nk = p.k_lead_total * p.Kr * KS;
    const size_t smem = 2 * (size_t)cp.buf_bytes + sizeof(float) * (TH * TW + (size_t)((nk + 3) & ~3)) + 16;
    if (smem > 200 * 1024) return FT_OK;
    CUtensorMap in_map, out_map;
    if (!plane_map(&in_map, Elem<T>::map, (int)sizeof(T), in, p.Nc, p.Nr, in_planes, BW, cp.SH)) return FT_OK;
    cp.store_tma = (p.vec_out && plane_map(&out_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, p.out, p.Mc, p.Mr, planes,
                                           TW, TH)) ? 1 : 0;
    if (!cp.store_tma) out_map = in_map;            // unused
    int *st = fastconv_status_word();
    cudaError_t e = st ? cudaSuccess : cudaErrorInvalidSymbol;
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(conv_tma_kernel<T, NTAP, SMALLR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
    if (e == cudaSuccess)   // as much shared memory as the SM has: more resident CTAs
        e = cudaFuncSetAttribute(conv_tma_kernel<T, NTAP, SMALLR>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    int per_sm = 0, dev = 0, nsm = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, conv_tma_kernel<T, NTAP, SMALLR>, kThreads, smem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        ft::set_cuda_error(e);
        return FT_ERR_CUDA;
    }
    if (per_sm < 1) return FT_OK;
    cp.status = st;
    cp.extra_tx = ft::tma_extra_tx();
    const int64_t grid = std::min<int64_t>(total_tiles, (int64_t)per_sm * nsm);
    conv_tma_kernel<T, NTAP, SMALLR><<<(unsigned)grid, kThreads, smem, s>>>(in_map, out_map, cp);
    *used = true;
    return ft::check_launch();
}

template <typename T, int NTAP>
ft_status launch_tma_rows(const ConvParams &p, int64_t planes, cudaStream_t s, bool *used)
{
    return p.Kr >= conv_tma::OY ? launch_tma<T, NTAP, false>(p, planes, s, used)
                                : launch_tma<T, NTAP, true>(p, planes, s, used);
}

// taps per row rounded up to the next odd count (at most one zero tap per row)
template <typename T>
ft_status launch_conv_tma_t(const ConvParams &p, int64_t planes, cudaStream_t s, bool *used)
{
    *used = false;
    if (p.Kc > 17) return FT_OK;
    switch (p.Kc / 2) {
    case 0: return launch_tma_rows<T, 1>(p, planes, s, used);
    case 1: return launch_tma_rows<T, 3>(p, planes, s, used);
    case 2: return launch_tma_rows<T, 5>(p, planes, s, used);
    case 3: return launch_tma_rows<T, 7>(p, planes, s, used);
    case 4: return launch_tma_rows<T, 9>(p, planes, s, used);
    case 5: return launch_tma_rows<T, 11>(p, planes, s, used);
    case 6: return launch_tma_rows<T, 13>(p, planes, s, used);
    case 7: return launch_tma_rows<T, 15>(p, planes, s, used);
    default: return launch_tma_rows<T, 17>(p, planes, s, used);
    }
}

}  // namespace ft_conv
