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
//
// Kernels of up to 17 columns use the persistent TMA-fed kernel of fastconv_tma.cu
// when the input rows meet the copy engine's rules, else (4..129 rows) conv_fma_kernel:
// asynchronous zero-filling copies for the staging and a branch-free schedule of the
// multiply-adds.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "conv.cuh"

namespace {

using namespace ft_conv;

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
    const int KS = (Kc + 3) & ~3;        // kernel row stride in shared memory (zero-padded)
    float *ks = sm + SH * SW;            // kernel slice, Kr * KS floats
    const float4 *ks4 = reinterpret_cast<const float4 *>(ks);

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
        for (int i = tid; i < Kr * KS; i += kThreads) {
            const int a = i / KS, b = i - a * KS;
            ks[i] = b < Kc ? __ldg(kk + a * Kc + b) : 0.f;
        }

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
            // kernel taps four at a time (one broadcast 16-byte shared load feeds 16
            // FMAs); taps past Kc are zero in shared memory
#pragma unroll
            for (int y = 0; y < OY; ++y) {
                const int a = y + Kr - 1 - ir;
                if (a < 0 || a >= Kr) continue;
                const float4 *krow = ks4 + a * (KS / 4);
#pragma unroll
                for (int b4 = 0; b4 <= PADC / 4; ++b4) {
                    if (4 * b4 >= Kc) break;
                    const float4 k4 = krow[b4];
                    const float kv[4] = {k4.x, k4.y, k4.z, k4.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int b = 4 * b4 + j;
                        if (b > PADC) break;     // compile time: tap b reads window index c - b + PADC
#pragma unroll
                        for (int c = 0; c < 4; ++c) acc[y][c] = fmaf(kv[j], win[c - b + PADC], acc[y][c]);
                    }
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

// ---------------------------------------------------------------------------
// FMA-bound plane kernel (kernels of 4..17 rows and up to 17 columns)
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *ptr)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(ptr));
}

// 16-byte asynchronous global -> shared copy; bytes = 0 writes zeros and reads nothing
__device__ __forceinline__ void cp_async16(void *dst, const void *src, int bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// A CTA owns TH = 8 * OY output rows x 128 columns; thread (warp w, lane l) computes
// rows OY * w .. + OY - 1 and columns 4l .. 4l + 3.  The zero-padded input tile
// arrives by cp.async (out-of-image 16-byte groups are zero-filled by the copy, so
// every copy of the tile is in flight at once) and the kernel slice is stored with
// rows zero-padded to whole float4 groups.  Staged input row ir (0 .. OY + Kr - 2 for
// the thread) feeds output row y through kernel row a = y + Kr - 1 - ir; with
// Kr >= OY the valid (ir, y) pairs form three phases whose bounds are known at
// compile time except for the middle one's length (rows OY - 1 .. Kr - 1, where
// every output row is fed), so the multiply-add stream has no branches: each window
// of PADC + 4 floats is loaded once and one broadcast 16-byte load of the kernel feeds
// 16 FMAs.  Order per output: input rows ascending, taps ascending (FP32 FMA).
template <int NTAP, int OY>
__global__ void __launch_bounds__(kThreads, OY == 8 ? 2 : 3)
conv_fma_kernel(const ConvParams p)
{
    constexpr int PADC = (NTAP - 1 + 3) & ~3;
    constexpr int TW = 128;
    constexpr int TH = 8 * OY;
    constexpr int SW = TW + PADC;
    constexpr int SW4 = SW / 4;
    constexpr int KS = (NTAP + 3) & ~3;  // kernel row stride, floats
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);

    const int Kr = (int)p.Kr, Kc = (int)p.Kc;
    const int SH = TH + Kr - 1;
    float *ks = sm + SH * SW;
    const float4 *ks4 = reinterpret_cast<const float4 *>(ks);

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

    const int c0 = 4 * (tid & 31);
    const int r0 = OY * (tid >> 5);
    float acc[OY][4];
#pragma unroll
    for (int y = 0; y < OY; ++y)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[y][c] = 0.f;

    bool first = true;
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
        if (!inside) continue;           // uniform over the CTA
        if (!first) __syncthreads();
        first = false;

        const float *src = p.in + q * p.Nr * p.Nc;
        const float *kk = p.ker + R * p.Kr * p.Kc;
        for (int i = tid; i < Kr * KS; i += kThreads) {
            const int a = i / KS, b = i - a * KS;
            ks[i] = b < Kc ? __ldg(kk + a * Kc + b) : 0.f;
        }
        const int64_t iy0 = oy0 - (Kr - 1), ix0 = ox0 - PADC;
        if (p.vec_in) {
            for (int i = tid; i < SH * SW4; i += kThreads) {
                const int r = i / SW4, c4 = i - r * SW4;
                const int64_t gy = iy0 + r, gx = ix0 + 4 * c4;
                const bool ok = gy >= 0 && gy < p.Nr && gx >= 0 && gx < p.Nc;
                cp_async16(smem4 + i, ok ? src + gy * p.Nc + gx : src, ok ? 16 : 0);
            }
            cp_async_wait_all();
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

        const float *base = sm + r0 * SW + c0;
        float win[PADC + 4];
        // phase 1: input rows 0 .. OY - 2 feed output rows 0 .. ir
#pragma unroll
        for (int ir = 0; ir < OY - 1; ++ir) {
            load_window<PADC>(win, base + ir * SW);
#pragma unroll
            for (int y = 0; y <= ir; ++y) fma_row<NTAP, PADC>(acc[y], win, ks4 + (y + Kr - 1 - ir) * (KS / 4));
        }
        // phase 2: input rows OY - 1 .. Kr - 1 feed every output row
        for (int ir = OY - 1; ir < Kr; ++ir) {
            load_window<PADC>(win, base + ir * SW);
            const float4 *kb = ks4 + (Kr - 1 - ir) * (KS / 4);
#pragma unroll
            for (int y = 0; y < OY; ++y) fma_row<NTAP, PADC>(acc[y], win, kb + y * (KS / 4));
        }
        // phase 3: input rows Kr - 1 + t, t = 1 .. OY - 1, feed output rows t .. OY - 1
#pragma unroll
        for (int t3 = 1; t3 < OY; ++t3) {
            load_window<PADC>(win, base + (Kr - 1 + t3) * SW);
#pragma unroll
            for (int y = t3; y < OY; ++y) fma_row<NTAP, PADC>(acc[y], win, ks4 + (y - t3) * (KS / 4));
        }
    }

    // stage the output tile in shared memory, then store coalesced rows
    __syncthreads();
#pragma unroll
    for (int y = 0; y < OY; ++y)
        *reinterpret_cast<float4 *>(sm + (r0 + y) * TW + c0) = make_float4(acc[y][0], acc[y][1], acc[y][2], acc[y][3]);
    __syncthreads();
    float *dst = p.out + plane * p.Mr * p.Mc;
    const int64_t rows = p.Mr - oy0 < TH ? p.Mr - oy0 : TH;
    const int64_t cols = p.Mc - ox0 < TW ? p.Mc - ox0 : TW;
    if (p.vec_out) {
        for (int i = tid; i < TH * TW / 4; i += kThreads) {
            const int r = i / (TW / 4), c = 4 * (i - r * (TW / 4));
            if (r < rows && c < cols)
                *reinterpret_cast<float4 *>(dst + (oy0 + r) * p.Mc + ox0 + c) =
                    *reinterpret_cast<const float4 *>(sm + r * TW + c);
        }
    } else {
        for (int i = tid; i < TH * TW; i += kThreads) {
            const int r = i / TW, c = i - r * TW;
            if (r < rows && c < cols) dst[(oy0 + r) * p.Mc + ox0 + c] = sm[i];
        }
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

// Streaming kernel for small kernels (memory-bound): one warp per 128-column strip
// and RB output rows of one output plane, no shared memory and no barriers.  Lane l
// owns output columns ox0 + 4l .. 4l + 3.  Every input row the strip needs is loaded
// once per warp up front (16-byte loads; all loads in flight together); the KC - 1
// columns to the left come from lane l - 1 by shuffle (lane 0 loads them).  The KR
// previous rows of each of the KL input planes stay in registers.
// Grid: x = groups of 8 warps within a plane (a warp per strip x row block, row blocks
// fastest), y and z = the output plane (z counts 65535 planes), so that a warp finds its
// work with one 32-bit division and its input planes without any (lead_plane).
// main_strips: strips of 128 columns done as above; when the output's last strip has
// at most 4 columns it is not one of them: warps past main_strips * nrb take it with a
// lane per output row (32 rows per warp), so that it costs 1/4 of a warp per 8 rows
// instead of one (for example 257-column planes: 2 main strips and a 1-column tail).
template <int KL, int KR, int KC, int RB>
__global__ void __launch_bounds__(kThreads)
conv_rows_kernel(const ConvParams p, int nrb, int main_strips, int warps_per_plane, int64_t planes)
{
    constexpr int NROW = RB + KR - 1;            // input rows per warp
    constexpr int WN = KC + 3;                   // window: KC - 1 halo + 4 own columns
    const int lane = threadIdx.x & 31;
    const int wi = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    const int64_t plane = (int64_t)blockIdx.z * 65535 + blockIdx.y;
    if (wi >= warps_per_plane || plane >= planes) return;      // warp-uniform

    // input plane of each leading kernel index (-1: outside the input)
    int64_t q[KL];
#pragma unroll
    for (int R = 0; R < KL; ++R) q[R] = lead_plane(p, plane, R);

    if (wi >= main_strips * nrb) {
        // the narrow last strip: output row m, columns ox0 .. ox0 + w - 1 (w <= 4),
        // terms in the order of the main path (R, kernel row a, kernel column b)
        const int64_t m = (int64_t)(wi - main_strips * nrb) * 32 + lane;
        if (m >= p.Mr) return;
        const int64_t ox0 = (int64_t)main_strips * 128;
        const int w = (int)(p.Mc - ox0);
        float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int R = 0; R < KL; ++R) {
            if (q[R] < 0) continue;
            const float *src = p.in + q[R] * p.Nr * p.Nc;
#pragma unroll
            for (int a = 0; a < KR; ++a) {
                const int64_t gy = m - a;
                if (gy < 0 || gy >= p.Nr) continue;
#pragma unroll
                for (int b = 0; b < KC; ++b) {
                    const float kv = __ldg(p.ker + (R * KR + a) * KC + b);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int64_t gx = ox0 + c - b;
                        if (c < w && gx >= 0 && gx < p.Nc) o[c] = fmaf(kv, __ldg(src + gy * p.Nc + gx), o[c]);
                    }
                }
            }
        }
        float *orow = p.out + (plane * p.Mr + m) * p.Mc + ox0;
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (c < w) orow[c] = o[c];
        return;
    }
    const int strip = wi / nrb;
    const int64_t m0 = (int64_t)(wi - strip * nrb) * RB;
    const int64_t ox0 = (int64_t)strip * 128;
    const int64_t c0 = ox0 + 4 * lane;
    float kr[KL][KR][KC];
#pragma unroll
    for (int R = 0; R < KL; ++R)
#pragma unroll
        for (int a = 0; a < KR; ++a)
#pragma unroll
            for (int b = 0; b < KC; ++b) kr[R][a][b] = __ldg(p.ker + (R * KR + a) * KC + b);

    // phase 1: all loads (own 4 columns; lane 0 also the KC - 1 columns to the left)
    float own[KL][NROW][4];
    float left[KL][NROW][KC > 1 ? KC - 1 : 1];
#pragma unroll
    for (int R = 0; R < KL; ++R) {
        const float *src = q[R] >= 0 ? p.in + q[R] * p.Nr * p.Nc : nullptr;
#pragma unroll
        for (int t = 0; t < NROW; ++t) {
            const int64_t gy = m0 - (KR - 1) + t;
            const bool rok = src != nullptr && gy >= 0 && gy < p.Nr;
            const float *row = rok ? src + gy * p.Nc : nullptr;
            if (rok && p.vec_in && c0 + 4 <= p.Nc) {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(row + c0));
                own[R][t][0] = v.x; own[R][t][1] = v.y; own[R][t][2] = v.z; own[R][t][3] = v.w;
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c) own[R][t][c] = (rok && c0 + c < p.Nc) ? __ldg(row + c0 + c) : 0.f;
            }
#pragma unroll
            for (int b = 0; b < KC - 1; ++b) {
                const int64_t gx = ox0 - (KC - 1) + b;
                left[R][t][b] = (lane == 0 && rok && gx >= 0 && gx < p.Nc) ? __ldg(row + gx) : 0.f;
            }
        }
    }

    // phase 2: windows, sums, stores
    float win[KL][KR][WN];
    float *dst = p.out + plane * p.Mr * p.Mc;
#pragma unroll
    for (int t = 0; t < NROW; ++t) {
#pragma unroll
        for (int R = 0; R < KL; ++R) {
#pragma unroll
            for (int a = 0; a < KR - 1; ++a)
#pragma unroll
                for (int w = 0; w < WN; ++w) win[R][a][w] = win[R][a + 1][w];
#pragma unroll
            for (int b = 0; b < KC - 1; ++b) {
                const float up = __shfl_up_sync(0xffffffffu, own[R][t][4 - (KC - 1) + b], 1);
                win[R][KR - 1][b] = lane == 0 ? left[R][t][b] : up;
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) win[R][KR - 1][KC - 1 + c] = own[R][t][c];
        }
        if (t < KR - 1) continue;
        const int64_t m = m0 + t - (KR - 1);      // output row; window slot a holds row m - (KR-1-a)
        float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int R = 0; R < KL; ++R)
#pragma unroll
            for (int a = 0; a < KR; ++a)          // kernel row a uses input row m - a (slot KR-1-a)
#pragma unroll
                for (int b = 0; b < KC; ++b)
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        o[c] = fmaf(kr[R][a][b], win[R][KR - 1 - a][c - b + KC - 1], o[c]);
        if (m < p.Mr) {
            float *orow = dst + m * p.Mc;
            if (p.vec_out && c0 + 4 <= p.Mc) {
                *reinterpret_cast<float4 *>(orow + c0) = make_float4(o[0], o[1], o[2], o[3]);
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (c0 + c < p.Mc) orow[c0 + c] = o[c];
            }
        }
    }
}

template <int KL, int KR, int KC>
ft_status launch_rows(const ConvParams &p, int64_t planes, cudaStream_t s)
{
    // two leading taps hold twice the rows in registers: half the rows per warp
    constexpr int RB = KL == 1 ? 8 : 4;
    const int64_t nstrips = ft::ceil_div(p.Mc, 128);
    const int64_t nrb = ft::ceil_div(p.Mr, RB);
    const bool tail = nstrips > 1 && p.Mc - (nstrips - 1) * 128 <= 4;
    const int64_t main_strips = tail ? nstrips - 1 : nstrips;
    const int64_t wpp = main_strips * nrb + (tail ? ft::ceil_div(p.Mr, 32) : 0);
    const int64_t bx = ft::ceil_div(wpp, kThreads / 32);
    const int64_t bz = ft::ceil_div(planes, 65535);
    if (wpp > 0x7fffffffLL || bx > 0x7fffffffLL || bz > 65535) return FT_ERR_UNSUPPORTED;
    const dim3 grid((unsigned)bx, (unsigned)std::min<int64_t>(planes, 65535), (unsigned)bz);
    conv_rows_kernel<KL, KR, KC, RB><<<grid, kThreads, 0, s>>>(p, (int)nrb, (int)main_strips, (int)wpp, planes);
    return ft::check_launch();
}

template <int KL>
ft_status launch_rows_kl(const ConvParams &p, int64_t planes, cudaStream_t s)
{
    switch (p.Kr * 4 + p.Kc) {
    case 4 * 1 + 1: return launch_rows<KL, 1, 1>(p, planes, s);
    case 4 * 1 + 2: return launch_rows<KL, 1, 2>(p, planes, s);
    case 4 * 1 + 3: return launch_rows<KL, 1, 3>(p, planes, s);
    case 4 * 2 + 1: return launch_rows<KL, 2, 1>(p, planes, s);
    case 4 * 2 + 2: return launch_rows<KL, 2, 2>(p, planes, s);
    case 4 * 2 + 3: return launch_rows<KL, 2, 3>(p, planes, s);
    case 4 * 3 + 1: return launch_rows<KL, 3, 1>(p, planes, s);
    case 4 * 3 + 2: return launch_rows<KL, 3, 2>(p, planes, s);
    default: return launch_rows<KL, 3, 3>(p, planes, s);
    }
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
    const size_t smem = sizeof(float) * ((size_t)(TH + p.Kr - 1) * (TW + PADC) + (size_t)(p.Kr * ((p.Kc + 3) & ~3)));
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

template <int NTAP, int OY>
ft_status launch_fma(const ConvParams &p0, int64_t planes, cudaStream_t s)
{
    constexpr int PADC = (NTAP - 1 + 3) & ~3;
    constexpr int TW = 128, TH = 8 * OY;
    ConvParams p = p0;
    const int64_t tiles_y = ft::ceil_div(p.Mr, TH);
    p.tiles_x = ft::ceil_div(p.Mc, TW);
    p.tiles_per_plane = tiles_y * p.tiles_x;
    const int64_t blocks = planes * p.tiles_per_plane;
    if (blocks > 0x7fffffffLL) return FT_ERR_UNSUPPORTED;
    const size_t smem =
        sizeof(float) * ((size_t)(TH + p.Kr - 1) * (TW + PADC) + (size_t)p.Kr * ((NTAP + 3) & ~3));
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(conv_fma_kernel<NTAP, OY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) {
            ft::set_cuda_error(e);
            return FT_ERR_CUDA;
        }
    }
    conv_fma_kernel<NTAP, OY><<<(unsigned)blocks, kThreads, smem, s>>>(p);
    return ft::check_launch();
}

// 64-row tiles (kernels up to 9 columns, whose registers allow them) need Kr >= 8 and
// enough tiles for two CTAs per SM; else 32-row tiles
template <int NTAP>
ft_status launch_fma_oy(const ConvParams &p, int64_t planes, cudaStream_t s)
{
    if constexpr (NTAP <= 9) {
        if (p.Kr < 8) return launch_fma<NTAP, 4>(p, planes, s);
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const int64_t tiles64 = planes * ft::ceil_div(p.Mr, 64) * ft::ceil_div(p.Mc, 128);
        if (tiles64 >= 2 * (int64_t)(nsm > 0 ? nsm : 1)) return launch_fma<NTAP, 8>(p, planes, s);
    }
    return launch_fma<NTAP, 4>(p, planes, s);
}

// taps per row rounded up to the next odd count (at most one zero tap per row)
ft_status launch_fma_taps(const ConvParams &p, int64_t planes, cudaStream_t s)
{
    switch (p.Kc / 2) {
    case 0: return launch_fma_oy<1>(p, planes, s);
    case 1: return launch_fma_oy<3>(p, planes, s);
    case 2: return launch_fma_oy<5>(p, planes, s);
    case 3: return launch_fma_oy<7>(p, planes, s);
    case 4: return launch_fma_oy<9>(p, planes, s);
    case 5: return launch_fma_oy<11>(p, planes, s);
    case 6: return launch_fma_oy<13>(p, planes, s);
    case 7: return launch_fma_oy<15>(p, planes, s);
    default: return launch_fma_oy<17>(p, planes, s);
    }
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

// plane decomposition of a rank-nd full convolution (shared by every entry point)
static ft_status make_conv_params(const void *input, const int64_t *dims, int nd, const float *kernel,
                                  const int64_t *kdims, float *out, ConvParams &p, int64_t &planes, int64_t &tot_out)
{
    if (!input || !dims || !kernel || !kdims || !out) return FT_ERR_INVALID_ARG;
    int64_t odims[FT_MAX_NDIM];
    ft_status st = fastconv_out_dims(nd, dims, kdims, odims);
    if (st != FT_OK) return st;
    // overflow guard: every size must stay below 2^62
    const int64_t lim = (int64_t)1 << 62;
    int64_t tot_in = 1, tot_k = 1;
    tot_out = 1;
    for (int d = 0; d < nd; ++d) {
        if (odims[d] > lim / tot_out || dims[d] > lim / tot_in || kdims[d] > lim / tot_k)
            return FT_ERR_UNSUPPORTED;
        tot_in *= dims[d];
        tot_k *= kdims[d];
        tot_out *= odims[d];
    }
    p = ConvParams{};
    p.in = static_cast<const float *>(input);
    p.ker = kernel;
    p.out = out;
    p.nlead = nd >= 2 ? nd - 2 : 0;
    p.k_lead_total = 1;
    planes = 1;
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
    p.vec_out = ((reinterpret_cast<uintptr_t>(out) & 15) == 0 && (p.Mc & 3) == 0) ? 1 : 0;
    return FT_OK;
}

static ft_status conv_nd_impl(const float *input, const int64_t *dims, int nd, const float *kernel,
                              const int64_t *kdims, float *out, cudaStream_t s)
{
    ConvParams p;
    int64_t planes = 0, tot_out = 0;
    const ft_status st0 = make_conv_params(input, dims, nd, kernel, kdims, out, p, planes, tot_out);
    if (st0 != FT_OK) return st0;
    const bool tiled = p.Kc <= 65 && p.Kr <= 129;
    if (!tiled) {
        if (tot_out / 256 + 1 > 0x7fffffffLL) return FT_ERR_UNSUPPORTED;
        const unsigned blocks = (unsigned)ft::ceil_div(tot_out, kThreads);
        conv_direct_kernel<<<blocks, kThreads, 0, s>>>(p, tot_out);
        return ft::check_launch();
    }
    // small kernels (at most 2 leading taps, plane kernel up to 3 x 3): memory-bound.
    // Batches of 2-D planes take the copy-engine kernel (measured faster there), single
    // planes and two leading taps the streaming rows kernel
    if (p.k_lead_total <= 2 && p.Kr <= 3 && p.Kc <= 3) {
        if (planes >= 4 && p.k_lead_total == 1) {
            bool used = false;
            const ft_status st = launch_conv_tma(p, planes, s, &used);
            if (st != FT_OK || used) return st;
        }
        if (p.k_lead_total == 1) return launch_rows_kl<1>(p, planes, s);
        return launch_rows_kl<2>(p, planes, s);
    }
    if (p.Mr == 1) return launch_by_pad<1, 8>(p, planes, s);          // rank 1 (one row)
    if (p.Kc <= 17) {
        // persistent TMA-fed kernel when the input rows allow it, else (4+ rows) the
        // cp.async-staged kernel
        bool used = false;
        const ft_status st = launch_conv_tma(p, planes, s, &used);
        if (st != FT_OK || used) return st;
        if (p.Kr >= 4) return launch_fma_taps(p, planes, s);
    }
    if (p.Kr * p.Kc <= 16) return launch_by_pad<4, 1>(p, planes, s);  // small, memory-bound
    return launch_by_pad<8, 1>(p, planes, s);                           // wide or flat kernels
}

extern "C" ft_status fastconv_nd(const float *input, const int64_t *dims, int nd,
                                 const float *kernel, const int64_t *kdims, float *out,
                                 void *stream)
{
    FT_API_RANGE;
    return conv_nd_impl(input, dims, nd, kernel, kdims, out, ft::as_stream(stream));
}

namespace {

template <typename T> __device__ __forceinline__ float widen(T v) { return (float)v; }
template <> __device__ __forceinline__ float widen(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float widen(__nv_bfloat16 v) { return __bfloat162float(v); }

// exact conversion of n elements to FP32 (the fallback of fastconv_nd_typed)
template <typename T>
__global__ void __launch_bounds__(kThreads) widen_kernel(const T *__restrict__ in, int64_t n, float *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
        out[i] = widen(in[i]);
}

}  // namespace

extern "C" ft_status fastconv_nd_typed(const void *input, int in_dtype, const int64_t *dims, int nd,
                                       const float *kernel, const int64_t *kdims, float *out, float *scratch,
                                       void *stream)
{
    FT_API_RANGE;
    cudaStream_t s = ft::as_stream(stream);
    if (in_dtype == FT_F32) return conv_nd_impl(static_cast<const float *>(input), dims, nd, kernel, kdims, out, s);
    if (in_dtype != FT_U8 && in_dtype != FT_I16 && in_dtype != FT_F16 && in_dtype != FT_BF16)
        return FT_ERR_INVALID_ARG;
    ConvParams p;
    int64_t planes = 0, tot_out = 0;
    ft_status st = make_conv_params(input, dims, nd, kernel, kdims, out, p, planes, tot_out);
    if (st != FT_OK) return st;
    // fused: the copy engine stages the input in its own type and the kernel widens it
    if (p.Mr > 1 && p.Kc <= 17) {
        p.in = nullptr;
        p.in_t = input;
        p.in_dtype = in_dtype;
        p.vec_in = 0;
        bool used = false;
        st = in_dtype == FT_U8 ? launch_conv_tma_u8(p, planes, s, &used) : launch_conv_tma_16(p, planes, s, &used);
        if (st != FT_OK || used) return st;
    }
    // otherwise an exact FP32 copy of the input in `scratch`, then the FP32 path
    if (!scratch) return FT_ERR_WORKSPACE;
    int64_t n = 1;
    for (int d = 0; d < nd; ++d) n *= dims[d];
    const unsigned blocks = (unsigned)std::min<int64_t>(ft::ceil_div(n, kThreads), 152 * 32);
    switch (in_dtype) {
    case FT_U8: widen_kernel<<<blocks, kThreads, 0, s>>>(static_cast<const unsigned char *>(input), n, scratch); break;
    case FT_I16: widen_kernel<<<blocks, kThreads, 0, s>>>(static_cast<const short *>(input), n, scratch); break;
    case FT_F16: widen_kernel<<<blocks, kThreads, 0, s>>>(static_cast<const __half *>(input), n, scratch); break;
    default: widen_kernel<<<blocks, kThreads, 0, s>>>(static_cast<const __nv_bfloat16 *>(input), n, scratch); break;
    }
    if ((st = ft::check_launch()) != FT_OK) return st;
    return conv_nd_impl(scratch, dims, nd, kernel, kdims, out, s);
}

// Separable kernel k = f_0 (x) f_1 (x) ... : one 1-D full convolution per axis, each a
// plane pass of the tiled kernels with a kernel of one row or one column (the work per
// output drops from prod(K) to sum(K) multiply-adds).
extern "C" ft_status fastconv_separable(const float *input, const int64_t *dims, int nd,
                                        const float *const *factors, const int64_t *kdims, float *out,
                                        float *scratch, void *stream)
{
    FT_API_RANGE;
    if (!input || !dims || !factors || !kdims || !out) return FT_ERR_INVALID_ARG;
    int64_t odims[FT_MAX_NDIM];
    ft_status st = fastconv_out_dims(nd, dims, kdims, odims);
    if (st != FT_OK) return st;
    for (int d = 0; d < nd; ++d)
        if (!factors[d]) return FT_ERR_INVALID_ARG;
    if (nd >= 2 && !scratch) return FT_ERR_INVALID_ARG;
    if (scratch == input || scratch == out || out == input) return FT_ERR_INVALID_ARG;
    cudaStream_t s = ft::as_stream(stream);
    int64_t cur[FT_MAX_NDIM];
    for (int d = 0; d < nd; ++d) cur[d] = dims[d];
    const float *src = input;
    for (int d = 0; d < nd; ++d) {
        float *dst = ((nd - 1 - d) % 2 == 0) ? out : scratch;     // the last pass writes `out`
        int64_t outer = 1, inner = 1;
        for (int e = 0; e < d; ++e) outer *= cur[e];
        for (int e = d + 1; e < nd; ++e) inner *= cur[e];
        if (inner == 1) {
            const int64_t pd[2] = {outer, cur[d]}, pk[2] = {1, kdims[d]};
            st = conv_nd_impl(src, pd, 2, factors[d], pk, dst, s);
        } else {
            const int64_t pd[3] = {outer, cur[d], inner}, pk[3] = {1, kdims[d], 1};
            st = conv_nd_impl(src, pd, 3, factors[d], pk, dst, s);
        }
        if (st != FT_OK) return st;
        cur[d] += kdims[d] - 1;
        src = dst;
    }
    return FT_OK;
}

// Rank-1 test of a host kernel: the fibres through its largest entry, scaled, are the
// factors when their outer product reproduces the kernel to rel_tol * max |k|.
extern "C" int fastconv_factor(const float *kernel, const int64_t *kdims, int nd, double rel_tol, float *factors)
{
    if (!kernel || !kdims || !factors || nd < 1 || nd > FT_MAX_NDIM || !(rel_tol >= 0.0)) return -1;
    int64_t total = 1, stride[FT_MAX_NDIM];
    for (int d = nd - 1; d >= 0; --d) {
        if (kdims[d] < 1 || kdims[d] > ((int64_t)1 << 20)) return -1;
        stride[d] = total;
        total *= kdims[d];
        if (total > ((int64_t)1 << 26)) return -1;
    }
    int64_t m = 0;
    double vmax = 0.0;
    for (int64_t i = 0; i < total; ++i)
        if (std::fabs((double)kernel[i]) > vmax) {
            vmax = std::fabs((double)kernel[i]);
            m = i;
        }
    int64_t off[FT_MAX_NDIM + 1];
    off[0] = 0;
    for (int d = 0; d < nd; ++d) off[d + 1] = off[d] + kdims[d];
    if (vmax == 0.0) {                   // the zero kernel: zero factors
        for (int64_t i = 0; i < off[nd]; ++i) factors[i] = 0.f;
        return 1;
    }
    const double v = (double)kernel[m];
    int64_t mi[FT_MAX_NDIM];
    for (int d = 0; d < nd; ++d) mi[d] = (m / stride[d]) % kdims[d];
    // factor d: the fibre along d through the largest entry; the first factor also
    // carries 1 / v^(nd-1) (the product of the fibres counts v nd times)
    double scale = 1.0;
    for (int d = 1; d < nd; ++d) scale /= v;
    std::vector<double> f((size_t)off[nd]);
    for (int d = 0; d < nd; ++d)
        for (int64_t i = 0; i < kdims[d]; ++i) {
            const double x = kernel[m + (i - mi[d]) * stride[d]];
            f[(size_t)(off[d] + i)] = d == 0 ? x * scale : x;
        }
    for (int64_t i = 0; i < total; ++i) {
        double prod = 1.0;
        for (int d = 0; d < nd; ++d) prod *= f[(size_t)(off[d] + (i / stride[d]) % kdims[d])];
        if (std::fabs(prod - (double)kernel[i]) > rel_tol * vmax) return 0;
    }
    for (int64_t i = 0; i < off[nd]; ++i) factors[i] = (float)f[(size_t)i];
    return 1;
}
