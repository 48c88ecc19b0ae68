// Stage 1 of the multi-scale TTC/FOE solve: the fused tile kernel (Sec. V-A, V-B).
//
// One CTA (256 threads) owns a tile of TR x TC level-0 cubes of one frame pair and
// produces, for every pyramid level l, ten FP32 partial sums of the cubes of level l
// whose corner lies in the tile:
//   0 Ex^2, 1 Ex Ey, 2 Ey^2, 3 G Ex, 4 G Ey, 5 G^2, 6 Ex Et, 7 Ey Et, 8 G Et, 9 Et^2
// with Ex, Ey, Et the 2x2x2 first differences of Sec. II (scaled by 4, and by 4^l at
// level l because the pyramid keeps block sums, not means; the scale is removed in
// FP64 by the merge kernel) and G = x Ex + y Ey (Sec. V-A).
//
// Level 0 is streamed from global memory: each thread owns 4 columns in the left
// half of the tile and the same 4 columns in the right half, and walks 8 rows (plus
// one row of overlap).  The two halves ride in the two lanes of packed FP32 pairs
// (add/sub/mul/fma .f32x2), so every arithmetic instruction serves two cubes.
// uint8 pixels become floats exactly through the mantissa (2^23 + b, minus 2^23).
// The same loads give the level-1 pixels (2x2 block sums, exact for uint8), which go
// to shared memory together with a halo of HB = 2^(levels-1) level-0 rows/columns
// (read again from L2) so that every coarser cube of the tile sees its neighbours.
// Levels >= 2 are built by 2x2 sums in shared memory.  Level-1 cubes use the same
// strip scheme from shared memory; coarser levels use one thread per cube.
// All tile geometry is compile-time (template on the level count).
#pragma once

#include "common.cuh"

namespace ttc_tile {

constexpr int TR = 64;          // level-0 cube rows per tile
constexpr int TC = 256;         // level-0 cube columns per tile (two halves of 128)
constexpr int HALF = TC / 2;
constexpr int NT = 256;         // threads per CTA
constexpr int NSUM = 10;

// level-0 rows whose loads are in flight ahead of the arithmetic, and the minimum
// number of resident CTAs per SM the register allocation must allow
#ifndef FT_TTC_PF
#define FT_TTC_PF 2
#endif
#ifndef FT_TTC_MINB
#define FT_TTC_MINB 1
#endif

struct TileParams {
    const unsigned char *prev;  // first frame of pair 0
    const unsigned char *cur;   // second frame of pair 0
    int64_t pair_stride;        // bytes from pair p to pair p + 1
    int64_t pitch;              // bytes between rows
    int H, W;
    int tiles_x, ntiles;
    int vec;                    // 1: frame rows allow 4-byte (u8) / 16-byte (f32) loads
    float *partials;            // [pair][level][tile][NSUM]
};

// compile-time geometry for a level count L
template <int L>
struct Geo {
    static constexpr int HB = L > 1 ? (1 << (L - 1)) : 0;
    __host__ __device__ static constexpr int R(int l) { return (TR + HB) >> l; }            // pixel rows of level l
    __host__ __device__ static constexpr int C(int l) { return (TC + HB) >> l; }            // pixel columns of level l
    __host__ __device__ static constexpr int S(int l) { return (C(l) + 3) & ~3; }           // row stride (floats)
    __host__ __device__ static constexpr int off(int l)                                     // float offset of level l
    {
        int o = NSUM * NT;
        for (int k = 1; k < l; ++k) o += 2 * R(k) * S(k);
        return o;
    }
    __host__ __device__ static constexpr int floats() { return off(L); }
};

// ---------------------------------------------------------------------------
// packed FP32 pairs
// ---------------------------------------------------------------------------

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    unsigned long long r;
    const unsigned long long x = *reinterpret_cast<const unsigned long long *>(&a);
    const unsigned long long y = *reinterpret_cast<const unsigned long long *>(&b);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
    return *reinterpret_cast<const float2 *>(&r);
}

// the ten products of two cubes (one per lane of the pair)
__device__ __forceinline__ void accum2(float2 acc[NSUM], float2 ex, float2 ey, float2 et, float2 x, float2 y)
{
    const float2 g = fma2(x, ex, mul2(y, ey));
    acc[0] = fma2(ex, ex, acc[0]);
    acc[1] = fma2(ex, ey, acc[1]);
    acc[2] = fma2(ey, ey, acc[2]);
    acc[3] = fma2(g, ex, acc[3]);
    acc[4] = fma2(g, ey, acc[4]);
    acc[5] = fma2(g, g, acc[5]);
    acc[6] = fma2(ex, et, acc[6]);
    acc[7] = fma2(ey, et, acc[7]);
    acc[8] = fma2(g, et, acc[8]);
    acc[9] = fma2(et, et, acc[9]);
}

__device__ __forceinline__ void accum1(float acc[NSUM], float ex, float ey, float et, float x, float y)
{
    const float g = fmaf(x, ex, y * ey);
    acc[0] = fmaf(ex, ex, acc[0]);
    acc[1] = fmaf(ex, ey, acc[1]);
    acc[2] = fmaf(ey, ey, acc[2]);
    acc[3] = fmaf(g, ex, acc[3]);
    acc[4] = fmaf(g, ey, acc[4]);
    acc[5] = fmaf(g, g, acc[5]);
    acc[6] = fmaf(ex, et, acc[6]);
    acc[7] = fmaf(ey, et, acc[7]);
    acc[8] = fmaf(g, et, acc[8]);
    acc[9] = fmaf(et, et, acc[9]);
}

// Fixed-order CTA reduction of ten per-thread values to dst[0..9] (global).
// red: NSUM * NT floats of shared memory.  Called by all threads; ends with a barrier.
__device__ __forceinline__ void block_reduce(const float acc[NSUM], float *red, float *dst)
{
    const int tid = threadIdx.x;
#pragma unroll
    for (int s = 0; s < NSUM; ++s) red[s * NT + tid] = acc[s];
    __syncthreads();
    if (tid < NSUM * 16) {
        const int s = tid >> 4, l = tid & 15;
        float v = 0.f;
#pragma unroll
        for (int k = 0; k < NT / 16; ++k) v += red[s * NT + l + 16 * k];
#pragma unroll
        for (int o = 8; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (l == 0) dst[s] = v;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// pixel loads (branch-free on interior tiles so that all rows can be in flight)
// ---------------------------------------------------------------------------

// byte k of w as an exact float: 2^23 + b assembled in the mantissa (bias removed later)
__device__ __forceinline__ float u8biased(uint32_t w, int k)
{
    return __int_as_float(__byte_perm(w, 0x4B000000u, 0x7540u | (uint32_t)k));
}
__device__ __forceinline__ float2 unbias2(float2 v) { return add2(v, make_float2(-8388608.f, -8388608.f)); }

// raw loads of one level-0 row of both frames for one thread: 4 columns in the left
// half (l) and 4 in the right half (r) of the tile, plus the column right of the
// right half (only lane 31 uses it).  Zero outside the frame.
template <typename T0> struct RawRow;
template <> struct RawRow<unsigned char> { uint32_t al, ar, bl, br; float a4, b4; };
template <> struct RawRow<float> { float4 al, ar, bl, br; float a4, b4; };

__device__ __forceinline__ uint32_t bytes4(const unsigned char *row, int col, int W, bool rowok)
{
    uint32_t w = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const bool ok = rowok && col + k < W;
        const uint32_t v = __ldg(row + (ok ? col + k : 0));
        w |= (ok ? v : 0u) << (8 * k);
    }
    return w;
}

__device__ __forceinline__ float4 floats4(const float *row, int col, int W, bool rowok)
{
    float v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const bool ok = rowok && col + k < W;
        const float x = __ldg(row + (ok ? col + k : 0));
        v[k] = ok ? x : 0.f;
    }
    return make_float4(v[0], v[1], v[2], v[3]);
}

template <bool ROWCHK, bool COLCHK, bool VEC>
__device__ __forceinline__ void load_raw(const TileParams &p, const unsigned char *fa, const unsigned char *fb,
                                         int gy, int gcl, RawRow<unsigned char> &r)
{
    const bool rowok = !ROWCHK || gy < p.H;
    const int gyc = ROWCHK ? min(gy, p.H - 1) : gy;
    const unsigned char *ra = fa + (int64_t)gyc * p.pitch;
    const unsigned char *rb = fb + (int64_t)gyc * p.pitch;
    const int gcr = gcl + HALF;
    if (!COLCHK && VEC) {
        const uint32_t m = rowok ? 0xffffffffu : 0u;
        r.al = __ldg(reinterpret_cast<const unsigned int *>(ra + gcl)) & m;
        r.ar = __ldg(reinterpret_cast<const unsigned int *>(ra + gcr)) & m;
        r.bl = __ldg(reinterpret_cast<const unsigned int *>(rb + gcl)) & m;
        r.br = __ldg(reinterpret_cast<const unsigned int *>(rb + gcr)) & m;
    } else {
        r.al = bytes4(ra, gcl, p.W, rowok);
        r.ar = bytes4(ra, gcr, p.W, rowok);
        r.bl = bytes4(rb, gcl, p.W, rowok);
        r.br = bytes4(rb, gcr, p.W, rowok);
    }
    const int c4 = gcr + 4;
    const bool ok4 = rowok && (!COLCHK || c4 < p.W);
    const int c4c = ok4 ? c4 : 0;
    const uint32_t va = __ldg(ra + c4c), vb = __ldg(rb + c4c);
    r.a4 = ok4 ? (float)va : 0.f;
    r.b4 = ok4 ? (float)vb : 0.f;
}

template <bool ROWCHK, bool COLCHK, bool VEC>
__device__ __forceinline__ void load_raw(const TileParams &p, const float *fa, const float *fb, int gy, int gcl,
                                         RawRow<float> &r)
{
    const bool rowok = !ROWCHK || gy < p.H;
    const int gyc = ROWCHK ? min(gy, p.H - 1) : gy;
    const int64_t pe = p.pitch / 4;
    const float *ra = fa + (int64_t)gyc * pe;
    const float *rb = fb + (int64_t)gyc * pe;
    const int gcr = gcl + HALF;
    if (!COLCHK && VEC) {
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 al = __ldg(reinterpret_cast<const float4 *>(ra + gcl));
        const float4 ar = __ldg(reinterpret_cast<const float4 *>(ra + gcr));
        const float4 bl = __ldg(reinterpret_cast<const float4 *>(rb + gcl));
        const float4 br = __ldg(reinterpret_cast<const float4 *>(rb + gcr));
        r.al = rowok ? al : z;
        r.ar = rowok ? ar : z;
        r.bl = rowok ? bl : z;
        r.br = rowok ? br : z;
    } else {
        r.al = floats4(ra, gcl, p.W, rowok);
        r.ar = floats4(ra, gcr, p.W, rowok);
        r.bl = floats4(rb, gcl, p.W, rowok);
        r.br = floats4(rb, gcr, p.W, rowok);
    }
    const int c4 = gcr + 4;
    const bool ok4 = rowok && (!COLCHK || c4 < p.W);
    const int c4c = ok4 ? c4 : 0;
    const float va = __ldg(ra + c4c), vb = __ldg(rb + c4c);
    r.a4 = ok4 ? va : 0.f;
    r.b4 = ok4 ? vb : 0.f;
}

// the 4 own columns of each half as (left, right) pairs
__device__ __forceinline__ void unpack4(const RawRow<unsigned char> &r, float2 A[5], float2 B[5])
{
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        A[k] = unbias2(make_float2(u8biased(r.al, k), u8biased(r.ar, k)));
        B[k] = unbias2(make_float2(u8biased(r.bl, k), u8biased(r.br, k)));
    }
}
__device__ __forceinline__ void unpack4(const RawRow<float> &r, float2 A[5], float2 B[5])
{
    A[0] = make_float2(r.al.x, r.ar.x); A[1] = make_float2(r.al.y, r.ar.y);
    A[2] = make_float2(r.al.z, r.ar.z); A[3] = make_float2(r.al.w, r.ar.w);
    B[0] = make_float2(r.bl.x, r.br.x); B[1] = make_float2(r.bl.y, r.br.y);
    B[2] = make_float2(r.bl.z, r.br.z); B[3] = make_float2(r.bl.w, r.br.w);
}

// plus the neighbour column: left half from lane+1 (lane 31: the first right-half
// column, held by lane 0); right half from lane+1 (lane 31: its own extra load)
template <typename T0>
__device__ __forceinline__ void unpack5(const RawRow<T0> &r, int lane, float2 A[5], float2 B[5])
{
    unpack4(r, A, B);
    const int src = (lane + 1) & 31;
    const float a4l = __shfl_sync(0xffffffffu, lane == 0 ? A[0].y : A[0].x, src);
    const float b4l = __shfl_sync(0xffffffffu, lane == 0 ? B[0].y : B[0].x, src);
    const float a4r = __shfl_sync(0xffffffffu, A[0].y, src);
    const float b4r = __shfl_sync(0xffffffffu, B[0].y, src);
    A[4] = make_float2(a4l, lane == 31 ? r.a4 : a4r);
    B[4] = make_float2(b4l, lane == 31 ? r.b4 : b4r);
}

// masks the cubes outside the level (EDGE tiles only)
__device__ __forceinline__ void mask3(float2 &ex, float2 &ey, float2 &et, bool okl, bool okr)
{
    ex = make_float2(okl ? ex.x : 0.f, okr ? ex.y : 0.f);
    ey = make_float2(okl ? ey.x : 0.f, okr ? ey.y : 0.f);
    et = make_float2(okl ? et.x : 0.f, okr ? et.y : 0.f);
}

// one row step of the strip scheme: rows (previous = ps/pd, current = A/B) give the
// 4 cube pairs of the previous row.  Columns are streamed left to right so that only
// a two-column window of the intermediate sums is live.
template <bool EDGE>
__device__ __forceinline__ void strip_row(const float2 A[5], const float2 B[5], float2 ps[5], float2 pd[5],
                                          bool first, float2 x0, float yv, bool rowok, int jl, int jr,
                                          int Wlim, float2 acc[NSUM])
{
    const float2 y = make_float2(yv, yv);
    float2 cs_p, vd_p, td_p;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const float2 s = add2(A[k], B[k]);
        const float2 d = sub2(B[k], A[k]);
        if (!first) {
            const float2 cs = add2(s, ps[k]);     // column sum over 2 rows x 2 frames
            const float2 vd = sub2(s, ps[k]);     // row difference, both frames
            const float2 td = add2(d, pd[k]);     // time difference, both rows
            if (k > 0) {
                float2 ex = sub2(cs, cs_p);
                float2 ey = add2(vd_p, vd);
                float2 et = add2(td_p, td);
                if (EDGE) mask3(ex, ey, et, rowok && (jl + k - 1 < Wlim), rowok && (jr + k - 1 < Wlim));
                const float kk = (float)(k - 1);
                accum2(acc, ex, ey, et, add2(x0, make_float2(kk, kk)), y);
            }
            cs_p = cs;
            vd_p = vd;
            td_p = td;
        }
        ps[k] = s;
        pd[k] = d;
    }
}

// ---------------------------------------------------------------------------
// level 0 from global memory; interior pixels of levels 1, 2 and 3 from registers
// ---------------------------------------------------------------------------

template <typename T0, int L, bool EDGE, bool VEC>
__device__ __forceinline__ void level0(const TileParams &p, const T0 *fa, const T0 *fb, int R0, int C0,
                                       float *sm, float2 acc[NSUM])
{
    using G = Geo<L>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gcl = C0 + 4 * lane;
    const int gr0 = R0 + 8 * warp;
    // cube centre x = j + 1/2 - (W-1)/2 = j + 1 - W/2 at level 0
    const float xoff = 1.f - 0.5f * (float)p.W;
    const float yoff = 1.f - 0.5f * (float)p.H;
    const float2 x0 = make_float2((float)gcl + xoff, (float)(gcl + HALF) + xoff);

    constexpr int PF = FT_TTC_PF;                   // rows in flight
    RawRow<T0> raw[9];
#pragma unroll
    for (int r = 0; r < PF; ++r) load_raw<EDGE, EDGE, VEC>(p, fa, fb, gr0 + r, gcl, raw[r]);

    float2 ps[5], pd[5];
    float2 ha[2], hb[2], k2a, k2b, k3a, k3b;
#pragma unroll
    for (int r = 0; r < 9; ++r) {
        if (r + PF < 9) load_raw<EDGE, EDGE, VEC>(p, fa, fb, gr0 + r + PF, gcl, raw[r + PF]);
        float2 A[5], B[5];
        unpack5(raw[r], lane, A, B);
        const int i = gr0 + r - 1;
        strip_row<EDGE>(A, B, ps, pd, r == 0, x0, (float)i + yoff, i < p.H - 1, gcl, gcl + HALF, p.W - 1, acc);
        if (L > 1 && r < 8) {
            if ((r & 1) == 0) {
                ha[0] = add2(A[0], A[1]); ha[1] = add2(A[2], A[3]);
                hb[0] = add2(B[0], B[1]); hb[1] = add2(B[2], B[3]);
            } else {
                // level-1 pixels (rows 4w + m, columns 2 lane, 2 lane + 1 of each half)
                const float2 va0 = add2(ha[0], add2(A[0], A[1]));
                const float2 va1 = add2(ha[1], add2(A[2], A[3]));
                const float2 vb0 = add2(hb[0], add2(B[0], B[1]));
                const float2 vb1 = add2(hb[1], add2(B[2], B[3]));
                const int m = r >> 1;
                float *rowa = sm + G::off(1) + (4 * warp + m) * G::S(1);
                float *rowb = rowa + G::R(1) * G::S(1);
                *reinterpret_cast<float2 *>(rowa + 2 * lane) = make_float2(va0.x, va1.x);
                *reinterpret_cast<float2 *>(rowa + HALF / 2 + 2 * lane) = make_float2(va0.y, va1.y);
                *reinterpret_cast<float2 *>(rowb + 2 * lane) = make_float2(vb0.x, vb1.x);
                *reinterpret_cast<float2 *>(rowb + HALF / 2 + 2 * lane) = make_float2(vb0.y, vb1.y);
                if (L > 2) {
                    const float2 sa = add2(va0, va1), sb = add2(vb0, vb1);
                    if ((m & 1) == 0) {
                        k2a = sa;
                        k2b = sb;
                    } else {
                        // level-2 pixels (row 2w + m/2, column lane of each half)
                        const float2 l2a = add2(k2a, sa), l2b = add2(k2b, sb);
                        float *r2a = sm + G::off(2) + (2 * warp + (m >> 1)) * G::S(2);
                        float *r2b = r2a + G::R(2) * G::S(2);
                        r2a[lane] = l2a.x;
                        r2a[HALF / 4 + lane] = l2a.y;
                        r2b[lane] = l2b.x;
                        r2b[HALF / 4 + lane] = l2b.y;
                        if (L > 3) {
                            if (m == 1) {
                                k3a = l2a;
                                k3b = l2b;
                            } else {
                                // level-3 pixels (row w, column lane/2 of each half)
                                float2 v3a = add2(k3a, l2a), v3b = add2(k3b, l2b);
                                v3a.x += __shfl_xor_sync(0xffffffffu, v3a.x, 1);
                                v3a.y += __shfl_xor_sync(0xffffffffu, v3a.y, 1);
                                v3b.x += __shfl_xor_sync(0xffffffffu, v3b.x, 1);
                                v3b.y += __shfl_xor_sync(0xffffffffu, v3b.y, 1);
                                if ((lane & 1) == 0) {
                                    float *r3a = sm + G::off(3) + warp * G::S(3);
                                    float *r3b = r3a + G::R(3) * G::S(3);
                                    r3a[lane >> 1] = v3a.x;
                                    r3a[HALF / 8 + (lane >> 1)] = v3a.y;
                                    r3b[lane >> 1] = v3b.x;
                                    r3b[HALF / 8 + (lane >> 1)] = v3b.y;
                                }
                            }
                        }
                    }
                }
            }
        }
    }
}

// level-1 halo: pixel rows [TR/2, R1) over the columns of the two halves (two level-0
// rows per level-1 row, warp w takes halo rows w, w+8, ...), and columns
// [TC/2, C1) over rows [0, R1) (four level-0 columns per work item)
template <typename T0, int L, bool EDGE, bool VEC>
__device__ __forceinline__ void level1_halo(const TileParams &p, const T0 *fa, const T0 *fb, int R0, int C0, float *sm)
{
    using G = Geo<L>;
    constexpr int R1 = G::R(1), C1 = G::C(1), S1 = G::S(1);
    float *L1 = sm + G::off(1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gcl = C0 + 4 * lane;
    for (int h = warp; h < R1 - TR / 2; h += NT / 32) {
        RawRow<T0> r0, r1;
        load_raw<true, EDGE, VEC>(p, fa, fb, R0 + TR + 2 * h, gcl, r0);
        load_raw<true, EDGE, VEC>(p, fa, fb, R0 + TR + 2 * h + 1, gcl, r1);
        float2 A0[5], B0[5], A1[5], B1[5];
        unpack4(r0, A0, B0);
        unpack4(r1, A1, B1);
        const float2 va0 = add2(add2(A0[0], A0[1]), add2(A1[0], A1[1]));
        const float2 va1 = add2(add2(A0[2], A0[3]), add2(A1[2], A1[3]));
        const float2 vb0 = add2(add2(B0[0], B0[1]), add2(B1[0], B1[1]));
        const float2 vb1 = add2(add2(B0[2], B0[3]), add2(B1[2], B1[3]));
        float *rowa = L1 + (TR / 2 + h) * S1;
        float *rowb = rowa + R1 * S1;
        *reinterpret_cast<float2 *>(rowa + 2 * lane) = make_float2(va0.x, va1.x);
        *reinterpret_cast<float2 *>(rowa + HALF / 2 + 2 * lane) = make_float2(va0.y, va1.y);
        *reinterpret_cast<float2 *>(rowb + 2 * lane) = make_float2(vb0.x, vb1.x);
        *reinterpret_cast<float2 *>(rowb + HALF / 2 + 2 * lane) = make_float2(vb0.y, vb1.y);
    }
    constexpr int PR = (C1 - TC / 2 + 1) / 2;           // level-1 column pairs right of the halves
    constexpr int N = R1 * PR;
    const int64_t pe = p.pitch / (int64_t)sizeof(T0);
    for (int e = threadIdx.x; e < 2 * N; e += NT) {
        const int f = e >= N;
        const int q = e - f * N;
        const int r1 = q / PR, cp = q % PR;
        const T0 *fr = f ? fb : fa;
        const int gy = R0 + 2 * r1, gx = C0 + TC + 4 * cp;
        float v[2][4];
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const bool rowok = gy + dy < p.H;
            const T0 *row = fr + (int64_t)(rowok ? gy + dy : 0) * pe;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const bool ok = rowok && gx + k < p.W;
                const float x = (float)__ldg(row + (ok ? gx + k : 0));
                v[dy][k] = ok ? x : 0.f;
            }
        }
        const float s0 = (v[0][0] + v[0][1]) + (v[1][0] + v[1][1]);
        const float s1 = (v[0][2] + v[0][3]) + (v[1][2] + v[1][3]);
        *reinterpret_cast<float2 *>(L1 + f * R1 * S1 + r1 * S1 + TC / 2 + 2 * cp) = make_float2(s0, s1);
    }
}

// level-l pixels with row in [r_lo, R_l) or column in [c_lo, C_l) (the part not
// produced from registers): 2x2 sums of level l-1 in shared memory
template <int L, int l>
__device__ __forceinline__ void build_halo(float *sm, int r_lo, int c_lo)
{
    using G = Geo<L>;
    constexpr int R = G::R(l), C = G::C(l), S = G::S(l);
    constexpr int Rs = G::R(l - 1), Ss = G::S(l - 1);
    const float *src = sm + G::off(l - 1);
    float *dst = sm + G::off(l);
    const int nb = (R - r_lo) * C;          // bottom strip
    const int nr = r_lo * (C - c_lo);       // right strip
    const int n = nb + nr;
    for (int e = threadIdx.x; e < 2 * n; e += NT) {
        const int f = e >= n;
        const int q = e - f * n;
        int r, c;
        if (q < nb) {
            r = r_lo + q / C;
            c = q % C;
        } else {
            const int q2 = q - nb;
            r = q2 / (C - c_lo);
            c = c_lo + q2 % (C - c_lo);
        }
        const float *s0 = src + f * Rs * Ss + (2 * r) * Ss + 2 * c;
        const float2 u = *reinterpret_cast<const float2 *>(s0);
        const float2 w = *reinterpret_cast<const float2 *>(s0 + Ss);
        dst[f * R * S + r * S + c] = (u.x + u.y) + (w.x + w.y);
    }
}

// cubes of level l (1 <= l <= 5) from shared memory by the strip scheme: a thread owns
// 4 columns in each half of the level's tile and RPT consecutive cube rows
template <int L, int l, bool EDGE>
__device__ __forceinline__ void strip_cubes(const TileParams &p, const float *sm, int R0, int C0, float2 acc[NSUM])
{
    using G = Geo<L>;
    constexpr int S = G::S(l), R = G::R(l);
    constexpr int NR = TR >> l;                  // cube rows of the tile at level l
    constexpr int HC = (TC >> l) / 2;            // cube columns per half
    constexpr int CG = HC / 4;                   // column groups per half
    constexpr int RG = NT / CG;                  // row groups available
    constexpr int RPT = NR > RG ? NR / RG : 1;   // cube rows per thread
    constexpr int ACTIVE = CG * (NR / RPT);
    const int tid = threadIdx.x;
    if (tid >= ACTIVE) return;
    const int cg = tid % CG, rg = tid / CG;
    const int j0 = 4 * cg, i0 = rg * RPT;
    const int Hl = p.H >> l, Wl = p.W >> l;
    const int gi0 = (R0 >> l) + i0, gjl = (C0 >> l) + j0, gjr = gjl + HC;
    const float pl = (float)(1 << l);
    // cube centre x = j + 1/2 - (W - 2^l) / 2^(l+1)
    const float xoff = 0.5f - ((float)p.W - pl) / (2.f * pl);
    const float yoff = 0.5f - ((float)p.H - pl) / (2.f * pl);
    const float2 x0 = make_float2((float)gjl + xoff, (float)gjr + xoff);
    const float *La = sm + G::off(l);
    const float *Lb = La + R * S;
    float2 ps[5], pd[5];
#pragma unroll
    for (int r = 0; r <= RPT; ++r) {
        const float *ra = La + (i0 + r) * S + j0;
        const float *rb = Lb + (i0 + r) * S + j0;
        const float4 al = *reinterpret_cast<const float4 *>(ra);
        const float4 ar = *reinterpret_cast<const float4 *>(ra + HC);
        const float4 bl = *reinterpret_cast<const float4 *>(rb);
        const float4 br = *reinterpret_cast<const float4 *>(rb + HC);
        const float2 A[5] = {make_float2(al.x, ar.x), make_float2(al.y, ar.y), make_float2(al.z, ar.z),
                             make_float2(al.w, ar.w), make_float2(ra[4], ra[HC + 4])};
        const float2 B[5] = {make_float2(bl.x, br.x), make_float2(bl.y, br.y), make_float2(bl.z, br.z),
                             make_float2(bl.w, br.w), make_float2(rb[4], rb[HC + 4])};
        const int gi = gi0 + r - 1;
        strip_row<EDGE>(A, B, ps, pd, r == 0, x0, (float)gi + yoff, gi < Hl - 1, gjl, gjr, Wl - 1, acc);
    }
}

// cubes of level l from shared memory, one per thread and iteration (l = 6)
template <int L, int l>
__device__ __forceinline__ void cube_loop(const TileParams &p, const float *sm, int R0, int C0, float acc[NSUM])
{
    using G = Geo<L>;
    constexpr int S = G::S(l), R = G::R(l);
    constexpr int nr = TR >> l, nc = TC >> l;
    const int Hl = p.H >> l, Wl = p.W >> l;
    const int i0 = R0 >> l, j0 = C0 >> l;
    const float pl = (float)(1 << l);
    const float xoff = 0.5f - ((float)p.W - pl) / (2.f * pl);
    const float yoff = 0.5f - ((float)p.H - pl) / (2.f * pl);
    const float *La = sm + G::off(l);
    for (int e = threadIdx.x; e < nr * nc; e += NT) {
        const int i = e / nc, j = e % nc;
        const int gi = i0 + i, gj = j0 + j;
        if (gi >= Hl - 1 || gj >= Wl - 1) continue;
        const float *pa = La + i * S + j;
        const float *pb = pa + R * S;
        const float a00 = pa[0], a01 = pa[1], a10 = pa[S], a11 = pa[S + 1];
        const float b00 = pb[0], b01 = pb[1], b10 = pb[S], b11 = pb[S + 1];
        const float ex = ((a01 - a00) + (a11 - a10)) + ((b01 - b00) + (b11 - b10));
        const float ey = ((a10 - a00) + (a11 - a01)) + ((b10 - b00) + (b11 - b01));
        const float et = ((b00 - a00) + (b01 - a01)) + ((b10 - a10) + (b11 - a11));
        accum1(acc, ex, ey, et, (float)gj + xoff, (float)gi + yoff);
    }
}

__device__ __forceinline__ void fold(const float2 acc2[NSUM], float acc[NSUM])
{
#pragma unroll
    for (int s = 0; s < NSUM; ++s) acc[s] = acc2[s].x + acc2[s].y;
}

// pixels of levels l.. L-1 not produced from registers
template <int L, int l>
__device__ __forceinline__ void build_levels(float *sm)
{
    if constexpr (l < L) {
        if constexpr (l <= 3) build_halo<L, l>(sm, TR >> (l + 1), TC >> (l + 1));
        else build_halo<L, l>(sm, 0, 0);
        __syncthreads();
        build_levels<L, l + 1>(sm);
    }
}

// cubes of levels l .. L-1, one tile reduction each
template <int L, int l>
__device__ __forceinline__ void coarse_cubes(const TileParams &p, float *sm, int R0, int C0, float *partial,
                                             int64_t lstride)
{
    if constexpr (l < L) {
        float acc[NSUM];
        if constexpr (l <= 5) {
            float2 acc2[NSUM];
#pragma unroll
            for (int s = 0; s < NSUM; ++s) acc2[s] = make_float2(0.f, 0.f);
            const bool edge = ((R0 >> l) + (TR >> l) > (p.H >> l) - 1) || ((C0 >> l) + (TC >> l) > (p.W >> l) - 1);
            if (edge) strip_cubes<L, l, true>(p, sm, R0, C0, acc2);
            else strip_cubes<L, l, false>(p, sm, R0, C0, acc2);
            fold(acc2, acc);
        } else {
#pragma unroll
            for (int s = 0; s < NSUM; ++s) acc[s] = 0.f;
            cube_loop<L, l>(p, sm, R0, C0, acc);
        }
        block_reduce(acc, sm, partial + l * lstride);
        coarse_cubes<L, l + 1>(p, sm, R0, C0, partial, lstride);
    }
}

template <typename T0, int L, bool VEC>
__global__ void __launch_bounds__(NT, FT_TTC_MINB)
ttc_tile_kernel(const TileParams p)
{
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);

    const int64_t bid = blockIdx.x;
    const int pair = (int)(bid / p.ntiles);
    const int tile = (int)(bid - (int64_t)pair * p.ntiles);
    const int ty = tile / p.tiles_x, tx = tile - ty * p.tiles_x;
    const int R0 = ty * TR, C0 = tx * TC;
    const T0 *fa = reinterpret_cast<const T0 *>(p.prev + (int64_t)pair * p.pair_stride);
    const T0 *fb = reinterpret_cast<const T0 *>(p.cur + (int64_t)pair * p.pair_stride);
    float *partial = p.partials + ((int64_t)pair * L * p.ntiles + tile) * NSUM;
    const int64_t lstride = (int64_t)p.ntiles * NSUM;

    float2 acc2[NSUM];
    float acc[NSUM];
#pragma unroll
    for (int s = 0; s < NSUM; ++s) acc2[s] = make_float2(0.f, 0.f);

    // level 0; all rows and columns read lie inside the frame unless EDGE
    const bool edge0 = (R0 + TR > p.H - 1) || (C0 + TC > p.W - 1);
    if (edge0) {
        level0<T0, L, true, VEC>(p, fa, fb, R0, C0, sm, acc2);
        if constexpr (L > 1) level1_halo<T0, L, true, VEC>(p, fa, fb, R0, C0, sm);
    } else {
        level0<T0, L, false, VEC>(p, fa, fb, R0, C0, sm, acc2);
        if constexpr (L > 1) level1_halo<T0, L, false, VEC>(p, fa, fb, R0, C0, sm);
    }
    fold(acc2, acc);
    block_reduce(acc, sm, partial);              // its barriers also publish level 1..3 pixels

    if constexpr (L > 2) build_levels<L, 2>(sm);
    if constexpr (L > 1) coarse_cubes<L, 1>(p, sm, R0, C0, partial, lstride);
}

inline size_t smem_bytes(int levels)
{
    switch (levels) {
    case 1: return sizeof(float) * Geo<1>::floats();
    case 2: return sizeof(float) * Geo<2>::floats();
    case 3: return sizeof(float) * Geo<3>::floats();
    case 4: return sizeof(float) * Geo<4>::floats();
    case 5: return sizeof(float) * Geo<5>::floats();
    case 6: return sizeof(float) * Geo<6>::floats();
    default: return sizeof(float) * Geo<7>::floats();
    }
}

template <typename T0, int L, bool VEC>
cudaError_t launch_one(const TileParams &p, unsigned blocks, cudaStream_t s)
{
    const size_t smem = sizeof(float) * Geo<L>::floats();
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(ttc_tile_kernel<T0, L, VEC>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    ttc_tile_kernel<T0, L, VEC><<<blocks, NT, smem, s>>>(p);
    return cudaGetLastError();
}

template <typename T0, bool VEC>
cudaError_t launch_vec(const TileParams &p, int levels, unsigned blocks, cudaStream_t s)
{
    switch (levels) {
    case 1: return launch_one<T0, 1, VEC>(p, blocks, s);
    case 2: return launch_one<T0, 2, VEC>(p, blocks, s);
    case 3: return launch_one<T0, 3, VEC>(p, blocks, s);
    case 4: return launch_one<T0, 4, VEC>(p, blocks, s);
    case 5: return launch_one<T0, 5, VEC>(p, blocks, s);
    case 6: return launch_one<T0, 6, VEC>(p, blocks, s);
    default: return launch_one<T0, 7, VEC>(p, blocks, s);
    }
}

template <typename T0>
cudaError_t launch(const TileParams &p, int levels, unsigned blocks, cudaStream_t s)
{
    return p.vec ? launch_vec<T0, true>(p, levels, blocks, s) : launch_vec<T0, false>(p, levels, blocks, s);
}

}  // namespace ttc_tile
