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
// pixel loads
// ---------------------------------------------------------------------------

// byte k of w as an exact float: 2^23 + b assembled in the mantissa, minus 2^23 later
__device__ __forceinline__ float u8biased(uint32_t w, int k)
{
    return __int_as_float(__byte_perm(w, 0x4B000000u, 0x7540u | (uint32_t)k));
}

// 4 consecutive pixels (zero beyond W) as biased floats (u8) or plain floats (f32)
__device__ __forceinline__ void load4raw(const unsigned char *row, int col, int W, int vec, float v[4])
{
    uint32_t w;
    if (vec && col + 4 <= W) {
        w = __ldg(reinterpret_cast<const unsigned int *>(row + col));
    } else {
        w = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (col + k < W) w |= (uint32_t)__ldg(row + col + k) << (8 * k);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = u8biased(w, k);
}

__device__ __forceinline__ void load4raw(const float *row, int col, int W, int vec, float v[4])
{
    if (vec && col + 4 <= W) {
        const float4 f = __ldg(reinterpret_cast<const float4 *>(row + col));
        v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = (col + k < W) ? __ldg(row + col + k) : 0.f;
    }
}

// bias removed from a packed pair of raw values
__device__ __forceinline__ float2 unbias(float2 v, unsigned char) { return add2(v, make_float2(-8388608.f, -8388608.f)); }
__device__ __forceinline__ float2 unbias(float2 v, float) { return v; }
__device__ __forceinline__ float load1(const unsigned char *row, int col, int W)
{
    return col < W ? (float)__ldg(row + col) : 0.f;
}
__device__ __forceinline__ float load1(const float *row, int col, int W) { return col < W ? __ldg(row + col) : 0.f; }

// One level-0 row of both frames for this thread: 5 columns (4 own + 1 neighbour) in
// the left half (lane .x) and the right half (lane .y) of the tile, unbiased.
template <typename T0, bool EDGE>
__device__ __forceinline__ void load_row0(const TileParams &p, const T0 *fa, const T0 *fb, int gy, int gcl,
                                          int lane, float2 A[5], float2 B[5])
{
    if (EDGE && gy >= p.H) {
#pragma unroll
        for (int k = 0; k < 5; ++k) A[k] = B[k] = make_float2(0.f, 0.f);
        return;
    }
    const int64_t pe = p.pitch / (int64_t)sizeof(T0);
    const T0 *ra = fa + (int64_t)gy * pe;
    const T0 *rb = fb + (int64_t)gy * pe;
    const int gcr = gcl + HALF;
    float al[4], ar[4], bl[4], br[4];
    load4raw(ra, gcl, p.W, p.vec, al);
    load4raw(ra, gcr, p.W, p.vec, ar);
    load4raw(rb, gcl, p.W, p.vec, bl);
    load4raw(rb, gcr, p.W, p.vec, br);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        A[k] = unbias(make_float2(al[k], ar[k]), T0());
        B[k] = unbias(make_float2(bl[k], br[k]), T0());
    }
    // neighbour column: left half from lane+1 (lane 31: the first right-half column,
    // held by lane 0); right half from lane+1 (lane 31: one extra load)
    const int src = (lane + 1) & 31;
    const float a4l = __shfl_sync(0xffffffffu, lane == 0 ? A[0].y : A[0].x, src);
    const float b4l = __shfl_sync(0xffffffffu, lane == 0 ? B[0].y : B[0].x, src);
    float a4r = __shfl_sync(0xffffffffu, A[0].y, src);
    float b4r = __shfl_sync(0xffffffffu, B[0].y, src);
    if (lane == 31) {
        a4r = load1(ra, gcr + 4, p.W);
        b4r = load1(rb, gcr + 4, p.W);
    }
    A[4] = make_float2(a4l, a4r);
    B[4] = make_float2(b4l, b4r);
}

// ---------------------------------------------------------------------------
// level 0 (global memory) + level-1 pixels of the tile interior
// ---------------------------------------------------------------------------

template <typename T0, int L, bool EDGE>
__device__ __forceinline__ void level0(const TileParams &p, const T0 *fa, const T0 *fb, int R0, int C0,
                                       float *L1, float2 acc[NSUM])
{
    using G = Geo<L>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gcl = C0 + 4 * lane;
    const int gr0 = R0 + 8 * warp;
    // cube centre x = j + 1/2 - (W-1)/2 = j + 1 - W/2 (level 0)
    const float xoff = 1.f - 0.5f * (float)p.W;
    const float yoff = 1.f - 0.5f * (float)p.H;
    float2 xk[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
        xk[k] = make_float2((float)(gcl + k) + xoff, (float)(gcl + HALF + k) + xoff);
    float2 ps[5], pd[5], ha[2], hb[2];
#pragma unroll
    for (int r = 0; r < 9; ++r) {
        const int gy = gr0 + r;
        float2 A[5], B[5];
        load_row0<T0, EDGE>(p, fa, fb, gy, gcl, lane, A, B);
        float2 s[5], d[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            s[k] = add2(A[k], B[k]);
            d[k] = sub2(B[k], A[k]);
        }
        if (r > 0) {
            const int i = gy - 1;
            const float yv = (float)i + yoff;
            const float2 y = make_float2(yv, yv);
            float2 cs[5], vd[5], td[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                cs[k] = add2(s[k], ps[k]);       // 2 rows x 2 frames, per column
                vd[k] = sub2(s[k], ps[k]);       // row difference, both frames
                td[k] = add2(d[k], pd[k]);       // time difference, both rows
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float2 ex = sub2(cs[k + 1], cs[k]);
                float2 ey = add2(vd[k], vd[k + 1]);
                float2 et = add2(td[k], td[k + 1]);
                if (EDGE) {
                    const bool rok = i < p.H - 1;
                    const bool okl = rok && (gcl + k < p.W - 1);
                    const bool okr = rok && (gcl + HALF + k < p.W - 1);
                    ex = make_float2(okl ? ex.x : 0.f, okr ? ex.y : 0.f);
                    ey = make_float2(okl ? ey.x : 0.f, okr ? ey.y : 0.f);
                    et = make_float2(okl ? et.x : 0.f, okr ? et.y : 0.f);
                }
                accum2(acc, ex, ey, et, xk[k], y);
            }
        }
        if (L > 1 && r < 8) {
            if ((r & 1) == 0) {
                ha[0] = add2(A[0], A[1]); ha[1] = add2(A[2], A[3]);
                hb[0] = add2(B[0], B[1]); hb[1] = add2(B[2], B[3]);
            } else {
                const float2 va0 = add2(ha[0], add2(A[0], A[1]));
                const float2 va1 = add2(ha[1], add2(A[2], A[3]));
                const float2 vb0 = add2(hb[0], add2(B[0], B[1]));
                const float2 vb1 = add2(hb[1], add2(B[2], B[3]));
                const int r1 = 4 * warp + (r >> 1);
                float *rowa = L1 + r1 * G::S(1);
                float *rowb = rowa + G::R(1) * G::S(1);
                *reinterpret_cast<float2 *>(rowa + 2 * lane) = make_float2(va0.x, va1.x);
                *reinterpret_cast<float2 *>(rowa + HALF / 2 + 2 * lane) = make_float2(va0.y, va1.y);
                *reinterpret_cast<float2 *>(rowb + 2 * lane) = make_float2(vb0.x, vb1.x);
                *reinterpret_cast<float2 *>(rowb + HALF / 2 + 2 * lane) = make_float2(vb0.y, vb1.y);
            }
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            ps[k] = s[k];
            pd[k] = d[k];
        }
    }
}

// level-1 halo: pixel rows [TR/2, R1) x all columns, and rows [0, TR/2) x columns
// [TC/2, C1), two level-1 pixels (four level-0 columns) per work item
template <typename T0, int L>
__device__ __forceinline__ void level1_halo(const TileParams &p, const T0 *fa, const T0 *fb, int R0, int C0, float *L1)
{
    using G = Geo<L>;
    constexpr int R1 = G::R(1), C1 = G::C(1), S1 = G::S(1);
    constexpr int PB = (C1 + 1) / 2;                    // column pairs, bottom strip
    constexpr int PR = (C1 - TC / 2 + 1) / 2;           // column pairs, right strip
    constexpr int NB = (R1 - TR / 2) * PB;
    constexpr int NR = (TR / 2) * PR;
    constexpr int N = NB + NR;
    const int64_t pe = p.pitch / (int64_t)sizeof(T0);
    for (int e = threadIdx.x; e < 2 * N; e += NT) {
        const int f = e >= N;
        const int q = e - f * N;
        int r1, c1;
        if (q < NB) {
            r1 = TR / 2 + q / PB;
            c1 = 2 * (q % PB);
        } else {
            const int q2 = q - NB;
            r1 = q2 / PR;
            c1 = TC / 2 + 2 * (q2 % PR);
        }
        const T0 *fr = f ? fb : fa;
        const int gy = R0 + 2 * r1, gx = C0 + 2 * c1;
        float v0 = 0.f, v1 = 0.f;
        if (gy + 1 < p.H) {
            float t0[4], t1[4];
            load4raw(fr + (int64_t)gy * pe, gx, p.W, p.vec, t0);
            load4raw(fr + (int64_t)(gy + 1) * pe, gx, p.W, p.vec, t1);
            const float2 a = unbias(make_float2(t0[0], t0[2]), T0());
            const float2 b = unbias(make_float2(t0[1], t0[3]), T0());
            const float2 c = unbias(make_float2(t1[0], t1[2]), T0());
            const float2 d = unbias(make_float2(t1[1], t1[3]), T0());
            const float2 v = add2(add2(a, b), add2(c, d));
            v0 = v.x;
            v1 = v.y;
        }
        *reinterpret_cast<float2 *>(L1 + f * R1 * S1 + r1 * S1 + c1) = make_float2(v0, v1);
    }
}

// level-1 cubes of the tile from shared memory: thread = 4 columns x 2 rows in each half
template <int L, bool EDGE>
__device__ __forceinline__ void level1_cubes(const TileParams &p, const float *L1, int R0, int C0, float2 acc[NSUM])
{
    using G = Geo<L>;
    constexpr int S1 = G::S(1), R1 = G::R(1);
    constexpr int H1C = TC / 4;                  // cube columns per half at level 1 (64)
    const int cg = threadIdx.x & 15;             // column group (4 columns)
    const int rg = threadIdx.x >> 4;             // row group (2 rows)
    const int j0 = 4 * cg, i0 = 2 * rg;          // tile-local level-1 cube indices
    const int Hl = p.H >> 1, Wl = p.W >> 1;
    const int gi0 = (R0 >> 1) + i0, gj0 = (C0 >> 1) + j0;
    const float xoff = 0.5f - (float)(p.W - 2) * 0.25f;
    const float yoff = 0.5f - (float)(p.H - 2) * 0.25f;
    float2 xk[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) xk[k] = make_float2((float)(gj0 + k) + xoff, (float)(gj0 + H1C + k) + xoff);
    float2 ps[5], pd[5];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const float *ra = L1 + (i0 + r) * S1 + j0;
        const float *rb = ra + R1 * S1;
        const float4 al = *reinterpret_cast<const float4 *>(ra);
        const float4 ar = *reinterpret_cast<const float4 *>(ra + H1C);
        const float4 bl = *reinterpret_cast<const float4 *>(rb);
        const float4 br = *reinterpret_cast<const float4 *>(rb + H1C);
        float2 A[5] = {make_float2(al.x, ar.x), make_float2(al.y, ar.y), make_float2(al.z, ar.z),
                       make_float2(al.w, ar.w), make_float2(ra[4], ra[H1C + 4])};
        float2 B[5] = {make_float2(bl.x, br.x), make_float2(bl.y, br.y), make_float2(bl.z, br.z),
                       make_float2(bl.w, br.w), make_float2(rb[4], rb[H1C + 4])};
        float2 s[5], d[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            s[k] = add2(A[k], B[k]);
            d[k] = sub2(B[k], A[k]);
        }
        if (r > 0) {
            const int gi = gi0 + r - 1;
            const float yv = (float)gi + yoff;
            const float2 y = make_float2(yv, yv);
            float2 cs[5], vd[5], td[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                cs[k] = add2(s[k], ps[k]);
                vd[k] = sub2(s[k], ps[k]);
                td[k] = add2(d[k], pd[k]);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float2 ex = sub2(cs[k + 1], cs[k]);
                float2 ey = add2(vd[k], vd[k + 1]);
                float2 et = add2(td[k], td[k + 1]);
                if (EDGE) {
                    const bool rok = gi < Hl - 1;
                    const bool okl = rok && (gj0 + k < Wl - 1);
                    const bool okr = rok && (gj0 + H1C + k < Wl - 1);
                    ex = make_float2(okl ? ex.x : 0.f, okr ? ex.y : 0.f);
                    ey = make_float2(okl ? ey.x : 0.f, okr ? ey.y : 0.f);
                    et = make_float2(okl ? et.x : 0.f, okr ? et.y : 0.f);
                }
                accum2(acc, ex, ey, et, xk[k], y);
            }
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            ps[k] = s[k];
            pd[k] = d[k];
        }
    }
}

// cubes of level l >= 2 from shared memory, one per thread and iteration
template <int L, int l>
__device__ __forceinline__ void levelN_cubes(const TileParams &p, const float *Ll, int R0, int C0, float acc[NSUM])
{
    using G = Geo<L>;
    constexpr int S = G::S(l), R = G::R(l);
    constexpr int nr = TR >> l, nc = TC >> l;
    const int Hl = p.H >> l, Wl = p.W >> l;
    const int i0 = R0 >> l, j0 = C0 >> l;
    const float pl = (float)(1 << l);
    // cube centre: x = j + 1/2 - (W - 2^l) / 2^(l+1)
    const float xoff = 0.5f - ((float)p.W - pl) / (2.f * pl);
    const float yoff = 0.5f - ((float)p.H - pl) / (2.f * pl);
    for (int e = threadIdx.x; e < nr * nc; e += NT) {
        const int i = e / nc, j = e % nc;
        const int gi = i0 + i, gj = j0 + j;
        if (gi >= Hl - 1 || gj >= Wl - 1) continue;
        const float *pa = Ll + i * S + j;
        const float *pb = pa + R * S;
        const float a00 = pa[0], a01 = pa[1], a10 = pa[S], a11 = pa[S + 1];
        const float b00 = pb[0], b01 = pb[1], b10 = pb[S], b11 = pb[S + 1];
        const float ex = ((a01 - a00) + (a11 - a10)) + ((b01 - b00) + (b11 - b10));
        const float ey = ((a10 - a00) + (a11 - a01)) + ((b10 - b00) + (b11 - b01));
        const float et = ((b00 - a00) + (b01 - a01)) + ((b10 - a10) + (b11 - a11));
        accum1(acc, ex, ey, et, (float)gj + xoff, (float)gi + yoff);
    }
}

// level l >= 2 pixels: 2x2 sums of level l-1 (both frames)
template <int L, int l>
__device__ __forceinline__ void build_level(float *sm)
{
    using G = Geo<L>;
    constexpr int R = G::R(l), C = G::C(l), S = G::S(l);
    constexpr int Rs = G::R(l - 1), Ss = G::S(l - 1);
    const float *src = sm + G::off(l - 1);
    float *dst = sm + G::off(l);
    for (int e = threadIdx.x; e < 2 * R * C; e += NT) {
        const int f = e / (R * C), q = e % (R * C);
        const int r = q / C, c = q % C;
        const float *s0 = src + f * Rs * Ss + (2 * r) * Ss + 2 * c;
        dst[f * R * S + r * S + c] = (s0[0] + s0[1]) + (s0[Ss] + s0[Ss + 1]);
    }
}

template <int L, int l>
struct CoarseLevels {
    // levels l .. L-1: build pixels, then reduce cubes
    __device__ __forceinline__ static void build(float *sm)
    {
        if constexpr (l < L) {
            build_level<L, l>(sm);
            __syncthreads();
            CoarseLevels<L, l + 1>::build(sm);
        }
    }
    __device__ __forceinline__ static void cubes(const TileParams &p, float *sm, int R0, int C0, float *partial,
                                                 int64_t lstride)
    {
        if constexpr (l < L) {
            float acc[NSUM];
#pragma unroll
            for (int s = 0; s < NSUM; ++s) acc[s] = 0.f;
            levelN_cubes<L, l>(p, sm + Geo<L>::off(l), R0, C0, acc);
            block_reduce(acc, sm, partial + l * lstride);
            CoarseLevels<L, l + 1>::cubes(p, sm, R0, C0, partial, lstride);
        }
    }
};

__device__ __forceinline__ void fold(const float2 acc2[NSUM], float acc[NSUM])
{
#pragma unroll
    for (int s = 0; s < NSUM; ++s) acc[s] = acc2[s].x + acc2[s].y;
}

template <typename T0, int L>
__global__ void __launch_bounds__(NT)
ttc_tile_kernel(const TileParams p)
{
    using G = Geo<L>;
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
    float *L1 = sm + G::off(1);

    float2 acc2[NSUM];
    float acc[NSUM];
#pragma unroll
    for (int s = 0; s < NSUM; ++s) acc2[s] = make_float2(0.f, 0.f);

    // level 0; every loaded row and column lies inside the frame unless EDGE
    const bool edge0 = (R0 + TR > p.H - 1) || (C0 + TC > p.W - 1);
    if (edge0) level0<T0, L, true>(p, fa, fb, R0, C0, L1, acc2);
    else level0<T0, L, false>(p, fa, fb, R0, C0, L1, acc2);
    if constexpr (L > 1) level1_halo<T0, L>(p, fa, fb, R0, C0, L1);
    fold(acc2, acc);
    block_reduce(acc, sm, partial);             // its barriers also publish level 1

    if constexpr (L > 1) {
        CoarseLevels<L, 2>::build(sm);
#pragma unroll
        for (int s = 0; s < NSUM; ++s) acc2[s] = make_float2(0.f, 0.f);
        const bool edge1 = ((R0 >> 1) + TR / 2 > (p.H >> 1) - 1) || ((C0 >> 1) + TC / 2 > (p.W >> 1) - 1);
        if (edge1) level1_cubes<L, true>(p, L1, R0, C0, acc2);
        else level1_cubes<L, false>(p, L1, R0, C0, acc2);
        fold(acc2, acc);
        block_reduce(acc, sm, partial + lstride);
        CoarseLevels<L, 2>::cubes(p, sm, R0, C0, partial, lstride);
    }
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

template <typename T0, int L>
cudaError_t launch_one(const TileParams &p, unsigned blocks, cudaStream_t s)
{
    const size_t smem = sizeof(float) * Geo<L>::floats();
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(ttc_tile_kernel<T0, L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    ttc_tile_kernel<T0, L><<<blocks, NT, smem, s>>>(p);
    return cudaGetLastError();
}

template <typename T0>
cudaError_t launch(const TileParams &p, int levels, unsigned blocks, cudaStream_t s)
{
    switch (levels) {
    case 1: return launch_one<T0, 1>(p, blocks, s);
    case 2: return launch_one<T0, 2>(p, blocks, s);
    case 3: return launch_one<T0, 3>(p, blocks, s);
    case 4: return launch_one<T0, 4>(p, blocks, s);
    case 5: return launch_one<T0, 5>(p, blocks, s);
    case 6: return launch_one<T0, 6>(p, blocks, s);
    default: return launch_one<T0, 7>(p, blocks, s);
    }
}

}  // namespace ttc_tile
