// Stage 1 of the multi-scale TTC/FOE solve (Sec. V-A, V-B): one streaming pass per
// pyramid level.
//
// Pass l reads the level-l images of both frames of every pair and produces
//   - ten FP32 partial sums per tile of TR x TC cubes (0 Ex^2, 1 Ex Ey, 2 Ey^2,
//     3 G Ex, 4 G Ey, 5 G^2, 6 Ex Et, 7 Ey Et, 8 G Et, 9 Et^2), with Ex, Ey, Et the
//     2x2x2 first differences of Sec. II scaled by 4 (and by 4^l, because the pyramid
//     images hold 2x2 block sums rather than means; the merge kernel removes the
//     scale in FP64) and G = x Ex + y Ey (Sec. V-A);
//   - from the same loads, the level-(l+1) image (2x2 block sums, floor cropping,
//     Sec. V-B) of each frame, written once per frame: uint16 for uint8 input up to
//     level 4 (exact: at most 255 * 4^4), float otherwise (exact up to 2^24).
// A thread owns 4 columns in the left half of the tile and the same 4 columns in the
// right half and walks 8 rows (plus one row of overlap); the two halves ride in the
// two lanes of packed FP32 pairs (add/sub/mul/fma .f32x2).  Integer pixels become
// floats exactly through the mantissa (2^23 + v assembled by a byte permute, minus
// 2^23).  The tile sums are reduced in a fixed order through shared memory.
#pragma once

#include "common.cuh"

namespace ttc_pass {

constexpr int TR = 64;          // cube rows per tile (large levels; small levels use 16)
constexpr int TR_SMALL = 16;
constexpr int TC = 256;         // cube columns per tile (two halves of 128)
constexpr int HALF = TC / 2;
constexpr int NT = 256;         // threads per CTA
constexpr int NSUM = 10;

#ifndef FT_TTC_PF
#define FT_TTC_PF 2             // rows whose loads are issued ahead of the arithmetic
#endif
#ifndef FT_TTC_MINB
#define FT_TTC_MINB 2           // resident CTAs per SM the register allocation must allow
#endif

// tile sets of one launch
enum TileSet { SET_INTERIOR = 0, SET_EDGES = 1, SET_BOTTOM = 2, SET_RIGHT = 3, SET_ALL = 4 };

struct PassParams {
    const unsigned char *prev;  // level-l image, first frame of pair 0
    const unsigned char *cur;   // level-l image, second frame of pair 0
    int64_t pair_stride;        // bytes from pair p to pair p + 1
    int64_t pitch;              // bytes between rows of the level-l images
    int H, W;                   // level-l image size
    int tiles_x, tiles_y, ntiles;
    int tr;                     // cube rows per tile: 64 (8 per warp) or 16 (2 per warp)
    int set;                    // which tiles this launch covers (TileSet)
    int vec;                    // 1: rows allow vector loads
    int padded;                 // 1: images padded past the last tile (context images)
    float xoff, yoff;           // cube centre: x = j + xoff, y = i + yoff
    float *partials;            // this level: [pair][tile][NSUM]
    unsigned char *next;        // level-(l+1) image of frame 0, or null
    int64_t next_fstride;       // bytes between frames of `next`
    int64_t next_pitch;         // bytes between rows of `next`
    int write_prev;             // 0: video (frame t+1 of pair t is shared); 1: independent pairs;
                                // -1: the first frame's level l+1 exists already (not written)
    unsigned char *next_cur;    // non-null: level-(l+1) image of the second frame (one pair per launch
                                // item); null: the frame after the first one in `next`
    int64_t frame_bytes;        // bytes readable from a frame's first pixel (checked builds)
    int64_t next_bytes;         // bytes writable from a next-level image's first pixel (checked builds)
    int *status;                // the call's status word (checked builds: bit 1 on an access out of bounds)
};

// Checked builds (FASTTTC_CHECK=1 at build time defines FT_CHECK): every global read of a
// frame and every store of a next-level pixel is compared with the extent the call gave;
// one outside it sets bit 1 of the status word (FT_FLAG_BOUNDS in the records) and is
// skipped (reads give zero).  Release builds compile the checks away.
#ifndef FT_CHECK
#define FT_CHECK 0
#endif

__device__ __forceinline__ bool in_extent(const PassParams &p, const void *base, const void *addr, int bytes,
                                          int64_t extent)
{
    const int64_t off = reinterpret_cast<const unsigned char *>(addr) - reinterpret_cast<const unsigned char *>(base);
    if (off >= 0 && off + bytes <= extent) return true;
    if (p.status) atomicOr(p.status, 2);
    return false;
}

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

// Fixed-order CTA reduction of ten per-thread values to dst[0..9] (global):
// shared-memory transpose, 16-way strided sums, 16-lane shuffle tree.
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
}

// ---------------------------------------------------------------------------
// pixel types
// ---------------------------------------------------------------------------

// exact float of an unsigned integer v < 2^23 held in bytes of w: the selector puts
// v in the low mantissa bytes under the exponent of 2^23; the bias is removed later
__device__ __forceinline__ float biased(uint32_t w, uint32_t sel)
{
    return __int_as_float(__byte_perm(w, 0x4B000000u, sel));
}
__device__ __forceinline__ float2 unbias2(float2 v) { return add2(v, make_float2(-8388608.f, -8388608.f)); }

template <typename T> struct Pix;

template <> struct Pix<unsigned char> {
    using Vec = uint32_t;                       // 4 pixels
    static constexpr bool INT = true;
    __device__ static Vec ld4(const unsigned char *p) { return __ldg(reinterpret_cast<const unsigned int *>(p)); }
    __device__ static Vec zero() { return 0u; }
    __device__ static float elem_biased(const Vec &v, int k) { return biased(v, 0x7540u | (uint32_t)k); }
    __device__ static float ld1(const unsigned char *p) { return (float)__ldg(p); }
};

template <> struct Pix<unsigned short> {
    using Vec = uint2;                          // 4 pixels
    static constexpr bool INT = true;
    __device__ static Vec ld4(const unsigned short *p) { return __ldg(reinterpret_cast<const uint2 *>(p)); }
    __device__ static Vec zero() { return make_uint2(0u, 0u); }
    __device__ static float elem_biased(const Vec &v, int k)
    {
        return biased(k < 2 ? v.x : v.y, (k & 1) ? 0x7532u : 0x7510u);
    }
    __device__ static float ld1(const unsigned short *p) { return (float)__ldg(p); }
};

template <> struct Pix<float> {
    using Vec = float4;
    static constexpr bool INT = false;
    __device__ static Vec ld4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
    __device__ static Vec zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    __device__ static float elem_biased(const Vec &v, int k)
    {
        return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w;
    }
    __device__ static float ld1(const float *p) { return __ldg(p); }
};

// raw loads of one row of both frames: 4 columns in each half + the column right of
// the right half (used by lane 31 only); zero outside the image
template <typename T> struct RawRow {
    typename Pix<T>::Vec al, ar, bl, br;
    float a4, b4;
};

// element loads with bounds checks; whole groups inside the row use one vector load
// (vec: the rows allow it)
__device__ __forceinline__ uint32_t load4_checked(const unsigned char *row, int col, int W, bool rowok, int vec)
{
    if (vec && rowok && col + 4 <= W) return __ldg(reinterpret_cast<const unsigned int *>(row + col));
    uint32_t w = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const bool ok = rowok && col + k < W;
        const uint32_t v = __ldg(row + (ok ? col + k : 0));
        w |= (ok ? v : 0u) << (8 * k);
    }
    return w;
}
__device__ __forceinline__ uint2 load4_checked(const unsigned short *row, int col, int W, bool rowok, int vec)
{
    if (vec && rowok && col + 4 <= W) return __ldg(reinterpret_cast<const uint2 *>(row + col));
    uint32_t v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const bool ok = rowok && col + k < W;
        const uint32_t x = __ldg(row + (ok ? col + k : 0));
        v[k] = ok ? x : 0u;
    }
    return make_uint2(v[0] | (v[1] << 16), v[2] | (v[3] << 16));
}
__device__ __forceinline__ float4 load4_checked(const float *row, int col, int W, bool rowok, int vec)
{
    if (vec && rowok && col + 4 <= W) return __ldg(reinterpret_cast<const float4 *>(row + col));
    float v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const bool ok = rowok && col + k < W;
        const float x = __ldg(row + (ok ? col + k : 0));
        v[k] = ok ? x : 0.f;
    }
    return make_float4(v[0], v[1], v[2], v[3]);
}

template <typename T, bool ROWCHK, bool COLCHK, bool VEC>
__device__ __forceinline__ void load_raw(const PassParams &p, const T *fa, const T *fb, int gy, int gcl, RawRow<T> &r)
{
    const bool rowok = !ROWCHK || gy < p.H;
    const int gyc = ROWCHK ? min(gy, p.H - 1) : gy;
    const int64_t pe = p.pitch / (int64_t)sizeof(T);
    const T *ra = fa + (int64_t)gyc * pe;
    const T *rb = fb + (int64_t)gyc * pe;
    const int gcr = gcl + HALF;
    if (!COLCHK && VEC) {
        const typename Pix<T>::Vec z = Pix<T>::zero();
        if (FT_CHECK) {
            constexpr int VB = 4 * (int)sizeof(T);
            const bool ok = in_extent(p, fa, ra + gcl, VB, p.frame_bytes) &&
                            in_extent(p, fa, ra + gcr, VB, p.frame_bytes) &&
                            in_extent(p, fb, rb + gcl, VB, p.frame_bytes) &&
                            in_extent(p, fb, rb + gcr, VB, p.frame_bytes);
            if (!ok) {
                r.al = r.ar = r.bl = r.br = z;
                r.a4 = r.b4 = 0.f;
                return;
            }
        }
        const typename Pix<T>::Vec al = Pix<T>::ld4(ra + gcl), ar = Pix<T>::ld4(ra + gcr);
        const typename Pix<T>::Vec bl = Pix<T>::ld4(rb + gcl), br = Pix<T>::ld4(rb + gcr);
        r.al = rowok ? al : z;
        r.ar = rowok ? ar : z;
        r.bl = rowok ? bl : z;
        r.br = rowok ? br : z;
    } else {
        // every element these loads may touch lies in the row's first W pixels
        if (FT_CHECK && !(in_extent(p, fa, ra, (int)sizeof(T), p.frame_bytes) &&
                          in_extent(p, fa, ra + (p.W - 1), (int)sizeof(T), p.frame_bytes) &&
                          in_extent(p, fb, rb, (int)sizeof(T), p.frame_bytes) &&
                          in_extent(p, fb, rb + (p.W - 1), (int)sizeof(T), p.frame_bytes))) {
            r.al = r.ar = r.bl = r.br = Pix<T>::zero();
            r.a4 = r.b4 = 0.f;
            return;
        }
        r.al = load4_checked(ra, gcl, p.W, rowok, p.vec);
        r.ar = load4_checked(ra, gcr, p.W, rowok, p.vec);
        r.bl = load4_checked(rb, gcl, p.W, rowok, p.vec);
        r.br = load4_checked(rb, gcr, p.W, rowok, p.vec);
    }
    const int c4 = gcr + 4;
    const bool ok4 = rowok && (!COLCHK || c4 < p.W);
    const int c4c = ok4 ? c4 : 0;
    if (FT_CHECK && !(in_extent(p, fa, ra + c4c, (int)sizeof(T), p.frame_bytes) &&
                      in_extent(p, fb, rb + c4c, (int)sizeof(T), p.frame_bytes))) {
        r.a4 = r.b4 = 0.f;
        return;
    }
    const float va = Pix<T>::ld1(ra + c4c), vb = Pix<T>::ld1(rb + c4c);
    r.a4 = ok4 ? va : 0.f;
    r.b4 = ok4 ? vb : 0.f;
}

// (left, right) float pairs of the 5 columns; the neighbour column of the left half
// comes from lane+1 (lane 31: the first right-half column, held by lane 0), that of
// the right half from lane+1 (lane 31: its own load)
template <typename T>
__device__ __forceinline__ void unpack5(const RawRow<T> &r, int lane, float2 A[5], float2 B[5])
{
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        A[k] = make_float2(Pix<T>::elem_biased(r.al, k), Pix<T>::elem_biased(r.ar, k));
        B[k] = make_float2(Pix<T>::elem_biased(r.bl, k), Pix<T>::elem_biased(r.br, k));
        if (Pix<T>::INT) {
            A[k] = unbias2(A[k]);
            B[k] = unbias2(B[k]);
        }
    }
    const int src = (lane + 1) & 31;
    const float a4l = __shfl_sync(0xffffffffu, lane == 0 ? A[0].y : A[0].x, src);
    const float b4l = __shfl_sync(0xffffffffu, lane == 0 ? B[0].y : B[0].x, src);
    const float a4r = __shfl_sync(0xffffffffu, A[0].y, src);
    const float b4r = __shfl_sync(0xffffffffu, B[0].y, src);
    A[4] = make_float2(a4l, lane == 31 ? r.a4 : a4r);
    B[4] = make_float2(b4l, lane == 31 ? r.b4 : b4r);
}

__device__ __forceinline__ void mask3(float2 &ex, float2 &ey, float2 &et, bool okl, bool okr)
{
    ex = make_float2(okl ? ex.x : 0.f, okr ? ex.y : 0.f);
    ey = make_float2(okl ? ey.x : 0.f, okr ? ey.y : 0.f);
    et = make_float2(okl ? et.x : 0.f, okr ? et.y : 0.f);
}

// One row step: previous row (ps = prev + cur, pd = cur - prev, per column) and the
// current row A (prev frame), B (cur frame) give the 4 cube pairs of the previous
// row.  Columns are streamed left to right (two-column window of intermediates).
template <bool MASK>
__device__ __forceinline__ void strip_row(const float2 A[5], const float2 B[5], float2 ps[5], float2 pd[5],
                                          bool first, float2 x0, float yv, bool rowok, int jl, int jr,
                                          int jlo, int jhi, float2 acc[NSUM])
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
                if (MASK) {
                    const int cl = jl + k - 1, cr = jr + k - 1;
                    mask3(ex, ey, et, rowok && cl >= jlo && cl < jhi, rowok && cr >= jlo && cr < jhi);
                }
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

// Running state of one thread's strip between rows.
struct Strip {
    float2 ps[5];   // previous row: prev + cur per column (biased by 2^23 for integer pixels)
    float2 pd[5];   // previous row: cur - prev per column
    float2 phs[4];  // previous row: horizontal differences of ps
};

// One row step, from the raw pixels of the row: with A = prev frame (unbiased), and
// the cur frame left biased by 2^23 for integer pixels (sums stay exact below 2^24),
//   s = A + B, d = B - A per column; hs = s[k+1] - s[k];
//   Ex = hs(row i) + hs(row i+1), Ey = vd[k] + vd[k+1] with vd = s(i+1) - s(i),
//   Et = td[k] + td[k+1] with td = d(i) + d(i+1)
// (the 2x2x2 first differences of Sec. II, times 4).  The neighbour column's s and d
// come from lane+1 (lane 31 of the right half: its own extra pixel).  Returns the
// unbiased prev-frame pixels and d of the row's 4 own columns for the pyramid.
template <typename T, bool MASK>
__device__ __forceinline__ void row_step(const RawRow<T> &r, int lane, Strip &st, bool first, const float2 xk[4],
                                         float2 y, bool rowok, int jl, int jr, int jlo, int jhi, float2 acc[NSUM],
                                         float2 Aout[4], float2 Dout[4])
{
    constexpr float BIAS = Pix<T>::INT ? 8388608.f : 0.f;
    float2 s[5], d[5];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 ab = make_float2(Pix<T>::elem_biased(r.al, k), Pix<T>::elem_biased(r.ar, k));
        const float2 bb = make_float2(Pix<T>::elem_biased(r.bl, k), Pix<T>::elem_biased(r.br, k));
        const float2 a = Pix<T>::INT ? unbias2(ab) : ab;
        s[k] = add2(a, bb);
        d[k] = sub2(bb, ab);
        Aout[k] = a;
        Dout[k] = d[k];
    }
    const int src = (lane + 1) & 31;
    const float s4l = __shfl_sync(0xffffffffu, lane == 0 ? s[0].y : s[0].x, src);
    const float d4l = __shfl_sync(0xffffffffu, lane == 0 ? d[0].y : d[0].x, src);
    const float s4r = __shfl_sync(0xffffffffu, s[0].y, src);
    const float d4r = __shfl_sync(0xffffffffu, d[0].y, src);
    s[4] = make_float2(s4l, lane == 31 ? (r.a4 + r.b4) + BIAS : s4r);
    d[4] = make_float2(d4l, lane == 31 ? r.b4 - r.a4 : d4r);
    float2 hs[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) hs[k] = sub2(s[k + 1], s[k]);
    if (!first) {
        float2 vd_p, td_p;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const float2 vd = sub2(s[k], st.ps[k]);
            const float2 td = add2(d[k], st.pd[k]);
            if (k > 0) {
                float2 ex = add2(hs[k - 1], st.phs[k - 1]);
                float2 ey = add2(vd_p, vd);
                float2 et = add2(td_p, td);
                if (MASK) {
                    const int cl = jl + k - 1, cr = jr + k - 1;
                    mask3(ex, ey, et, rowok && cl >= jlo && cl < jhi, rowok && cr >= jlo && cr < jhi);
                }
                accum2(acc, ex, ey, et, xk[k - 1], y);
            }
            vd_p = vd;
            td_p = td;
        }
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        st.ps[k] = s[k];
        st.pd[k] = d[k];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) st.phs[k] = hs[k];
}

// 2x2 block sums of the next level from two rows' unbiased prev pixels A and
// differences D (cur = A + D), for the even row (a = true: keep) and the odd row
// (returns prev-frame sums va0, va1 and cur-frame sums vb0, vb1 of the thread's two
// level-(l+1) columns, as (left, right) pairs)
struct Pyr {
    float2 ha[2], hd[2];
};

__device__ __forceinline__ void pyr_even(Pyr &py, const float2 A[4], const float2 D[4])
{
    py.ha[0] = add2(A[0], A[1]);
    py.ha[1] = add2(A[2], A[3]);
    py.hd[0] = add2(D[0], D[1]);
    py.hd[1] = add2(D[2], D[3]);
}

__device__ __forceinline__ void pyr_odd(const Pyr &py, const float2 A[4], const float2 D[4], float2 &va0, float2 &va1,
                                        float2 &vb0, float2 &vb1)
{
    va0 = add2(py.ha[0], add2(A[0], A[1]));
    va1 = add2(py.ha[1], add2(A[2], A[3]));
    const float2 vd0 = add2(py.hd[0], add2(D[0], D[1]));
    const float2 vd1 = add2(py.hd[1], add2(D[2], D[3]));
    vb0 = add2(va0, vd0);
    vb1 = add2(va1, vd1);
}

// level-(l+1) pixels (row r1, columns c and c+1) of one frame from the thread's 2x2
// block sums, written if they exist (r1 < H/2, column < W/2)
template <typename Tout, bool EDGE>
__device__ __forceinline__ void store_next(const PassParams &p, unsigned char *img, int64_t pitch, int r1, int c,
                                           float v0, float v1, int Hn, int Wn)
{
    if (EDGE && (r1 >= Hn || c >= Wn)) return;
    const bool two = !EDGE || c + 1 < Wn;
    Tout *row = reinterpret_cast<Tout *>(img + (int64_t)r1 * pitch);
    if (FT_CHECK && !in_extent(p, img, row + c, (two ? 2 : 1) * (int)sizeof(Tout), p.next_bytes)) return;
    if (two) {
        if (sizeof(Tout) == 2) {
            // exact integers < 2^16: their bits are the low mantissa bits of 2^23 + v
            const uint32_t lo = __float_as_uint(v0 + 8388608.f) & 0xffffu;
            const uint32_t hi = __float_as_uint(v1 + 8388608.f) << 16;
            *reinterpret_cast<uint32_t *>(row + c) = lo | hi;
        } else {
            *reinterpret_cast<float2 *>(row + c) = make_float2(v0, v1);
        }
    } else {
        row[c] = sizeof(Tout) == 2 ? (Tout)(__float_as_uint(v0 + 8388608.f) & 0xffffu) : (Tout)v0;
    }
}

// R0, C0: first cube row / column the tile reads; cubes outside [ilo, ihi) x [jlo, jhi)
// are masked (MASK only)
template <typename Tin, typename Tout, bool ROWCHK, bool COLCHK, bool MASK, bool WRITE, int RPW>
__device__ __forceinline__ void pass_body(const PassParams &p, const Tin *fa, const Tin *fb, int pair, int R0,
                                          int C0, int ilo, int ihi, int jlo, int jhi, float2 acc[NSUM])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gcl = C0 + 4 * lane;
    const int gr0 = R0 + RPW * warp;
    const float2 x0 = make_float2((float)gcl + p.xoff, (float)(gcl + HALF) + p.xoff);
    const int Hn = p.H >> 1, Wn = p.W >> 1;
    // consecutive pairs of a video share frames (frame t+1 of pair t is frame t+1 of
    // the next pair): the first frame is written by pair 0 only; independent pairs
    // own two frames each
    const bool wprev = WRITE && (p.write_prev == 1 || (p.write_prev == 0 && pair == 0));
    const int64_t fprev = p.write_prev == 1 ? 2 * (int64_t)pair : (int64_t)pair;
    unsigned char *nprev = WRITE && wprev ? p.next + fprev * p.next_fstride : nullptr;
    unsigned char *ncur = WRITE ? (p.next_cur ? p.next_cur : p.next + (fprev + 1) * p.next_fstride) : nullptr;

    constexpr int PF = COLCHK ? 1 : (FT_TTC_PF < RPW ? FT_TTC_PF : RPW);
    RawRow<Tin> raw[RPW + 1];
#pragma unroll
    for (int r = 0; r < PF; ++r) load_raw<Tin, ROWCHK, COLCHK, !COLCHK>(p, fa, fb, gr0 + r, gcl, raw[r]);

    float2 xk[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) xk[k] = add2(x0, make_float2((float)k, (float)k));
    float2 y = make_float2((float)(gr0 - 1) + p.yoff, (float)(gr0 - 1) + p.yoff);
    Strip st;
    Pyr py;
#pragma unroll
    for (int r = 0; r <= RPW; ++r) {
        if (r + PF <= RPW) load_raw<Tin, ROWCHK, COLCHK, !COLCHK>(p, fa, fb, gr0 + r + PF, gcl, raw[r + PF]);
        float2 A[4], D[4];
        const int i = gr0 + r - 1;
        row_step<Tin, MASK>(raw[r], lane, st, r == 0, xk, y, i >= ilo && i < ihi, gcl, gcl + HALF, jlo, jhi, acc,
                            A, D);
        y = add2(y, make_float2(1.f, 1.f));
        if (WRITE && r < RPW) {
            if ((r & 1) == 0) {
                pyr_even(py, A, D);
            } else {
                float2 va0, va1, vb0, vb1;
                pyr_odd(py, A, D, va0, va1, vb0, vb1);
                const int r1 = (gr0 >> 1) + (r >> 1);
                const int cl = gcl >> 1, cr = (gcl + HALF) >> 1;
                store_next<Tout, MASK>(p, ncur, p.next_pitch, r1, cl, vb0.x, vb1.x, Hn, Wn);
                store_next<Tout, MASK>(p, ncur, p.next_pitch, r1, cr, vb0.y, vb1.y, Hn, Wn);
                if (wprev) {
                    store_next<Tout, MASK>(p, nprev, p.next_pitch, r1, cl, va0.x, va1.x, Hn, Wn);
                    store_next<Tout, MASK>(p, nprev, p.next_pitch, r1, cr, va0.y, va1.y, Hn, Wn);
                }
            }
        }
    }
}

// Tile sets.  Interior tiles read only inside the image: vector loads, no masks.
// Images of levels >= 1 live in the context, padded past the last tile row and
// column: their last tile row and column (SET_EDGES) are shifted inwards (origin
// H - 1 - TR rounded up to even, W - 1 - TC rounded up to a multiple of 4) so that
// they cover the rest of the image with vector loads, read at most one row and three
// columns into the padding, and mask every cube outside their own tile or the image;
// pyramid pixels they share with a neighbour are written twice with the same value.
// Level 0 reads the caller's frames, which have no padding: its last tile row clamps
// rows past the image (SET_BOTTOM; vector loads, columns inside), its last tile
// column checks every element group (SET_RIGHT), and SET_ALL (narrow images or
// frames whose rows do not allow vector loads) checks everything.
__device__ __forceinline__ void decode_tile(const PassParams &p, int64_t bid, int &pair, int &ty, int &tx)
{
    int n;
    switch (p.set) {
    case SET_INTERIOR: n = (p.tiles_y - 1) * (p.tiles_x - 1); break;
    case SET_EDGES: n = p.tiles_x + p.tiles_y - 1; break;
    case SET_BOTTOM: n = p.tiles_x - 1; break;
    case SET_RIGHT: n = p.tiles_y; break;
    default: n = p.ntiles; break;
    }
    pair = (int)(bid / n);
    const int t = (int)(bid - (int64_t)pair * n);
    switch (p.set) {
    case SET_INTERIOR: ty = t / (p.tiles_x - 1); tx = t - ty * (p.tiles_x - 1); break;
    case SET_EDGES:
        if (t < p.tiles_x) { ty = p.tiles_y - 1; tx = t; }
        else { ty = t - p.tiles_x; tx = p.tiles_x - 1; }
        break;
    case SET_BOTTOM: ty = p.tiles_y - 1; tx = t; break;
    case SET_RIGHT: ty = t; tx = p.tiles_x - 1; break;
    default: ty = t / p.tiles_x; tx = t - ty * p.tiles_x; break;
    }
}

inline int64_t set_size(const PassParams &p)
{
    switch (p.set) {
    case SET_INTERIOR: return (int64_t)(p.tiles_y - 1) * (p.tiles_x - 1);
    case SET_EDGES: return p.tiles_x + p.tiles_y - 1;
    case SET_BOTTOM: return p.tiles_x - 1;
    case SET_RIGHT: return p.tiles_y;
    default: return p.ntiles;
    }
}

// ROWCHK / COLCHK: bounds checks on rows / element groups; MASK: cubes outside the
// tile or the image are masked; SHIFT: edge tiles move inwards (padded images)
template <typename Tin, typename Tout, bool WRITE, bool ROWCHK, bool COLCHK, bool MASK, bool SHIFT, int RPW>
__global__ void __launch_bounds__(NT, RPW == 2 ? 3 : FT_TTC_MINB)
ttc_pass_kernel(const PassParams p)
{
    __shared__ float red[NSUM * NT];
    int pair, ty, tx;
    decode_tile(p, blockIdx.x, pair, ty, tx);
    const int tile = ty * p.tiles_x + tx;
    constexpr int TRL = 8 * RPW;            // cube rows of this kernel's tiles
    const int ilo = ty * TRL, jlo = tx * TC;
    int R0 = ilo, C0 = jlo;
    if (SHIFT) {
        R0 = min(R0, (p.H - 1 - TRL + 1) & ~1);
        C0 = min(C0, (p.W - 1 - TC + 3) & ~3);
    }
    const Tin *fa = reinterpret_cast<const Tin *>(p.prev + (int64_t)pair * p.pair_stride);
    const Tin *fb = reinterpret_cast<const Tin *>(p.cur + (int64_t)pair * p.pair_stride);

    float2 acc2[NSUM];
#pragma unroll
    for (int s = 0; s < NSUM; ++s) acc2[s] = make_float2(0.f, 0.f);
    pass_body<Tin, Tout, ROWCHK, COLCHK, MASK, WRITE, RPW>(p, fa, fb, pair, R0, C0, ilo, min(ilo + TRL, p.H - 1),
                                                           jlo, min(jlo + TC, p.W - 1), acc2);
    float acc[NSUM];
#pragma unroll
    for (int s = 0; s < NSUM; ++s) acc[s] = acc2[s].x + acc2[s].y;
    block_reduce(acc, red, p.partials + ((int64_t)pair * p.ntiles + tile) * NSUM);
}

template <typename Tin, typename Tout, bool WRITE, bool ROWCHK, bool COLCHK, bool MASK, bool SHIFT, int RPW>
int launch_set(PassParams p, int set, int npairs, cudaStream_t s)
{
    p.set = set;
    const int64_t n = set_size(p) * npairs;
    if (n <= 0) return 0;
    ttc_pass_kernel<Tin, Tout, WRITE, ROWCHK, COLCHK, MASK, SHIFT, RPW><<<(unsigned)n, NT, 0, s>>>(p);
    return 1;
}

// launches the pass; adds the number of kernels launched to *count.  RPW: cube rows
// per warp (tiles of 8 * RPW rows)
template <typename Tin, typename Tout, bool WRITE, int RPW>
void launch_rpw(const PassParams &p, int npairs, cudaStream_t s, int *count)
{
    constexpr int TRL = 8 * RPW;
    const bool big = p.H >= TRL + 2 && p.W >= TC + 4;
    int n = 0;
    if (p.padded && big) {
        n += launch_set<Tin, Tout, WRITE, false, false, false, false, RPW>(p, SET_INTERIOR, npairs, s);
        n += launch_set<Tin, Tout, WRITE, false, false, true, true, RPW>(p, SET_EDGES, npairs, s);
    } else if (p.vec && big) {
        n += launch_set<Tin, Tout, WRITE, false, false, false, false, RPW>(p, SET_INTERIOR, npairs, s);
        n += launch_set<Tin, Tout, WRITE, true, false, true, false, RPW>(p, SET_BOTTOM, npairs, s);
        n += launch_set<Tin, Tout, WRITE, true, true, true, false, RPW>(p, SET_RIGHT, npairs, s);
    } else {
        n += launch_set<Tin, Tout, WRITE, true, true, true, false, RPW>(p, SET_ALL, npairs, s);
    }
    *count += n;
}

template <typename Tin, typename Tout, bool WRITE>
cudaError_t launch_w(const PassParams &p, int npairs, cudaStream_t s, int *count)
{
    if (p.tr == 64) launch_rpw<Tin, Tout, WRITE, 8>(p, npairs, s, count);
    else launch_rpw<Tin, Tout, WRITE, 2>(p, npairs, s, count);
    return cudaGetLastError();
}

template <typename Tin, typename Tout>
cudaError_t launch(const PassParams &p, int npairs, cudaStream_t s, int *count)
{
    return p.next ? launch_w<Tin, Tout, true>(p, npairs, s, count) : launch_w<Tin, Tout, false>(p, npairs, s, count);
}

// ---------------------------------------------------------------------------
// batches of frame pairs of different sizes: one launch per level and tile class
// over a work list of (pair, tile) items
// ---------------------------------------------------------------------------

// descs: pass parameters of every pair at this level (pair-local: prev/cur, partials
// and next-level images of that pair only); prefix: npairs + 1 running item counts
// of this tile class.  CHECK = false: interior tiles (vector loads, no masks);
// CHECK = true: edge tiles (element checks, masks).
template <typename Tin, typename Tout, bool WRITE, bool CHECK, int RPW>
__global__ void __launch_bounds__(NT, RPW == 2 ? 3 : FT_TTC_MINB)
ttc_batch_kernel(const PassParams *__restrict__ descs, const int *__restrict__ prefix, int npairs)
{
    __shared__ float red[NSUM * NT];
    constexpr int TRL = 8 * RPW;
    const int item = blockIdx.x;
    int lo = 0, hi = npairs - 1;                 // last pair whose first item <= item
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(prefix + mid) <= item) lo = mid;
        else hi = mid - 1;
    }
    const PassParams &p = descs[lo];
    const int local = item - __ldg(prefix + lo);
    int ty, tx;
    if (!CHECK) {
        ty = local / (p.tiles_x - 1);
        tx = local - ty * (p.tiles_x - 1);
    } else if (p.set == SET_ALL) {
        ty = local / p.tiles_x;
        tx = local - ty * p.tiles_x;
    } else if (local < p.tiles_x) {
        ty = p.tiles_y - 1;
        tx = local;
    } else {
        ty = local - p.tiles_x;
        tx = p.tiles_x - 1;
    }
    const int tile = ty * p.tiles_x + tx;
    const int R0 = ty * TRL, C0 = tx * TC;
    const Tin *fa = reinterpret_cast<const Tin *>(p.prev);
    const Tin *fb = reinterpret_cast<const Tin *>(p.cur);
    float2 acc2[NSUM];
#pragma unroll
    for (int s = 0; s < NSUM; ++s) acc2[s] = make_float2(0.f, 0.f);
    pass_body<Tin, Tout, CHECK, CHECK, CHECK, WRITE, RPW>(p, fa, fb, 0, R0, C0, R0, min(R0 + TRL, p.H - 1), C0,
                                                          min(C0 + TC, p.W - 1), acc2);
    float acc[NSUM];
#pragma unroll
    for (int s = 0; s < NSUM; ++s) acc[s] = acc2[s].x + acc2[s].y;
    block_reduce(acc, red, p.partials + (int64_t)tile * NSUM);
}

template <typename Tin, typename Tout, bool WRITE, int RPW>
void launch_batch_rpw(const PassParams *descs, const int *pre_int, const int *pre_edge, int n_int, int n_edge,
                      int npairs, cudaStream_t s, int *count)
{
    if (n_int > 0) {
        ttc_batch_kernel<Tin, Tout, WRITE, false, RPW><<<n_int, NT, 0, s>>>(descs, pre_int, npairs);
        ++*count;
    }
    if (n_edge > 0) {
        ttc_batch_kernel<Tin, Tout, WRITE, true, RPW><<<n_edge, NT, 0, s>>>(descs, pre_edge, npairs);
        ++*count;
    }
}

template <typename Tin, typename Tout>
cudaError_t launch_batch(const PassParams *descs, const int *pre_int, const int *pre_edge, int n_int, int n_edge,
                         int npairs, bool write, int rpw, cudaStream_t s, int *count)
{
    if (write) {
        if (rpw == 8) launch_batch_rpw<Tin, Tout, true, 8>(descs, pre_int, pre_edge, n_int, n_edge, npairs, s, count);
        else launch_batch_rpw<Tin, Tout, true, 2>(descs, pre_int, pre_edge, n_int, n_edge, npairs, s, count);
    } else {
        if (rpw == 8) launch_batch_rpw<Tin, Tout, false, 8>(descs, pre_int, pre_edge, n_int, n_edge, npairs, s, count);
        else launch_batch_rpw<Tin, Tout, false, 2>(descs, pre_int, pre_edge, n_int, n_edge, npairs, s, count);
    }
    return cudaGetLastError();
}

}  // namespace ttc_pass
