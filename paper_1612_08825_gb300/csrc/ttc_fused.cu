// All pyramid levels of uint8 frame pairs in one persistent launch (Sec. II stencil,
// Sec. V-A G and the ten sums, Sec. V-B 2x2 block-sum pyramid); the scheme is described
// in ttc_fused.cuh.
//
// Per item a CTA of 256 threads runs, between CTA barriers:
//   A  the level-0 cubes of the 64 x 256 tile from the copy-engine buffer (the copy-engine
//      pass's arithmetic), writing both frames' level-1 pixels of the tile's 32 rows into
//      the level-1 ring; the 8 level-1 columns right of the tile from the extra box;
//      the level-0 tile reduction;
//   B  the level-1 cubes (4 rows x 2 columns in each half of the tile per thread) from the
//      ring, and from the same words the level-2 and level-3 pixels of the tile's rows;
//      the level-1 reduction;
//   D  the level-2, 3 and 4 cubes by three groups of threads (warp 6 first forms the
//      level-4 pixels); one reduction of the three levels.
// Rings hold packed (first frame | second frame << 16) uint16 block sums; row r of level
// l lives in slot r mod (64 / 2^l + 1).  The partials of level l carry the scale of the
// block sums (4^l) and of the stencil (4); levels 0..3 carry 2^16 more (pixels scaled by
// 256 in the arithmetic), level 4 not.
#include <algorithm>

#include "common.cuh"
#include "tma.cuh"
#include "ttc_pass.cuh"
#include "ttc_tma.cuh"
#include "ttc_fused.cuh"

namespace ttc_fused {
namespace {

using namespace ttc_pass;
using namespace ft_tma;
using ttc_tma::BOX;
using ttc_tma::BUF;
using ttc_tma::BW;
using ttc_tma::FRAME;
using ttc_tma::Raw8;
using ttc_tma::Strip8;
using ttc_tma::TX;
using ttc_tma::XW;

// rings: slots (the tile's new rows plus the row above them) x row stride in words
constexpr int S1 = 33, RS1 = 136;       // 128 + 8 columns
constexpr int S2 = 17, RS2 = 68;        // 64 + 4
constexpr int S3 = 9, RS3 = 36;         // 32 + 2, padded to 16-byte rows
constexpr int S4 = 5, RS4 = 20;         // 16 + 1, padded
constexpr int RING_WORDS = S1 * RS1 + S2 * RS2 + S3 * RS3 + S4 * RS4;

enum Kind { K_TILE = 0, K_PRO = 1, K_END = 2 };

struct Item {
    Geom g;
    int kind, pair, tx, j;
};

constexpr int SMEM = 2 * BUF + RING_WORDS * 4 + NSUM * NT * 4 + 2 * 8 + 2 * (int)sizeof(Item);

template <int N>
__device__ __forceinline__ int slot(int row)           // row >= -1
{
    return (row + N) % N;
}

// packed (first | second << 16) word of two level-(l+1) pixels held as 2^23 + v floats
__device__ __forceinline__ uint32_t pack(float a, float b)
{
    return __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x5410u);
}

// ---------------------------------------------------------------------------
// phase A: level 0 (the copy-engine pass's tile body, next level into the ring)
// ---------------------------------------------------------------------------

// UNR: unroll factor of the row loop
template <bool MASK, bool FOLD, int UNR>
__device__ __forceinline__ void tile0(const Geom &g, const unsigned char *buf, int j, int C0, uint32_t *ring1,
                                      float2 acc[NSUM])
{
    constexpr int RPW = FOLD ? 4 : 8;           // cube rows per warp
    constexpr int DR = FOLD ? TR / 2 : 0;       // row offset of the pair's second lane
    const int R0 = j * TR;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gcl = C0 + 4 * lane;
    const int gcr = FOLD ? gcl : gcl + HALF;
    const int gr0 = R0 + RPW * warp;
    const float xo = g.xoff[0], yo = g.yoff[0];
    const float2 x0 = make_float2((float)gcl + xo, (float)gcr + xo);
    const int ihi = min(R0 + TR, g.H - 1), jhi = min(C0 + TC, g.W - 1);
    const int ccl = 2 * lane, ccr = FOLD ? 2 * lane : HALF / 2 + 2 * lane;   // ring columns
    const int jm = j % S1;

    float2 xk[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) xk[k] = add2(x0, make_float2((float)k, (float)k));
    float2 y = make_float2((float)(gr0 - 1) + yo, (float)(gr0 - 1 + DR) + yo);
    Strip8 st;
    float2 hb[2], ha[2];
    Raw8 nxt;
    ttc_tma::row_from_smem<FOLD>(buf, RPW * warp, lane, nxt);
#pragma unroll(UNR)
    for (int r = 0; r <= RPW; ++r) {
        const Raw8 cur = nxt;
        if (r < RPW) ttc_tma::row_from_smem<FOLD>(buf, RPW * warp + r + 1, lane, nxt);
        float2 A[4], B[4];
        const int i = gr0 + r - 1;
        ttc_tma::row_step8<MASK, FOLD>(cur, lane, st, r == 0, xk, y, i >= R0 && i < ihi,
                                       i + DR >= R0 && i + DR < ihi, gcl, gcr, C0, jhi, acc, A, B);
        y = add2(y, make_float2(1.f, 1.f));
        if (r < RPW) {
            const float2 b0 = add2(B[0], B[1]), b1 = add2(B[2], B[3]);
            const float2 a0 = add2(A[0], A[1]), a1 = add2(A[2], A[3]);
            if ((r & 1) == 0) {
                hb[0] = b0;
                hb[1] = b1;
                ha[0] = a0;
                ha[1] = a1;
            } else {
                // tile-local level-1 rows of the two lanes; global row 32 j + q sits in
                // slot (q - j) mod 33
                const int q1 = (RPW / 2) * warp + (r >> 1), q2 = q1 + DR / 2;
                int s1 = q1 - jm, s2 = q2 - jm;
                s1 += s1 < 0 ? S1 : 0;
                s2 += s2 < 0 ? S1 : 0;
                const float2 v0 = ttc_tma::unscale_block(add2(hb[0], b0));
                const float2 v1 = ttc_tma::unscale_block(add2(hb[1], b1));
                const float2 u0 = ttc_tma::unscale_block(add2(ha[0], a0));
                const float2 u1 = ttc_tma::unscale_block(add2(ha[1], a1));
                *reinterpret_cast<uint2 *>(ring1 + s1 * RS1 + ccl) = make_uint2(pack(u0.x, v0.x), pack(u1.x, v1.x));
                *reinterpret_cast<uint2 *>(ring1 + s2 * RS1 + ccr) = make_uint2(pack(u0.y, v0.y), pack(u1.y, v1.y));
            }
        }
    }
}

// level-1 columns 128..135 of the tile's 32 rows, from the extra box (level-0 columns
// 256..271): one per thread
__device__ __forceinline__ void l1_extra(const unsigned char *buf, int j, uint32_t *ring1)
{
    const int t = threadIdx.x, q = t >> 3, e = t & 7;
    const int o = 2 * q * XW + 2 * e;
    uint32_t v[2];
#pragma unroll
    for (int f = 0; f < 2; ++f) {
        const unsigned char *x = buf + f * FRAME + 2 * BOX;
        const uint32_t w0 = *reinterpret_cast<const unsigned short *>(x + o);
        const uint32_t w1 = *reinterpret_cast<const unsigned short *>(x + o + XW);
        v[f] = (w0 & 0xffu) + (w0 >> 8) + (w1 & 0xffu) + (w1 >> 8);
    }
    ring1[slot<S1>(32 * j + q) * RS1 + 128 + e] = v[0] | (v[1] << 16);
}

// ---------------------------------------------------------------------------
// phases B, D: cubes of levels >= 1 from a ring
// ---------------------------------------------------------------------------

// A packed word's two pixels as the (left, right) lanes of two float pairs.  SC: as
// 2^23 + 256 v (one byte permute; exact for v < 2^15, i.e. levels 1..3), so that every
// stencil sum and difference is a multiple of 256 below 2^26 and exact, and the ten
// products are 2^16 times the unscaled ones; otherwise as v itself (level 4, sums up to
// 2^16), with the bias removed.
template <bool SC>
__device__ __forceinline__ void px2(uint32_t wl, uint32_t wr, float2 &A, float2 &B)
{
    if (SC) {
        A = make_float2(__int_as_float(__byte_perm(wl, 0x4B000000u, 0x7104u)),
                        __int_as_float(__byte_perm(wr, 0x4B000000u, 0x7104u)));
        B = make_float2(__int_as_float(__byte_perm(wl, 0x4B000000u, 0x7324u)),
                        __int_as_float(__byte_perm(wr, 0x4B000000u, 0x7324u)));
    } else {
        const float2 bias = make_float2(8388608.f, 8388608.f);
        A = sub2(make_float2(__int_as_float(__byte_perm(wl, 0x4B000000u, 0x7410u)),
                             __int_as_float(__byte_perm(wr, 0x4B000000u, 0x7410u))), bias);
        B = sub2(make_float2(__int_as_float(__byte_perm(wl, 0x4B000000u, 0x7432u)),
                             __int_as_float(__byte_perm(wr, 0x4B000000u, 0x7432u))), bias);
    }
}

// The cubes of RB rows i0 .. i0+RB-1 of one level, columns cl, cl+1 (left lane) and cr,
// cr+1 (right lane) of the ring; gcl, gcr: the level's columns of cl, cr.  The window is
// RB + 1 pixel rows x 3 columns per lane; the previous row is carried as partial cube
// values (hs = s[k+1] - s[k], hp = s[k+1] + s[k], dp = d[k+1] + d[k], s = first + second,
// d = second - first), so Ex = hs + hs', Ey = hp - hp', Et = dp + dp' (the 2x2x2 first
// differences of Sec. II, times 4, times 256 with SC).  MASK: cubes outside the level
// image (rows < 0 or > Hk - 2, columns > Wk - 2) are zeroed.  PYR (level 1, RB = 4): the
// window rows 1..4 of columns cl, cl+1 and cr, cr+1 are 2 x 2 blocks of level-2 pixels:
// the first row pair's to l2a[0] / l2a[32], the second's to l2b[0] / l2b[32]; returns in
// tl, tr the sum of each lane's two level-2 pixels (half of a level-3 pixel).
template <int RB, bool MASK, bool SC, bool PYR>
__device__ __forceinline__ void ring_lr(const uint32_t *ring, int RS, int NS, int i0, int cl, int cr, int gcl,
                                        int gcr, int Hk, int Wk, float xo, float yo, float2 acc[NSUM],
                                        uint32_t *l2a = nullptr, uint32_t *l2b = nullptr, uint32_t *tl = nullptr,
                                        uint32_t *tr = nullptr)
{
    int sl = (i0 + NS) % NS;
    const float2 xk[2] = {make_float2((float)gcl + xo, (float)gcr + xo),
                          make_float2((float)(gcl + 1) + xo, (float)(gcr + 1) + xo)};
    float2 phs[2], php[2], pdp[2];
    uint32_t kl0 = 0, kl1 = 0, kr0 = 0, kr1 = 0, sl2 = 0, sr2 = 0;
#pragma unroll
    for (int r = 0; r <= RB; ++r) {
        const uint32_t *row = ring + sl * RS;
        const uint2 L = *reinterpret_cast<const uint2 *>(row + cl);
        const uint2 R = *reinterpret_cast<const uint2 *>(row + cr);
        const uint32_t L2 = row[cl + 2], R2 = row[cr + 2];
        float2 A[3], B[3];
        px2<SC>(L.x, R.x, A[0], B[0]);
        px2<SC>(L.y, R.y, A[1], B[1]);
        px2<SC>(L2, R2, A[2], B[2]);
        float2 s[3], d[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            s[k] = add2(A[k], B[k]);
            d[k] = sub2(B[k], A[k]);
        }
        float2 hs[2], hp[2], dp[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            hs[k] = sub2(s[k + 1], s[k]);
            hp[k] = add2(s[k + 1], s[k]);
            dp[k] = add2(d[k + 1], d[k]);
        }
        if (r > 0) {
            const int i = i0 + r - 1;
            const float yv = (float)i + yo;
            const float2 y = make_float2(yv, yv);
            const bool rowok = i >= 0 && i <= Hk - 2;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                float2 ex = add2(hs[k], phs[k]);
                float2 ey = sub2(hp[k], php[k]);
                float2 et = add2(dp[k], pdp[k]);
                if (MASK) mask3(ex, ey, et, rowok && gcl + k <= Wk - 2, rowok && gcr + k <= Wk - 2);
                accum2(acc, ex, ey, et, xk[k], y);
            }
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            phs[k] = hs[k];
            php[k] = hp[k];
            pdp[k] = dp[k];
        }
        if (PYR) {
            if (r == 1 || r == 3) {
                kl0 = L.x;
                kl1 = L.y;
                kr0 = R.x;
                kr1 = R.y;
            } else if (r == 2 || r == 4) {
                // packed sums: each half stays below 2^16 (4 x 1020)
                const uint32_t vl = (kl0 + L.x) + (kl1 + L.y), vr = (kr0 + R.x) + (kr1 + R.y);
                uint32_t *dst = r == 2 ? l2a : l2b;
                dst[0] = vl;
                dst[32] = vr;
                sl2 += vl;
                sr2 += vr;
            }
        }
        sl = sl + 1 == NS ? 0 : sl + 1;
    }
    if (PYR) {
        *tl = sl2;
        *tr = sr2;
    }
}

// one (masked) variant per level: a second, unmasked copy of each costs more in
// instruction-cache misses than the masks cost in issue slots
template <int RB, bool SC, bool PYR>
__device__ __forceinline__ void ring_cubes(const uint32_t *ring, int RS, int NS, int i0, int cl, int cr, int gcl,
                                           int gcr, int Hk, int Wk, float xo, float yo, float2 acc[NSUM],
                                           uint32_t *l2a = nullptr, uint32_t *l2b = nullptr,
                                           uint32_t *tl = nullptr, uint32_t *tr = nullptr)
{
    ring_lr<RB, true, SC, PYR>(ring, RS, NS, i0, cl, cr, gcl, gcr, Hk, Wk, xo, yo, acc, l2a, l2b, tl, tr);
}

// ---------------------------------------------------------------------------
// prologue of a unit that starts at tile row j0 > 0: the rows above the unit's first
// tile that its cubes need (level 1: 32 j0 - 1, level 2: 16 j0 - 1, level 3: 8 j0 - 1,
// level 4: 4 j0 - 1), from the 16 level-0 rows above it (buffer rows 0..15)
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t pair_sum(const unsigned char *f, int row, int c)
{
    // level-0 columns 2c, 2c+1 of buffer row `row` (main boxes, then the extra box)
    const unsigned char *p = c < 64 ? f + row * BW + 2 * c
                             : c < 128 ? f + BOX + row * BW + 2 * (c - 64)
                                       : f + 2 * BOX + row * XW + 2 * (c - 128);
    const uint32_t w = *reinterpret_cast<const unsigned short *>(p);
    return (w & 0xffu) + (w >> 8);
}

__device__ void prologue(const unsigned char *buf, int j0, uint32_t *ring1, uint32_t *ring2, uint32_t *ring3,
                         uint32_t *ring4)
{
    const int t = threadIdx.x;
    for (int o = t; o < 8 * 136; o += NT) {
        const int q = o / 136, c = o - q * 136;
        const uint32_t a = pair_sum(buf, 2 * q, c) + pair_sum(buf, 2 * q + 1, c);
        const uint32_t b = pair_sum(buf + FRAME, 2 * q, c) + pair_sum(buf + FRAME, 2 * q + 1, c);
        ring1[slot<S1>(32 * j0 - 8 + q) * RS1 + c] = a | (b << 16);
    }
    __syncthreads();
    for (int o = t; o < 4 * 68; o += NT) {
        const int q = o / 68, c = o - q * 68;
        const int ra = 32 * j0 - 8 + 2 * q;
        const uint32_t *a = ring1 + slot<S1>(ra) * RS1 + 2 * c, *b = ring1 + slot<S1>(ra + 1) * RS1 + 2 * c;
        ring2[slot<S2>(16 * j0 - 4 + q) * RS2 + c] = (a[0] + a[1]) + (b[0] + b[1]);
    }
    __syncthreads();
    if (t < 2 * 34) {
        const int q = t / 34, c = t - q * 34;
        const int ra = 16 * j0 - 4 + 2 * q;
        const uint32_t *a = ring2 + slot<S2>(ra) * RS2 + 2 * c, *b = ring2 + slot<S2>(ra + 1) * RS2 + 2 * c;
        ring3[slot<S3>(8 * j0 - 2 + q) * RS3 + c] = (a[0] + a[1]) + (b[0] + b[1]);
    }
    __syncthreads();
    if (t < 17) {
        const int ra = 8 * j0 - 2;
        const uint32_t *a = ring3 + slot<S3>(ra) * RS3 + 2 * t, *b = ring3 + slot<S3>(ra + 1) * RS3 + 2 * t;
        ring4[slot<S4>(4 * j0 - 1) * RS4 + t] = (a[0] + a[1]) + (b[0] + b[1]);
    }
}

// second frame's level-l pixels of the tile's rows into the caller's pyramid block
__device__ __forceinline__ void pyr_out(const Geom &g, int l, const uint32_t *ring, int RS, int NS, int j, int C0,
                                        int t0, int nt)
{
    const int nr = TR >> l, nc = TC >> l;
    const int Hl = g.H >> l, Wl = g.W >> l;
    unsigned char *img = g.pyr + g.pyr_off[l];
    for (int o = threadIdx.x - t0; o < nr * nc; o += nt) {
        const int q = o / nc, c = o - q * nc;
        const int row = nr * j + q, col = (C0 >> l) + c;
        if (row < Hl && col < Wl)
            reinterpret_cast<unsigned short *>(img + row * g.pyr_pitch[l])[col] =
                (unsigned short)(ring[(row % NS) * RS + c] >> 16);
    }
}

// ---------------------------------------------------------------------------
// one tile of all levels
// ---------------------------------------------------------------------------

// Fixed-order reduction of levels 2, 3, 4 held by thread groups [0,128), [128,192),
// [192,208): eight lanes per (level, sum), then a 3-step shuffle tree; dst: this thread's
// output (t < 240, t % 8 == 0) or null
__device__ __forceinline__ void reduce_levels(const float acc[NSUM], float *red, float *dst)
{
    const int tid = threadIdx.x;
#pragma unroll
    for (int s = 0; s < NSUM; ++s) red[s * NT + tid] = acc[s];
    __syncthreads();
    float v = 0.f;
    if (tid < 30 * 8) {
        const int o = tid >> 3, sub = tid & 7;
        const int lv = o / NSUM, s = o - lv * NSUM;
        const int lo = lv == 0 ? 0 : lv == 1 ? 128 : 192, n = lv == 0 ? 16 : lv == 1 ? 8 : 2;
        for (int m = 0; m < n; ++m) v += red[s * NT + lo + sub + 8 * m];
    }
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    if (dst) *dst = v;
}

__device__ __forceinline__ void fold(const float2 acc2[NSUM], float acc[NSUM])
{
#pragma unroll
    for (int s = 0; s < NSUM; ++s) acc[s] = acc2[s].x + acc2[s].y;
}

__device__ __forceinline__ void zero(float2 acc2[NSUM])
{
#pragma unroll
    for (int s = 0; s < NSUM; ++s) acc2[s] = make_float2(0.f, 0.f);
}

// Every read of the item's descriptor (smem) happens before the item's last barrier: the
// copy-issuing thread rewrites it for the item after next right after that barrier.
__device__ void tile(const Item &it, const unsigned char *buf, uint32_t *ring1, uint32_t *ring2, uint32_t *ring3,
                     uint32_t *ring4, float *red)
{
    const Geom &g = it.g;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int j = it.j, C0 = it.tx * TC, R0 = j * TR;
    const int tileno = j * g.tiles_x + it.tx;
    const int nlev = g.nlev;
    float2 acc2[NSUM];
    float acc[NSUM];

    // A: level 0
    zero(acc2);
    const bool edge = (R0 + TR > g.H - 1) || (C0 + TC > g.W - 1);
    const bool narrow = g.W - 1 - C0 <= HALF;
    if (narrow) tile0<true, true, 5>(g, buf, j, C0, ring1, acc2);
    else if (edge) tile0<true, false, 9>(g, buf, j, C0, ring1, acc2);
    else tile0<false, false, 9>(g, buf, j, C0, ring1, acc2);
    l1_extra(buf, j, ring1);
    fold(acc2, acc);
    block_reduce(acc, red, g.part[0] + (int64_t)tileno * NSUM);

    // B: level 1 (a warp per 4 rows; a lane 2 columns in each 64-column half), the tile's
    // level-2 pixels from the same words and its level-3 pixels from lane pairs
    zero(acc2);
    {
        const int c = 2 * lane;
        uint32_t *l2a = ring2 + slot<S2>(16 * j + 2 * warp) * RS2 + lane;
        uint32_t *l2b = ring2 + slot<S2>(16 * j + 2 * warp + 1) * RS2 + lane;
        uint32_t tl, tr;
        ring_cubes<4, true, true>(ring1, RS1, S1, 32 * j - 1 + 4 * warp, c, 64 + c, (C0 >> 1) + c,
                                  (C0 >> 1) + 64 + c, g.H >> 1, g.W >> 1, g.xoff[1], g.yoff[1], acc2, l2a, l2b,
                                  &tl, &tr);
        const uint32_t ol = __shfl_xor_sync(0xffffffffu, tl, 1), orr = __shfl_xor_sync(0xffffffffu, tr, 1);
        if ((lane & 1) == 0) {
            uint32_t *l3 = ring3 + slot<S3>(8 * j + warp) * RS3 + (lane >> 1);
            l3[0] = tl + ol;
            l3[16] = tr + orr;
        }
    }
    if (tid < 64) {
        // level-2 columns 64..67 from level-1 columns 128..135
        const int rr = tid >> 2, c = tid & 3;
        const uint32_t *a = ring1 + slot<S1>(32 * j + 2 * rr) * RS1 + 128 + 2 * c;
        const uint32_t *b = ring1 + slot<S1>(32 * j + 2 * rr + 1) * RS1 + 128 + 2 * c;
        ring2[slot<S2>(16 * j + rr) * RS2 + 64 + c] = (a[0] + a[1]) + (b[0] + b[1]);
    } else if (tid < 80) {
        // level-3 columns 32, 33 from level-1 columns 128..135
        const int u = tid - 64, rr = u >> 1, c = u & 1;
        uint32_t v = 0;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const uint4 x = *reinterpret_cast<const uint4 *>(ring1 + slot<S1>(32 * j + 4 * rr + m) * RS1 + 128 + 4 * c);
            v += (x.x + x.y) + (x.z + x.w);
        }
        ring3[slot<S3>(8 * j + rr) * RS3 + 32 + c] = v;
    }
    fold(acc2, acc);
    // the tile buffer is free (level 0 is done): it serves as this reduction's scratch
    block_reduce(acc, reinterpret_cast<float *>(const_cast<unsigned char *>(buf)),
                 g.part[1] + (int64_t)tileno * NSUM);

    if (nlev < 3) {
        if (g.pyr) pyr_out(g, 1, ring1, RS1, S1, j, C0, 0, NT);
        __syncthreads();
        return;
    }

    // D: levels 2, 3, 4 by three groups of threads (half-warps, groups of 8 and 4 lanes
    // per row band; two columns per lane in each half of the level's tile width)
    zero(acc2);
    if (tid < 128) {
        const int grp = tid >> 4, c = 2 * (tid & 15);
        ring_cubes<2, true, false>(ring2, RS2, S2, 16 * j - 1 + 2 * grp, c, 32 + c, (C0 >> 2) + c,
                                   (C0 >> 2) + 32 + c, g.H >> 2, g.W >> 2, g.xoff[2], g.yoff[2], acc2);
    } else if (tid < 192) {
        if (nlev > 3) {
            const int u = tid - 128, grp = u >> 3, c = 2 * (u & 7);
            ring_cubes<1, true, false>(ring3, RS3, S3, 8 * j - 1 + grp, c, 16 + c, (C0 >> 3) + c,
                                       (C0 >> 3) + 16 + c, g.H >> 3, g.W >> 3, g.xoff[3], g.yoff[3], acc2);
        }
    } else if (warp == 6) {
        if (nlev > 4) {
            for (int o = lane; o < 4 * 17; o += 32) {
                const int rr = o / 17, c = o - rr * 17;
                const uint32_t *a = ring3 + slot<S3>(8 * j + 2 * rr) * RS3 + 2 * c;
                const uint32_t *b = ring3 + slot<S3>(8 * j + 2 * rr + 1) * RS3 + 2 * c;
                ring4[slot<S4>(4 * j + rr) * RS4 + c] = (a[0] + a[1]) + (b[0] + b[1]);
            }
            __syncwarp();
            if (lane < 16) {
                const int grp = lane >> 2, c = 2 * (lane & 3);
                ring_cubes<1, false, false>(ring4, RS4, S4, 4 * j - 1 + grp, c, 8 + c, (C0 >> 4) + c,
                                            (C0 >> 4) + 8 + c, g.H >> 4, g.W >> 4, g.xoff[4], g.yoff[4], acc2);
            }
            if (g.pyr) pyr_out(g, 4, ring4, RS4, S4, j, C0, 6 * 32, 32);
        }
    }
    if (g.pyr) {
        pyr_out(g, 1, ring1, RS1, S1, j, C0, 0, NT);
        pyr_out(g, 2, ring2, RS2, S2, j, C0, 0, NT);
        if (nlev > 3) pyr_out(g, 3, ring3, RS3, S3, j, C0, 0, NT);
    }
    fold(acc2, acc);
    float *dst = nullptr;
    if (tid < 240 && (tid & 7) == 0) {
        const int o = tid >> 3, lv = 2 + o / NSUM, s = o % NSUM;
        if (lv < nlev) dst = g.part[lv] + (int64_t)tileno * NSUM + s;
    }
    reduce_levels(acc, red, dst);
}

// ---------------------------------------------------------------------------
// units
// ---------------------------------------------------------------------------

__device__ __forceinline__ void unit_of(const VideoUnits &u, int t, int &pair, int &tx, int &j0, int &len)
{
    const int per_pair = u.g.tiles_x * u.nseg;
    pair = t / per_pair;
    const int r = t - pair * per_pair;
    tx = r / u.nseg;
    const int sg = r - tx * u.nseg;
    j0 = sg * u.seg;
    len = min(u.seg, u.g.tiles_y - j0);
}

__device__ __forceinline__ void geom_of(const VideoUnits &u, int pair, Geom &o)
{
    o = u.g;
    const int64_t off = (int64_t)pair * u.g.ntiles * NSUM;
#pragma unroll
    for (int l = 0; l < MAXLEV; ++l) o.part[l] = u.g.part[l] ? u.g.part[l] + off : nullptr;
}

__device__ __forceinline__ const CUtensorMap *maps_of(const VideoUnits &u, int pair, int &z)
{
    z = pair;
    return u.m;
}

__device__ __forceinline__ void unit_of(const BatchUnits &u, int t, int &pair, int &tx, int &j0, int &len)
{
    const int4 v = __ldg(u.units + t);
    pair = v.x;
    tx = v.y;
    j0 = v.z;
    len = v.w;
}

__device__ __forceinline__ void geom_of(const BatchUnits &u, int pair, Geom &o) { o = u.geoms[pair]; }

__device__ __forceinline__ const CUtensorMap *maps_of(const BatchUnits &u, int pair, int &z)
{
    z = 0;
    return u.maps + 4 * (int64_t)pair;
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------

template <class U, bool GLOBAL_MAPS>
__global__ void __launch_bounds__(NT, 2)
ttc_fused_kernel(const __grid_constant__ U units, int *status, int *counter, unsigned extra_tx)
{
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *bufs = smem;
    uint32_t *ring1 = reinterpret_cast<uint32_t *>(smem + 2 * BUF);
    uint32_t *ring2 = ring1 + S1 * RS1;
    uint32_t *ring3 = ring2 + S2 * RS2;
    uint32_t *ring4 = ring3 + S3 * RS3;
    float *red = reinterpret_cast<float *>(ring4 + S4 * RS4);
    uint64_t *bar = reinterpret_cast<uint64_t *>(red + NSUM * NT);
    Item *info = reinterpret_cast<Item *>(bar + 2);
    const int tid = threadIdx.x;
    // the copy engine writes 128-byte aligned boxes; refuse (and report) otherwise
    if (smem_addr(bufs) & 127) {
        if (tid == 0) atomicOr(status, 1);
        return;
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // thread 0's walk over its units (tickets in increasing order) and the items of each
    int u_pair = 0, u_tx = 0, u_next = 0, u_end = 0;
    bool done = false;          // the end marker has been issued
    // the pair whose geometry each slot's descriptor holds, and the last pair whose maps
    // this thread has fenced: consecutive items are mostly tiles of one strip, so the
    // 192-byte copy and the fences are made only when the pair changes
    int pair0 = -1, pair1 = -1, fenced = -1;
    auto issue_next = [&](int slot_b) -> bool {   // true: a copy is in flight for slot_b
        Item &it = info[slot_b];
        int kind = K_TILE, j = 0;
        if (u_next >= u_end) {
            const int t = atomicAdd(counter, 1);
            if (t >= units.total) {
                it.kind = K_END;
                done = true;
                mbar_arrive(&bar[slot_b]);
                return false;
            }
            int j0, len;
            unit_of(units, t, u_pair, u_tx, j0, len);
            u_next = j0;
            u_end = j0 + len;
            if (j0 > 0) {
                kind = K_PRO;
                j = j0;
            }
        }
        if (kind == K_TILE) j = u_next++;
        if ((slot_b ? pair1 : pair0) != u_pair) {
            geom_of(units, u_pair, it.g);
            if (slot_b) pair1 = u_pair;
            else pair0 = u_pair;
        }
        it.kind = kind;
        it.pair = u_pair;
        it.tx = u_tx;
        it.j = j;
        int z;
        const CUtensorMap *m = maps_of(units, u_pair, z);
        if (GLOBAL_MAPS && fenced != u_pair) {
            for (int k = 0; k < 4; ++k) ttc_tma::tensormap_acquire(m + k);
            fenced = u_pair;
        }
        unsigned char *buf = bufs + slot_b * BUF;
        const int x = u_tx * TC, y = kind == K_PRO ? j * TR - 16 : j * TR;
        // generic-proxy accesses of this buffer (earlier items) are ordered before the copies
        fence_proxy_async();
        mbar_expect_tx(&bar[slot_b], TX + extra_tx);
        tma_load_3d(buf, m + 0, x, y, z, &bar[slot_b]);
        tma_load_3d(buf + BOX, m + 0, x + BW, y, z, &bar[slot_b]);
        tma_load_3d(buf + 2 * BOX, m + 2, x + 2 * BW, y, z, &bar[slot_b]);
        tma_load_3d(buf + FRAME, m + 1, x, y, z, &bar[slot_b]);
        tma_load_3d(buf + FRAME + BOX, m + 1, x + BW, y, z, &bar[slot_b]);
        tma_load_3d(buf + FRAME + 2 * BOX, m + 3, x + 2 * BW, y, z, &bar[slot_b]);
        return true;
    };

    if (tid == 0) issue_next(0);
    for (int k = 0;; ++k) {
        const int b = k & 1;
        // one item ahead into the other buffer: every read of it (and of its descriptor)
        // by the previous item came before that item's last barrier
        bool inflight = false;
        if (tid == 0 && !done) inflight = issue_next(b ^ 1);
        const bool ok = mbar_wait(&bar[b], (k >> 1) & 1);
        if (__syncthreads_or(!ok)) {
            // give up on this CTA: report, let the copies in flight land, return
            if (tid == 0) {
                atomicOr(status, 1);
                if (inflight) mbar_wait(&bar[b ^ 1], ((k + 1) >> 1) & 1);
            }
            __syncthreads();
            return;
        }
        const int kind = info[b].kind;
        if (kind == K_END) break;
        const unsigned char *buf = bufs + b * BUF;
        if (kind == K_PRO) prologue(buf, info[b].j, ring1, ring2, ring3, ring4);
        else tile(info[b], buf, ring1, ring2, ring3, ring4, red);
    }
}

template <class U, bool GLOBAL_MAPS>
cudaError_t launch_units(const U &u, int *status, int *counter, cudaStream_t s)
{
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::min(u.total, 2 * std::max(nsm, 1));
    if (grid <= 0) return cudaSuccess;
    auto k = ttc_fused_kernel<U, GLOBAL_MAPS>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    if (e != cudaSuccess) return e;
    k<<<grid, NT, SMEM, s>>>(u, status, counter, ft::tma_extra_tx());
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_video(const VideoUnits &u, int *status, int *counter, cudaStream_t s)
{
    return launch_units<VideoUnits, false>(u, status, counter, s);
}

cudaError_t launch_batch(const BatchUnits &u, int *status, int *counter, cudaStream_t s)
{
    return launch_units<BatchUnits, true>(u, status, counter, s);
}

}  // namespace ttc_fused
