// Multi-scale time to contact / focus of expansion on sm_103a (Sec. V-A, V-B).
//
// Stage 1, ttc_tile_kernel (one CTA per level-0 tile of TR x TC cubes per pair):
//   - level 0: each thread streams 9 rows x 5 columns of both frames straight from
//     global memory (4-byte / 16-byte vector loads), forms the 2x2x2 first
//     differences Ex, Ey, Et (scaled by 4, exact for uint8 frames), G = x Ex + y Ey
//     and the ten products in FP32, and accumulates them in registers;
//   - the same loads give the 2x2 block sums of level 1 (exact for uint8), written
//     to shared memory together with a halo of 2^(levels-1) level-0 rows/columns;
//   - levels 2..L-1 are built in shared memory by 2x2 sums, and their cubes are
//     processed from shared memory;
//   - each level's per-thread sums are reduced in a fixed order (shared-memory
//     transpose, 16-way strided FP32 sums, 16-lane shuffle tree) to ten FP32
//     partials per (pair, level, tile).
// Stage 2, ttc_solve_kernel (one warp per pair and level): FP64 merge of the tile
// partials in a fixed order, scaling to level-l mean-image units, and the FP64
// solve of the normal equations (Eq. final_TTC).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "common.cuh"

namespace {

constexpr int TR = 64;          // level-0 cube rows per tile
constexpr int TC = 128;         // level-0 cube columns per tile
constexpr int NT = 256;         // threads per CTA (8 warps x 32 lanes)
constexpr int NSUM = 10;

struct TileParams {
    const unsigned char *prev;  // first frame of pair 0
    const unsigned char *cur;   // second frame of pair 0
    int64_t pair_stride;        // bytes from pair p to pair p + 1
    int64_t pitch;              // bytes between rows
    int H, W, levels, HB;       // HB: halo rows/cols (2^(levels-1), or 0 for one level)
    int tiles_x, ntiles;
    int vec;                    // 1: rows allow vector loads
    float xoff[FT_MAX_LEVELS];  // x = j + xoff[l] for cube column j of level l
    float yoff[FT_MAX_LEVELS];
    float *partials;            // [pair][level][tile][NSUM]
};

// ---------------------------------------------------------------------------
// pixel loads
// ---------------------------------------------------------------------------

__device__ __forceinline__ float u8f(uint32_t w, int k)
{
    // byte k of w as a float, exact: 2^23 + b in the mantissa, then subtract 2^23
    return __int_as_float(__byte_perm(w, 0x4B000000u, 0x7540u | (uint32_t)k)) - 8388608.f;
}

// four pixels of row `row` at columns col..col+3 (zero outside [0, W))
__device__ __forceinline__ void load4(const unsigned char *row, int col, int W, int vec, float v[4])
{
    if (vec && col + 4 <= W) {
        const uint32_t w = __ldg(reinterpret_cast<const unsigned int *>(row + col));
        v[0] = u8f(w, 0); v[1] = u8f(w, 1); v[2] = u8f(w, 2); v[3] = u8f(w, 3);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = (col + k < W) ? (float)__ldg(row + col + k) : 0.f;
    }
}

__device__ __forceinline__ void load4(const float *row, int col, int W, int vec, float v[4])
{
    if (vec && col + 4 <= W) {
        const float4 f = __ldg(reinterpret_cast<const float4 *>(row + col));
        v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = (col + k < W) ? __ldg(row + col + k) : 0.f;
    }
}

__device__ __forceinline__ float load1(const unsigned char *row, int col, int W)
{
    return col < W ? (float)__ldg(row + col) : 0.f;
}
__device__ __forceinline__ float load1(const float *row, int col, int W)
{
    return col < W ? __ldg(row + col) : 0.f;
}

// ---------------------------------------------------------------------------
// the ten products of one cube
// ---------------------------------------------------------------------------

__device__ __forceinline__ void accum(float acc[NSUM], float ex, float ey, float et, float x, float y)
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

// Fixed-order CTA reduction of ten per-thread values to dst[0..9].
// red: NSUM * NT floats of shared memory.  Called by all threads.
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
// stage 1: fused pyramid + stencil + G + products + tile reduction
// ---------------------------------------------------------------------------

template <typename T0, bool EDGE>
__device__ __forceinline__ void level0_rows(const TileParams &p, const T0 *fa, const T0 *fb,
                                            int R0, int C0, float *L1, int C1S, int R1S,
                                            float acc[NSUM])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gc = C0 + 4 * lane;            // first pixel column of this thread
    const int gr0 = R0 + 8 * warp;           // first pixel row of this thread
    const int64_t pitch_e = p.pitch / (int64_t)sizeof(T0);
    const bool pyr = p.levels > 1;
    float ps[5], pd[5];                      // previous row: prev + cur and cur - prev
    float ha[2], hb[2];                      // horizontal pair sums of the even row
    const float x0 = (float)gc + p.xoff[0];
#pragma unroll
    for (int r = 0; r < 9; ++r) {
        const int gy = gr0 + r;
        float a[5], b[5];
        if (!EDGE || gy < p.H) {
            const T0 *ra = fa + (int64_t)gy * pitch_e;
            const T0 *rb = fb + (int64_t)gy * pitch_e;
            load4(ra, gc, p.W, p.vec, a);
            load4(rb, gc, p.W, p.vec, b);
            float a4 = __shfl_down_sync(0xffffffffu, a[0], 1);
            float b4 = __shfl_down_sync(0xffffffffu, b[0], 1);
            if (lane == 31) {
                a4 = load1(ra, gc + 4, p.W);
                b4 = load1(rb, gc + 4, p.W);
            }
            a[4] = a4;
            b[4] = b4;
        } else {
#pragma unroll
            for (int k = 0; k < 5; ++k) a[k] = b[k] = 0.f;
        }
        float s[5], d[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            s[k] = a[k] + b[k];
            d[k] = b[k] - a[k];
        }
        if (r > 0) {
            const int i = gy - 1;            // cube row
            const float y = (float)i + p.yoff[0];
            float cs[5], vd[5], td[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                cs[k] = s[k] + ps[k];        // column sums over 2 rows x 2 frames
                vd[k] = s[k] - ps[k];        // row differences summed over frames
                td[k] = d[k] + pd[k];        // time differences summed over rows
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float ex = cs[k + 1] - cs[k];
                float ey = vd[k] + vd[k + 1];
                float et = td[k] + td[k + 1];
                if (EDGE) {
                    const bool ok = (i < p.H - 1) && (gc + k < p.W - 1);
                    ex = ok ? ex : 0.f;
                    ey = ok ? ey : 0.f;
                    et = ok ? et : 0.f;
                }
                accum(acc, ex, ey, et, x0 + (float)k, y);
            }
        }
        if (pyr && r < 8) {
            if ((r & 1) == 0) {
                ha[0] = a[0] + a[1]; ha[1] = a[2] + a[3];
                hb[0] = b[0] + b[1]; hb[1] = b[2] + b[3];
            } else {
                const int r1 = 4 * warp + (r >> 1);
                float2 va = make_float2(ha[0] + (a[0] + a[1]), ha[1] + (a[2] + a[3]));
                float2 vb = make_float2(hb[0] + (b[0] + b[1]), hb[1] + (b[2] + b[3]));
                *reinterpret_cast<float2 *>(L1 + r1 * C1S + 2 * lane) = va;
                *reinterpret_cast<float2 *>(L1 + R1S * C1S + r1 * C1S + 2 * lane) = vb;
            }
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            ps[k] = s[k];
            pd[k] = d[k];
        }
    }
}

template <typename T0>
__global__ void __launch_bounds__(NT)
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
    const int64_t pitch_e = p.pitch / (int64_t)sizeof(T0);

    // shared layout: red[NSUM*NT] | level l = 1..L-1: [2 frames][R_l][S_l]
    // (R_l x C_l pixels per frame, row stride S_l = C_l rounded up to even so that
    // float2 stores stay 8-byte aligned)
    float *red = sm;
    float *lev[FT_MAX_LEVELS];
    int Rl[FT_MAX_LEVELS], Cl[FT_MAX_LEVELS], Sl[FT_MAX_LEVELS];
    {
        float *ptr = red + NSUM * NT;
        for (int l = 1; l < p.levels; ++l) {
            Rl[l] = (TR + p.HB) >> l;
            Cl[l] = (TC + p.HB) >> l;
            Sl[l] = (Cl[l] + 1) & ~1;
            lev[l] = ptr;
            ptr += 2 * Rl[l] * Sl[l];
        }
    }
    float *partial = p.partials + ((int64_t)pair * p.levels * p.ntiles + tile) * NSUM;
    const int64_t lstride = (int64_t)p.ntiles * NSUM;   // next level, same pair and tile

    float acc[NSUM];
#pragma unroll
    for (int s = 0; s < NSUM; ++s) acc[s] = 0.f;

    // ---- level 0 (registers) and level-1 interior (shared) ----
    const bool edge = (R0 + TR + 1 > p.H - 1) || (C0 + TC + 1 > p.W - 1);
    float *L1 = p.levels > 1 ? lev[1] : nullptr;
    const int C1S = p.levels > 1 ? Sl[1] : 0, R1S = p.levels > 1 ? Rl[1] : 0;
    if (edge) level0_rows<T0, true>(p, fa, fb, R0, C0, L1, C1S, R1S, acc);
    else level0_rows<T0, false>(p, fa, fb, R0, C0, L1, C1S, R1S, acc);

    // ---- level-1 halo: rows [TR/2, R1) all columns; columns [TC/2, C1) rows [0, TR/2) ----
    if (p.levels > 1) {
        const int hr = Rl[1] - TR / 2, hc = Cl[1] - TC / 2;
        const int n_bottom = hr * Cl[1];
        const int n_right = (TR / 2) * hc;
        for (int e = threadIdx.x; e < 2 * (n_bottom + n_right); e += NT) {
            const int f = e >= (n_bottom + n_right);
            const int q = e - f * (n_bottom + n_right);
            int r1, c1;
            if (q < n_bottom) { r1 = TR / 2 + q / Cl[1]; c1 = q % Cl[1]; }
            else { const int q2 = q - n_bottom; r1 = q2 / hc; c1 = TC / 2 + q2 % hc; }
            const T0 *fr = f ? fb : fa;
            const int gy = R0 + 2 * r1, gx = C0 + 2 * c1;
            float v = 0.f;
            if (gy + 1 < p.H && gx + 1 < p.W) {
                const T0 *row0 = fr + (int64_t)gy * pitch_e;
                const T0 *row1 = row0 + pitch_e;
                v = ((float)row0[gx] + (float)row0[gx + 1]) + ((float)row1[gx] + (float)row1[gx + 1]);
            }
            L1[f * Rl[1] * Sl[1] + r1 * Sl[1] + c1] = v;
        }
    }

    block_reduce(acc, red, partial);          // level 0 (also orders the L1 writes)

    // ---- levels 2..L-1: 2x2 sums in shared memory ----
    for (int l = 2; l < p.levels; ++l) {
        const float *src = lev[l - 1];
        float *dst = lev[l];
        const int R = Rl[l], C = Cl[l], S = Sl[l], Ss = Sl[l - 1], Rs = Rl[l - 1];
        for (int e = threadIdx.x; e < 2 * R * C; e += NT) {
            const int f = e / (R * C), q = e - f * R * C;
            const int r = q / C, c = q - r * C;
            const float *s0 = src + f * Rs * Ss + (2 * r) * Ss + 2 * c;
            dst[f * R * S + r * S + c] = (s0[0] + s0[1]) + (s0[Ss] + s0[Ss + 1]);
        }
        __syncthreads();
    }

    // ---- cubes of levels 1..L-1 from shared memory ----
    for (int l = 1; l < p.levels; ++l) {
#pragma unroll
        for (int s = 0; s < NSUM; ++s) acc[s] = 0.f;
        const float *La = lev[l];
        const float *Lb = lev[l] + Rl[l] * Sl[l];
        const int C = Sl[l];
        const int nr = TR >> l, nc = TC >> l;
        const int Hl = p.H >> l, Wl = p.W >> l;
        const int i0 = R0 >> l, j0 = C0 >> l;
        for (int e = threadIdx.x; e < nr * nc; e += NT) {
            const int i = e / nc, j = e - i * nc;
            const int gi = i0 + i, gj = j0 + j;
            if (gi >= Hl - 1 || gj >= Wl - 1) continue;
            const float *pa = La + i * C + j;
            const float *pb = Lb + i * C + j;
            const float a00 = pa[0], a01 = pa[1], a10 = pa[C], a11 = pa[C + 1];
            const float b00 = pb[0], b01 = pb[1], b10 = pb[C], b11 = pb[C + 1];
            const float ex = ((a01 - a00) + (a11 - a10)) + ((b01 - b00) + (b11 - b10));
            const float ey = ((a10 - a00) + (a11 - a01)) + ((b10 - b00) + (b11 - b01));
            const float et = ((b00 - a00) + (b01 - a01)) + ((b10 - a10) + (b11 - a11));
            accum(acc, ex, ey, et, (float)gj + p.xoff[l], (float)gi + p.yoff[l]);
        }
        block_reduce(acc, red, partial + l * lstride);
    }
}

// ---------------------------------------------------------------------------
// stage 2: FP64 merge of the tile partials + solve
// ---------------------------------------------------------------------------

struct SolveParams {
    const float *partials;
    int ntiles, levels, npairs, mode;
    double inv_scale[FT_MAX_LEVELS];  // 1 / (16 * 16^l): level-l sums -> mean-image units
    int64_t ncubes[FT_MAX_LEVELS];
    ttc_level_result *out;
};

__device__ void solve_one(const double s[NSUM], int mode, int level, ttc_level_result *r)
{
    double th[3] = {0.0, 0.0, 0.0};
    int flags = 0;
    if (mode == FT_MODE_TTC) {
        if (!(s[5] > 0.0)) flags |= FT_FLAG_SINGULAR;
        else th[2] = -s[8] / s[5];
    } else {
        // M [A B C]^T = -[s6 s7 s8]^T with M = [[s0 s1 s3] [s1 s2 s4] [s3 s4 s5]],
        // scaled to unit diagonal, inverted by its adjugate (Sec. V-A).
        const double m[3][3] = {{s[0], s[1], s[3]}, {s[1], s[2], s[4]}, {s[3], s[4], s[5]}};
        double dsc[3];
        for (int i = 0; i < 3; ++i) {
            if (!(m[i][i] > 0.0)) flags |= FT_FLAG_SINGULAR;
            dsc[i] = m[i][i] > 0.0 ? rsqrt(m[i][i]) : 0.0;
        }
        if (!flags) {
            double u[3][3];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) u[i][j] = dsc[i] * m[i][j] * dsc[j];
            const double rhs[3] = {-s[6] * dsc[0], -s[7] * dsc[1], -s[8] * dsc[2]};
            const double c00 = u[1][1] * u[2][2] - u[1][2] * u[2][1];
            const double c01 = u[0][2] * u[2][1] - u[0][1] * u[2][2];
            const double c02 = u[0][1] * u[1][2] - u[0][2] * u[1][1];
            const double c10 = u[1][2] * u[2][0] - u[1][0] * u[2][2];
            const double c11 = u[0][0] * u[2][2] - u[0][2] * u[2][0];
            const double c12 = u[0][2] * u[1][0] - u[0][0] * u[1][2];
            const double c20 = u[1][0] * u[2][1] - u[1][1] * u[2][0];
            const double c21 = u[0][1] * u[2][0] - u[0][0] * u[2][1];
            const double c22 = u[0][0] * u[1][1] - u[0][1] * u[1][0];
            const double det = u[0][0] * c00 + u[0][1] * c10 + u[0][2] * c20;
            if (!(det > 1e-12)) {
                flags |= FT_FLAG_SINGULAR;
            } else {
                th[0] = dsc[0] * ((c00 * rhs[0] + c01 * rhs[1] + c02 * rhs[2]) / det);
                th[1] = dsc[1] * ((c10 * rhs[0] + c11 * rhs[1] + c12 * rhs[2]) / det);
                th[2] = dsc[2] * ((c20 * rhs[0] + c21 * rhs[1] + c22 * rhs[2]) / det);
            }
        }
    }
    r->level = level;
    r->flags = flags;
    const double qnan = __longlong_as_double(0x7ff8000000000000LL);
    if (flags & FT_FLAG_SINGULAR) {
        r->A = r->B = r->C = r->ttc = r->x0 = r->y0 = r->resid = qnan;
        return;
    }
    const double A = th[0], B = th[1], C = th[2];
    r->A = A;
    r->B = B;
    r->C = C;
    const double scale = (double)(1 << level);
    if (C == 0.0) {
        r->flags |= FT_FLAG_C_ZERO;
        r->ttc = __longlong_as_double(0x7ff0000000000000LL);
        r->x0 = r->y0 = qnan;
    } else {
        r->ttc = 1.0 / C;
        r->x0 = -A / C * scale;
        r->y0 = -B / C * scale;
        if (C < 0.0) r->flags |= FT_FLAG_RECEDING;
    }
    // sum (A Ex + B Ey + C G + Et)^2 = th' M th + 2 th' [s6 s7 s8] + s9
    const double m0 = s[0] * A + s[1] * B + s[3] * C;
    const double m1 = s[1] * A + s[2] * B + s[4] * C;
    const double m2 = s[3] * A + s[4] * B + s[5] * C;
    const double res = (A * m0 + B * m1 + C * m2) + 2.0 * (A * s[6] + B * s[7] + C * s[8]) + s[9];
    r->resid = s[9] > 0.0 ? res / s[9] : 0.0;
}

__global__ void __launch_bounds__(32)
ttc_solve_kernel(const SolveParams p)
{
    const int item = blockIdx.x;                 // pair * levels + level
    const int pair = item / p.levels, l = item - pair * p.levels;
    const int lane = threadIdx.x;
    const float *src = p.partials + ((int64_t)pair * p.levels + l) * p.ntiles * NSUM;
    double acc[NSUM];
#pragma unroll
    for (int s = 0; s < NSUM; ++s) acc[s] = 0.0;
    for (int t = lane; t < p.ntiles; t += 32)
#pragma unroll
        for (int s = 0; s < NSUM; ++s) acc[s] += (double)src[t * NSUM + s];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1)
#pragma unroll
        for (int s = 0; s < NSUM; ++s) acc[s] += __shfl_xor_sync(0xffffffffu, acc[s], o);
    if (lane == 0) {
        ttc_level_result r;
        for (int s = 0; s < NSUM; ++s) r.sums[s] = acc[s] * p.inv_scale[l];
        r.n = p.ncubes[l];
        solve_one(r.sums, p.mode, l, &r);
        p.out[item] = r;
    }
}

// ---------------------------------------------------------------------------
// materialised level-0 derivatives (debug / inspection surface)
// ---------------------------------------------------------------------------

template <typename T0>
__global__ void __launch_bounds__(256)
ttc_derivatives_kernel(const T0 *fa, const T0 *fb, int H, int W, int64_t pitch_e, float xoff,
                       float yoff, float *Ex, float *Ey, float *Et, float *G)
{
    const int j = blockIdx.x * 32 + (threadIdx.x & 31);
    const int i = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (i >= H - 1 || j >= W - 1) return;
    const T0 *a0 = fa + (int64_t)i * pitch_e + j, *a1 = a0 + pitch_e;
    const T0 *b0 = fb + (int64_t)i * pitch_e + j, *b1 = b0 + pitch_e;
    const float a00 = (float)a0[0], a01 = (float)a0[1], a10 = (float)a1[0], a11 = (float)a1[1];
    const float b00 = (float)b0[0], b01 = (float)b0[1], b10 = (float)b1[0], b11 = (float)b1[1];
    const float ex = 0.25f * (((a01 - a00) + (a11 - a10)) + ((b01 - b00) + (b11 - b10)));
    const float ey = 0.25f * (((a10 - a00) + (a11 - a01)) + ((b10 - b00) + (b11 - b01)));
    const float et = 0.25f * (((b00 - a00) + (b01 - a01)) + ((b10 - a10) + (b11 - a11)));
    const int64_t o = (int64_t)i * (W - 1) + j;
    Ex[o] = ex;
    Ey[o] = ey;
    Et[o] = et;
    if (G) G[o] = fmaf((float)j + xoff, ex, ((float)i + yoff) * ey);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

int elem_size(int dtype) { return dtype == FT_U8 ? 1 : dtype == FT_F32 ? 4 : 0; }

ft_status check_frames(int dtype, int H, int W, int64_t pitch)
{
    const int es = elem_size(dtype);
    if (es == 0) return FT_ERR_INVALID_ARG;
    if (H < 2 || W < 2) return FT_ERR_SHAPE;
    if (pitch < (int64_t)W * es || pitch % es != 0) return FT_ERR_SHAPE;
    return FT_OK;
}

ft_status check_levels(int H, int W, int levels)
{
    if (levels < 1) return FT_ERR_INVALID_ARG;
    if (levels > FT_MAX_LEVELS) return FT_ERR_UNSUPPORTED;
    for (int l = 0; l < levels; ++l)
        if ((H >> l) < 2 || (W >> l) < 2) return FT_ERR_SHAPE;
    return FT_OK;
}

void tiling(int H, int W, int &tiles_x, int &tiles_y)
{
    tiles_y = (int)ft::ceil_div(H - 1, TR);
    tiles_x = (int)ft::ceil_div(W - 1, TC);
}

size_t tile_smem_bytes(int levels)
{
    const int HB = levels > 1 ? 1 << (levels - 1) : 0;
    size_t floats = (size_t)NSUM * NT;
    for (int l = 1; l < levels; ++l) floats += 2 * (size_t)((TR + HB) >> l) * ((((TC + HB) >> l) + 1) & ~1);
    return floats * sizeof(float);
}

}  // namespace

struct ttc_ctx {
    int max_H, max_W, max_levels, max_pairs;
    int max_tiles;
    float *partials;
    size_t partial_bytes;
    // geometry of the last ttc_partial_sums call
    int H, W, levels, npairs, ntiles;
    bool ready;
};

extern "C" ft_status ttc_ctx_create(ttc_ctx **ctx, int max_H, int max_W, int max_levels, int max_pairs)
{
    if (!ctx) return FT_ERR_INVALID_ARG;
    *ctx = nullptr;
    if (max_pairs < 1 || max_levels < 1) return FT_ERR_INVALID_ARG;
    if (max_H < 2 || max_W < 2) return FT_ERR_SHAPE;
    if (max_levels > FT_MAX_LEVELS) return FT_ERR_UNSUPPORTED;
    int tx, ty;
    tiling(max_H, max_W, tx, ty);
    const size_t bytes = (size_t)max_pairs * max_levels * (size_t)tx * ty * NSUM * sizeof(float);
    float *buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, bytes);
    if (e != cudaSuccess) {
        ft::set_cuda_error(e);
        return FT_ERR_CUDA;
    }
    ttc_ctx *c = new (std::nothrow) ttc_ctx();
    if (!c) {
        cudaFree(buf);
        return FT_ERR_CUDA;
    }
    c->max_H = max_H;
    c->max_W = max_W;
    c->max_levels = max_levels;
    c->max_pairs = max_pairs;
    c->max_tiles = tx * ty;
    c->partials = buf;
    c->partial_bytes = bytes;
    c->ready = false;
    *ctx = c;
    return FT_OK;
}

extern "C" void ttc_ctx_destroy(ttc_ctx *ctx)
{
    if (!ctx) return;
    cudaFree(ctx->partials);
    delete ctx;
}

extern "C" size_t ttc_ctx_workspace_bytes(const ttc_ctx *ctx) { return ctx ? ctx->partial_bytes : 0; }

namespace {

ft_status launch_partials(ttc_ctx *ctx, const void *prev, const void *cur, int64_t pair_stride,
                          int npairs, int dtype, int H, int W, int64_t pitch, int levels,
                          cudaStream_t s)
{
    if (!ctx || !prev || !cur) return FT_ERR_INVALID_ARG;
    if (npairs < 1) return FT_ERR_SHAPE;
    ft_status st = check_frames(dtype, H, W, pitch);
    if (st != FT_OK) return st;
    if ((st = check_levels(H, W, levels)) != FT_OK) return st;
    int tx, ty;
    tiling(H, W, tx, ty);
    const int ntiles = tx * ty;
    if ((size_t)npairs * levels * ntiles > (size_t)ctx->max_pairs * ctx->max_levels * ctx->max_tiles)
        return FT_ERR_WORKSPACE;
    if ((int64_t)npairs * ntiles > 0x7fffffffLL) return FT_ERR_UNSUPPORTED;

    TileParams p{};
    p.prev = static_cast<const unsigned char *>(prev);
    p.cur = static_cast<const unsigned char *>(cur);
    p.pair_stride = pair_stride;
    p.pitch = pitch;
    p.H = H;
    p.W = W;
    p.levels = levels;
    p.HB = levels > 1 ? 1 << (levels - 1) : 0;
    p.tiles_x = tx;
    p.ntiles = ntiles;
    const uintptr_t al = dtype == FT_U8 ? 3 : 15;
    p.vec = ((reinterpret_cast<uintptr_t>(prev) & al) == 0 && (reinterpret_cast<uintptr_t>(cur) & al) == 0 &&
             (pitch & (int64_t)al) == 0 && (pair_stride & (int64_t)al) == 0) ? 1 : 0;
    for (int l = 0; l < levels; ++l) {
        // cube centre x = j + 1/2 - cx_l, cx_l = (W - 2^l) / 2^(l+1): the level-0 image
        // centre (W-1)/2 expressed in level-l pixel indices
        const double pl = (double)(1 << l);
        p.xoff[l] = (float)(0.5 - ((double)W - pl) / (2.0 * pl));
        p.yoff[l] = (float)(0.5 - ((double)H - pl) / (2.0 * pl));
    }
    p.partials = ctx->partials;
    const size_t smem = tile_smem_bytes(levels);
    const unsigned blocks = (unsigned)((int64_t)npairs * ntiles);
    cudaError_t e = cudaSuccess;
    if (dtype == FT_U8) {
        if (smem > 48 * 1024)
            e = cudaFuncSetAttribute(ttc_tile_kernel<unsigned char>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) ttc_tile_kernel<unsigned char><<<blocks, NT, smem, s>>>(p);
    } else {
        if (smem > 48 * 1024)
            e = cudaFuncSetAttribute(ttc_tile_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) ttc_tile_kernel<float><<<blocks, NT, smem, s>>>(p);
    }
    if (e != cudaSuccess) {
        ft::set_cuda_error(e);
        return FT_ERR_CUDA;
    }
    st = ft::check_launch();
    if (st != FT_OK) return st;
    ctx->H = H;
    ctx->W = W;
    ctx->levels = levels;
    ctx->npairs = npairs;
    ctx->ntiles = ntiles;
    ctx->ready = true;
    return FT_OK;
}

ft_status launch_solve(ttc_ctx *ctx, int mode, ttc_level_result *out, cudaStream_t s)
{
    if (!ctx || !out) return FT_ERR_INVALID_ARG;
    if (mode != FT_MODE_TTC && mode != FT_MODE_FOE) return FT_ERR_INVALID_ARG;
    if (!ctx->ready) return FT_ERR_INVALID_ARG;
    SolveParams sp{};
    sp.partials = ctx->partials;
    sp.ntiles = ctx->ntiles;
    sp.levels = ctx->levels;
    sp.npairs = ctx->npairs;
    sp.mode = mode;
    for (int l = 0; l < ctx->levels; ++l) {
        sp.inv_scale[l] = std::ldexp(1.0, -4 - 4 * l);
        sp.ncubes[l] = (int64_t)((ctx->H >> l) - 1) * (int64_t)((ctx->W >> l) - 1);
    }
    sp.out = out;
    ttc_solve_kernel<<<(unsigned)(ctx->npairs * ctx->levels), 32, 0, s>>>(sp);
    return ft::check_launch();
}

}  // namespace

extern "C" ft_status ttc_partial_sums(ttc_ctx *ctx, const void *frames, int64_t frame_stride_bytes, int T,
                                      int dtype, int H, int W, int64_t pitch_bytes, int levels, void *stream)
{
    if (!ctx || !frames) return FT_ERR_INVALID_ARG;
    if (T < 2) return FT_ERR_SHAPE;
    if (frame_stride_bytes < 0) return FT_ERR_INVALID_ARG;
    const unsigned char *f0 = static_cast<const unsigned char *>(frames);
    return launch_partials(ctx, f0, f0 + frame_stride_bytes, frame_stride_bytes, T - 1, dtype, H, W,
                           pitch_bytes, levels, ft::as_stream(stream));
}

extern "C" ft_status ttc_reduce_solve(ttc_ctx *ctx, int mode, ttc_level_result *out, void *stream)
{
    return launch_solve(ctx, mode, out, ft::as_stream(stream));
}

extern "C" ft_status ttc_solve(ttc_ctx *ctx, const void *prev, const void *cur, int dtype, int H, int W,
                               int64_t pitch_bytes, int levels, int mode, ttc_level_result *out,
                               void *stream)
{
    if (!ctx || !prev || !cur || !out) return FT_ERR_INVALID_ARG;
    if (mode != FT_MODE_TTC && mode != FT_MODE_FOE) return FT_ERR_INVALID_ARG;
    ft_status st = launch_partials(ctx, prev, cur, 0, 1, dtype, H, W, pitch_bytes, levels,
                                   ft::as_stream(stream));
    if (st != FT_OK) return st;
    return launch_solve(ctx, mode, out, ft::as_stream(stream));
}

extern "C" ft_status ttc_solve_sequence(ttc_ctx *ctx, const void *frames, int64_t frame_stride_bytes, int T,
                                        int dtype, int H, int W, int64_t pitch_bytes, int levels, int mode,
                                        ttc_level_result *out, void *stream)
{
    if (!ctx || !frames || !out) return FT_ERR_INVALID_ARG;
    if (mode != FT_MODE_TTC && mode != FT_MODE_FOE) return FT_ERR_INVALID_ARG;
    ft_status st = ttc_partial_sums(ctx, frames, frame_stride_bytes, T, dtype, H, W, pitch_bytes, levels, stream);
    if (st != FT_OK) return st;
    return launch_solve(ctx, mode, out, ft::as_stream(stream));
}

extern "C" ft_status ttc_derivatives(const void *prev, const void *cur, int dtype, int H, int W,
                                     int64_t pitch_bytes, float *Ex, float *Ey, float *Et, float *G,
                                     void *stream)
{
    if (!prev || !cur || !Ex || !Ey || !Et) return FT_ERR_INVALID_ARG;
    ft_status st = check_frames(dtype, H, W, pitch_bytes);
    if (st != FT_OK) return st;
    const dim3 grid((unsigned)ft::ceil_div(W - 1, 32), (unsigned)ft::ceil_div(H - 1, 8));
    if (grid.y > 65535) return FT_ERR_UNSUPPORTED;
    const float xoff = (float)(0.5 - ((double)W - 1.0) / 2.0);
    const float yoff = (float)(0.5 - ((double)H - 1.0) / 2.0);
    cudaStream_t s = ft::as_stream(stream);
    if (dtype == FT_U8)
        ttc_derivatives_kernel<unsigned char><<<grid, 256, 0, s>>>(
            static_cast<const unsigned char *>(prev), static_cast<const unsigned char *>(cur), H, W,
            pitch_bytes, xoff, yoff, Ex, Ey, Et, G);
    else
        ttc_derivatives_kernel<float><<<grid, 256, 0, s>>>(
            static_cast<const float *>(prev), static_cast<const float *>(cur), H, W, pitch_bytes / 4, xoff,
            yoff, Ex, Ey, Et, G);
    return ft::check_launch();
}

extern "C" int ttc_select_level(const ttc_level_result *r, int levels, int rule)
{
    if (!r || levels < 1 || (rule != 0 && rule != 1)) return -2;
    auto usable = [](const ttc_level_result &x) {
        return !(x.flags & (FT_FLAG_SINGULAR | FT_FLAG_C_ZERO)) && x.ttc > 0.0;
    };
    int l = -1;
    for (int i = 0; i < levels; ++i)
        if (usable(r[i])) { l = i; break; }
    if (l < 0) return -1;
    while (l + 1 < levels && usable(r[l + 1])) {
        const double kc = rule == 0 ? r[l].ttc : r[l].resid;
        const double kn = rule == 0 ? r[l + 1].ttc : r[l + 1].resid;
        if (!(kn < kc)) break;
        ++l;
    }
    return l;
}
