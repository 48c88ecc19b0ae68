// Stage 2 of the TTC/FOE solve (Sec. V-A, Eq. final_TTC): the FP64 merge of a
// (pair, level)'s tile partials in a fixed order and the solve of the normal
// equations, shared by the merge kernels.
#pragma once

#include "common.cuh"
#include "ttc_pass.cuh"

namespace ttc_merge {

using ttc_pass::NSUM;

// partials and cube count of one (pair, level) of a batch
struct SolveDesc {
    int64_t poff;                     // floats into the partials
    int64_t ncubes;
    int ntiles, level;
    int shift;                        // the partials are 2^shift times the block-sum sums
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

// One warp: FP64 merge of ntiles FP32 tile partials in a fixed order (lane-strided, then
// a shuffle tree); every lane ends with the ten totals.
__device__ __forceinline__ void merge_sums(const float *src, int ntiles, double acc[NSUM])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int s = 0; s < NSUM; ++s) acc[s] = 0.0;
    for (int t = lane; t < ntiles; t += 32)
#pragma unroll
        for (int s = 0; s < NSUM; ++s) acc[s] += (double)src[t * NSUM + s];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1)
#pragma unroll
        for (int s = 0; s < NSUM; ++s) acc[s] += __shfl_xor_sync(0xffffffffu, acc[s], o);
}

// One thread: the merged sums scaled to level-l mean-image units, the solve, the status
// flags, the record.
__device__ __forceinline__ void solve_record(const double *acc, int l, double inv_scale, int64_t ncubes, int mode,
                                             const int *status, ttc_level_result *out)
{
    ttc_level_result r;
    for (int s = 0; s < NSUM; ++s) r.sums[s] = acc[s] * inv_scale;
    r.n = ncubes;
    solve_one(r.sums, mode, l, &r);
    // status word: bit 0 a wait gave up, bit 1 a checked build found an access out of bounds
    const int st = *status;
    if (st & 1) r.flags |= FT_FLAG_TIMEOUT;
    if (st & 2) r.flags |= FT_FLAG_BOUNDS;
    *out = r;
}

// Most (pair, level) items per CTA of the merge kernels: a warp merges each, then the
// lanes of the first warp solve them side by side (FP64 runs at a small fraction of the
// FP32 rate on this part, so a solve gets one lane, not a warp)
constexpr int MERGE_ITEMS = 16;

}  // namespace ttc_merge
