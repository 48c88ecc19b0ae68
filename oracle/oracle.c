/*
 * FP64 CPU oracle for FastConv and the multi-scale time-to-contact (TTC) pipeline.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this code.  It shares nothing with the CUDA path:
 * no headers, no helpers, no tables.  Every function is a plain, slow,
 * loop-by-loop statement of the definition it cites, in double precision.
 *
 * Paper: "Accelerated Convolutions for Efficient Multi-Scale Time to Contact
 * Computation in Julia" (Amini, Horn, Edelman).
 *
 * Readings of the paper that this file fixes:
 *  - Eq. conv2 is read as the full linear convolution (kernel flipped, output
 *    extent N + K - 1 per dimension), the operation FastConv replaces in Sec. IV-D.
 *  - The derivative stencils are the 2x2x2 time-averaged first differences whose
 *    single-frame slices are the 2x2 mask of Sec. II (1/2 [[-1, 1], [-1, 1]]).
 *  - x and y are measured from the principal point, x to the right (column),
 *    y downward (row), in pixels of the level being processed.
 *  - Down-sampling (Sec. V-B) is a 2x2 block mean with floor cropping.
 *  - C > 0 means approaching: TTC = 1/C frames (Eq. final_TTC).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_MAX_ND 8

enum { OR_FLAG_SINGULAR = 1, OR_FLAG_C_ZERO = 2, OR_FLAG_RECEDING = 4 };

/* One result per pyramid level (mirrored by a numpy dtype in oracle/__init__.py). */
typedef struct {
    double sums[10];     /* see oracle_sums for the order */
    double abssums[10];  /* error-bound scale of each sum: sum of |term|, with G replaced
                            by |x Ex| + |y Ey| in the four G terms (see oracle_sums) */
    double A, B, C;      /* Eq. final_TTC parameters, level-l pixel units */
    double ttc;          /* 1/C, frames */
    double x0, y0;       /* FOE, level-0 pixels from the principal point */
    double resid;        /* relative residual of the least-squares fit */
    int64_t n;           /* number of 2x2x2 cubes summed */
    int32_t level;
    int32_t flags;
} oracle_result;

/* ------------------------------------------------------------------------ */
/* Sec. III/IV: convolution                                                  */
/* ------------------------------------------------------------------------ */

/* Output extent of the full convolution: N_d + K_d - 1.  Returns 0 on success. */
int oracle_conv_out_dims(int nd, const int64_t *dims, const int64_t *kdims, int64_t *out_dims)
{
    if (nd < 1 || nd > ORACLE_MAX_ND) return -1;
    for (int d = 0; d < nd; ++d) {
        if (dims[d] < 1 || kdims[d] < 1) return -1;
        out_dims[d] = dims[d] + kdims[d] - 1;
    }
    return 0;
}

/* Row-major multi-index of a linear index (last dimension fastest). */
static void unravel(int64_t lin, const int64_t *dims, int nd, int64_t *idx)
{
    for (int d = nd - 1; d >= 0; --d) {
        idx[d] = lin % dims[d];
        lin /= dims[d];
    }
}

/*
 * Eq. conv2, full linear convolution:  out[p] = sum_r k[r] * E[p - r], summed over
 * every kernel index r for which p - r is inside the input.  This is the same sum
 * as sum_q E[q] k[p - q] over the input indices q.  Evaluated at the given output
 * linear indices only.  out_abs (nullable) receives sum_r |k[r] E[p - r]|.
 */
int oracle_fastconv_points(const double *E, const int64_t *dims, int nd,
                           const double *k, const int64_t *kdims,
                           const int64_t *points, int64_t npoints,
                           double *out, double *out_abs)
{
    int64_t odims[ORACLE_MAX_ND];
    if (oracle_conv_out_dims(nd, dims, kdims, odims) != 0) return -1;
    int64_t ksize = 1;
    for (int d = 0; d < nd; ++d) ksize *= kdims[d];
    int64_t p[ORACLE_MAX_ND], r[ORACLE_MAX_ND];
    for (int64_t s = 0; s < npoints; ++s) {
        unravel(points[s], odims, nd, p);
        double acc = 0.0, acc_abs = 0.0;
        for (int64_t rl = 0; rl < ksize; ++rl) {
            unravel(rl, kdims, nd, r);
            int64_t q = 0;
            int inside = 1;
            for (int d = 0; d < nd; ++d) {
                int64_t qd = p[d] - r[d];
                if (qd < 0 || qd >= dims[d]) { inside = 0; break; }
                q = q * dims[d] + qd;
            }
            if (!inside) continue;
            double term = E[q] * k[rl];
            acc += term;
            acc_abs += fabs(term);
        }
        out[s] = acc;
        if (out_abs) out_abs[s] = acc_abs;
    }
    return 0;
}

/* Full convolution at every output index. */
int oracle_fastconv_nd(const double *E, const int64_t *dims, int nd,
                       const double *k, const int64_t *kdims,
                       double *out, double *out_abs)
{
    int64_t odims[ORACLE_MAX_ND];
    if (oracle_conv_out_dims(nd, dims, kdims, odims) != 0) return -1;
    int64_t total = 1;
    for (int d = 0; d < nd; ++d) total *= odims[d];
    int64_t *pts = (int64_t *)malloc(sizeof(int64_t) * (size_t)(total > 0 ? total : 1));
    if (!pts) return -2;
    for (int64_t i = 0; i < total; ++i) pts[i] = i;
    int rc = oracle_fastconv_points(E, dims, nd, k, kdims, pts, total, out, out_abs);
    free(pts);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Sec. V-B: down-sampling by 2x2 block averaging                            */
/* ------------------------------------------------------------------------ */

/* (H/2) x (W/2) image of 2x2 block means; an odd last row or column is dropped. */
void oracle_downsample(const double *in, int H, int W, double *out)
{
    int h = H / 2, w = W / 2;
    for (int i = 0; i < h; ++i)
        for (int j = 0; j < w; ++j) {
            double s = in[(int64_t)(2 * i) * W + 2 * j] + in[(int64_t)(2 * i) * W + 2 * j + 1]
                     + in[(int64_t)(2 * i + 1) * W + 2 * j] + in[(int64_t)(2 * i + 1) * W + 2 * j + 1];
            out[(int64_t)i * w + j] = s / 4.0;
        }
}

/* ------------------------------------------------------------------------ */
/* Sec. II, Eq. Emag and Eq. Eangle: gradient magnitude and direction         */
/* ------------------------------------------------------------------------ */

/* Single image E (H x W): at every 2x2 block centre, Ex and Ey from the Sec. II mask
 * 1/2 [[-1, 1], [-1, 1]] (and its transpose), then |E| = sqrt(Ex^2 + Ey^2) and
 * theta = four-quadrant inverse tangent of (Ey, Ex), in [-pi, pi].  Outputs
 * (H-1) x (W-1); either may be NULL. */
void oracle_gradient(const double *E, int H, int W, double *mag, double *dir)
{
    int w = W - 1;
    for (int i = 0; i < H - 1; ++i)
        for (int j = 0; j < W - 1; ++j) {
            const double a = E[(int64_t)i * W + j], b = E[(int64_t)i * W + j + 1];
            const double c = E[(int64_t)(i + 1) * W + j], d = E[(int64_t)(i + 1) * W + j + 1];
            const double ex = 0.5 * ((b - a) + (d - c));
            const double ey = 0.5 * ((c - a) + (d - b));
            if (mag) mag[(int64_t)i * w + j] = sqrt(ex * ex + ey * ey);
            if (dir) dir[(int64_t)i * w + j] = atan2(ey, ex);
        }
}

/* ------------------------------------------------------------------------ */
/* Sec. II / V-A: 2x2x2 spatio-temporal derivative estimates                 */
/* ------------------------------------------------------------------------ */

/*
 * For the cube with corner (i, j) spanning rows i..i+1, columns j..j+1 and the two
 * frames E0 (time t) and E1 (time t+1):
 *   Ex = mean of the four first differences along x (column j -> j+1),
 *   Ey = mean of the four first differences along y (row i -> i+1),
 *   Et = mean of the four first differences along t (E0 -> E1).
 * Outputs are (H-1) x (W-1), located at the cube centre (i + 1/2, j + 1/2, t + 1/2).
 */
void oracle_derivatives(const double *E0, const double *E1, int H, int W,
                        double *Ex, double *Ey, double *Et)
{
    int w = W - 1;
    for (int i = 0; i < H - 1; ++i)
        for (int j = 0; j < W - 1; ++j) {
            const double *f[2] = { E0, E1 };
            double ex = 0.0, ey = 0.0, et = 0.0;
            for (int t = 0; t < 2; ++t)
                for (int a = 0; a < 2; ++a) {
                    /* x differences along rows i and i+1 */
                    ex += f[t][(int64_t)(i + a) * W + j + 1] - f[t][(int64_t)(i + a) * W + j];
                    /* y differences along columns j and j+1 */
                    ey += f[t][(int64_t)(i + 1) * W + j + a] - f[t][(int64_t)i * W + j + a];
                }
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b)
                    et += E1[(int64_t)(i + a) * W + j + b] - E0[(int64_t)(i + a) * W + j + b];
            Ex[(int64_t)i * w + j] = ex / 4.0;
            Ey[(int64_t)i * w + j] = ey / 4.0;
            Et[(int64_t)i * w + j] = et / 4.0;
        }
}

/* ------------------------------------------------------------------------ */
/* Sec. V-A: radial gradient G and the least-squares sums                    */
/* ------------------------------------------------------------------------ */

/* Neumaier-compensated running sum. */
typedef struct { double s, c; } csum;

static void csum_add(csum *a, double v)
{
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}

/*
 * G = x Ex + y Ey with x = j + 1/2 - cx, y = i + 1/2 - cy (cube centre relative to
 * the principal point (cx, cy) in pixel-index coordinates).  The ten sums over all
 * cubes, in this order:
 *   0 Ex^2   1 Ex Ey   2 Ey^2   3 G Ex   4 G Ey   5 G^2
 *   6 Ex Et  7 Ey Et   8 G Et   9 Et^2
 * 0..8 are the entries of the 3x3 normal equations; 9 feeds the fit residual.
 */
void oracle_sums(const double *Ex, const double *Ey, const double *Et, int h, int w,
                 double cx, double cy, double sums[10], double abssums[10])
{
    csum acc[10];
    double aacc[10];
    memset(acc, 0, sizeof(acc));
    memset(aacc, 0, sizeof(aacc));
    for (int i = 0; i < h; ++i)
        for (int j = 0; j < w; ++j) {
            int64_t o = (int64_t)i * w + j;
            double ex = Ex[o], ey = Ey[o], et = Et[o];
            double x = (double)j + 0.5 - cx;
            double y = (double)i + 0.5 - cy;
            double G = x * ex + y * ey;
            double term[10] = { ex * ex, ex * ey, ey * ey, G * ex, G * ey, G * G,
                                ex * et, ey * et, G * et, et * et };
            /* magnitudes the rounding error of a finite-precision evaluation scales
               with: G = x Ex + y Ey rounds relative to |x Ex| + |y Ey|, not to |G| */
            double Gm = fabs(x * ex) + fabs(y * ey);
            double mag[10] = { fabs(ex * ex), fabs(ex * ey), ey * ey, Gm * fabs(ex), Gm * fabs(ey), Gm * Gm,
                               fabs(ex * et), fabs(ey * et), Gm * fabs(et), et * et };
            for (int s = 0; s < 10; ++s) {
                csum_add(&acc[s], term[s]);
                aacc[s] += mag[s];
            }
        }
    for (int s = 0; s < 10; ++s) {
        sums[s] = acc[s].s + acc[s].c;
        if (abssums) abssums[s] = aacc[s];
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. V-A: solve the normal equations; Eq. final_TTC                       */
/* ------------------------------------------------------------------------ */

/*
 * mode 0: motion along the optical axis only (A = B = 0): the third normal
 *         equation gives C = -sum(G Et) / sum(G^2).
 * mode 1: the 3x3 system  M [A B C]^T = -[sum Ex Et, sum Ey Et, sum G Et]^T  is
 *         solved with the inverse of M (adjugate / determinant), after scaling M
 *         to unit diagonal.  The system is declared singular when the determinant
 *         of the unit-diagonal matrix is <= 1e-12.
 * Then TTC = 1/C, x0 = -A/C, y0 = -B/C; the FOE is reported in level-0 pixels
 * (multiplied by 2^level).
 */
void oracle_solve(const double s[10], int mode, int level, oracle_result *r)
{
    double nanv = NAN;
    double th[3] = { 0.0, 0.0, 0.0 };
    int flags = 0;
    if (mode == 0) {
        if (!(s[5] > 0.0)) flags |= OR_FLAG_SINGULAR;
        else th[2] = -s[8] / s[5];
    } else {
        double M[3][3] = { { s[0], s[1], s[3] }, { s[1], s[2], s[4] }, { s[3], s[4], s[5] } };
        double b[3] = { -s[6], -s[7], -s[8] };
        double D[3];
        for (int i = 0; i < 3; ++i) {
            if (!(M[i][i] > 0.0)) flags |= OR_FLAG_SINGULAR;
            else D[i] = 1.0 / sqrt(M[i][i]);
        }
        if (!flags) {
            double S[3][3], bs[3];
            for (int i = 0; i < 3; ++i) {
                bs[i] = D[i] * b[i];
                for (int j = 0; j < 3; ++j) S[i][j] = D[i] * M[i][j] * D[j];
            }
            /* adjugate (cofactor transpose) of S */
            double adj[3][3];
            adj[0][0] = S[1][1] * S[2][2] - S[1][2] * S[2][1];
            adj[0][1] = S[0][2] * S[2][1] - S[0][1] * S[2][2];
            adj[0][2] = S[0][1] * S[1][2] - S[0][2] * S[1][1];
            adj[1][0] = S[1][2] * S[2][0] - S[1][0] * S[2][2];
            adj[1][1] = S[0][0] * S[2][2] - S[0][2] * S[2][0];
            adj[1][2] = S[0][2] * S[1][0] - S[0][0] * S[1][2];
            adj[2][0] = S[1][0] * S[2][1] - S[1][1] * S[2][0];
            adj[2][1] = S[0][1] * S[2][0] - S[0][0] * S[2][1];
            adj[2][2] = S[0][0] * S[1][1] - S[0][1] * S[1][0];
            double det = S[0][0] * adj[0][0] + S[0][1] * adj[1][0] + S[0][2] * adj[2][0];
            if (!(det > 1e-12)) {
                flags |= OR_FLAG_SINGULAR;
            } else {
                for (int i = 0; i < 3; ++i) {
                    double v = 0.0;
                    for (int j = 0; j < 3; ++j) v += adj[i][j] * bs[j];
                    th[i] = D[i] * (v / det);
                }
            }
        }
    }
    r->level = level;
    r->flags = flags;
    if (flags & OR_FLAG_SINGULAR) {
        r->A = r->B = r->C = r->ttc = r->x0 = r->y0 = r->resid = nanv;
        return;
    }
    double A = th[0], B = th[1], C = th[2];
    r->A = A; r->B = B; r->C = C;
    double scale = ldexp(1.0, level);
    if (C == 0.0) {
        r->flags |= OR_FLAG_C_ZERO;
        r->ttc = INFINITY;
        r->x0 = r->y0 = nanv;
    } else {
        r->ttc = 1.0 / C;
        r->x0 = -A / C * scale;
        r->y0 = -B / C * scale;
        if (C < 0.0) r->flags |= OR_FLAG_RECEDING;
    }
    /* sum (A Ex + B Ey + C G + Et)^2 = th' M th + 2 th' [s6 s7 s8] + s9 */
    double M[3][3] = { { s[0], s[1], s[3] }, { s[1], s[2], s[4] }, { s[3], s[4], s[5] } };
    double q = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) q += th[i] * M[i][j] * th[j];
    double res = q + 2.0 * (A * s[6] + B * s[7] + C * s[8]) + s[9];
    r->resid = s[9] > 0.0 ? res / s[9] : 0.0;
}

/* ------------------------------------------------------------------------ */
/* The whole per-pair chain                                                  */
/* ------------------------------------------------------------------------ */

/*
 * Per level l = 0..levels-1: the level-l images are the l-fold 2x2 block means of
 * the input frames; derivatives, G and the sums are taken over all cubes of level l
 * with the principal point at cx_l = (W - 2^l) / 2^(l+1), cy_l = (H - 2^l) / 2^(l+1)
 * (the centre of the level-0 image expressed in level-l pixel indices); then the
 * solve.  Returns 0, or -1 if some level would be smaller than 2x2.
 */
int oracle_ttc_pair(const double *E0, const double *E1, int H, int W, int levels, int mode,
                    oracle_result *res)
{
    if (levels < 1 || H < 2 || W < 2) return -1;
    for (int l = 0; l < levels; ++l)
        if ((H >> l) < 2 || (W >> l) < 2) return -1;
    size_t n0 = (size_t)H * (size_t)W;
    double *a = (double *)malloc(n0 * sizeof(double));
    double *b = (double *)malloc(n0 * sizeof(double));
    double *ta = (double *)malloc(n0 * sizeof(double));
    double *tb = (double *)malloc(n0 * sizeof(double));
    double *ex = (double *)malloc(n0 * sizeof(double));
    double *ey = (double *)malloc(n0 * sizeof(double));
    double *et = (double *)malloc(n0 * sizeof(double));
    if (!a || !b || !ta || !tb || !ex || !ey || !et) {
        free(a); free(b); free(ta); free(tb); free(ex); free(ey); free(et);
        return -2;
    }
    memcpy(a, E0, n0 * sizeof(double));
    memcpy(b, E1, n0 * sizeof(double));
    int h = H, w = W;
    for (int l = 0; l < levels; ++l) {
        if (l > 0) {
            oracle_downsample(a, h, w, ta);
            oracle_downsample(b, h, w, tb);
            h /= 2; w /= 2;
            double *t;
            t = a; a = ta; ta = t;
            t = b; b = tb; tb = t;
        }
        oracle_derivatives(a, b, h, w, ex, ey, et);
        double p = ldexp(1.0, l);
        double cx = ((double)W - p) / (2.0 * p);
        double cy = ((double)H - p) / (2.0 * p);
        oracle_result *r = &res[l];
        memset(r, 0, sizeof(*r));
        oracle_sums(ex, ey, et, h - 1, w - 1, cx, cy, r->sums, r->abssums);
        oracle_solve(r->sums, mode, l, r);
        r->n = (int64_t)(h - 1) * (int64_t)(w - 1);
    }
    free(a); free(b); free(ta); free(tb); free(ex); free(ey); free(et);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sec. V-B: multi-scale selection                                           */
/* ------------------------------------------------------------------------ */

/*
 * Start at the finest usable level and move to the next coarser level while the
 * estimate there is usable and smaller ("improved (ie. reduced)"):
 *   rule 0: the quantity compared is the TTC itself;
 *   rule 1: the quantity compared is the relative fit residual.
 * A level is usable when it is not singular, C != 0 and TTC > 0.
 * Returns the chosen level, or -1 when no level is usable.
 */
int oracle_select_level(const oracle_result *r, int levels, int rule)
{
    int l = -1;
    for (int i = 0; i < levels; ++i) {
        int ok = !(r[i].flags & (OR_FLAG_SINGULAR | OR_FLAG_C_ZERO)) && r[i].ttc > 0.0;
        if (ok) { l = i; break; }
    }
    if (l < 0) return -1;
    while (l + 1 < levels) {
        const oracle_result *nx = &r[l + 1];
        int ok = !(nx->flags & (OR_FLAG_SINGULAR | OR_FLAG_C_ZERO)) && nx->ttc > 0.0;
        if (!ok) break;
        double kc = rule == 0 ? r[l].ttc : r[l].resid;
        double kn = rule == 0 ? nx->ttc : nx->resid;
        if (!(kn < kc)) break;
        ++l;
    }
    return l;
}

/* Size of oracle_result, checked by the Python wrapper. */
int oracle_result_size(void) { return (int)sizeof(oracle_result); }
