// Multi-scale time to contact / focus of expansion on sm_103a (Sec. V-A, V-B).
//
// Stage 1 (ttc_pass.cuh): one streaming pass per pyramid level, fusing the 2x2x2
// stencil, G, the ten products and the tile reduction with the 2x2 block sums of
// the next level; it leaves ten FP32 partial sums per (level, pair, tile).
// Stage 2 (ttc_solve_kernel, one warp per pair and level): FP64 merge of the tile
// partials in a fixed order, scaling to level-l mean-image units, and the FP64
// solve of the normal equations (Eq. final_TTC).
// Also here: the materialised level-0 derivatives, the context and the C ABI.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "ttc_pass.cuh"
#include "ttc_merge.cuh"
#include "ttc_tma.cuh"
#include "ttc_fused.cuh"

#include <cudaTypedefs.h>

namespace {

using ttc_pass::NSUM;
using ttc_merge::SolveDesc;
using ttc_merge::merge_sums;
using ttc_merge::solve_record;
using ttc_pass::TR;
using ttc_pass::TC;

// ---------------------------------------------------------------------------
// stage 2: FP64 merge of the tile partials + solve
// ---------------------------------------------------------------------------

struct SolveParams {
    const float *partials;
    int levels, npairs, mode;
    int ntiles[FT_MAX_LEVELS];        // tiles of level l
    int64_t poff[FT_MAX_LEVELS];      // level l partials start here: [pair][tile][NSUM]
    double inv_scale[FT_MAX_LEVELS];  // 1 / (16 * 16^l): level-l sums -> mean-image units
    int64_t ncubes[FT_MAX_LEVELS];
    const int *status;                // nonzero: a stage-1 wait gave up
    ttc_level_result *out;
    int skip;                         // pairs [0, skip) are not written
};

__global__ void __launch_bounds__(32 * ttc_merge::MERGE_ITEMS)
ttc_solve_kernel(const SolveParams p)
{
    __shared__ double ssum[ttc_merge::MERGE_ITEMS][NSUM];
    const int MI = blockDim.x >> 5;                           // items of this CTA
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int total = p.npairs * p.levels;
    const int item = blockIdx.x * MI + warp;                  // pair * levels + level
    if (item < total) {
        const int pair = item / p.levels, l = item - pair * p.levels;
        if (pair >= p.skip) {
            double acc[NSUM];
            merge_sums(p.partials + p.poff[l] + (int64_t)pair * p.ntiles[l] * NSUM, p.ntiles[l], acc);
            if (lane == 0)
                for (int s = 0; s < NSUM; ++s) ssum[warp][s] = acc[s];
        }
    }
    __syncthreads();
    const int it = blockIdx.x * MI + lane;
    if (warp == 0 && lane < MI && it < total) {
        const int pair = it / p.levels, l = it - pair * p.levels;
        if (pair >= p.skip) solve_record(ssum[lane], l, p.inv_scale[l], p.ncubes[l], p.mode, p.status, p.out + it);
    }
}

__global__ void __launch_bounds__(32 * ttc_merge::MERGE_ITEMS)
ttc_batch_solve_kernel(const float *partials, const SolveDesc *sd, int total, int mode, const int *status,
                       ttc_level_result *out)
{
    __shared__ double ssum[ttc_merge::MERGE_ITEMS][NSUM];
    const int MI = blockDim.x >> 5;                           // items of this CTA
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int item = blockIdx.x * MI + warp;                  // pair * levels + level
    if (item < total) {
        const SolveDesc d = sd[item];
        double acc[NSUM];
        merge_sums(partials + d.poff, d.ntiles, acc);
        if (lane == 0)
            for (int s = 0; s < NSUM; ++s) ssum[warp][s] = acc[s];
    }
    __syncthreads();
    const int it = blockIdx.x * MI + lane;
    if (warp == 0 && lane < MI && it < total) {
        const SolveDesc d = sd[it];
        solve_record(ssum[lane], d.level, ldexp(1.0, -4 - 4 * d.level - d.shift), d.ncubes, mode, status, out + it);
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

// atan2(y, x) in FP32 for the gradient direction: with t = min(|x|, |y|) / max(|x|, |y|)
// in [0, 1], atan(t) = t P(t^2) with P the degree-8 minimax polynomial of
// csrc/fit_atan.py (FP32 evaluation error 9.5e-8 on [0, 1]); then atan2 follows from the
// octant: pi/2 - a when |y| > |x|, pi - a when x < 0, the sign of y.  Total error below
// 5e-7 rad (t within about half an ulp; the two subtractions round once each).  atan2(0, 0)
// gives +-0 (x = +0) or +-pi (x = -0), NaN inputs give NaN.
__device__ __forceinline__ float atan2_poly(float y, float x)
{
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    // t = mn / mx: approximate reciprocal, then one correction of the quotient with its
    // exact residual (fma), which leaves t within about half an ulp; mx of at least 2^-100
    // (any gradient of real images) keeps the reciprocal finite, smaller mx divides exactly
    float t = 0.f;
    if (mx >= 7.8886091e-31f) {
        const float rc = __fdividef(1.f, mx);
        const float q = mn * rc;
        t = fmaf(fmaf(-q, mx, mn), rc, q);
    } else if (mx > 0.f) {
        t = mn / mx;
    }
    const float s = t * t;
    float p = 2.456720220e-03f;
    p = fmaf(p, s, -1.440133899e-02f);
    p = fmaf(p, s, 3.978119045e-02f);
    p = fmaf(p, s, -7.234854251e-02f);
    p = fmaf(p, s, 1.049894467e-01f);
    p = fmaf(p, s, -1.416122913e-01f);
    p = fmaf(p, s, 1.998590678e-01f);
    p = fmaf(p, s, -3.333259821e-01f);
    p = fmaf(p, s, 9.999998808e-01f);
    float r = p * t;
    if (ay > ax) r = 1.57079632679489662f - r;
    if (signbit(x)) r = 3.14159265358979324f - r;
    r = copysignf(r, y);
    return (x != x || y != y) ? x + y : r;
}

// Gradient magnitude and direction (Sec. II, Eq. Emag, Eq. Eangle) of image blockIdx.z
// of a batch: a thread owns one output column and walks GR_ROWS output rows, keeping
// the previous pixel row in registers; the right neighbour pixel comes from the next
// lane (the last lane of a warp loads its own).  Stores are coalesced rows.  One image
// of 1080p is a single short wave (latency-bound); batches fill the GPU.
constexpr int GR_ROWS = 8;

template <typename T, bool MAG, bool DIR>
__global__ void __launch_bounds__(256)
ttc_gradient_kernel(const T *__restrict__ img, int H, int W, int64_t pitch_e, int64_t image_stride_e,
                    float *__restrict__ mag, float *__restrict__ dir)
{
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * 256 + threadIdx.x;      // output column
    const int i0 = blockIdx.y * GR_ROWS;               // first output row
    const bool inside = j < W - 1;
    const int jc = inside ? j : W - 2;                 // clamped column for loads
    const int nrows = min(GR_ROWS, H - 1 - i0);        // output rows of this block (>= 1)
    const bool own = lane == 31 || jc + 1 >= W - 1;    // the right neighbour is not in the next lane
    // image blockIdx.z of the batch; this thread's first output of each kind
    img += (int64_t)blockIdx.z * image_stride_e;
    const int64_t o0 = ((int64_t)blockIdx.z * (H - 1) + i0) * (W - 1) + j;
    // all pixel loads first (rows i0 .. i0 + nrows; rows past the image repeat the last)
    float c0[GR_ROWS + 1], c1[GR_ROWS + 1];
    const T *row = img + (int64_t)i0 * pitch_e + jc;
#pragma unroll
    for (int r = 0; r <= GR_ROWS; ++r) {
        c0[r] = (float)__ldg(row);
        c1[r] = own ? (float)__ldg(row + 1) : 0.f;
        if (r < nrows) row += pitch_e;
    }
#pragma unroll
    for (int r = 0; r <= GR_ROWS; ++r) {
        const float n = __shfl_down_sync(0xffffffffu, c0[r], 1);
        if (!own) c1[r] = n;
    }
    if (!inside) return;
    float *pm = MAG ? mag + o0 : nullptr;
    float *pd = DIR ? dir + o0 : nullptr;
#pragma unroll
    for (int r = 0; r < GR_ROWS; ++r) {
        if (r >= nrows) break;
        const float ex = 0.5f * ((c1[r] - c0[r]) + (c1[r + 1] - c0[r + 1]));
        const float ey = 0.5f * ((c0[r + 1] - c0[r]) + (c1[r + 1] - c1[r]));
        if (MAG) {
            *pm = sqrtf(ex * ex + ey * ey);
            pm += W - 1;
        }
        if (DIR) {
            *pd = atan2_poly(ey, ex);
            pd += W - 1;
        }
    }
}

template <typename T>
void launch_gradient(const T *img, int H, int W, int64_t pitch_e, int64_t stride_e, float *mag, float *dir,
                     dim3 grid, cudaStream_t s)
{
    if (mag && dir) ttc_gradient_kernel<T, true, true><<<grid, 256, 0, s>>>(img, H, W, pitch_e, stride_e, mag, dir);
    else if (mag) ttc_gradient_kernel<T, true, false><<<grid, 256, 0, s>>>(img, H, W, pitch_e, stride_e, mag, dir);
    else ttc_gradient_kernel<T, false, true><<<grid, 256, 0, s>>>(img, H, W, pitch_e, stride_e, mag, dir);
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

// level-l image (l >= 1) of one frame in a batch: row pitch and bytes, the same in
// the context workspace and in caller-owned pyramid blocks
void batch_level_image(int H, int W, int l, int dtype, int64_t *pitch, int64_t *bytes)
{
    const int es = (dtype == FT_U8 && l <= 4) ? 2 : 4;
    *pitch = ((int64_t)(W >> l) * es + 15) / 16 * 16;
    *bytes = (*pitch * (H >> l) + 255) / 256 * 256;
}

// Per-level geometry of one request: tiles, partial-sum offsets, and the layout of
// the level images kept in the context (level l >= 1 of every frame).
struct Geometry {
    int levels, npairs, nframes;
    int H[FT_MAX_LEVELS], W[FT_MAX_LEVELS];
    int tiles_x[FT_MAX_LEVELS], tiles_y[FT_MAX_LEVELS], ntiles[FT_MAX_LEVELS];
    int tr[FT_MAX_LEVELS];            // cube rows per tile
    int64_t poff[FT_MAX_LEVELS];      // floats
    int esize[FT_MAX_LEVELS];         // bytes per pixel of the level-l image (l >= 1)
    int64_t pitch[FT_MAX_LEVELS];     // bytes
    int64_t fstride[FT_MAX_LEVELS];   // bytes between frames
    int64_t ioff[FT_MAX_LEVELS];      // bytes, start of level l images
    int shift[FT_MAX_LEVELS];         // the level's partials are 2^shift times the block-sum sums
    int64_t partial_floats, image_bytes;
};

// force_tr: 0 picks the tile height per level (16 rows when 64-row tiles would give
// fewer than ~4 waves of CTAs, so that small levels run as many short CTAs)
// plan_pairs: the pair count that decides the tile height per level (0: npairs), so that
// chunks of a sequence use the tiles of the whole sequence
void geometry(int H, int W, int levels, int dtype, int npairs, int nframes, Geometry &g, int force_tr = 0,
              int plan_pairs = 0)
{
    g.levels = levels;
    g.npairs = npairs;
    g.nframes = nframes;
    int64_t po = 0, io = 0;
    for (int l = 0; l < levels; ++l) {
        g.H[l] = H >> l;
        g.W[l] = W >> l;
        g.tiles_x[l] = (int)ft::ceil_div(g.W[l] - 1, TC);
        int tr = TR;
        if (force_tr) tr = force_tr;
        else if ((int64_t)(plan_pairs ? plan_pairs : npairs) * ft::ceil_div(g.H[l] - 1, TR) * g.tiles_x[l] < 1216)
            tr = ttc_pass::TR_SMALL;
        g.tr[l] = tr;
        g.shift[l] = 0;
        g.tiles_y[l] = (int)ft::ceil_div(g.H[l] - 1, tr);
        g.ntiles[l] = g.tiles_y[l] * g.tiles_x[l];
        g.poff[l] = po;
        po += (int64_t)npairs * g.ntiles[l] * NSUM;
        if (l == 0) {
            g.esize[0] = dtype == FT_U8 ? 1 : 4;
            g.pitch[0] = g.fstride[0] = g.ioff[0] = 0;
            continue;
        }
        // uint8 frames: exact block sums fit uint16 up to level 4 (255 * 4^4)
        g.esize[l] = (dtype == FT_U8 && l <= 4) ? 2 : 4;
        // padded so that every tile of the pass reads inside the allocation: shifted
        // edge tiles read up to row H and column W + 2 (tiles_y * tr >= H - 1,
        // tiles_x * TC >= W - 1)
        g.pitch[l] = (((int64_t)(g.tiles_x[l] * TC + 8) * g.esize[l]) + 15) / 16 * 16;
        g.fstride[l] = ((g.pitch[l] * (g.tiles_y[l] * g.tr[l] + 2)) + 255) / 256 * 256;
        g.ioff[l] = io;
        io += g.fstride[l] * nframes;
    }
    g.partial_floats = po;
    g.image_bytes = io;
}

// Geometry of the all-levels kernel: every level's partials on the level-0 tile grid
// (64 x 256 cubes), no level images.
void geometry_fused(int H, int W, int levels, int npairs, Geometry &g)
{
    g.levels = levels;
    g.npairs = npairs;
    g.nframes = 0;
    const int tx = (int)ft::ceil_div(W - 1, TC), ty = (int)ft::ceil_div(H - 1, TR);
    for (int l = 0; l < levels; ++l) {
        g.H[l] = H >> l;
        g.W[l] = W >> l;
        g.tiles_x[l] = tx;
        g.tiles_y[l] = ty;
        g.ntiles[l] = tx * ty;
        g.tr[l] = TR;
        g.poff[l] = (int64_t)l * npairs * tx * ty * NSUM;
        g.shift[l] = l <= 3 ? 16 : 0;     // levels 0..3: pixels scaled by 256 in the kernel's arithmetic
        g.esize[l] = l == 0 ? 1 : 2;
        g.pitch[l] = g.fstride[l] = g.ioff[l] = 0;
    }
    g.partial_floats = (int64_t)levels * npairs * tx * ty * NSUM;
    g.image_bytes = 0;
}

// the all-levels kernel takes uint8 pairs of 2..5 levels whose frames the copy engine
// can address (16-byte aligned frames, pitch and pair stride)
bool fused_eligible(int dtype, int levels, const void *prev, const void *cur, int64_t pitch, int64_t pair_stride,
                    int npairs)
{
    if (dtype != FT_U8 || levels < 2 || levels > ttc_fused::MAXLEV) return false;
    if ((reinterpret_cast<uintptr_t>(prev) & 15) || (reinterpret_cast<uintptr_t>(cur) & 15) || (pitch & 15))
        return false;
    if (npairs > 1 && (pair_stride <= 0 || (pair_stride & 15))) return false;
    return ft::tensor_map_encoder() != nullptr;
}

// cube centre offsets of level l: x = j + 1/2 - cx_l with cx_l = (W - 2^l) / 2^(l+1),
// the level-0 image centre (W-1)/2 in level-l pixel indices
float centre_off(int n, int l)
{
    const double pl = (double)(1 << l);
    return (float)(0.5 - ((double)n - pl) / (2.0 * pl));
}

}  // namespace

namespace {

// key of a batch frame's tensor map: the map is a function of these values only
struct MapKey {
    const void *base;
    int W, H, bw;
    int64_t pitch;
    bool operator==(const MapKey &o) const
    {
        return base == o.base && W == o.W && H == o.H && bw == o.bw && pitch == o.pitch;
    }
};
struct MapKeyHash {
    size_t operator()(const MapKey &k) const
    {
        size_t h = std::hash<const void *>()(k.base);
        h = h * 1000003u ^ (size_t)k.W;
        h = h * 1000003u ^ (size_t)k.H;
        h = h * 1000003u ^ (size_t)k.bw;
        return h * 1000003u ^ (size_t)k.pitch;
    }
};

}  // namespace

struct ttc_ctx {
    int max_H, max_W, max_levels, max_pairs;
    float *partials;
    unsigned char *images;
    int *status;              // stage-1 timeout flag
    int64_t partial_cap;      // floats
    int64_t image_cap;        // bytes
    size_t bytes;
    Geometry g;               // of the last ttc_partial_sums call
    bool ready;
    cudaEvent_t ev0_start, ev0_end;   // optional timing of the level-0 pass
    int launches;                     // kernels launched by the last ttc_partial_sums
    // batches of pairs of different sizes
    ttc_pass::PassParams *d_descs;    // [max_levels][max_pairs]
    int *d_prefix;                    // [max_levels][2][max_pairs + 1]
    SolveDesc *d_sdesc;               // [max_pairs * max_levels]
    CUtensorMap *d_maps;              // [max_pairs][4]: level-0 maps of pairs the TMA kernel takes
    int2 *d_items;                    // [items_cap]: (pair, tile) of the TMA kernel's level-0 items
    ttc_fused::Geom *d_geoms;         // [max_pairs]: pairs of the all-levels kernel
    int4 *d_units;                    // [items_cap]: its units (pair, strip, first tile row, tiles)
    size_t items_cap;
    size_t off_maps, off_items, off_geoms, off_units;   // byte offsets of those arrays in the staging buffers
    unsigned char *h_stage;           // pinned staging buffer of the arrays: the half in use
    unsigned char *h_stage_buf[2];    // two halves, used alternately by prepares
    size_t stage_bytes;
    cudaEvent_t stage_ev_buf[2];      // the last upload from each half
    bool stage_pending_buf[2];
    int stage_idx;                    // the half the next prepare fills
    // tensor maps of batch frames, by (base, W, H, pitch, box width): a serving loop's frames
    // live in a few fixed slots, so most prepares find their maps here instead of encoding them
    std::unordered_map<MapKey, CUtensorMap, MapKeyHash> map_cache;
    struct {
        int npairs, levels, dtype;
        int rpw[FT_MAX_LEVELS], in_es[FT_MAX_LEVELS], out_es[FT_MAX_LEVELS];
        int n_int[FT_MAX_LEVELS], n_edge[FT_MAX_LEVELS];
        int n_tma;                    // level-0 items of the TMA kernel (uint8 pairs it can read)
        int n_units;                  // units of the all-levels kernel
        bool ready;
    } b;
    int plan_rpw[FT_MAX_LEVELS];      // tile rows per warp per level for batches (0: automatic)
    ttc_pair_desc *h_pairs;           // host copy of the prepared batch (for the autotuner)
    // sequences in host memory: two device buffers of frame chunks, a results buffer,
    // copy streams and their events (allocated on first use)
    unsigned char *ring;
    size_t ring_bytes;                // per buffer
    ttc_level_result *ring_out;
    size_t ring_out_records;
    cudaStream_t cstream[2];
    cudaEvent_t ev_start, ev_copied[2], ev_free[2];
    cudaEvent_t ev_ring_done;         // the last host-sequence call has finished with the ring
    bool ring_ready;                  // streams and events exist
    bool ring_used;                   // ev_ring_done has been recorded
};

extern "C" ft_status ttc_ctx_create(ttc_ctx **ctx, int max_H, int max_W, int max_levels, int max_pairs)
{
    FT_API_RANGE;
    if (!ctx) return FT_ERR_INVALID_ARG;
    *ctx = nullptr;
    if (max_pairs < 1 || max_levels < 1) return FT_ERR_INVALID_ARG;
    if (max_H < 2 || max_W < 2) return FT_ERR_SHAPE;
    if (max_levels > FT_MAX_LEVELS) return FT_ERR_UNSUPPORTED;
    int lv = 0;
    while (lv < max_levels && (max_H >> lv) >= 2 && (max_W >> lv) >= 2) ++lv;
    // the larger of the two layouts: a video of max_pairs + 1 frames or max_pairs
    // independent pairs (two frames each); float frames need the wider images
    // any tile height a later call may pick
    Geometry g, g16;
    geometry(max_H, max_W, lv, FT_F32, max_pairs, 2 * max_pairs, g, TR);
    geometry(max_H, max_W, lv, FT_F32, max_pairs, 2 * max_pairs, g16, ttc_pass::TR_SMALL);
    Geometry gf;
    geometry_fused(max_H, max_W, std::min(lv, ttc_fused::MAXLEV), max_pairs, gf);
    const int64_t pf = std::max(std::max(g.partial_floats, g16.partial_floats), gf.partial_floats);
    const int64_t ib = std::max(g.image_bytes, g16.image_bytes);
    float *part = nullptr;
    unsigned char *img = nullptr;
    // the partials, then 256 bytes holding the status word
    const size_t cbytes = 256;
    cudaError_t e = cudaMalloc(&part, (size_t)pf * sizeof(float) + cbytes);
    if (e == cudaSuccess && ib > 0) e = cudaMalloc(&img, (size_t)ib);
    if (e != cudaSuccess) {
        ft::set_cuda_error(e);
        cudaFree(part);
        return FT_ERR_CUDA;
    }
    ttc_ctx *c = new (std::nothrow) ttc_ctx();
    if (!c) {
        cudaFree(part);
        cudaFree(img);
        return FT_ERR_CUDA;
    }
    c->max_H = max_H;
    c->max_W = max_W;
    c->max_levels = max_levels;
    c->max_pairs = max_pairs;
    c->partials = part;
    c->images = img;
    c->status = reinterpret_cast<int *>(part + pf);
    c->partial_cap = pf;
    c->image_cap = ib;
    c->bytes = (size_t)pf * sizeof(float) + cbytes + (size_t)ib;
    c->ready = false;
    // batch descriptors
    const size_t nd = (size_t)max_levels * max_pairs;
    const size_t b_desc = nd * sizeof(ttc_pass::PassParams);
    const size_t b_pre = (size_t)max_levels * 2 * (max_pairs + 1) * sizeof(int);
    const size_t b_sd = nd * sizeof(SolveDesc);
    // level-0 tensor maps (64-byte aligned) and the TMA kernel's item table
    const size_t tiles0 = (size_t)ft::ceil_div(max_H - 1, TR) * (size_t)ft::ceil_div(max_W - 1, TC);
    c->items_cap = tiles0 * (size_t)max_pairs;
    c->off_maps = (b_desc + b_pre + b_sd + 127) / 128 * 128;
    c->off_items = c->off_maps + (size_t)max_pairs * 4 * sizeof(CUtensorMap);
    c->off_geoms = (c->off_items + c->items_cap * sizeof(int2) + 127) / 128 * 128;
    c->off_units = (c->off_geoms + (size_t)max_pairs * sizeof(ttc_fused::Geom) + 127) / 128 * 128;
    c->stage_bytes = c->off_units + c->items_cap * sizeof(int4);
    unsigned char *dbuf = nullptr;
    e = cudaMalloc(&dbuf, c->stage_bytes);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaHostAlloc(&c->h_stage_buf[k], c->stage_bytes, cudaHostAllocMapped | cudaHostAllocPortable);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->stage_ev_buf[k], cudaEventDisableTiming);
    }
    c->h_stage = c->h_stage_buf[0];
    c->h_pairs = new (std::nothrow) ttc_pair_desc[max_pairs];
    if (e != cudaSuccess || !c->h_pairs) {
        ft::set_cuda_error(e != cudaSuccess ? e : cudaErrorMemoryAllocation);
        cudaFree(dbuf);
        for (int k = 0; k < 2; ++k) {
            if (c->h_stage_buf[k]) cudaFreeHost(c->h_stage_buf[k]);
            if (c->stage_ev_buf[k]) cudaEventDestroy(c->stage_ev_buf[k]);
        }
        delete[] c->h_pairs;
        cudaFree(part);
        cudaFree(img);
        delete c;
        return FT_ERR_CUDA;
    }
    // copy streams and events of host-frame sequences (no device memory: the ring
    // itself is sized by ttc_ctx_reserve_host)
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = cudaStreamCreateWithFlags(&c->cstream[b], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_copied[b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_free[b], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_start, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_ring_done, cudaEventDisableTiming);
    c->ring_ready = e == cudaSuccess;
    if (e != cudaSuccess) ft::set_cuda_error(e);
    c->d_descs = reinterpret_cast<ttc_pass::PassParams *>(dbuf);
    c->d_prefix = reinterpret_cast<int *>(dbuf + b_desc);
    c->d_sdesc = reinterpret_cast<SolveDesc *>(dbuf + b_desc + b_pre);
    c->d_maps = reinterpret_cast<CUtensorMap *>(dbuf + c->off_maps);
    c->d_items = reinterpret_cast<int2 *>(dbuf + c->off_items);
    c->d_geoms = reinterpret_cast<ttc_fused::Geom *>(dbuf + c->off_geoms);
    c->d_units = reinterpret_cast<int4 *>(dbuf + c->off_units);
    c->bytes += c->stage_bytes;
    *ctx = c;
    if (!c->ring_ready) {
        ttc_ctx_destroy(c);
        *ctx = nullptr;
        return FT_ERR_CUDA;
    }
    return FT_OK;
}

extern "C" void ttc_ctx_destroy(ttc_ctx *ctx)
{
    if (!ctx) return;
    for (int k = 0; k < 2; ++k)
        if (ctx->stage_pending_buf[k]) cudaEventSynchronize(ctx->stage_ev_buf[k]);
    cudaFree(ctx->partials);
    cudaFree(ctx->images);
    cudaFree(ctx->d_descs);
    for (int k = 0; k < 2; ++k) {
        if (ctx->h_stage_buf[k]) cudaFreeHost(ctx->h_stage_buf[k]);
        if (ctx->stage_ev_buf[k]) cudaEventDestroy(ctx->stage_ev_buf[k]);
    }
    if (ctx->ring_used) cudaEventSynchronize(ctx->ev_ring_done);
    for (int b = 0; b < 2; ++b) {
        if (ctx->cstream[b]) {
            cudaStreamSynchronize(ctx->cstream[b]);
            cudaStreamDestroy(ctx->cstream[b]);
        }
        if (ctx->ev_copied[b]) cudaEventDestroy(ctx->ev_copied[b]);
        if (ctx->ev_free[b]) cudaEventDestroy(ctx->ev_free[b]);
    }
    if (ctx->ev_start) cudaEventDestroy(ctx->ev_start);
    if (ctx->ev_ring_done) cudaEventDestroy(ctx->ev_ring_done);
    if (ctx->ring) cudaFree(ctx->ring);
    if (ctx->ring_out) cudaFree(ctx->ring_out);
    delete[] ctx->h_pairs;
    delete ctx;
}

extern "C" size_t ttc_ctx_workspace_bytes(const ttc_ctx *ctx) { return ctx ? ctx->bytes : 0; }

extern "C" int ttc_ctx_last_launch_count(const ttc_ctx *ctx) { return ctx ? ctx->launches : 0; }

extern "C" ft_status ttc_ctx_set_level0_events(ttc_ctx *ctx, void *start, void *end)
{
    if (!ctx || (!start) != (!end)) return FT_ERR_INVALID_ARG;
    ctx->ev0_start = static_cast<cudaEvent_t>(start);
    ctx->ev0_end = static_cast<cudaEvent_t>(end);
    return FT_OK;
}

namespace {

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link)
// 3-D map over npairs frames of H x W uint8 pixels (box: bw columns x TR+1 rows x 1)
bool u8_frame_map(CUtensorMap *m, const void *base, int W, int H, int npairs, int64_t pitch, int64_t pstride,
                  int bw)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = ft::tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)npairs};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch, (cuuint64_t)pstride};
    const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)(TR + 1), 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<void *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// the tensor map of one batch frame (one pair coordinate), from the context's cache or
// encoded and cached
bool batch_frame_map(ttc_ctx *ctx, CUtensorMap *m, const void *base, int W, int H, int64_t pitch, int bw)
{
    const MapKey k{base, W, H, bw, pitch};
    const auto it = ctx->map_cache.find(k);
    if (it != ctx->map_cache.end()) {
        *m = it->second;
        return true;
    }
    if (!u8_frame_map(m, base, W, H, 1, pitch, (pitch * H + 15) / 16 * 16, bw)) return false;
    if (ctx->map_cache.size() >= 4096) ctx->map_cache.clear();
    ctx->map_cache.emplace(k, *m);
    return true;
}

// the persistent TMA level-0 kernel over a set of work items: two CTAs per SM
template <class Items, bool GLOBAL_MAPS>
cudaError_t launch_tma_items_w(const Items &it, bool write, int *status, cudaStream_t s)
{
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::min(it.total, 2 * std::max(nsm, 1));
    if (grid <= 0) return cudaSuccess;
    const unsigned extra = ft::tma_extra_tx();
    cudaError_t e;
    if (write) {
        auto k = ttc_tma::ttc_pass_tma_kernel<true, Items, GLOBAL_MAPS>;
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, ttc_tma::SMEM);
        if (e == cudaSuccess) k<<<grid, ttc_pass::NT, ttc_tma::SMEM, s>>>(it, status, extra);
    } else {
        auto k = ttc_tma::ttc_pass_tma_kernel<false, Items, GLOBAL_MAPS>;
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, ttc_tma::SMEM);
        if (e == cudaSuccess) k<<<grid, ttc_pass::NT, ttc_tma::SMEM, s>>>(it, status, extra);
    }
    return e == cudaSuccess ? cudaGetLastError() : e;
}

cudaError_t launch_tma_items(const ttc_tma::VideoItems &it, bool write, int *status, cudaStream_t s)
{
    return launch_tma_items_w<ttc_tma::VideoItems, false>(it, write, status, s);
}

cudaError_t launch_tma_items(const ttc_tma::BatchItems &it, bool write, int *status, cudaStream_t s)
{
    return launch_tma_items_w<ttc_tma::BatchItems, true>(it, write, status, s);
}

// level 0 of uint8 frames by the persistent TMA kernel; false when the frames do not
// meet the copy engine's alignment rules (the caller then uses the load path)
bool launch_level0_tma(const ttc_pass::PassParams &p, const void *prev, const void *cur, int64_t pair_stride,
                       int npairs, int *status, cudaStream_t s, cudaError_t *err)
{
    *err = cudaSuccess;
    const int64_t pitch = p.pitch;
    if ((reinterpret_cast<uintptr_t>(prev) & 15) || (reinterpret_cast<uintptr_t>(cur) & 15) || (pitch & 15))
        return false;
    int64_t ps = pair_stride;
    if (npairs == 1) ps = (pitch * p.H + 15) / 16 * 16;
    else if (ps <= 0 || (ps & 15)) return false;
    ttc_tma::VideoItems it{};
    if (!u8_frame_map(&it.m[0], prev, p.W, p.H, npairs, pitch, ps, ttc_tma::BW) ||
        !u8_frame_map(&it.m[1], cur, p.W, p.H, npairs, pitch, ps, ttc_tma::BW) ||
        !u8_frame_map(&it.m[2], prev, p.W, p.H, npairs, pitch, ps, ttc_tma::XW) ||
        !u8_frame_map(&it.m[3], cur, p.W, p.H, npairs, pitch, ps, ttc_tma::XW))
        return false;
    it.p = p;
    it.total = npairs * p.ntiles;
    *err = launch_tma_items(it, p.next != nullptr, status, s);
    return true;
}

template <typename Tin>
cudaError_t launch_pass(const ttc_pass::PassParams &p, int out_esize, int npairs, cudaStream_t s, int *count)
{
    if (out_esize == 2) return ttc_pass::launch<Tin, unsigned short>(p, npairs, s, count);
    return ttc_pass::launch<Tin, float>(p, npairs, s, count);
}

// Long videos (consecutive pairs sharing frames) keep the per-level passes: there each
// frame's pyramid is built once and the level-0 pass runs alone, which measured faster
// than the all-levels kernel once a video gives every CTA of the grid more than 64
// level-0 tiles (1080p, 299 pairs: 1.10 against 1.16 ms per step).  Decided on the pair
// count of the whole sequence, so that the chunks of a host sequence take the same path.
int sm_count();
bool per_level_video(int independent, int seq_pairs, int H, int W)
{
    if (independent) return false;
    const int64_t tiles = (int64_t)seq_pairs * ft::ceil_div(W - 1, TC) * ft::ceil_div(H - 1, TR);
    return tiles > 64 * 2 * (int64_t)sm_count();
}

// SM count of the current device (grid sizes of the persistent kernels)
int sm_count()
{
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return std::max(nsm, 1);
}

// (pair, level) items per CTA of the merge kernels: enough to spread them over every SM
// (the FP64 merges of one SM run one after another), at most MERGE_ITEMS
int merge_items_per_cta(int items)
{
    return (int)std::min<int64_t>(ttc_merge::MERGE_ITEMS, std::max<int64_t>(1, ft::ceil_div(items, sm_count())));
}

// Tiles per unit of the all-levels kernel: whole strips when there are at least four
// units per CTA of the grid, else shorter runs (each below the top of its strip starts
// with a prologue).
int fused_segment(int64_t strips, int tiles_y)
{
    const int64_t per = strips * tiles_y / (4 * 2 * (int64_t)sm_count());
    return (int)std::min<int64_t>(tiles_y, std::max<int64_t>(1, per));
}

void fused_geom(ttc_fused::Geom &fg, const Geometry &g, int H, int W, int levels, float *partials)
{
    fg = ttc_fused::Geom{};
    fg.H = H;
    fg.W = W;
    fg.tiles_x = g.tiles_x[0];
    fg.tiles_y = g.tiles_y[0];
    fg.ntiles = g.ntiles[0];
    fg.nlev = levels;
    for (int l = 0; l < levels; ++l) {
        fg.xoff[l] = centre_off(W, l);
        fg.yoff[l] = centre_off(H, l);
        fg.part[l] = partials + g.poff[l];
    }
}

// All levels of npairs uint8 pairs by the all-levels kernel (pair p is (prev + p *
// pair_stride, cur + p * pair_stride)).  False when the frames' tensor maps cannot be
// made (the caller then takes the per-level passes); *st is the call's status otherwise.
bool launch_fused(ttc_ctx *ctx, const void *prev, const void *cur, int64_t pair_stride, int npairs, int H, int W,
                  int64_t pitch, int levels, cudaStream_t s, ft_status *st)
{
    Geometry g;
    geometry_fused(H, W, levels, npairs, g);
    *st = FT_OK;
    const int64_t ps = npairs == 1 ? (pitch * H + 15) / 16 * 16 : pair_stride;
    ttc_fused::VideoUnits u{};
    if (!u8_frame_map(&u.m[0], prev, W, H, npairs, pitch, ps, ttc_tma::BW) ||
        !u8_frame_map(&u.m[1], cur, W, H, npairs, pitch, ps, ttc_tma::BW) ||
        !u8_frame_map(&u.m[2], prev, W, H, npairs, pitch, ps, ttc_tma::XW) ||
        !u8_frame_map(&u.m[3], cur, W, H, npairs, pitch, ps, ttc_tma::XW))
        return false;
    if (g.partial_floats > ctx->partial_cap) {
        *st = FT_ERR_WORKSPACE;
        return true;
    }
    fused_geom(u.g, g, H, W, levels, ctx->partials);
    u.npairs = npairs;
    u.seg = fused_segment((int64_t)npairs * u.g.tiles_x, u.g.tiles_y);
    u.nseg = (int)ft::ceil_div(u.g.tiles_y, u.seg);
    const int64_t total = (int64_t)npairs * u.g.tiles_x * u.nseg;
    if (total > 0x7fffffffLL) {
        *st = FT_ERR_UNSUPPORTED;
        return true;
    }
    u.total = (int)total;
    // the status word and the unit ticket start at zero
    cudaError_t e = cudaMemsetAsync(ctx->status, 0, 2 * sizeof(int), s);
    if (e == cudaSuccess && ctx->ev0_start) e = cudaEventRecord(ctx->ev0_start, s);
    if (e == cudaSuccess) e = ttc_fused::launch_video(u, ctx->status, ctx->status + 1, s);
    if (e == cudaSuccess && ctx->ev0_end) e = cudaEventRecord(ctx->ev0_end, s);
    if (e != cudaSuccess) {
        ft::set_cuda_error(e);
        *st = FT_ERR_CUDA;
        return true;
    }
    ctx->g = g;
    ctx->ready = true;
    ctx->launches = 1;
    return true;
}

// all levels of npairs pairs: pair p is (prev + p * pair_stride, cur + p * pair_stride);
// independent = 0 for the consecutive pairs of a video (frame t+1 shared)
// the levels kernel takes levels 1 .. L-1 in one launch when their images have one pixel
// type: uint16 (uint8 frames, at most 5 levels) or float (float frames)
// all levels of npairs pairs: pair p is (prev + p * pair_stride, cur + p * pair_stride);
// independent = 0 for the consecutive pairs of a video (frame t+1 shared)
ft_status launch_partials(ttc_ctx *ctx, const void *prev, const void *cur, int64_t pair_stride, int npairs,
                          int independent, int dtype, int H, int W, int64_t pitch, int levels, cudaStream_t s,
                          int plan_pairs = 0)
{
    if (!ctx || !prev || !cur) return FT_ERR_INVALID_ARG;
    if (npairs < 1) return FT_ERR_SHAPE;
    ft_status st = check_frames(dtype, H, W, pitch);
    if (st != FT_OK) return st;
    if ((st = check_levels(H, W, levels)) != FT_OK) return st;
    if (npairs > ctx->max_pairs || levels > ctx->max_levels || H > ctx->max_H || W > ctx->max_W)
        return FT_ERR_WORKSPACE;
    if (fused_eligible(dtype, levels, prev, cur, pitch, pair_stride, npairs) &&
        !per_level_video(independent, plan_pairs ? plan_pairs : npairs, H, W)) {
        if (launch_fused(ctx, prev, cur, pair_stride, npairs, H, W, pitch, levels, s, &st)) return st;
    }
    Geometry g;
    geometry(H, W, levels, dtype, npairs, independent ? 2 * npairs : npairs + 1, g, 0, plan_pairs);
    if (g.partial_floats > ctx->partial_cap || g.image_bytes > ctx->image_cap) return FT_ERR_WORKSPACE;
    for (int l = 0; l < levels; ++l)
        if ((int64_t)npairs * g.ntiles[l] > 0x7fffffffLL) return FT_ERR_UNSUPPORTED;

    int launches = 0;
    const uintptr_t al = dtype == FT_U8 ? 3 : 15;
    const int vec0 = ((reinterpret_cast<uintptr_t>(prev) & al) == 0 && (reinterpret_cast<uintptr_t>(cur) & al) == 0 &&
                      (pitch & (int64_t)al) == 0 && (pair_stride & (int64_t)al) == 0) ? 1 : 0;
    ttc_pass::PassParams pp[FT_MAX_LEVELS];
    int out_es[FT_MAX_LEVELS];
    for (int l = 0; l < levels; ++l) {
        ttc_pass::PassParams &p = pp[l];
        p = ttc_pass::PassParams{};
        if (l == 0) {
            p.prev = static_cast<const unsigned char *>(prev);
            p.cur = static_cast<const unsigned char *>(cur);
            p.pair_stride = pair_stride;
            p.pitch = pitch;
            p.frame_bytes = pitch * (H - 1) + (int64_t)W * g.esize[0];
        } else {
            p.prev = ctx->images + g.ioff[l];
            p.cur = p.prev + g.fstride[l];
            p.pair_stride = independent ? 2 * g.fstride[l] : g.fstride[l];
            p.pitch = g.pitch[l];
            p.frame_bytes = g.fstride[l];
        }
        p.status = ctx->status;
        p.H = g.H[l];
        p.W = g.W[l];
        p.tiles_x = g.tiles_x[l];
        p.tiles_y = g.tiles_y[l];
        p.tr = g.tr[l];
        p.ntiles = g.ntiles[l];
        // cube centre x = j + 1/2 - cx_l, cx_l = (W - 2^l) / 2^(l+1): the level-0 image
        // centre (W-1)/2 expressed in level-l pixel indices
        const double pl = (double)(1 << l);
        p.xoff = (float)(0.5 - ((double)W - pl) / (2.0 * pl));
        p.yoff = (float)(0.5 - ((double)H - pl) / (2.0 * pl));
        p.partials = ctx->partials + g.poff[l];
        out_es[l] = 4;
        if (l + 1 < levels) {
            p.next = ctx->images + g.ioff[l + 1];
            p.next_fstride = g.fstride[l + 1];
            p.next_pitch = g.pitch[l + 1];
            p.next_bytes = g.fstride[l + 1];
            out_es[l] = g.esize[l + 1];
        }
        p.write_prev = independent;
        p.vec = l == 0 ? vec0 : 1;
        p.padded = l == 0 ? 0 : 1;
    }
    cudaError_t e = cudaMemsetAsync(ctx->status, 0, sizeof(int), s);
    if (e == cudaSuccess && ctx->ev0_start) e = cudaEventRecord(ctx->ev0_start, s);
    if (e != cudaSuccess) {
        ft::set_cuda_error(e);
        return FT_ERR_CUDA;
    }
    for (int l = 0; l < levels; ++l) {
        const ttc_pass::PassParams &p = pp[l];
        const int in_es = g.esize[l];
        bool done = false;
        if (l == 0 && dtype == FT_U8 && g.tr[0] == TR && (out_es[0] == 2 || !p.next)) {
            done = launch_level0_tma(p, prev, cur, pair_stride, npairs, ctx->status, s, &e);
            if (done) {
                ++launches;
                g.shift[0] = 16;            // pixels scaled by 256 in the TMA pass
            }
        }
        if (done) {
        } else if (in_es == 1) e = launch_pass<unsigned char>(p, out_es[l], npairs, s, &launches);
        else if (in_es == 2) e = launch_pass<unsigned short>(p, out_es[l], npairs, s, &launches);
        else e = launch_pass<float>(p, out_es[l], npairs, s, &launches);
        if (e == cudaSuccess && l == 0 && ctx->ev0_end) e = cudaEventRecord(ctx->ev0_end, s);
        if (e != cudaSuccess) {
            ft::set_cuda_error(e);
            return FT_ERR_CUDA;
        }
    }
    ctx->g = g;
    ctx->ready = true;
    ctx->launches = launches;
    return FT_OK;
}

ft_status launch_solve(ttc_ctx *ctx, int mode, ttc_level_result *out, cudaStream_t s, int skip = 0)
{
    if (!ctx || !out) return FT_ERR_INVALID_ARG;
    if (mode != FT_MODE_TTC && mode != FT_MODE_FOE) return FT_ERR_INVALID_ARG;
    if (!ctx->ready) return FT_ERR_INVALID_ARG;
    const Geometry &g = ctx->g;
    SolveParams sp{};
    sp.partials = ctx->partials;
    sp.levels = g.levels;
    sp.npairs = g.npairs;
    sp.mode = mode;
    for (int l = 0; l < g.levels; ++l) {
        sp.ntiles[l] = g.ntiles[l];
        sp.poff[l] = g.poff[l];
        sp.inv_scale[l] = std::ldexp(1.0, -4 - 4 * l - g.shift[l]);
        sp.ncubes[l] = (int64_t)(g.H[l] - 1) * (int64_t)(g.W[l] - 1);
    }
    sp.status = ctx->status;
    sp.out = out;
    sp.skip = skip;
    const int items = g.npairs * g.levels;
    const int mi = merge_items_per_cta(items);
    ttc_solve_kernel<<<(unsigned)ft::ceil_div(items, mi), 32 * mi, 0, s>>>(sp);
    return ft::check_launch();
}

}  // namespace

extern "C" ft_status ttc_partial_sums(ttc_ctx *ctx, const void *frames, int64_t frame_stride_bytes, int T,
                                      int dtype, int H, int W, int64_t pitch_bytes, int levels, void *stream)
{
    FT_API_RANGE;
    if (!ctx || !frames) return FT_ERR_INVALID_ARG;
    if (T < 2) return FT_ERR_SHAPE;
    if (frame_stride_bytes < 0) return FT_ERR_INVALID_ARG;
    const unsigned char *f0 = static_cast<const unsigned char *>(frames);
    return launch_partials(ctx, f0, f0 + frame_stride_bytes, frame_stride_bytes, T - 1, 0, dtype, H, W,
                           pitch_bytes, levels, ft::as_stream(stream));
}

extern "C" ft_status ttc_reduce_solve(ttc_ctx *ctx, int mode, ttc_level_result *out, void *stream)
{
    FT_API_RANGE;
    return launch_solve(ctx, mode, out, ft::as_stream(stream));
}

namespace {

// the merge + solve as its own launch (when the levels kernel did not run it)
ft_status solve_after(ttc_ctx *ctx, int mode, ttc_level_result *out, cudaStream_t s)
{
    const ft_status st = launch_solve(ctx, mode, out, s);
    if (st == FT_OK) ++ctx->launches;
    return st;
}

}  // namespace

extern "C" ft_status ttc_solve(ttc_ctx *ctx, const void *prev, const void *cur, int dtype, int H, int W,
                               int64_t pitch_bytes, int levels, int mode, ttc_level_result *out,
                               void *stream)
{
    FT_API_RANGE;
    if (!ctx || !prev || !cur || !out) return FT_ERR_INVALID_ARG;
    if (mode != FT_MODE_TTC && mode != FT_MODE_FOE) return FT_ERR_INVALID_ARG;
    ft_status st = launch_partials(ctx, prev, cur, 0, 1, 0, dtype, H, W, pitch_bytes, levels,
                                   ft::as_stream(stream));
    if (st != FT_OK) return st;
    return solve_after(ctx, mode, out, ft::as_stream(stream));
}

// ---------------------------------------------------------------------------
// batches of pairs of different sizes
// ---------------------------------------------------------------------------

namespace {

// Ranges of the staging buffer a prepare uploads, in 16-byte words.
struct StageRanges {
    const int4 *src[5];         // pinned host staging (addressable from kernels under unified addressing)
    int4 *dst[5];               // device staging
    long long start[6];         // word prefix over the ranges
    int nr;
};

// Copies the staged arrays of a prepare from pinned host memory to the device staging
// buffer.  A kernel rather than copy-engine copies: a small copy on the compute stream
// would otherwise queue behind the frame uploads that another stream has pending on the
// same copy engine (a serving loop's next tick), delaying the kernels that read it.
__global__ void __launch_bounds__(256) stage_copy_kernel(const StageRanges r)
{
    const long long total = r.start[r.nr];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        int k = 0;
        while (k + 1 < r.nr && i >= r.start[k + 1]) ++k;
        const long long w = i - r.start[k];
        r.dst[k][w] = r.src[k][w];
    }
    // the tensor maps among these words are read by later kernels through the tensor-map
    // proxy (after their acquire fence): release this thread's generic-proxy stores to it
    asm volatile("fence.proxy.tensormap::generic.release.gpu;" ::: "memory");
}

ft_status batch_prepare_impl(ttc_ctx *ctx, const ttc_pair_desc *pairs, int npairs, int dtype, int levels,
                             cudaStream_t s)
{
    if (!ctx || !pairs) return FT_ERR_INVALID_ARG;
    if (dtype != FT_U8 && dtype != FT_F32) return FT_ERR_INVALID_ARG;
    if (npairs < 1 || levels < 1) return FT_ERR_INVALID_ARG;
    if (levels > FT_MAX_LEVELS) return FT_ERR_UNSUPPORTED;
    if (npairs > ctx->max_pairs || levels > ctx->max_levels) return FT_ERR_WORKSPACE;
    for (int p = 0; p < npairs; ++p) {
        const ttc_pair_desc &d = pairs[p];
        if (!d.prev || !d.cur) return FT_ERR_INVALID_ARG;
        if ((reinterpret_cast<uintptr_t>(d.prev_pyramid) & 15) || (reinterpret_cast<uintptr_t>(d.cur_pyramid) & 15))
            return FT_ERR_INVALID_ARG;
        if (d.prev_pyramid && d.prev_pyramid == d.cur_pyramid) return FT_ERR_INVALID_ARG;
        ft_status st = check_frames(dtype, d.H, d.W, d.pitch_bytes);
        if (st != FT_OK) return st;
        if ((st = check_levels(d.H, d.W, levels)) != FT_OK) return st;
        if (d.H > ctx->max_H || d.W > ctx->max_W) return FT_ERR_WORKSPACE;
    }
    // tile rows per warp per level: the plan, or 2 when 64-row tiles give few CTAs
    int rpw[FT_MAX_LEVELS];
    for (int l = 0; l < levels; ++l) {
        if (ctx->plan_rpw[l]) {
            rpw[l] = ctx->plan_rpw[l];
            continue;
        }
        int64_t t64 = 0;
        for (int p = 0; p < npairs; ++p)
            t64 += ft::ceil_div((pairs[p].H >> l) - 1, TR) * ft::ceil_div((pairs[p].W >> l) - 1, TC);
        rpw[l] = t64 < 1216 ? 2 : 8;
    }
    const size_t nd = (size_t)ctx->max_levels * ctx->max_pairs;
    // the half of the staging buffer this prepare fills: free once its last upload (two
    // prepares ago) has run
    const int si = ctx->stage_idx;
    ctx->h_stage = ctx->h_stage_buf[si];
    if (ctx->stage_pending_buf[si]) {
        cudaError_t e = cudaEventSynchronize(ctx->stage_ev_buf[si]);
        if (e != cudaSuccess) {
            ft::set_cuda_error(e);
            return FT_ERR_CUDA;
        }
        ctx->stage_pending_buf[si] = false;
    }
    // level 0 of uint8 pairs whose frames the copy engine can address (16-byte aligned
    // frames and pitch) runs the persistent TMA kernel when the plan has 64-row tiles
    const bool tma_level0 = dtype == FT_U8 && rpw[0] == 8 && ft::tensor_map_encoder() != nullptr;
    CUtensorMap *hmaps = reinterpret_cast<CUtensorMap *>(ctx->h_stage + ctx->off_maps);
    int2 *hitems = reinterpret_cast<int2 *>(ctx->h_stage + ctx->off_items);
    int64_t n_tma = 0;
    ttc_pass::PassParams *hd = reinterpret_cast<ttc_pass::PassParams *>(ctx->h_stage);
    int *hpre = reinterpret_cast<int *>(ctx->h_stage + nd * sizeof(ttc_pass::PassParams));
    SolveDesc *hsd = reinterpret_cast<SolveDesc *>(ctx->h_stage + nd * sizeof(ttc_pass::PassParams) +
                                                    (size_t)ctx->max_levels * 2 * (ctx->max_pairs + 1) * sizeof(int));
    const int es0 = dtype == FT_U8 ? 1 : 4;
    int64_t poff = 0, ioff = 0;
    int in_es[FT_MAX_LEVELS], out_es[FT_MAX_LEVELS];
    int64_t n_int[FT_MAX_LEVELS] = {0}, n_edge[FT_MAX_LEVELS] = {0};
    // uint8 pairs of 2..5 levels whose frames the copy engine can address take the
    // all-levels kernel (any tile plan: its tiles are fixed); a caller's first-frame
    // pyramid is not read (the kernel forms every level from level 0, giving the same
    // block sums), the second frame's pyramid is written when a block is given
    ttc_fused::Geom *hgeoms = reinterpret_cast<ttc_fused::Geom *>(ctx->h_stage + ctx->off_geoms);
    int4 *hunits = reinterpret_cast<int4 *>(ctx->h_stage + ctx->off_units);
    const bool fused_dt = dtype == FT_U8 && levels >= 2 && levels <= ttc_fused::MAXLEV &&
                          ft::tensor_map_encoder() != nullptr;
    int n_fused = 0;
    int64_t fused_tiles = 0;
    std::vector<int> fused_pairs;
    // per pair: level images and partials, level by level.  A frame's level images
    // live in the caller's pyramid block when the descriptor gives one, else in the
    // context workspace (images + ioff).
    for (int p = 0; p < npairs; ++p) {
        const ttc_pair_desc &d = pairs[p];
        int64_t img_pitch[FT_MAX_LEVELS], img_fs[FT_MAX_LEVELS];
        int64_t prev_off[FT_MAX_LEVELS], cur_off[FT_MAX_LEVELS];   // workspace offsets, -1: caller block
        int64_t pyr_off[FT_MAX_LEVELS];                             // offsets in a pyramid block
        int64_t po = 0;
        const int64_t ioff_pair = ioff;
        for (int l = 1; l < levels; ++l) {
            batch_level_image(d.H, d.W, l, dtype, &img_pitch[l], &img_fs[l]);
            pyr_off[l] = po;
            po += img_fs[l];
            prev_off[l] = d.prev_pyramid ? -1 : ioff;
            if (!d.prev_pyramid) ioff += img_fs[l];
            cur_off[l] = d.cur_pyramid ? -1 : ioff;
            if (!d.cur_pyramid) ioff += img_fs[l];
        }
        auto prev_img = [&](int l) -> unsigned char * {
            return prev_off[l] >= 0 ? ctx->images + prev_off[l] : nullptr;
        };
        auto cur_img = [&](int l) -> unsigned char * {
            return cur_off[l] >= 0 ? ctx->images + cur_off[l]
                                   : static_cast<unsigned char *>(d.cur_pyramid) + pyr_off[l];
        };
        const bool aligned16 = (reinterpret_cast<uintptr_t>(d.prev) & 15) == 0 &&
                               (reinterpret_cast<uintptr_t>(d.cur) & 15) == 0 && (d.pitch_bytes & 15) == 0;
        if (fused_dt && aligned16) {
            bool ok = batch_frame_map(ctx, &hmaps[4 * p + 0], d.prev, d.W, d.H, d.pitch_bytes, ttc_tma::BW) &&
                      batch_frame_map(ctx, &hmaps[4 * p + 1], d.cur, d.W, d.H, d.pitch_bytes, ttc_tma::BW) &&
                      batch_frame_map(ctx, &hmaps[4 * p + 2], d.prev, d.W, d.H, d.pitch_bytes, ttc_tma::XW) &&
                      batch_frame_map(ctx, &hmaps[4 * p + 3], d.cur, d.W, d.H, d.pitch_bytes, ttc_tma::XW);
            if (ok) {
                Geometry gf;
                geometry_fused(d.H, d.W, levels, 1, gf);
                fused_geom(hgeoms[p], gf, d.H, d.W, levels, ctx->partials + poff);
                if (d.cur_pyramid) {
                    hgeoms[p].pyr = static_cast<unsigned char *>(d.cur_pyramid);
                    for (int l = 1; l < levels; ++l) {
                        hgeoms[p].pyr_off[l] = pyr_off[l];
                        hgeoms[p].pyr_pitch[l] = img_pitch[l];
                    }
                }
                // the per-level kernels skip this pair: empty item ranges, unused descriptors
                for (int l = 0; l < levels; ++l) {
                    hd[(size_t)l * ctx->max_pairs + p] = ttc_pass::PassParams{};
                    int *pi = hpre + ((size_t)l * 2 + 0) * (ctx->max_pairs + 1);
                    int *pe = hpre + ((size_t)l * 2 + 1) * (ctx->max_pairs + 1);
                    pi[p] = pi[p + 1] = (int)n_int[l];
                    pe[p] = pe[p + 1] = (int)n_edge[l];
                    SolveDesc sd;
                    sd.poff = poff + gf.poff[l];
                    sd.ncubes = (int64_t)(gf.H[l] - 1) * (gf.W[l] - 1);
                    sd.ntiles = gf.ntiles[l];
                    sd.level = l;
                    sd.shift = gf.shift[l];
                    hsd[(size_t)p * levels + l] = sd;
                    in_es[l] = l == 0 ? es0 : 2;
                    out_es[l] = l + 1 <= 4 ? 2 : 4;
                }
                poff += gf.partial_floats;
                // this pair's level images were counted in the workspace: give them back
                ioff = ioff_pair;
                fused_pairs.push_back(p);
                fused_tiles += gf.ntiles[0];
                ++n_fused;
                continue;
            }
        }
        bool tma = tma_level0 && aligned16;
        if (tma) {
            tma = batch_frame_map(ctx, &hmaps[4 * p + 0], d.prev, d.W, d.H, d.pitch_bytes, ttc_tma::BW) &&
                  batch_frame_map(ctx, &hmaps[4 * p + 1], d.cur, d.W, d.H, d.pitch_bytes, ttc_tma::BW) &&
                  batch_frame_map(ctx, &hmaps[4 * p + 2], d.prev, d.W, d.H, d.pitch_bytes, ttc_tma::XW) &&
                  batch_frame_map(ctx, &hmaps[4 * p + 3], d.cur, d.W, d.H, d.pitch_bytes, ttc_tma::XW);
        }
        const uintptr_t al = dtype == FT_U8 ? 3 : 15;
        const int vec0 = ((reinterpret_cast<uintptr_t>(d.prev) & al) == 0 &&
                          (reinterpret_cast<uintptr_t>(d.cur) & al) == 0 && (d.pitch_bytes & (int64_t)al) == 0)
                             ? 1 : 0;
        for (int l = 0; l < levels; ++l) {
            ttc_pass::PassParams q{};
            const int H = d.H >> l, W = d.W >> l, tr = 8 * rpw[l];
            q.H = H;
            q.W = W;
            q.tiles_x = (int)ft::ceil_div(W - 1, TC);
            q.tiles_y = (int)ft::ceil_div(H - 1, tr);
            q.ntiles = q.tiles_x * q.tiles_y;
            q.tr = tr;
            if (l == 0) {
                q.prev = static_cast<const unsigned char *>(d.prev);
                q.cur = static_cast<const unsigned char *>(d.cur);
                q.pitch = d.pitch_bytes;
                q.vec = vec0;
                q.frame_bytes = d.pitch_bytes * (d.H - 1) + (int64_t)d.W * es0;
            } else {
                q.prev = prev_off[l] >= 0 ? ctx->images + prev_off[l]
                                          : static_cast<const unsigned char *>(d.prev_pyramid) + pyr_off[l];
                q.cur = cur_img(l);
                q.pitch = img_pitch[l];
                q.vec = 1;
                q.frame_bytes = img_fs[l];
            }
            q.status = ctx->status;
            q.set = q.vec ? ttc_pass::SET_EDGES : ttc_pass::SET_ALL;
            const double pl = (double)(1 << l);
            q.xoff = (float)(0.5 - ((double)d.W - pl) / (2.0 * pl));
            q.yoff = (float)(0.5 - ((double)d.H - pl) / (2.0 * pl));
            q.partials = ctx->partials + poff;
            q.write_prev = d.prev_pyramid ? -1 : 1;
            if (l + 1 < levels) {
                q.next = prev_img(l + 1);
                q.next_cur = cur_img(l + 1);
                q.next_pitch = img_pitch[l + 1];
                q.next_bytes = img_fs[l + 1];
            }
            hd[(size_t)l * ctx->max_pairs + p] = q;
            const bool by_tma = l == 0 && tma;
            const int ni = by_tma ? 0 : q.vec ? (q.tiles_y - 1) * (q.tiles_x - 1) : 0;
            const int ne = by_tma ? 0 : q.vec ? q.tiles_x + q.tiles_y - 1 : q.ntiles;
            if (by_tma) {
                if (n_tma + q.ntiles > (int64_t)ctx->items_cap) return FT_ERR_WORKSPACE;
                for (int t = 0; t < q.ntiles; ++t) hitems[n_tma + t] = make_int2(p, t);
                n_tma += q.ntiles;
            }
            int *pi = hpre + ((size_t)l * 2 + 0) * (ctx->max_pairs + 1);
            int *pe = hpre + ((size_t)l * 2 + 1) * (ctx->max_pairs + 1);
            pi[p] = (int)n_int[l];
            pe[p] = (int)n_edge[l];
            n_int[l] += ni;
            n_edge[l] += ne;
            pi[p + 1] = (int)n_int[l];
            pe[p + 1] = (int)n_edge[l];
            SolveDesc sd;
            sd.poff = poff;
            sd.ncubes = (int64_t)(H - 1) * (W - 1);
            sd.ntiles = q.ntiles;
            sd.level = l;
            sd.shift = by_tma ? 16 : 0;       // the TMA kernel's pixels are scaled by 256
            hsd[(size_t)p * levels + l] = sd;
            poff += (int64_t)q.ntiles * NSUM;
            in_es[l] = l == 0 ? es0 : ((dtype == FT_U8 && l <= 4) ? 2 : 4);
            out_es[l] = (dtype == FT_U8 && l + 1 <= 4) ? 2 : 4;
        }
    }
    if (poff > ctx->partial_cap || ioff > ctx->image_cap) return FT_ERR_WORKSPACE;
    // units of the all-levels kernel: strips cut into runs of `seg` tiles, longest first
    // (the kernel hands them out in order, so the long ones start early)
    int64_t n_units = 0;
    if (n_fused > 0) {
        int max_ty = 1;
        for (int p : fused_pairs) max_ty = std::max(max_ty, hgeoms[p].tiles_y);
        const int seg = (int)std::min<int64_t>(max_ty, std::max<int64_t>(1, fused_tiles / (8 * (int64_t)sm_count())));
        for (int p : fused_pairs) {
            const ttc_fused::Geom &fg = hgeoms[p];
            for (int tx = 0; tx < fg.tiles_x; ++tx)
                for (int j0 = 0; j0 < fg.tiles_y; j0 += seg) {
                    if (n_units >= (int64_t)ctx->items_cap) return FT_ERR_WORKSPACE;
                    hunits[n_units++] = make_int4(p, tx, j0, std::min(seg, fg.tiles_y - j0));
                }
        }
        std::stable_sort(hunits, hunits + n_units, [](const int4 &a, const int4 &b) { return a.w > b.w; });
    }
    for (int l = 0; l < levels; ++l)
        if (n_int[l] > 0x7fffffffLL || n_edge[l] > 0x7fffffffLL) return FT_ERR_UNSUPPORTED;
    if (n_tma > 0x7fffffffLL) return FT_ERR_UNSUPPORTED;
    // one kernel uploads the used parts of the staging buffer (every part starts on a
    // 128-byte boundary; sizes rounded up to 16 bytes stay inside their part)
    unsigned char *dstage = reinterpret_cast<unsigned char *>(ctx->d_descs);
    StageRanges r{};
    auto add = [&](size_t off, size_t bytes) {
        if (bytes == 0) return;
        r.src[r.nr] = reinterpret_cast<const int4 *>(ctx->h_stage + off);
        r.dst[r.nr] = reinterpret_cast<int4 *>(dstage + off);
        r.start[r.nr + 1] = r.start[r.nr] + (long long)((bytes + 15) / 16);
        ++r.nr;
    };
    add(0, ctx->off_maps);
    if (n_tma > 0 || n_units > 0) add(ctx->off_maps, (size_t)npairs * 4 * sizeof(CUtensorMap));
    if (n_tma > 0) add(ctx->off_items, (size_t)n_tma * sizeof(int2));
    if (n_units > 0) add(ctx->off_geoms, (size_t)npairs * sizeof(ttc_fused::Geom));
    if (n_units > 0) add(ctx->off_units, (size_t)n_units * sizeof(int4));
    const long long words = r.start[r.nr];
    const int grid = (int)std::min<long long>(std::max<long long>(1, (words + 255) / 256), 2LL * sm_count());
    stage_copy_kernel<<<grid, 256, 0, s>>>(r);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(ctx->stage_ev_buf[si], s);
    if (e != cudaSuccess) {
        ft::set_cuda_error(e);
        return FT_ERR_CUDA;
    }
    ctx->stage_pending_buf[si] = true;
    ctx->stage_idx = si ^ 1;
    if (pairs != ctx->h_pairs)
        for (int p = 0; p < npairs; ++p) ctx->h_pairs[p] = pairs[p];
    ctx->b.npairs = npairs;
    ctx->b.levels = levels;
    ctx->b.dtype = dtype;
    ctx->b.n_tma = (int)n_tma;
    ctx->b.n_units = (int)n_units;
    for (int l = 0; l < levels; ++l) {
        ctx->b.rpw[l] = rpw[l];
        ctx->b.in_es[l] = in_es[l];
        ctx->b.out_es[l] = out_es[l];
        ctx->b.n_int[l] = (int)n_int[l];
        ctx->b.n_edge[l] = (int)n_edge[l];
    }
    ctx->b.ready = true;
    return FT_OK;
}

template <typename Tin>
cudaError_t batch_level(ttc_ctx *ctx, int l, int *count, cudaStream_t s)
{
    const auto &b = ctx->b;
    const ttc_pass::PassParams *descs = ctx->d_descs + (size_t)l * ctx->max_pairs;
    const int *pi = ctx->d_prefix + ((size_t)l * 2 + 0) * (ctx->max_pairs + 1);
    const int *pe = ctx->d_prefix + ((size_t)l * 2 + 1) * (ctx->max_pairs + 1);
    const bool write = l + 1 < b.levels;
    if (b.out_es[l] == 2)
        return ttc_pass::launch_batch<Tin, unsigned short>(descs, pi, pe, b.n_int[l], b.n_edge[l], b.npairs, write,
                                                           b.rpw[l], s, count);
    return ttc_pass::launch_batch<Tin, float>(descs, pi, pe, b.n_int[l], b.n_edge[l], b.npairs, write, b.rpw[l], s,
                                              count);
}

// launches of one prepared batch
ft_status batch_run_impl(ttc_ctx *ctx, int mode, ttc_level_result *out, cudaStream_t s)
{
    if (!ctx || !out) return FT_ERR_INVALID_ARG;
    if (mode != FT_MODE_TTC && mode != FT_MODE_FOE) return FT_ERR_INVALID_ARG;
    if (!ctx->b.ready) return FT_ERR_INVALID_ARG;
    const auto &b = ctx->b;
    int count = 0;
    // the status word and the all-levels kernel's unit ticket start at zero
    cudaError_t e = cudaMemsetAsync(ctx->status, 0, 2 * sizeof(int), s);
    if (e == cudaSuccess && b.n_units > 0) {
        const ttc_fused::BatchUnits u{ctx->d_geoms, ctx->d_maps, ctx->d_units, b.n_units};
        e = ttc_fused::launch_batch(u, ctx->status, ctx->status + 1, s);
        ++count;
    }
    for (int l = 0; l < b.levels && e == cudaSuccess; ++l) {
        if (l == 0 && b.n_tma > 0) {
            ttc_tma::BatchItems it{ctx->d_descs, ctx->d_maps, ctx->d_items, b.n_tma};
            e = launch_tma_items(it, b.levels > 1, ctx->status, s);
            ++count;
            if (e != cudaSuccess) break;
        }
        if (b.in_es[l] == 1) e = batch_level<unsigned char>(ctx, l, &count, s);
        else if (b.in_es[l] == 2) e = batch_level<unsigned short>(ctx, l, &count, s);
        else e = batch_level<float>(ctx, l, &count, s);
    }
    if (e == cudaSuccess) {
        const int items = b.npairs * b.levels, mi = merge_items_per_cta(items);
        ttc_batch_solve_kernel<<<(unsigned)ft::ceil_div(items, mi), 32 * mi, 0, s>>>(ctx->partials, ctx->d_sdesc,
                                                                                     items, mode, ctx->status, out);
        e = cudaGetLastError();
        ++count;
    }
    if (e != cudaSuccess) {
        ft::set_cuda_error(e);
        return FT_ERR_CUDA;
    }
    ctx->launches = count;
    return FT_OK;
}

}  // namespace

extern "C" ft_status ttc_batch_prepare(ttc_ctx *ctx, const ttc_pair_desc *pairs, int npairs, int dtype, int levels,
                                       void *stream)
{
    FT_API_RANGE;
    return batch_prepare_impl(ctx, pairs, npairs, dtype, levels, ft::as_stream(stream));
}

extern "C" ft_status ttc_batch_run(ttc_ctx *ctx, int mode, ttc_level_result *out, void *stream)
{
    FT_API_RANGE;
    return batch_run_impl(ctx, mode, out, ft::as_stream(stream));
}

extern "C" ft_status ttc_batch_autotune(ttc_ctx *ctx, int mode, ttc_level_result *out, int reps, int *rows_per_tile,
                                        void *stream)
{
    FT_API_RANGE;
    if (!ctx || !out || reps < 1) return FT_ERR_INVALID_ARG;
    if (!ctx->b.ready) return FT_ERR_INVALID_ARG;
    cudaStream_t s = ft::as_stream(stream);
    const int npairs = ctx->b.npairs, levels = ctx->b.levels, dtype = ctx->b.dtype;
    // candidate plans (cube rows per warp per level: 8 -> 64-row tiles, 2 -> 16-row
    // tiles): 64-row tiles down to level k and 16-row tiles below, for k = levels .. 0.
    // 64-row tiles at level 0 let uint8 batches use the copy-engine kernel; small levels
    // may run more, shorter CTAs.  Each plan is timed on the whole prepared batch.
    cudaEvent_t ev[2];
    cudaError_t e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    if (e != cudaSuccess) {
        ft::set_cuda_error(e);
        return FT_ERR_CUDA;
    }
    float best_ms = 0.f;
    int best_k = -1;
    ft_status st = FT_OK;
    for (int k = levels; k >= 0 && st == FT_OK && e == cudaSuccess; --k) {
        for (int l = 0; l < levels; ++l) ctx->plan_rpw[l] = l < k ? 8 : 2;
        st = batch_prepare_impl(ctx, ctx->h_pairs, npairs, dtype, levels, s);
        float ms = 0.f;
        for (int r = 0; r <= reps && st == FT_OK; ++r) {       // the first run warms up
            if (r == 1) e = cudaEventRecord(ev[0], s);
            if (e == cudaSuccess) st = batch_run_impl(ctx, mode, out, s);
        }
        if (st != FT_OK) break;
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
        if (e == cudaSuccess && (best_k < 0 || ms < best_ms)) {
            best_ms = ms;
            best_k = k;
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (e != cudaSuccess) {
        ft::set_cuda_error(e);
        st = FT_ERR_CUDA;
    }
    if (st != FT_OK) {
        for (int l = 0; l < FT_MAX_LEVELS; ++l) ctx->plan_rpw[l] = 0;
        return st;
    }
    for (int l = 0; l < levels; ++l) {
        ctx->plan_rpw[l] = l < best_k ? 8 : 2;
        if (rows_per_tile) rows_per_tile[l] = 8 * ctx->plan_rpw[l];
    }
    return batch_prepare_impl(ctx, ctx->h_pairs, npairs, dtype, levels, s);
}

extern "C" ft_status ttc_pyramid_layout(int H, int W, int levels, int dtype, int64_t *offsets, int64_t *pitches,
                                        int64_t *bytes)
{
    if (!bytes || (dtype != FT_U8 && dtype != FT_F32)) return FT_ERR_INVALID_ARG;
    if (H < 2 || W < 2) return FT_ERR_SHAPE;
    const ft_status st = check_levels(H, W, levels);
    if (st != FT_OK) return st;
    int64_t po = 0;
    if (offsets) offsets[0] = 0;
    if (pitches) pitches[0] = 0;
    for (int l = 1; l < levels; ++l) {
        int64_t pitch, fs;
        batch_level_image(H, W, l, dtype, &pitch, &fs);
        if (offsets) offsets[l] = po;
        if (pitches) pitches[l] = pitch;
        po += fs;
    }
    *bytes = po;
    return FT_OK;
}

extern "C" ft_status ttc_batch_set_plan(ttc_ctx *ctx, const int *rows_per_tile, int levels)
{
    if (!ctx || levels < 1) return FT_ERR_INVALID_ARG;
    if (levels > FT_MAX_LEVELS) return FT_ERR_UNSUPPORTED;
    if (!rows_per_tile) {
        for (int l = 0; l < FT_MAX_LEVELS; ++l) ctx->plan_rpw[l] = 0;
        return FT_OK;
    }
    for (int l = 0; l < levels; ++l)
        if (rows_per_tile[l] != 8 * 8 && rows_per_tile[l] != 8 * 2) return FT_ERR_INVALID_ARG;
    for (int l = 0; l < FT_MAX_LEVELS; ++l) ctx->plan_rpw[l] = l < levels ? rows_per_tile[l] / 8 : 0;
    return FT_OK;
}

// ---------------------------------------------------------------------------
// ttc_solve without device allocation: scratch in a fixed static device array
// ---------------------------------------------------------------------------

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[FT_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kMaxDevices] = {};   // device address of g_noalloc_scratch, per device
void *g_noalloc_ctx[kMaxDevices] = {};    // the context that address belongs to

// cuCtxGetCurrent through the runtime's driver entry point (no libcuda link); null
// when unavailable
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
CtxGetCurrentFn ctx_get_current()
{
    static std::once_flag once;
    static CtxGetCurrentFn fn = nullptr;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrentFn>(f);
        cudaGetLastError();
    });
    return fn;
}

// Device address of the scratch array on the current device (in host code the array's
// name is only a host-side stand-in).  Looked up on the first call on a device and
// again whenever that device's current context has changed (a context destroyed and
// re-created reloads the module, which moves the array).
ft_status noalloc_scratch(unsigned char **base)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        ft::set_cuda_error(e);
        return FT_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return FT_ERR_UNSUPPORTED;
    // null before the runtime has made the device's context current on this thread:
    // the address is then looked up again on the next call
    CUcontext cur = nullptr;
    if (CtxGetCurrentFn get = ctx_get_current()) get(&cur);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev] || g_noalloc_ctx[dev] != static_cast<void *>(cur)) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            ft::set_cuda_error(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
            return FT_ERR_CUDA;
        }
        g_noalloc_addr[dev] = ptr;
        g_noalloc_ctx[dev] = cur;
    }
    *base = static_cast<unsigned char *>(g_noalloc_addr[dev]);
    return FT_OK;
}

}  // namespace

extern "C" ft_status ttc_solve_noalloc(const void *prev, const void *cur, int dtype, int H, int W,
                                       int64_t pitch_bytes, int levels, int mode, ttc_level_result *out,
                                       void *stream)
{
    if (!prev || !cur || !out) return FT_ERR_INVALID_ARG;
    if (mode != FT_MODE_TTC && mode != FT_MODE_FOE) return FT_ERR_INVALID_ARG;
    ft_status st = check_frames(dtype, H, W, pitch_bytes);
    if (st != FT_OK) return st;
    if ((st = check_levels(H, W, levels)) != FT_OK) return st;
    Geometry g, gf;
    geometry(H, W, levels, dtype, 1, 2, g);
    geometry_fused(H, W, std::min(levels, ttc_fused::MAXLEV), 1, gf);
    const int64_t pfl = std::max(g.partial_floats, gf.partial_floats);
    // layout: 256 bytes for the status word and unit ticket, the partials, the level images
    const int64_t pbytes = 256 + (pfl * (int64_t)sizeof(float) + 255) / 256 * 256;
    if (pbytes + g.image_bytes > (int64_t)FT_NOALLOC_SCRATCH_BYTES) return FT_ERR_WORKSPACE;
    unsigned char *base = nullptr;
    if ((st = noalloc_scratch(&base)) != FT_OK) return st;
    // a context on the stack whose workspace is the static array
    ttc_ctx c{};
    c.max_H = H;
    c.max_W = W;
    c.max_levels = levels;
    c.max_pairs = 1;
    c.status = reinterpret_cast<int *>(base);
    c.partials = reinterpret_cast<float *>(base + 256);
    c.images = base + pbytes;
    c.partial_cap = pfl;
    c.image_cap = g.image_bytes;
    c.bytes = FT_NOALLOC_SCRATCH_BYTES;
    c.ready = false;
    st = launch_partials(&c, prev, cur, 0, 1, 0, dtype, H, W, pitch_bytes, levels, ft::as_stream(stream));
    if (st != FT_OK) return st;
    return launch_solve(&c, mode, out, ft::as_stream(stream));
}

extern "C" ft_status ttc_solve_sequence(ttc_ctx *ctx, const void *frames, int64_t frame_stride_bytes, int T,
                                        int dtype, int H, int W, int64_t pitch_bytes, int levels, int mode,
                                        ttc_level_result *out, void *stream)
{
    FT_API_RANGE;
    if (!ctx || !frames || !out) return FT_ERR_INVALID_ARG;
    if (mode != FT_MODE_TTC && mode != FT_MODE_FOE) return FT_ERR_INVALID_ARG;
    if (T < 2) return FT_ERR_SHAPE;
    if (frame_stride_bytes < 0) return FT_ERR_INVALID_ARG;
    const unsigned char *f0 = static_cast<const unsigned char *>(frames);
    ft_status st = launch_partials(ctx, f0, f0 + frame_stride_bytes, frame_stride_bytes, T - 1, 0, dtype, H, W,
                                   pitch_bytes, levels, ft::as_stream(stream));
    if (st != FT_OK) return st;
    return solve_after(ctx, mode, out, ft::as_stream(stream));
}

namespace {

// Ring and records sizes a host-frame sequence needs.  Float frames: a frame's pyramid
// images are rounded differently when written as the first frame of a pair (block sums
// of its pixels) and as the second (first frame's sums plus the sums of the
// differences), and the level-l image of a second frame depends on the level-(l-1)
// image of the frame before it.  So that every record equals the whole-sequence call,
// a chunk after the first also computes the levels - 1 pairs before it (their records
// are not written).  uint8 sums are exact either way.
struct HostPlan {
    int lead, chunk, nchunks;
    size_t frame_bytes, buf_bytes, records;
};

ft_status host_plan(const ttc_ctx *ctx, int64_t frame_stride_bytes, int T, int dtype, int H, int W,
                    int64_t pitch_bytes, int levels, HostPlan *hp)
{
    if (T < 2) return FT_ERR_SHAPE;
    ft_status st = check_frames(dtype, H, W, pitch_bytes);
    if (st != FT_OK) return st;
    if ((st = check_levels(H, W, levels)) != FT_OK) return st;
    if (frame_stride_bytes < pitch_bytes * (H - 1) + (int64_t)W * elem_size(dtype)) return FT_ERR_SHAPE;
    if (H > ctx->max_H || W > ctx->max_W || levels > ctx->max_levels) return FT_ERR_WORKSPACE;
    const int npairs = T - 1;
    hp->lead = (dtype == FT_F32 && ctx->max_pairs > levels - 1) ? levels - 1 : 0;
    hp->chunk = std::min(std::min(FT_SEQ_CHUNK_PAIRS, ctx->max_pairs - hp->lead), npairs);
    hp->nchunks = (npairs + hp->chunk - 1) / hp->chunk;
    hp->frame_bytes = (size_t)(pitch_bytes * (H - 1) + (int64_t)W * elem_size(dtype));
    hp->buf_bytes = ((size_t)(hp->chunk + hp->lead) * (size_t)frame_stride_bytes + hp->frame_bytes + 255) / 256 * 256;
    hp->records = (size_t)npairs * levels;
    return FT_OK;
}

}  // namespace

extern "C" ft_status ttc_ctx_reserve_host(ttc_ctx *ctx, int64_t frame_stride_bytes, int T, int dtype, int H, int W,
                                          int64_t pitch_bytes, int levels)
{
    FT_API_RANGE;
    if (!ctx) return FT_ERR_INVALID_ARG;
    if (!ctx->ring_ready) return FT_ERR_CUDA;
    HostPlan hp;
    ft_status st = host_plan(ctx, frame_stride_bytes, T, dtype, H, W, pitch_bytes, levels, &hp);
    if (st != FT_OK) return st;
    if (hp.buf_bytes <= ctx->ring_bytes && hp.records <= ctx->ring_out_records) return FT_OK;
    // the buffers may still be in use by this context's last host-sequence call: wait for
    // that call only, then free and allocate in stream order on the context's first copy
    // stream (cudaFree would synchronise the whole device); other streams and contexts
    // keep running
    cudaStream_t cs = ctx->cstream[0];
    cudaError_t e = ctx->ring_used ? cudaEventSynchronize(ctx->ev_ring_done) : cudaSuccess;
    if (e == cudaSuccess && hp.buf_bytes > ctx->ring_bytes) {
        if (ctx->ring) e = cudaFreeAsync(ctx->ring, cs);
        ctx->bytes -= 2 * ctx->ring_bytes;
        ctx->ring = nullptr;
        ctx->ring_bytes = 0;
        if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void **>(&ctx->ring), 2 * hp.buf_bytes, cs);
        if (e == cudaSuccess) {
            ctx->ring_bytes = hp.buf_bytes;
            ctx->bytes += 2 * hp.buf_bytes;
        }
    }
    if (e == cudaSuccess && hp.records > ctx->ring_out_records) {
        if (ctx->ring_out) e = cudaFreeAsync(ctx->ring_out, cs);
        ctx->bytes -= ctx->ring_out_records * sizeof(ttc_level_result);
        ctx->ring_out = nullptr;
        ctx->ring_out_records = 0;
        if (e == cudaSuccess)
            e = cudaMallocAsync(reinterpret_cast<void **>(&ctx->ring_out), hp.records * sizeof(ttc_level_result), cs);
        if (e == cudaSuccess) {
            ctx->ring_out_records = hp.records;
            ctx->bytes += hp.records * sizeof(ttc_level_result);
        }
    }
    // the new buffers are usable from any stream once the copy stream has made them
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) {
        ft::set_cuda_error(e);
        return FT_ERR_CUDA;
    }
    return FT_OK;
}

extern "C" ft_status ttc_solve_sequence_host(ttc_ctx *ctx, const void *frames, int64_t frame_stride_bytes, int T,
                                             int dtype, int H, int W, int64_t pitch_bytes, int levels, int mode,
                                             ttc_level_result *out, void *stream)
{
    FT_API_RANGE;
    if (!ctx || !frames || !out) return FT_ERR_INVALID_ARG;
    if (mode != FT_MODE_TTC && mode != FT_MODE_FOE) return FT_ERR_INVALID_ARG;
    if (!ctx->ring_ready) return FT_ERR_CUDA;
    HostPlan hp;
    ft_status st = host_plan(ctx, frame_stride_bytes, T, dtype, H, W, pitch_bytes, levels, &hp);
    if (st != FT_OK) return st;
    // the ring is sized by ttc_ctx_reserve_host: nothing is allocated here
    if (hp.buf_bytes > ctx->ring_bytes || hp.records > ctx->ring_out_records) return FT_ERR_WORKSPACE;
    const int npairs = T - 1;
    const int lead = hp.lead, chunk = hp.chunk, nchunks = hp.nchunks;
    const size_t frame_bytes = hp.frame_bytes;
    cudaStream_t s = ft::as_stream(stream);
    const unsigned char *host = static_cast<const unsigned char *>(frames);
    cudaError_t e = cudaEventRecord(ctx->ev_start, s);
    int launches = 0;
    for (int k = 0; k < nchunks && e == cudaSuccess; ++k) {
        const int b = k & 1;
        const int p0 = k * chunk, n = std::min(chunk, npairs - p0);
        const int x = k > 0 ? std::min(lead, p0) : 0;   // extra pairs before the chunk
        const int f0 = p0 - x;                   // the chunk's first frame
        unsigned char *dev = ctx->ring + (size_t)b * ctx->ring_bytes;
        cudaStream_t cs = ctx->cstream[b];
        // the buffer is free once the chunk two back has been computed (or, for the
        // first two chunks, once the stream has reached this call)
        e = cudaStreamWaitEvent(cs, k < 2 ? ctx->ev_start : ctx->ev_free[b], 0);
        // and, on any stream, once the previous call has finished with the ring
        if (e == cudaSuccess && k < 2 && ctx->ring_used) e = cudaStreamWaitEvent(cs, ctx->ev_ring_done, 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dev, host + (size_t)f0 * frame_stride_bytes,
                                (size_t)(n + x) * frame_stride_bytes + frame_bytes, cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_copied[b], cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ctx->ev_copied[b], 0);
        if (e != cudaSuccess) break;
        st = launch_partials(ctx, dev, dev + frame_stride_bytes, frame_stride_bytes, n + x, 0, dtype, H, W,
                             pitch_bytes, levels, s, npairs);
        if (st != FT_OK) return st;
        launches += ctx->launches + 1;
        e = cudaEventRecord(ctx->ev_free[b], s);
        if (e != cudaSuccess) break;
        st = launch_solve(ctx, mode, ctx->ring_out + (size_t)f0 * levels, s, x);
        if (st != FT_OK) return st;
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, ctx->ring_out, (size_t)npairs * levels * sizeof(ttc_level_result),
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_ring_done, s);
    if (e == cudaSuccess) ctx->ring_used = true;
    if (e != cudaSuccess) {
        ft::set_cuda_error(e);
        return FT_ERR_CUDA;
    }
    ctx->launches = launches;
    return FT_OK;
}

extern "C" ft_status ttc_derivatives(const void *prev, const void *cur, int dtype, int H, int W,
                                     int64_t pitch_bytes, float *Ex, float *Ey, float *Et, float *G,
                                     void *stream)
{
    FT_API_RANGE;
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

extern "C" ft_status ttc_gradient_batch(const void *images, int n, int64_t image_stride_bytes, int dtype, int H,
                                        int W, int64_t pitch_bytes, float *mag, float *dir, void *stream)
{
    FT_API_RANGE;
    if (!images || (!mag && !dir)) return FT_ERR_INVALID_ARG;
    const ft_status st = check_frames(dtype, H, W, pitch_bytes);
    if (st != FT_OK) return st;
    const int es = elem_size(dtype);
    if (n < 1) return FT_ERR_SHAPE;
    if (n > 1 && image_stride_bytes < (int64_t)(H - 1) * pitch_bytes + (int64_t)W * es) return FT_ERR_SHAPE;
    if (n > 65535) return FT_ERR_UNSUPPORTED;
    if (image_stride_bytes % es) return FT_ERR_SHAPE;
    const dim3 grid((unsigned)ft::ceil_div(W - 1, 256), (unsigned)ft::ceil_div(H - 1, GR_ROWS), (unsigned)n);
    if (grid.y > 65535) return FT_ERR_UNSUPPORTED;
    cudaStream_t s = ft::as_stream(stream);
    if (dtype == FT_U8)
        launch_gradient(static_cast<const unsigned char *>(images), H, W, pitch_bytes, image_stride_bytes, mag, dir,
                        grid, s);
    else
        launch_gradient(static_cast<const float *>(images), H, W, pitch_bytes / 4, image_stride_bytes / 4, mag, dir,
                        grid, s);
    return ft::check_launch();
}

extern "C" ft_status ttc_gradient(const void *image, int dtype, int H, int W, int64_t pitch_bytes, float *mag,
                                  float *dir, void *stream)
{
    return ttc_gradient_batch(image, 1, 0, dtype, H, W, pitch_bytes, mag, dir, stream);
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
