// Pyramid levels 1 .. L-1 of every pair in one persistent launch (Sec. V-B: each level
// is computed from the down-sampled images of the level before), with the FP64 merge
// and solve of each pair (Sec. V-A) as soon as its last level is done.
//
// Work items are tiles of ttc_pass_kernel's pass (same arithmetic, same tiles, same
// reduction: results bitwise those of the per-level launches), numbered level-major:
// all level-1 tiles of all pairs, then level 2, ...  A CTA takes the next item from a
// global ticket counter.  Level l of a pair reads the level-l images that level l-1 of
// that pair (and, in a video, of the pair before, which wrote its first frame) writes,
// so each (level, pair) counts its finished tiles and a level-l item first waits until
// the counts it depends on are complete.  Tickets are handed out in order and every
// item depends only on items with smaller tickets, held by CTAs that are running, so the
// waits end (they are bounded all the same: on expiry the CTA sets the status word,
// counts the item as done without computing it, and the records carry FT_FLAG_TIMEOUT).
// The CTA that finishes the last tile of a pair's last level merges and solves that
// pair (one warp per level).
#pragma once

#include "tma.cuh"
#include "ttc_pass.cuh"
#include "ttc_merge.cuh"

namespace ttc_levels {

using namespace ttc_pass;
using namespace ttc_merge;

constexpr int MAXL = FT_MAX_LEVELS;

struct LevelsParams {
    // video (VIDEO = true): one descriptor per level, pair p at prev + p * pair_stride;
    // pair p's first frame is written by pair p - 1.  Batch: descriptor [level][pair]
    // (row stride desc_stride) and a (pair, tile) table for the items.
    PassParams lvl[MAXL];
    const PassParams *descs;
    int desc_stride;
    const int2 *items;        // batch: item t - begin[1] -> (pair, tile)
    int ntiles[MAXL];         // video: tiles per pair at each level
    int levels, npairs;
    int begin[MAXL + 1];      // first ticket of level l (l >= 1); begin[levels] = total
    int rpw[MAXL];            // tile rows per warp at each level (8 or 2)
    int *tickets;             // [0]: next ticket (zero before the launch)
    int *done;                // [level][npairs]: finished tiles (zero before the launch)
    int *status;              // set when a wait gives up
    // merge + solve (solve = 0: the caller solves with a separate launch)
    int solve, mode, skip;
    const float *partials;
    int64_t poff[MAXL];       // video: level-l partials start here ([pair][tile][NSUM])
    double inv_scale[MAXL];   // video
    int64_t ncubes[MAXL];     // video
    const void *sdesc;        // batch: per (pair, level) solve descriptors
    ttc_level_result *out;
};

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// bounded wait until *ctr >= need; false when the clock limit passed or the status word
// says an earlier wait gave up
__device__ __forceinline__ bool wait_count(const int *ctr, int need, const int *status)
{
    const long long t0 = clock64();
    while (ld_acquire(ctr) < need) {
        if (*reinterpret_cast<const volatile int *>(status)) return false;
        if (clock64() - t0 > ft_tma::WAIT_CYCLES) return false;
        __nanosleep(100);
    }
    return true;
}

// One tile of level l, reduced to its ten partials at dst: interior tiles read only
// inside the image (VAR 0); edge tiles of padded images (the context's own) shift
// inwards and mask (VAR 1); other edge tiles check every load (VAR 2).  A call, not
// inlined, one per variant: each gets the registers of a standalone pass kernel, and the
// persistent loop's state stays out of them.
#ifndef FT_LEVEL_TILE_CALL
#define FT_LEVEL_TILE_CALL 1    // 0: tile bodies inlined into the persistent loop
#endif
#if FT_LEVEL_TILE_CALL
#define FT_LEVEL_TILE_ATTR __noinline__
#else
#define FT_LEVEL_TILE_ATTR __forceinline__
#endif

template <typename Tin, int RPW, int VAR, bool CG>
__device__ FT_LEVEL_TILE_ATTR void level_tile(const PassParams &p, int pair, int ty, int tx, float *red, float *dst)
{
    constexpr int TRL = 8 * RPW;
    const int ilo = ty * TRL, jlo = tx * TC;
    const int ihi = min(ilo + TRL, p.H - 1), jhi = min(jlo + TC, p.W - 1);
    const Tin *fa = reinterpret_cast<const Tin *>(p.prev + (int64_t)pair * p.pair_stride);
    const Tin *fb = reinterpret_cast<const Tin *>(p.cur + (int64_t)pair * p.pair_stride);
    float2 acc2[NSUM];
#pragma unroll
    for (int s = 0; s < NSUM; ++s) acc2[s] = make_float2(0.f, 0.f);
    if (VAR == 0) {
        pass_body<Tin, Tin, false, false, false, true, RPW, CG>(p, fa, fb, pair, ilo, jlo, ilo, ihi, jlo, jhi, acc2);
    } else if (VAR == 1) {
        const int R0 = min(ilo, (p.H - 1 - TRL + 1) & ~1);
        const int C0 = min(jlo, (p.W - 1 - TC + 3) & ~3);
        pass_body<Tin, Tin, false, false, true, true, RPW, CG>(p, fa, fb, pair, R0, C0, ilo, ihi, jlo, jhi, acc2);
    } else {
        pass_body<Tin, Tin, true, true, true, true, RPW, CG>(p, fa, fb, pair, ilo, jlo, ilo, ihi, jlo, jhi, acc2);
    }
    float acc[NSUM];
#pragma unroll
    for (int s = 0; s < NSUM; ++s) acc[s] = acc2[s].x + acc2[s].y;
    block_reduce(acc, red, dst);
}

// CG: the level's images were written by this launch (levels >= 2): loads from L2.
// Level 1 was written by the level-0 launch before, and reads through L1.
template <typename Tin, int RPW, bool CG>
__device__ __forceinline__ void level_tile_any(const PassParams &p, int pair, int ty, int tx, float *red, float *dst)
{
    constexpr int TRL = 8 * RPW;
    const bool big = p.H >= TRL + 2 && p.W >= TC + 4;
    const bool edge = ty == p.tiles_y - 1 || tx == p.tiles_x - 1;
    if (!edge && big) level_tile<Tin, RPW, 0, CG>(p, pair, ty, tx, red, dst);
    else if (p.padded && big) level_tile<Tin, RPW, 1, CG>(p, pair, ty, tx, red, dst);
    else level_tile<Tin, RPW, 2, CG>(p, pair, ty, tx, red, dst);
}

// the pair's every level is done: merge and solve, one warp per level (a call, not
// inlined, for the same reason as level_tile)
template <bool VIDEO>
__device__ __noinline__ void solve_pair(const LevelsParams &lp, int pair)
{
    const int w = threadIdx.x >> 5;
    if (w >= lp.levels || pair < lp.skip) return;
    if (VIDEO) {
        merge_solve_cg(lp.partials + lp.poff[w] + (int64_t)pair * lp.ntiles[w] * NSUM, lp.ntiles[w], w,
                       lp.inv_scale[w], lp.ncubes[w], lp.mode, lp.status, lp.out + (int64_t)pair * lp.levels + w);
    } else {
        const SolveDesc &d = static_cast<const SolveDesc *>(lp.sdesc)[(int64_t)pair * lp.levels + w];
        merge_solve_cg(lp.partials + d.poff, d.ntiles, d.level, ldexp(1.0, -4 - 4 * d.level - d.shift), d.ncubes,
                       lp.mode, lp.status, lp.out + (int64_t)pair * lp.levels + w);
    }
}

template <typename Tin, bool VIDEO>
__global__ void __launch_bounds__(NT, FT_TTC_MINB)
ttc_levels_kernel(const __grid_constant__ LevelsParams lp)
{
    __shared__ float red[NSUM * NT];
    __shared__ int sh_t, sh_last, sh_ok;
    const int tid = threadIdx.x;
    const int total = lp.begin[lp.levels];
    if (tid == 0) sh_t = atomicAdd(lp.tickets, 1);
    __syncthreads();
    int t = sh_t;
    while (t < total) {
        // the next ticket, fetched while this item runs
        int tn = 0;
        if (tid == 0) tn = atomicAdd(lp.tickets, 1);
        int l = 1;
        while (l + 1 < lp.levels && t >= lp.begin[l + 1]) ++l;
        const int local = t - lp.begin[l];
        int pair, tile;
        if (VIDEO) {
            pair = local / lp.ntiles[l];
            tile = local - pair * lp.ntiles[l];
        } else {
            const int2 it = __ldg(lp.items + (t - lp.begin[1]));
            pair = it.x;
            tile = it.y;
        }
        const PassParams &p = VIDEO ? lp.lvl[l] : lp.descs[(int64_t)l * lp.desc_stride + pair];
        const int dpair = VIDEO ? pair : 0;          // pair index within the descriptor
        // the images of this level are complete once the level before has finished this
        // pair (and, in a video, the pair before, which wrote this pair's first frame)
        if (tid == 0) {
            bool ok = true;
            if (l >= 2) {
                const int *dprev = lp.done + (int64_t)(l - 1) * lp.npairs;
                const int need = VIDEO ? lp.ntiles[l - 1]
                                       : lp.descs[(int64_t)(l - 1) * lp.desc_stride + pair].ntiles;
                ok = wait_count(dprev + pair, need, lp.status);
                if (ok && VIDEO && pair > 0) ok = wait_count(dprev + pair - 1, need, lp.status);
                if (!ok) atomicExch(lp.status, 1);
            }
            sh_ok = ok;
        }
        // the acquire loads of thread 0 and this barrier order every later read of the
        // CTA after the writes the counts stand for
        __syncthreads();
        if (sh_ok) {
            const int ty = tile / p.tiles_x, tx = tile - ty * p.tiles_x;
            float *dst = p.partials + ((int64_t)dpair * p.ntiles + tile) * NSUM;
            if (l == 1) {
                if (lp.rpw[l] == 8) level_tile_any<Tin, 8, false>(p, dpair, ty, tx, red, dst);
                else level_tile_any<Tin, 2, false>(p, dpair, ty, tx, red, dst);
            } else {
                if (lp.rpw[l] == 8) level_tile_any<Tin, 8, true>(p, dpair, ty, tx, red, dst);
                else level_tile_any<Tin, 2, true>(p, dpair, ty, tx, red, dst);
            }
        }
        // every write of this item (next-level pixels, partials) before the count: the
        // barrier, then one thread's device-scope fence (cumulative over the writes the
        // barrier ordered before it) and the count
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            const int old = atomicAdd(lp.done + (int64_t)l * lp.npairs + pair, 1);
            sh_last = lp.solve && l == lp.levels - 1 && old + 1 == p.ntiles;
            // the pair's last count: every other item's writes are visible from here on
            if (sh_last) __threadfence();
            sh_t = tn;
        }
        __syncthreads();
        if (sh_last) solve_pair<VIDEO>(lp, pair);
        t = sh_t;
    }
}

}  // namespace ttc_levels
