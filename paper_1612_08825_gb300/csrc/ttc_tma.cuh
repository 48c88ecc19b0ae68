// Level-0 pass for uint8 frames with tiles delivered by the Tensor Memory Accelerator.
//
// The results of ttc_pass_kernel (Sec. II stencil, Sec. V-A G and sums, Sec. V-B
// next pyramid level; partial sums 2^16 times larger, bit for bit otherwise), with its
// own arithmetic and data movement: the kernel is persistent (a CTA
// walks tiles t = blockIdx.x, blockIdx.x + gridDim.x, ...) and one elected thread
// brings the next tile of both frames into shared memory with cp.async.bulk.tensor
// while the CTA computes the current one (two buffers, completion tracked by an
// mbarrier with an expected byte count).  A tile of 64 x 256 cubes needs 65 pixel
// rows x 257 columns of each frame; they arrive as two 128-column boxes and one
// 16-column box per frame.  Pixels outside the frame are zero-filled by the copy
// engine, so edge tiles need no bounds checks (their cubes outside the frame are
// masked).  Pixels enter the arithmetic scaled by 256 (see b256), which keeps every
// stencil value exact without removing a bias.  Every wait is bounded by a clock limit: on expiry the CTA sets a status
// word (reported by the merge kernel as FT_FLAG_TIMEOUT), waits a bounded time for
// its copies in flight, and returns.
#pragma once

#include "tma.cuh"
#include "ttc_pass.cuh"

namespace ttc_tma {

using namespace ttc_pass;

constexpr int ROWS = TR + 1;                              // pixel rows per tile
constexpr int BW = 128;                                   // main box width (bytes)
constexpr int XW = 16;                                    // extra box: columns 256..271
constexpr int BOX = ROWS * BW;                            // 8320 B
constexpr int XBOX = ROWS * XW;                           // 1040 B
constexpr int XBOX_PAD = (XBOX + 127) / 128 * 128;        // 1152 B
constexpr int FRAME = 2 * BOX + XBOX_PAD;                 // 17792 B, 128-B multiple
constexpr int BUF = 2 * FRAME;                            // both frames
constexpr unsigned TX = 2u * (2u * BOX + XBOX);           // bytes the copies deliver per tile

// A batch tile's descriptor and origin, written to shared memory by the thread that
// issues the tile's copies (before its arrive on the tile's barrier, whose completion
// the consumers wait for), so that the CTA reads them from there rather than every
// thread from global memory.
struct TileInfo {
    PassParams p;
    int pair, tile, R0, C0;
};

// two buffers, the reduction scratch, two barriers, two tile descriptors
constexpr int SMEM = 2 * BUF + NSUM * NT * 4 + 2 * 8 + 2 * (int)sizeof(TileInfo);

using namespace ft_tma;

// Where a work item's tile is: the pair's descriptor and tensor maps, the pair's index
// in that descriptor (frames of a video share one descriptor), and the tile's origin.
struct Loc {
    const PassParams *p;
    const CUtensorMap *m;       // four maps: prev main, cur main, prev extra, cur extra
    int z;                      // pair coordinate of the maps
    int pair;                   // pair index within the descriptor
    int tile, R0, C0;
};

// A video (or single pair): one descriptor and one set of maps for all pairs, the
// pair being the maps' third coordinate; items numbered pair-major.
struct VideoItems {
    CUtensorMap m[4];
    PassParams p;
    int total;                  // npairs * ntiles
    __device__ __forceinline__ void locate(int t, Loc &l) const
    {
        const int pair = t / p.ntiles, tile = t - pair * p.ntiles;
        const int ty = tile / p.tiles_x, tx = tile - ty * p.tiles_x;
        l.p = &p;
        l.m = m;
        l.z = pair;
        l.pair = pair;
        l.tile = tile;
        l.R0 = ty * TR;
        l.C0 = tx * TC;
    }
};

// A batch of independent pairs: pair j has its own descriptor and four maps in global
// memory (written before the launch); item t is tile items[t].y of pair items[t].x.
struct BatchItems {
    const PassParams *descs;
    const CUtensorMap *maps;
    const int2 *items;
    int total;
    __device__ __forceinline__ void locate(int t, Loc &l) const
    {
        const int2 it = __ldg(items + t);
        const PassParams *p = descs + it.x;
        const int tiles_x = p->tiles_x;
        const int ty = it.y / tiles_x, tx = it.y - ty * tiles_x;
        l.p = p;
        l.m = maps + 4 * (int64_t)it.x;
        l.z = 0;
        l.pair = 0;
        l.tile = it.y;
        l.R0 = ty * TR;
        l.C0 = tx * TC;
    }
};

// maps in global memory are read by the tensor-map proxy: order the earlier writes
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap *m)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(m))
                 : "memory");
}

// elected thread: copies of one tile of both frames into buffer `buf` (and, for a batch,
// the tile's descriptor into `info`)
template <bool GLOBAL_MAPS>
__device__ __forceinline__ void issue_tile(const Loc &l, unsigned extra_tx, unsigned char *buf, uint64_t *bar,
                                           TileInfo *info)
{
    if (GLOBAL_MAPS) {
        for (int k = 0; k < 4; ++k) tensormap_acquire(l.m + k);
        info->p = *l.p;
        info->pair = l.pair;
        info->tile = l.tile;
        info->R0 = l.R0;
        info->C0 = l.C0;
    }
    // generic-proxy reads of this buffer (previous tile) are ordered before the async writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, TX + extra_tx);
    tma_load_3d(buf, l.m + 0, l.C0, l.R0, l.z, bar);
    tma_load_3d(buf + BOX, l.m + 0, l.C0 + BW, l.R0, l.z, bar);
    tma_load_3d(buf + 2 * BOX, l.m + 2, l.C0 + 2 * BW, l.R0, l.z, bar);
    tma_load_3d(buf + FRAME, l.m + 1, l.C0, l.R0, l.z, bar);
    tma_load_3d(buf + FRAME + BOX, l.m + 1, l.C0 + BW, l.R0, l.z, bar);
    tma_load_3d(buf + FRAME + 2 * BOX, l.m + 3, l.C0 + 2 * BW, l.R0, l.z, bar);
}

// ---------------------------------------------------------------------------
// uint8 pixels scaled by 256: byte k of w becomes the float 2^23 + 256 v (v in the
// second mantissa byte).  Then s = A + B = 2^24 + 256 (a + b) and every later sum and
// difference of the stencil are multiples of 256 below 2^26, so they stay exact with
// no bias to remove; the stencil values are 256 times the unscaled ones, the ten
// products 2^16 times (removed in FP64 by the merge kernel).
// ---------------------------------------------------------------------------

__device__ __forceinline__ float b256(uint32_t w, uint32_t k)
{
    return __int_as_float(__byte_perm(w, 0x4B000000u, 0x7604u | (k << 4)));
}

// raw bytes of one row of both frames: 4 columns in each half, and the right
// neighbour of lane 31's columns in byte 0 of xa / xb (column 256 of the tile: the
// first column of the extra box).  Folded tiles (see tile_body) pair row i with row
// i + 32 of the same columns instead; lane 31's neighbours are then column 128 of those
// two rows (bytes 0 and 1 of xa / xb).
struct Raw8 {
    uint32_t al, ar, bl, br, xa, xb;
};

// one row of both frames for this thread, from the tile buffer (pixel row `row`)
template <bool FOLD>
__device__ __forceinline__ void row_from_smem(const unsigned char *buf, int row, int lane, Raw8 &r)
{
    const unsigned char *fa = buf, *fb = buf + FRAME;
    r.al = *reinterpret_cast<const uint32_t *>(fa + row * BW + 4 * lane);
    r.bl = *reinterpret_cast<const uint32_t *>(fb + row * BW + 4 * lane);
    if (FOLD) {
        r.ar = *reinterpret_cast<const uint32_t *>(fa + (row + 32) * BW + 4 * lane);
        r.br = *reinterpret_cast<const uint32_t *>(fb + (row + 32) * BW + 4 * lane);
        const uint32_t a0 = *reinterpret_cast<const uint32_t *>(fa + BOX + row * BW);
        const uint32_t a1 = *reinterpret_cast<const uint32_t *>(fa + BOX + (row + 32) * BW);
        const uint32_t b0 = *reinterpret_cast<const uint32_t *>(fb + BOX + row * BW);
        const uint32_t b1 = *reinterpret_cast<const uint32_t *>(fb + BOX + (row + 32) * BW);
        r.xa = __byte_perm(a0, a1, 0x0040u);
        r.xb = __byte_perm(b0, b1, 0x0040u);
    } else {
        r.ar = *reinterpret_cast<const uint32_t *>(fa + BOX + row * BW + 4 * lane);
        r.br = *reinterpret_cast<const uint32_t *>(fb + BOX + row * BW + 4 * lane);
        r.xa = *reinterpret_cast<const uint32_t *>(fa + 2 * BOX + row * XW);
        r.xb = *reinterpret_cast<const uint32_t *>(fb + 2 * BOX + row * XW);
    }
}

// The previous row's contribution to the cubes between it and the next row, per
// cube column k of the thread (0..3, as (left, right) pairs): hs = s[k+1] - s[k],
// hp = s[k+1] + s[k], dp = d[k+1] + d[k] (s = prev + cur, d = cur - prev).
struct Strip8 {
    float2 hs[4], hp[4], dp[4];
};

// One row step: the cubes between the previous row and this one,
//   Ex = hs(i) + hs(i+1),  Ey = hp(i+1) - hp(i),  Et = dp(i) + dp(i+1)
// (the 2x2x2 first differences of Sec. II, times 4 * 256), G and the ten products.
// The neighbour column's s and d come from lane+1 (lane 31 of the right half: the
// extra box).  Returns the row's scaled pixels of both frames for the pyramid.
template <bool MASK, bool FOLD>
__device__ __forceinline__ void row_step8(const Raw8 &r, int lane, Strip8 &st, bool first, const float2 xk[4],
                                          float2 y, bool rowok_l, bool rowok_r, int jl, int jr, int jlo, int jhi,
                                          float2 acc[NSUM], float2 A[4], float2 B[4])
{
    float2 s[5], d[5];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        A[k] = make_float2(b256(r.al, k), b256(r.ar, k));
        B[k] = make_float2(b256(r.bl, k), b256(r.br, k));
        s[k] = add2(A[k], B[k]);
        d[k] = sub2(B[k], A[k]);
    }
    const int src = (lane + 1) & 31;
    const float s4l = __shfl_sync(0xffffffffu, lane == 0 ? s[0].y : s[0].x, src);
    const float d4l = __shfl_sync(0xffffffffu, lane == 0 ? d[0].y : d[0].x, src);
    const float s4r = __shfl_sync(0xffffffffu, s[0].y, src);
    const float d4r = __shfl_sync(0xffffffffu, d[0].y, src);
    const float xa = b256(r.xa, 0), xb = b256(r.xb, 0);
    if (FOLD) {
        const float xa1 = b256(r.xa, 1), xb1 = b256(r.xb, 1);
        s[4] = make_float2(lane == 31 ? xa + xb : s4l, lane == 31 ? xa1 + xb1 : s4r);
        d[4] = make_float2(lane == 31 ? xb - xa : d4l, lane == 31 ? xb1 - xa1 : d4r);
    } else {
        s[4] = make_float2(s4l, lane == 31 ? xa + xb : s4r);
        d[4] = make_float2(d4l, lane == 31 ? xb - xa : d4r);
    }
    float2 hs[4], hp[4], dp[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        hs[k] = sub2(s[k + 1], s[k]);
        hp[k] = add2(s[k + 1], s[k]);
        dp[k] = add2(d[k + 1], d[k]);
    }
    if (!first) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float2 ex = add2(hs[k], st.hs[k]);
            float2 ey = sub2(hp[k], st.hp[k]);
            float2 et = add2(dp[k], st.dp[k]);
            if (MASK) {
                const int cl = jl + k, cr = jr + k;
                mask3(ex, ey, et, rowok_l && cl >= jlo && cl < jhi, rowok_r && cr >= jlo && cr < jhi);
            }
            accum2(acc, ex, ey, et, xk[k], y);
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        st.hs[k] = hs[k];
        st.hp[k] = hp[k];
        st.dp[k] = dp[k];
    }
}

// level-(l+1) pixels of a 2x2 block of scaled pixels: v = 2^25 + 256 sum; the uint16
// value is the low half of the float 2^23 + sum = v / 256 + (2^23 - 2^17)
__device__ __forceinline__ float2 unscale_block(float2 v)
{
    return fma2(v, make_float2(0.00390625f, 0.00390625f), make_float2(8257536.f, 8257536.f));
}

template <bool EDGE>
__device__ __forceinline__ void store_u16(const PassParams &p, unsigned char *img, int64_t pitch, int r1, int c,
                                          float t0, float t1, int Hn, int Wn)
{
    if (EDGE && (r1 >= Hn || c >= Wn)) return;
    const bool two = !EDGE || c + 1 < Wn;
    unsigned short *row = reinterpret_cast<unsigned short *>(img + (int64_t)r1 * pitch);
    if (FT_CHECK && !in_extent(p, img, row + c, two ? 4 : 2, p.next_bytes)) return;
    const uint32_t lo = __float_as_uint(t0) & 0xffffu, hi = __float_as_uint(t1) << 16;
    if (two) *reinterpret_cast<uint32_t *>(row + c) = lo | hi;
    else row[c] = (unsigned short)lo;
}

// One tile of 64 x 256 cubes.  A thread's packed pair of lanes normally holds the same
// 4 columns of the tile's left and right halves, and a warp walks 8 cube rows.  A tile
// whose cubes all lie in the left half (FOLD: the last, narrow tile column of an image)
// pairs each left-half row with the row 32 below it instead, so a warp walks 4 rows and
// the tile costs about half.
template <bool MASK, bool WRITE, bool FOLD>
__device__ __forceinline__ void tile_body(const PassParams &p, const unsigned char *buf, int pair, int R0, int C0,
                                          float2 acc[NSUM])
{
    constexpr int RPW = FOLD ? 4 : 8;           // cube rows per warp
    constexpr int DR = FOLD ? TR / 2 : 0;       // row offset of the pair's second lane
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gcl = C0 + 4 * lane;
    const int gcr = FOLD ? gcl : gcl + HALF;    // columns of the pair's second lane
    const int gr0 = R0 + RPW * warp;
    const float2 x0 = make_float2((float)gcl + p.xoff, (float)gcr + p.xoff);
    const int Hn = p.H >> 1, Wn = p.W >> 1;
    const int ihi = min(R0 + TR, p.H - 1), jhi = min(C0 + TC, p.W - 1);
    // consecutive pairs of a video share frames: the first frame's next level is written
    // by pair 0 only; independent pairs write both (write_prev 1) or only the second
    // (write_prev -1: the first frame's next level exists already)
    const bool wprev = WRITE && (p.write_prev == 1 || (p.write_prev == 0 && pair == 0));
    const int64_t fprev = p.write_prev == 1 ? 2 * (int64_t)pair : (int64_t)pair;
    unsigned char *nprev = wprev ? p.next + fprev * p.next_fstride : nullptr;
    unsigned char *ncur = WRITE ? (p.next_cur ? p.next_cur : p.next + (fprev + 1) * p.next_fstride) : nullptr;

    float2 xk[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) xk[k] = add2(x0, make_float2((float)k, (float)k));
    float2 y = make_float2((float)(gr0 - 1) + p.yoff, (float)(gr0 - 1 + DR) + p.yoff);
    Strip8 st;
    float2 hb[2], ha[2];            // horizontal pair sums of the even row (cur, prev)
    Raw8 nxt;
    row_from_smem<FOLD>(buf, RPW * warp, lane, nxt);
#pragma unroll
    for (int r = 0; r <= RPW; ++r) {
        const Raw8 cur = nxt;
        if (r < RPW) row_from_smem<FOLD>(buf, RPW * warp + r + 1, lane, nxt);
        float2 A[4], B[4];
        const int i = gr0 + r - 1;
        row_step8<MASK, FOLD>(cur, lane, st, r == 0, xk, y, i >= R0 && i < ihi, i + DR >= R0 && i + DR < ihi, gcl,
                              gcr, C0, jhi, acc, A, B);
        y = add2(y, make_float2(1.f, 1.f));
        if (WRITE && r < RPW) {
            const float2 b0 = add2(B[0], B[1]), b1 = add2(B[2], B[3]);
            float2 a0, a1;
            if (wprev) {
                a0 = add2(A[0], A[1]);
                a1 = add2(A[2], A[3]);
            }
            if ((r & 1) == 0) {
                hb[0] = b0;
                hb[1] = b1;
                if (wprev) {
                    ha[0] = a0;
                    ha[1] = a1;
                }
            } else {
                const int r1 = (gr0 >> 1) + (r >> 1), r2 = r1 + DR / 2;
                const int cl = gcl >> 1, cr = gcr >> 1;
                const float2 v0 = unscale_block(add2(hb[0], b0)), v1 = unscale_block(add2(hb[1], b1));
                store_u16<MASK>(p, ncur, p.next_pitch, r1, cl, v0.x, v1.x, Hn, Wn);
                store_u16<MASK>(p, ncur, p.next_pitch, r2, cr, v0.y, v1.y, Hn, Wn);
                if (wprev) {
                    const float2 u0 = unscale_block(add2(ha[0], a0)), u1 = unscale_block(add2(ha[1], a1));
                    store_u16<MASK>(p, nprev, p.next_pitch, r1, cl, u0.x, u1.x, Hn, Wn);
                    store_u16<MASK>(p, nprev, p.next_pitch, r2, cr, u0.y, u1.y, Hn, Wn);
                }
            }
        }
    }
}

template <bool WRITE, class Items, bool GLOBAL_MAPS>
__global__ void __launch_bounds__(NT, 2)
ttc_pass_tma_kernel(const __grid_constant__ Items items, int *status, unsigned extra_tx)
{
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *bufs = smem;
    float *red = reinterpret_cast<float *>(smem + 2 * BUF);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * BUF + NSUM * NT * 4);
    TileInfo *info = reinterpret_cast<TileInfo *>(smem + 2 * BUF + NSUM * NT * 4 + 2 * 8);
    const int tid = threadIdx.x;
    const int total = items.total;
    // the copy engine writes 128-byte aligned boxes; refuse (and report) otherwise
    if (smem_addr(bufs) & 127) {
        if (tid == 0) atomicExch(status, 2);
        return;
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int t0 = blockIdx.x;
    if (tid == 0 && t0 < total) {
        Loc l;
        items.locate(t0, l);
        issue_tile<GLOBAL_MAPS>(l, extra_tx, bufs, &bar[0], &info[0]);
    }

    int k = 0;
    for (int t = t0; t < total; t += gridDim.x, ++k) {
        const int b = k & 1;
        const int tn = t + gridDim.x;
        // the other buffer was released by the barrier inside the previous tile's reduction
        if (tid == 0 && tn < total) {
            Loc ln;
            items.locate(tn, ln);
            issue_tile<GLOBAL_MAPS>(ln, extra_tx, bufs + (b ^ 1) * BUF, &bar[b ^ 1], &info[b ^ 1]);
        }
        const bool ok = mbar_wait(&bar[b], (k >> 1) & 1);
        if (__syncthreads_or(!ok)) {
            // give up on this CTA: report, let the copies in flight land, return
            if (tid == 0) {
                atomicExch(status, 1);
                if (tn < total) mbar_wait(&bar[b ^ 1], ((k + 1) >> 1) & 1);
            }
            __syncthreads();
            return;
        }
        Loc l;
        if (GLOBAL_MAPS) {
            l.p = &info[b].p;
            l.pair = info[b].pair;
            l.tile = info[b].tile;
            l.R0 = info[b].R0;
            l.C0 = info[b].C0;
        } else {
            items.locate(t, l);
        }
        const PassParams &p = *l.p;
        float2 acc2[NSUM];
#pragma unroll
        for (int s = 0; s < NSUM; ++s) acc2[s] = make_float2(0.f, 0.f);
        const bool edge = (l.R0 + TR > p.H - 1) || (l.C0 + TC > p.W - 1);
        const bool fold = p.W - 1 - l.C0 <= HALF;          // every cube in the left half
        if (fold) tile_body<true, WRITE, true>(p, bufs + b * BUF, l.pair, l.R0, l.C0, acc2);
        else if (edge) tile_body<true, WRITE, false>(p, bufs + b * BUF, l.pair, l.R0, l.C0, acc2);
        else tile_body<false, WRITE, false>(p, bufs + b * BUF, l.pair, l.R0, l.C0, acc2);
        float acc[NSUM];
#pragma unroll
        for (int s = 0; s < NSUM; ++s) acc[s] = acc2[s].x + acc2[s].y;
        // no CTA barrier after the reduction: its own barrier (between the scratch writes
        // and reads) already follows every thread's reads of buffer b, which the next
        // tile's copy refills, and the next tile's barrier after its wait follows every
        // read of the scratch, which the next reduction rewrites.  The warp barrier keeps
        // the compiler from moving the next tile's code into this one (registers).
        block_reduce(acc, red, p.partials + ((int64_t)l.pair * p.ntiles + l.tile) * NSUM);
        __syncwarp();
    }
}

}  // namespace ttc_tma
