// Level-0 pass for uint8 frames with tiles delivered by the Tensor Memory Accelerator.
//
// Same arithmetic as ttc_pass_kernel (Sec. II stencil, Sec. V-A G and sums, Sec. V-B
// next pyramid level), different data movement: the kernel is persistent (a CTA
// walks tiles t = blockIdx.x, blockIdx.x + gridDim.x, ...) and one elected thread
// brings the next tile of both frames into shared memory with cp.async.bulk.tensor
// while the CTA computes the current one (two buffers, completion tracked by an
// mbarrier with an expected byte count).  A tile of 64 x 256 cubes needs 65 pixel
// rows x 257 columns of each frame; they arrive as two 128-column boxes and one
// 16-column box per frame.  Pixels outside the frame are zero-filled by the copy
// engine, so edge tiles need no bounds checks (their cubes outside the frame are
// masked).  Every wait is bounded by a clock limit: on expiry the CTA sets a status
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
constexpr int SMEM = 2 * BUF + NSUM * NT * 4 + 2 * 8;     // two buffers, reduction, barriers

struct TmaParams {
    PassParams p;               // geometry, partials, next level (prev/cur unused)
    int total;                  // npairs * ntiles
    int *status;                // set to 1 when a wait gives up
    unsigned extra_tx;          // added to the expected bytes (0; tests of the timeout path)
};

using namespace ft_tma;

// elected thread: copies of tile t of both frames into buffer `buf`
__device__ __forceinline__ void issue_tile(const TmaParams &tp, const CUtensorMap *ma, const CUtensorMap *mb,
                                           const CUtensorMap *xa, const CUtensorMap *xb, int t,
                                           unsigned char *buf, uint64_t *bar)
{
    const PassParams &p = tp.p;
    const int pair = t / p.ntiles, tile = t - pair * p.ntiles;
    const int ty = tile / p.tiles_x, tx = tile - ty * p.tiles_x;
    const int R0 = ty * TR, C0 = tx * TC;
    // generic-proxy reads of this buffer (previous tile) are ordered before the async writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, TX + tp.extra_tx);
    tma_load_3d(buf, ma, C0, R0, pair, bar);
    tma_load_3d(buf + BOX, ma, C0 + BW, R0, pair, bar);
    tma_load_3d(buf + 2 * BOX, xa, C0 + 2 * BW, R0, pair, bar);
    tma_load_3d(buf + FRAME, mb, C0, R0, pair, bar);
    tma_load_3d(buf + FRAME + BOX, mb, C0 + BW, R0, pair, bar);
    tma_load_3d(buf + FRAME + 2 * BOX, xb, C0 + 2 * BW, R0, pair, bar);
}

// one row of both frames for this thread, from the tile buffer (pixel row `row` of the tile)
__device__ __forceinline__ void row_from_smem(const unsigned char *buf, int row, int lane, RawRow<unsigned char> &r)
{
    const unsigned char *fa = buf, *fb = buf + FRAME;
    r.al = *reinterpret_cast<const uint32_t *>(fa + row * BW + 4 * lane);
    r.ar = *reinterpret_cast<const uint32_t *>(fa + BOX + row * BW + 4 * lane);
    r.bl = *reinterpret_cast<const uint32_t *>(fb + row * BW + 4 * lane);
    r.br = *reinterpret_cast<const uint32_t *>(fb + BOX + row * BW + 4 * lane);
    r.a4 = (float)fa[2 * BOX + row * XW];
    r.b4 = (float)fb[2 * BOX + row * XW];
}

template <bool MASK, bool WRITE>
__device__ __forceinline__ void tile_body(const PassParams &p, const unsigned char *buf, int pair, int R0, int C0,
                                          float2 acc[NSUM])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gcl = C0 + 4 * lane;
    const int gr0 = R0 + 8 * warp;
    const float2 x0 = make_float2((float)gcl + p.xoff, (float)(gcl + HALF) + p.xoff);
    const int Hn = p.H >> 1, Wn = p.W >> 1;
    const int ihi = min(R0 + TR, p.H - 1), jhi = min(C0 + TC, p.W - 1);
    const bool wprev = WRITE && (p.write_prev || pair == 0);
    const int64_t fprev = p.write_prev ? 2 * (int64_t)pair : (int64_t)pair;
    unsigned char *nprev = WRITE ? p.next + fprev * p.next_fstride : nullptr;
    unsigned char *ncur = WRITE ? nprev + p.next_fstride : nullptr;

    float2 xk[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) xk[k] = add2(x0, make_float2((float)k, (float)k));
    float2 y = make_float2((float)(gr0 - 1) + p.yoff, (float)(gr0 - 1) + p.yoff);
    Strip st;
    Pyr py;
    RawRow<unsigned char> nxt;
    row_from_smem(buf, 8 * warp, lane, nxt);
#pragma unroll
    for (int r = 0; r < 9; ++r) {
        const RawRow<unsigned char> cur = nxt;
        if (r < 8) row_from_smem(buf, 8 * warp + r + 1, lane, nxt);
        float2 A[4], D[4];
        const int i = gr0 + r - 1;
        row_step<unsigned char, MASK>(cur, lane, st, r == 0, xk, y, i >= R0 && i < ihi, gcl, gcl + HALF, C0, jhi,
                                      acc, A, D);
        y = add2(y, make_float2(1.f, 1.f));
        if (WRITE && r < 8) {
            if ((r & 1) == 0) {
                pyr_even(py, A, D);
            } else {
                float2 va0, va1, vb0, vb1;
                pyr_odd(py, A, D, va0, va1, vb0, vb1);
                const int r1 = (gr0 >> 1) + (r >> 1);
                const int cl = gcl >> 1, cr = (gcl + HALF) >> 1;
                store_next<unsigned short, MASK>(ncur, p.next_pitch, r1, cl, vb0.x, vb1.x, Hn, Wn);
                store_next<unsigned short, MASK>(ncur, p.next_pitch, r1, cr, vb0.y, vb1.y, Hn, Wn);
                if (wprev) {
                    store_next<unsigned short, MASK>(nprev, p.next_pitch, r1, cl, va0.x, va1.x, Hn, Wn);
                    store_next<unsigned short, MASK>(nprev, p.next_pitch, r1, cr, va0.y, va1.y, Hn, Wn);
                }
            }
        }
    }
}

template <bool WRITE>
__global__ void __launch_bounds__(NT, 2)
ttc_pass_tma_kernel(const __grid_constant__ CUtensorMap ma, const __grid_constant__ CUtensorMap mb,
                    const __grid_constant__ CUtensorMap xa, const __grid_constant__ CUtensorMap xb,
                    const TmaParams tp)
{
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *bufs = smem;
    float *red = reinterpret_cast<float *>(smem + 2 * BUF);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * BUF + NSUM * NT * 4);
    const PassParams &p = tp.p;
    const int tid = threadIdx.x;
    // the copy engine writes 128-byte aligned boxes; refuse (and report) otherwise
    if (smem_addr(bufs) & 127) {
        if (tid == 0) atomicExch(tp.status, 2);
        return;
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int t0 = blockIdx.x;
    if (tid == 0 && t0 < tp.total) issue_tile(tp, &ma, &mb, &xa, &xb, t0, bufs, &bar[0]);

    int k = 0;
    for (int t = t0; t < tp.total; t += gridDim.x, ++k) {
        const int b = k & 1;
        const int tn = t + gridDim.x;
        // the other buffer was released by the barrier inside the previous tile's reduction
        if (tid == 0 && tn < tp.total) issue_tile(tp, &ma, &mb, &xa, &xb, tn, bufs + (b ^ 1) * BUF, &bar[b ^ 1]);
        const bool ok = mbar_wait(&bar[b], (k >> 1) & 1);
        if (__syncthreads_or(!ok)) {
            // give up on this CTA: report, let the copies in flight land, return
            if (tid == 0) {
                atomicExch(tp.status, 1);
                if (tn < tp.total) mbar_wait(&bar[b ^ 1], ((k + 1) >> 1) & 1);
            }
            __syncthreads();
            return;
        }
        const int pair = t / p.ntiles, tile = t - pair * p.ntiles;
        const int ty = tile / p.tiles_x, tx = tile - ty * p.tiles_x;
        const int R0 = ty * TR, C0 = tx * TC;
        float2 acc2[NSUM];
#pragma unroll
        for (int s = 0; s < NSUM; ++s) acc2[s] = make_float2(0.f, 0.f);
        const bool edge = (R0 + TR > p.H - 1) || (C0 + TC > p.W - 1);
        if (edge) tile_body<true, WRITE>(p, bufs + b * BUF, pair, R0, C0, acc2);
        else tile_body<false, WRITE>(p, bufs + b * BUF, pair, R0, C0, acc2);
        float acc[NSUM];
#pragma unroll
        for (int s = 0; s < NSUM; ++s) acc[s] = acc2[s].x + acc2[s].y;
        // no CTA barrier after the reduction: its own barrier (between the scratch writes
        // and reads) already follows every thread's reads of buffer b, which the next
        // tile's copy refills, and the next tile's barrier after its wait follows every
        // read of the scratch, which the next reduction rewrites.  The warp barrier keeps
        // the compiler from moving the next tile's code into this one (registers).
        block_reduce(acc, red, p.partials + ((int64_t)pair * p.ntiles + tile) * NSUM);
        __syncwarp();
    }
}

}  // namespace ttc_tma
