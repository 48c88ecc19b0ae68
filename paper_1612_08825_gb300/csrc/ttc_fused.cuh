// All pyramid levels of uint8 frame pairs in one persistent launch (Sec. II, V-A, V-B):
// the interface between the host code (ttc.cu) and the kernel (ttc_fused.cu).
//
// The kernel walks units: a unit is a run of consecutive tiles of one tile column (a
// strip) of one pair, taken top to bottom.  A tile is the 64 x 256-cube level-0 tile of
// the copy-engine pass; from the same shared-memory copy of both frames the CTA forms the
// level-1 pixels (2x2 block sums) into a ring of rows in shared memory, and from there the
// cubes and pixels of every coarser level: the tile owns the level-l cubes of rows
// 64j/2^l - 1 .. 64j/2^l + 64/2^l - 2 and columns 256tx/2^l .. 256(tx+1)/2^l - 1, so each
// level-l cube of the pair belongs to exactly one tile.  The one pixel row of each level
// that a tile needs from above its own level-0 rows is the last row the tile above left
// in the ring; a unit that starts below the top of its strip first runs a prologue that
// computes those rows from the 16 level-0 rows above it.  No level image is written to
// global memory (unless the caller asks for the second frame's pyramid).  Results per
// (pair, level, tile) do not depend on how the strips are cut into units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ttc_pass.cuh"

namespace ttc_fused {

constexpr int MAXLEV = 5;       // levels 0..4: uint16 block sums hold up to 255 * 4^4

// One pair's geometry and outputs.
struct Geom {
    int H, W;                   // level-0 frame size
    int tiles_x, tiles_y;       // level-0 tiles of 64 x 256 cubes; every level uses this grid
    int ntiles;
    int nlev;                   // levels 0 .. nlev-1, 2 <= nlev <= MAXLEV
    float xoff[MAXLEV];         // cube centre at level l: x = j + xoff[l], y = i + yoff[l]
    float yoff[MAXLEV];
    float *part[MAXLEV];        // level-l partials of this pair, [tile][NSUM]
    unsigned char *pyr;         // null, or the second frame's pyramid block (levels 1..nlev-1, uint16)
    int64_t pyr_off[MAXLEV];    // byte offset and row pitch of level l in that block
    int64_t pyr_pitch[MAXLEV];
};

// A video or a single pair: one geometry, the pair being the tensor maps' third
// coordinate and pair p's partials at part[l] + p * ntiles * NSUM.  Unit u: pair
// u / (tiles_x * nseg), then strip, then segment of `seg` tiles.
struct VideoUnits {
    CUtensorMap m[4];           // prev main, cur main, prev extra, cur extra
    Geom g;
    int npairs;
    int seg;                    // tiles per unit
    int nseg;                   // units per strip, ceil(tiles_y / seg)
    int total;                  // npairs * tiles_x * nseg
};

// A batch of pairs of any sizes: per-pair geometry and four tensor maps in global
// memory; unit u is units[u] = (pair, strip, first tile row, tiles).
struct BatchUnits {
    const Geom *geoms;
    const CUtensorMap *maps;
    const int4 *units;
    int total;
};

// Launch on `s` with a grid of two CTAs per SM.  status: the call's status word (bit 0:
// a wait gave up); counter: the unit ticket, zero before the launch.
cudaError_t launch_video(const VideoUnits &u, int *status, int *counter, cudaStream_t s);
cudaError_t launch_batch(const BatchUnits &u, int *status, int *counter, cudaStream_t s);

}  // namespace ttc_fused
