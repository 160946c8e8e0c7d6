// batched.h -- plain (host and device) description of a batch of uneven 3D
// DFTs executed by one persistent launch (k_batched).
#pragma once

#include <stdint.h>

#include "geom.h"

namespace fft3 {

constexpr int kBatchMaxLine = 128; // longest line of a batched problem

enum BatchDecomp { BD_SLAB = 0, BD_PPP = 1 };

struct BatchCube {
    int64_t off;    // complex offset of the problem in `in` and `out`
    int n0, n1, n2;
    int lx, ly, lz; // indices of the x, y, z line plans in the LineRt table
    int decomp;     // BD_SLAB: 2D slabs then z lines; BD_PPP: x, y, z lines
    int nph;        // phases (2 or 3)
    int items[3];   // work items of each phase
    int lpt;        // columns per tile of the z phase
    int lpty;       // columns per tile of the y phase (pencil-pencil-pencil)
    int spi;        // slabs (BD_SLAB) or rows (BD_PPP) per phase-0 item
    int zpi;        // the slab executor: z tiles per z item
};

struct BatchItem {
    int cube, phase, index, pad;
};

struct BatchArgs {
    const float2 *in;
    float2 *out;
    const BatchCube *cubes;
    const BatchItem *items;
    int nitems;
    const LineRt *lines; // tw_off of each line plan indexes `tw`
    const float2 *tw;
    int *counters;       // [0] ticket; [1 + 3*cube + phase] finished items
    unsigned *err;
    long long wait_budget;
    int conj;
    int buf_elems;       // complex elements of each of the shared buffers
    int prefetch;        // 1: a third buffer stages the next item's first tile (cp.async)
};

// One launch of the segmented passes (k_segmented.cu): the lines of one
// length along dimension `dim` of the listed problems, LPT lines per tile.
struct SegArgs {
    const float2 *src;     // input of this pass (`in` for the x pass, `out` after)
    float2 *out;
    const BatchCube *cubes;
    const int *list;       // problem index of each listed slot
    const int64_t *tstart; // first tile of each slot
    const int *tcube;      // slot of every tile
    int64_t ntiles;
    int dim;               // 0: x lines (contiguous), 1: y lines, 2: z lines
    const float2 *tw;      // the line plan's twiddle table, tw_len entries
    int tw_len;
    int conj;
};

// One segment of the one-launch segmented executor (k_seg_all): the tiles of
// one line length along one dimension of the problems of one wave.
struct SegAllSeg {
    int64_t tile0;      // first tile of the segment within its step
    int64_t list_off, tstart_off, tcube_off; // offsets into the problem list, first-tile and slot tables
    int kidx;           // line kernel: 0 .. kSegLens-1 contiguous (x), kSegLens .. 2 kSegLens-1 strided (y, z)
    int dim;
    int tw_off;         // offset of the line's twiddle table in the block's shared copy
    int pad;
};

// The whole batch in one cooperative launch: steps separated by grid
// barriers; step s holds segments seg0[s] .. seg0[s+1]-1 and ntiles[s] tiles.
struct SegAllArgs {
    const float2 *in;
    float2 *out;
    const BatchCube *cubes;
    const int *list;
    const int64_t *tstart;
    const int *tcube;
    const SegAllSeg *segs;
    const int *seg0;
    const int64_t *ntiles;
    int nsteps;
    const float2 *tw;   // every line kernel's twiddle table, tw_len entries (copied to shared memory)
    int tw_len;
    int *barrier;       // grid-barrier arrivals (zero at launch)
    unsigned *err;
    long long wait_budget;
    int conj;
};

constexpr int kSegAllThreads = 256;

// The slab-by-slab executor (k_slabz.cu): the item executor's tables, and
// twiddle tables read through L1: tw_z[k] the offset of the table of the
// k-th plan of FFT3_SLABZ_Z_PLANS (z tiles), tw_w[k] that of the table w_N^m
// of the k-th length of FFT3_SLABZ_WARP_PLANS (rows and columns).
struct SlabZArgs {
    BatchArgs b;
    const float2 *tw;
    int tw_len;
    int tw_z[16];
    int tw_w[16];
};
__global__ void k_slabz(SlabZArgs z);
int slabz_smem_bytes(int buf_elems);

} // namespace fft3
