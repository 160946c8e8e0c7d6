// seg_plans.h -- compile-time line plans of the segmented batched passes
// (k_segmented.cu): for each line length of the batched workloads, the
// threads per line T, the lines per tile of the contiguous (x) and strided
// (y, z) kernels, and the radix list (Stockham stages, Section 2.1 Eq. ct).
#pragma once

#include "plans.h"

namespace fft3 {

// X(N, T, lines (x) or columns (y, z) per tile, radices...).  Two stages
// where the length allows (each stage is a round trip through shared memory;
// three-stage lists and lists chosen for 32-byte-aligned first-stage runs
// measured slower on the contiguous x lines).  Strided y and z lines: coalescing
// is across the tile's columns, so the lists keep registers low and threads busy.
#define FFT3_SEG_PLANS_CONTIG(X) \
    X(8, 1, 256, 8)              \
    X(16, 4, 64, 4, 4)           \
    X(24, 4, 64, 8, 3)           \
    X(32, 4, 64, 8, 4)           \
    X(40, 5, 32, 8, 5)           \
    X(48, 4, 64, 16, 3)          \
    X(64, 8, 32, 8, 8)           \
    X(80, 5, 32, 16, 5)          \
    X(96, 6, 32, 16, 2, 3)       \
    X(128, 8, 32, 16, 8)

#define FFT3_SEG_PLANS_STRIDED(X) \
    X(8, 1, 64, 8)                \
    X(16, 4, 32, 4, 4)            \
    X(24, 4, 32, 8, 3)            \
    X(32, 4, 32, 8, 4)            \
    X(40, 5, 32, 8, 5)            \
    X(48, 4, 32, 16, 3)           \
    X(64, 8, 32, 8, 8)            \
    X(80, 5, 32, 16, 5)           \
    X(96, 8, 32, 4, 8, 3)         \
    X(128, 8, 32, 16, 8)

// Contiguous (x) lines by the warp-shuffle line transform (warp_fft.cuh):
// X(N, R, L, D) with N = R * L, L / 2 lanes per line, 256-thread blocks of
// 512 / L lines and no shared memory.  D = 1 marks the default kernel of a
// length (the faster of its rows and the shared-memory kernel, timed on the
// 4096-cube workload's x lengths: 0.45-0.48 ms against 0.49-0.58 ms per
// 48 Mi-value batch); lengths without one keep the shared-memory kernel (64
// and 128 points, where it measured 1% faster).  Each length's first row is
// its faster warp-shuffle kernel.
#define FFT3_SEGW_PLANS(X) \
    X(8, 4, 2, 1)           \
    X(16, 4, 4, 1)          \
    X(16, 8, 2, 0)          \
    X(24, 3, 8, 1)          \
    X(24, 6, 4, 0)          \
    X(32, 4, 8, 1)          \
    X(32, 8, 4, 0)          \
    X(40, 10, 4, 1)         \
    X(40, 5, 8, 0)          \
    X(48, 6, 8, 1)          \
    X(48, 12, 4, 0)         \
    X(64, 8, 8, 0)          \
    X(64, 16, 4, 0)         \
    X(80, 10, 8, 1)         \
    X(80, 5, 16, 0)         \
    X(96, 6, 16, 1)         \
    X(96, 12, 8, 0)         \
    X(128, 8, 16, 0)        \
    X(128, 16, 8, 0)        \
    X(64, 4, 16, 0)         \
    X(128, 4, 32, 0)

// Rows and columns of the slab executor (k_slabz.cu) by the warp-shuffle
// transform: X(N, R, L), one variant per length, each within the 80 registers
// of three 256-thread blocks per multiprocessor.  The host derives the
// executor's line lengths and twiddle tables from the same list.
#define FFT3_SLABZ_WARP_PLANS(X) \
    X(8, 4, 2)                   \
    X(16, 4, 4)                  \
    X(24, 3, 8)                  \
    X(32, 4, 8)                  \
    X(40, 5, 8)                  \
    X(48, 6, 8)                  \
    X(64, 4, 16)                 \
    X(80, 5, 16)                 \
    X(96, 6, 16)                 \
    X(128, 4, 32)

// z tiles of the slab executor (k_slabz.cu): X(N, T, columns per tile,
// radices...), shared-memory column tiles like FFT3_SEG_PLANS_STRIDED, with T
// times the tile width chosen so that whole tiles fill 240-256 of the block's
// 256 threads, and two stages where the length allows (80 = 8 x 10 and
// 96 = 8 x 12, composite butterflies in registers).
#define FFT3_SLABZ_Z_PLANS(X) \
    X(8, 1, 64, 8)            \
    X(16, 4, 32, 4, 4)        \
    X(24, 4, 32, 8, 3)        \
    X(32, 4, 32, 8, 4)        \
    X(40, 5, 16, 8, 5)        \
    X(48, 4, 32, 16, 3)       \
    X(64, 8, 32, 8, 8)        \
    X(80, 10, 24, 8, 10)      \
    X(96, 12, 20, 8, 12)      \
    X(128, 8, 32, 16, 8)

// y and z lines (columns) by the warp-shuffle transform, the same rows.  None
// is a default: on the 4096-cube workload they measured slower than the
// shared-memory column kernels at 24-128 points (by 0-45%; within 3-9% faster
// at 16 and 40 points), so they run only when a tuning code asks for them.
#define FFT3_SEGW_PLANS_STRIDED(X) \
    X(8, 4, 2, 0)                   \
    X(16, 4, 4, 0)                  \
    X(16, 8, 2, 0)                  \
    X(24, 3, 8, 0)                  \
    X(24, 6, 4, 0)                  \
    X(32, 4, 8, 0)                  \
    X(32, 8, 4, 0)                  \
    X(40, 10, 4, 0)                 \
    X(40, 5, 8, 0)                  \
    X(48, 6, 8, 0)                  \
    X(48, 12, 4, 0)                 \
    X(64, 8, 8, 0)                  \
    X(64, 16, 4, 0)                 \
    X(80, 10, 8, 0)                 \
    X(80, 5, 16, 0)                 \
    X(96, 6, 16, 0)                 \
    X(96, 12, 8, 0)                 \
    X(128, 8, 16, 0)                \
    X(128, 16, 8, 0)

struct SegKernel {
    int n, T, lpt, nrad;
    int rad[4];
    const void *func;
    int warp; // 1: warp-shuffle kernel, T = lanes per line, rad = {R, L}, twiddles w_n^m (m < n)
    int dflt; // warp-shuffle kernel that is the default for its length
};

// The compiled lists (device translation unit) and their sizes.
const SegKernel *seg_kernels(bool contiguous, int *count);
const SegKernel *segw_kernels(int *count, bool contiguous = true);

// The one-launch executor (k_seg_all): its line kernel kidx is the index in
// the contiguous list, or the count of that list plus the index in the
// strided list; dynamic shared memory for a twiddle table of tw_len entries.
__global__ void k_seg_all(struct SegAllArgs a);
int seg_all_smem_bytes(int tw_len);

} // namespace fft3
