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

struct SegKernel {
    int n, T, lpt, nrad;
    int rad[4];
    const void *func;
};

// The compiled lists (device translation unit) and their sizes.
const SegKernel *seg_kernels(bool contiguous, int *count);

// The one-launch executor (k_seg_all): its line kernel kidx is the index in
// the contiguous list, or the count of that list plus the index in the
// strided list; dynamic shared memory for a twiddle table of tw_len entries.
__global__ void k_seg_all(struct SegAllArgs a);
int seg_all_smem_bytes(int tw_len);

} // namespace fft3
