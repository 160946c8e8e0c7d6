// seg_plans.h -- compile-time line plans of the segmented batched passes
// (k_segmented.cu): for each line length of the batched workloads, the
// threads per line T, the lines per tile of the contiguous (x) and strided
// (y, z) kernels, and the radix list (Stockham stages, Section 2.1 Eq. ct).
#pragma once

#include "plans.h"

namespace fft3 {

// X(N, T, lines per contiguous tile, columns per strided tile, radices...)
#define FFT3_SEG_PLANS(X)                  \
    X(8, 1, 256, 64, 8)                    \
    X(16, 4, 64, 32, 4, 4)                 \
    X(24, 4, 64, 32, 8, 3)                 \
    X(32, 4, 64, 32, 8, 4)                 \
    X(40, 5, 32, 32, 8, 5)                 \
    X(48, 4, 64, 32, 16, 3)                \
    X(64, 8, 32, 32, 8, 8)                 \
    X(80, 5, 32, 32, 16, 5)                \
    X(96, 6, 32, 32, 16, 2, 3)             \
    X(128, 8, 32, 32, 16, 8)

struct SegKernel {
    int n, T, lpt_c, lpt_s, nrad;
    int rad[4];
    const void *func_c; // contiguous lines (x)
    const void *func_s; // strided lines (y, z)
};

// The compiled list (device translation unit) and its size.
const SegKernel *seg_kernels(int *count);

} // namespace fft3
