// Fixed-plan pass kernels, second half of the plan list (short lines).
#include "k_fixed.cuh"

namespace fft3 {
extern const FixedKernels g_fixed_kernels_b[] = {FFT3_FIXED_PLANS_B(FFT3_KERNEL_ROW)};
extern const int g_fixed_kernels_b_count = sizeof(g_fixed_kernels_b) / sizeof(g_fixed_kernels_b[0]);
} // namespace fft3
