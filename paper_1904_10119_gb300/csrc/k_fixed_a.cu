// Fixed-plan pass kernels, first half of the plan list (long lines).
#include "k_fixed.cuh"

namespace fft3 {
extern const FixedKernels g_fixed_kernels_a[] = {FFT3_FIXED_PLANS_A(FFT3_KERNEL_ROW)};
extern const int g_fixed_kernels_a_count = sizeof(g_fixed_kernels_a) / sizeof(g_fixed_kernels_a[0]);
} // namespace fft3
