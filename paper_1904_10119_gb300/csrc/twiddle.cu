// twiddle.cu -- FP64 generation of the roots of unity used by every pass
// (Section 2.1: DFT_n = [w_n^{lk}] and the twiddle matrix Twid = [w_n^{kl}]),
// plus the split-BF16 helper of the tensor-core path.
//
// w_n^m = exp(sign * 2 pi i m / n) comes from root_fp64 (roots.cuh): an
// exactly reduced integer exponent and one FP64 sincospi.  Results are kept
// as doubles and rounded once to float32.
#include <cuda_bf16.h>
#include <stdint.h>

#include "roots.cuh"

namespace fft3 {

__global__ void k_roots(int n, int sign, const int64_t *m, int64_t count, double *o64, float2 *o32)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double2 w = root_fp64(m[i], n, sign);
        if (o64) {
            o64[2 * i] = w.x;
            o64[2 * i + 1] = w.y;
        }
        if (o32)
            o32[i] = make_float2((float)w.x, (float)w.y);
    }
}

__global__ void k_split_bf16(const float *x, int64_t count, uint16_t *hi, uint16_t *lo)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float v = x[i];
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
        hi[i] = __bfloat16_as_ushort(h);
        lo[i] = __bfloat16_as_ushort(l);
    }
}

} // namespace fft3
