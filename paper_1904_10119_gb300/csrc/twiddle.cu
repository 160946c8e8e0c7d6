// twiddle.cu -- FP64 generation of the roots of unity used by every pass
// (Section 2.1: DFT_n = [w_n^{lk}] and the twiddle matrix Twid = [w_n^{kl}]),
// plus the split-BF16 helper of the tensor-core path.
//
// w_n^m = exp(sign * 2 pi i m / n) is formed from an exactly reduced integer
// exponent: m mod n, then the quadrant q = floor(4m/n) and remainder
// rem = 4m - q*n are integers, so the only rounded quantities are the
// argument rem/(2n) of sincospi (one division, |error| <= 2^-53 relative)
// and sincospi itself.  The quarter-turn rotation by q is exact.  Results are
// kept as doubles and rounded once to float32.
#include <cuda_bf16.h>
#include <stdint.h>

namespace fft3 {

__global__ void k_roots(int n, int sign, const int64_t *m, int64_t count, double *o64, float2 *o32)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t mm = m[i] % n;
        if (mm < 0)
            mm += n;
        const int64_t q = (4 * mm) / n;
        const int64_t rem = 4 * mm - q * n;
        double s, c;
        sincospi((double)rem / (2.0 * (double)n), &s, &c);
        double re, im;
        switch (q & 3) {
        case 0: re = c; im = s; break;
        case 1: re = -s; im = c; break;
        case 2: re = -c; im = -s; break;
        default: re = s; im = -c; break;
        }
        im = sign < 0 ? -im : im;
        if (o64) {
            o64[2 * i] = re;
            o64[2 * i + 1] = im;
        }
        if (o32)
            o32[i] = make_float2((float)re, (float)im);
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
