// roots.cuh -- the two pieces every twiddle table of the library is made of
// (Section 2.1: DFT_n = [w_n^{lk}] and the twiddle matrix Twid = [w_n^{kl}]):
//
//   stage_twiddle_exponent: entry e of the stage-major table of a radix list
//     (fft_engine.cuh), the integer exponent m of w_n^m;
//   root_fp64: w_n^m = exp(sign * 2 pi i m / n) in FP64 from an exactly reduced
//     integer exponent: m mod n, then the quadrant q = floor(4m/n) and the
//     remainder rem = 4m - q*n are integers, so the only rounded quantities are
//     the argument rem/(2n) of sincospi (one division, |error| <= 2^-53
//     relative) and sincospi itself; the quarter-turn rotation by q is exact.
//
// The plan generator (twiddle.cu, exponents listed by the host planner) and
// the allocation-free path (capi.cu, exponents computed on the device) both
// call these, so their tables agree bit for bit.
#pragma once

#include <stdint.h>

namespace fft3 {

// Exponent of entry e of the stage-major table of a line of n points with
// radices rad[0..nst): stage s holds (R_s - 1) * NS_s entries, entry
// (r - 1) * NS_s + k being w_n^{r k n / (NS_s R_s)} (r in [1, R_s), k < NS_s).
// Returns -1 for e past the table.
__host__ __device__ inline int64_t stage_twiddle_exponent(int n, const int *rad, int nst, int64_t e)
{
    int64_t off = 0, ns = 1;
    for (int s = 0; s < nst; ++s) {
        const int64_t R = rad[s];
        const int64_t cnt = (R - 1) * ns;
        if (e < off + cnt) {
            const int64_t idx = e - off;
            const int64_t r = 1 + idx / ns, k = idx % ns;
            return r * k * ((int64_t)n / (ns * R)) % n;
        }
        off += cnt;
        ns *= R;
    }
    return -1;
}

#ifdef __CUDACC__
// w_n^m with the sign of the exponent given by `sign` (-1: forward roots).
__device__ __forceinline__ double2 root_fp64(int64_t m, int n, int sign)
{
    int64_t mm = m % n;
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
    return make_double2(re, sign < 0 ? -im : im);
}
#endif

} // namespace fft3
