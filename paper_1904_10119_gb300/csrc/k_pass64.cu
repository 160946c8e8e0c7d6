// k_pass64.cu -- complex128 (FP64) line passes with a compile-time radix list,
// the precision of the paper's experiments (Section 4: complex double): the
// Stockham stages of Section 2.1 (Eq. ct applied repeatedly, fft_engine.cuh)
// on double2 values with FP64 twiddles, one pass per dimension as in the
// pencil-pencil-pencil definition of Section 2.3.
//   k_pass_j64  contiguous lines (ij == 1, ok == 1), T threads per line, LPT
//               lines per tile, one padded line buffer in shared memory (the
//               first stage reads global memory, the last writes it).
//   k_pass_c64  strided lines (ic == 1, oc == 1), tiles of 8 adjacent
//               columns (128-byte rows), position-major shared layout.
// The runtime-radix FP64 kernel (k_pass_g64) covers the other lengths.
#include "pass_kernels.cuh"
#include "plans.h"

namespace fft3 {

struct G64Load1 {
    const double2 *p;
    bool valid, conj;
    __device__ __forceinline__ double2 operator()(int j) const
    {
        const double2 v = valid ? p[j] : make_double2(0.0, 0.0);
        return conj ? cconj(v) : v;
    }
};
struct G64Store1 {
    double2 *p;
    bool valid, conj;
    __device__ __forceinline__ void operator()(int k, double2 v) const
    {
        if (valid)
            p[k] = conj ? cconj(v) : v;
    }
};
struct G64Load {
    const double2 *p;
    int64_t s;
    bool valid, conj;
    __device__ __forceinline__ double2 operator()(int j) const
    {
        const double2 v = valid ? p[(int64_t)j * s] : make_double2(0.0, 0.0);
        return conj ? cconj(v) : v;
    }
};
struct G64Store {
    double2 *p;
    int64_t s;
    bool valid, conj;
    __device__ __forceinline__ void operator()(int k, double2 v) const
    {
        if (valid)
            p[(int64_t)k * s] = conj ? cconj(v) : v;
    }
};
template <int S>
struct Smem64Line { // padded line-major
    double2 *p;
    __device__ __forceinline__ double2 operator()(int j) const { return p[padpos(j)]; }
    __device__ __forceinline__ void operator()(int k, double2 v) const { p[padpos(k)] = v; }
};
template <int LPT>
struct Smem64Col { // element j of column l at p[j*LPT] (p = buffer + l)
    double2 *p;
    __device__ __forceinline__ double2 operator()(int j) const { return p[j * LPT]; }
    __device__ __forceinline__ void operator()(int k, double2 v) const { p[k * LPT] = v; }
};

__device__ __forceinline__ double2 *smem64()
{
    extern __shared__ __align__(16) unsigned char s64_raw[];
    return reinterpret_cast<double2 *>(s64_raw);
}

__device__ __forceinline__ void load_twiddles64(double2 *tw_s, const double2 *tw_g, int len)
{
    for (int i = threadIdx.x; i < len; i += blockDim.x)
        tw_s[i] = tw_g[i];
}

template <int N, int T, class Rad, int LPT>
__global__ void __launch_bounds__(T *LPT) k_pass_j64(PassArgs a)
{
    constexpr int S = line_pitch(N);
    double2 *tw = smem64();
    double2 *buf = tw + tw_slots(a.tw_len);
    load_twiddles64(tw, reinterpret_cast<const double2 *>(a.tw), a.tw_len);
    const double2 *in = reinterpret_cast<const double2 *>(a.in);
    double2 *out = reinterpret_cast<double2 *>(a.out);
    const int t = threadIdx.x % T, l = threadIdx.x / T;
    const bool conj = a.conj != 0;
    for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        __syncthreads();
        const TileId id = decode_tile(tile, a.tiles_c, a.g.A, LPT);
        const int64_t c = id.c0 + l;
        const bool valid = c < a.g.C;
        G64Load1 src{in + c * a.g.ic + id.a * a.g.ia + id.b * a.g.ib, valid, conj};
        G64Store1 dst{out + c * a.g.oc + id.a * a.g.oa + id.b * a.g.ob, valid, conj};
        Smem64Line<S> sm{buf + l * S};
        EngineFixed<N, T, 1, Rad>::template run<true, false>(t, src, sm, dst, (const double2 *)tw);
    }
}

template <int N, int T, class Rad, int LPT>
__global__ void __launch_bounds__(T *LPT) k_pass_c64(PassArgs a)
{
    double2 *tw = smem64();
    double2 *buf = tw + tw_slots(a.tw_len);
    load_twiddles64(tw, reinterpret_cast<const double2 *>(a.tw), a.tw_len);
    const double2 *in = reinterpret_cast<const double2 *>(a.in);
    double2 *out = reinterpret_cast<double2 *>(a.out);
    const int l = threadIdx.x % LPT, t = threadIdx.x / LPT;
    const bool conj = a.conj != 0;
    for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        __syncthreads();
        const TileId id = decode_tile(tile, a.tiles_c, a.g.A, LPT);
        const int64_t c = id.c0 + l;
        const bool valid = c < a.g.C;
        G64Load src{in + c * a.g.ic + id.a * a.g.ia + id.b * a.g.ib, a.g.ij, valid, conj};
        G64Store dst{out + c * a.g.oc + id.a * a.g.oa + id.b * a.g.ob, a.g.ok, valid, conj};
        Smem64Col<LPT> sm{buf + l};
        EngineFixed<N, T, 1, Rad>::template run<true, false>(t, src, sm, dst, (const double2 *)tw);
    }
}

template <int N, int T, class Rad>
constexpr const void *pass_c64_ptr()
{
    if constexpr (T * kLpt64Strided <= 1024)
        return (const void *)&k_pass_c64<N, T, Rad, kLpt64Strided>;
    else
        return nullptr;
}

#define FFT3_KERNEL64_ROW(ID, N, T, ...)                                                              \
    {ID, (const void *)&k_pass_j64<N, T, Radices<__VA_ARGS__>, lpt_j(T)>,                            \
     pass_c64_ptr<N, T, Radices<__VA_ARGS__>>()},

static const Fixed64Kernels g_fixed64[] = {FFT3_FIXED_PLANS_A(FFT3_KERNEL64_ROW)
                                               FFT3_FIXED_PLANS_B(FFT3_KERNEL64_ROW)};

const Fixed64Kernels *fixed64_kernels(int id)
{
    for (const Fixed64Kernels &k : g_fixed64)
        if (k.id == id)
            return &k;
    return nullptr;
}

} // namespace fft3
