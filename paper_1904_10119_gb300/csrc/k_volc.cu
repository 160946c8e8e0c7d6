// k_volc.cu -- compile-time specialised volumetric pass for strided lines
// (Section 3.2, Eq. cteinstein; Fig. cuboid): each line of n = A*B points is
// split over a cluster of P thread blocks holding it in elemental-cyclic order,
// with the single exchange done through distributed shared memory.
//
// Tile: LPT adjacent columns (lines) of the array, every line n points at
// element stride ij.  Block r of the cluster holds the rows
// i0 = r + P*u (u < A/P) of each line's matrix x~[i0, i1] = x[i0 + A*i1], i.e.
// the line elements j with j mod P = r: n/P rows of LPT*8 contiguous bytes.
//   (I)   DFT_B on its A/P rows of every column, in place in T0
//         (T0[(u*B + i1)*LPT + l]),
//   (II)  twiddle w_n^{i0*k1},
//   (III) cluster barrier; gather the columns k1 = r + P*v (v < B/P) of every
//         block's T0 from distributed shared memory into T1
//         (T1[(v*A + i0)*LPT + l]); cluster barrier,
//   (IV)  DFT_A on its B/P columns of every line, in place in T1, and store
//         y[k1 + B*k0], the line elements k with k mod P = r.
// Shared memory per block: 2 * LPT * n/P complex values plus the twiddles, so
// a 1024-point line split over 4 blocks needs a quarter of the single-block
// tile and several blocks fit on an SM while every row is still LPT*8 bytes.
#include <cooperative_groups.h>

#include "pass_kernels.cuh"
#include "plans.h"

namespace cg = cooperative_groups;

namespace fft3 {

template <int N, int A, int B, int P, int LPT, int TA, class RadA, int TB, class RadB>
__global__ void __launch_bounds__(LPT *(A / P) * TB) k_volc(PassArgs a)
{
    static_assert(A % P == 0 && B % P == 0, "one exchange needs P | A and P | B");
    static_assert(LPT * (A / P) * TB == LPT * (B / P) * TA, "both sub-DFTs use every thread");
    constexpr int AP = A / P, BP = B / P;
    constexpr int THREADS = LPT * AP * TB;
    extern __shared__ float2 smem[];
    cg::cluster_group cluster = cg::this_cluster();
    const int r = (int)cluster.block_rank();
    float2 *tw = smem;                        // [table B | table A | w_n^m]
    float2 *T0 = smem + a.tw_len;             // AP*B*LPT
    float2 *T1 = T0 + AP * B * LPT;           // BP*A*LPT
    load_twiddles(tw, a.tw, a.tw_len);
    const float2 *twB = tw + a.L[0].tw_off;
    const float2 *twA = tw + a.L[1].tw_off;
    const float2 *W = tw + a.tw_split_off;
    const bool conj = a.conj != 0;
    const int tid = threadIdx.x;
    const int l = tid % LPT;
    const int64_t cid = blockIdx.x / P, ncl = gridDim.x / P;
    for (int64_t tile = cid; tile < a.ntiles; tile += ncl) {
        __syncthreads();
        const TileId id = decode_tile(tile, a.tiles_c, a.g.A, LPT);
        const bool valid = id.c0 + l < a.g.C;
        const float2 *ib = a.in + id.c0 + l + id.a * a.g.ia + id.b * a.g.ib;
        // load rows j = (r + P*u) + A*i1 of this block's share
#pragma unroll 4
        for (int e = tid; e < AP * B * LPT; e += THREADS) {
            const int row = e / LPT; // = u*B + i1
            const int u = row / B, i1 = row - u * B;
            const int64_t j = r + P * u + A * i1;
            float2 v = valid ? ib[j * a.g.ij] : make_float2(0.f, 0.f);
            T0[e] = conj ? cconj(v) : v;
        }
        __syncthreads();
        { // (I) DFT_B on sub-lines (u, l): thread (l, u, t)
            const int sub = tid / LPT, u = sub / TB, t = sub % TB;
            SmemCol<LPT> sl{T0 + u * B * LPT + l};
            EngineFixed<B, TB, 1, RadB>::template run<false, true>(t, sl, sl, sl, twB);
        }
        __syncthreads();
        // (II) twiddles w_n^{i0 k1}, i0 = r + P*u
        for (int e = tid; e < AP * B * LPT; e += THREADS) {
            const int row = e / LPT, u = row / B, k1 = row - u * B;
            const int i0 = r + P * u;
            T0[e] = cmul(T0[e], W[(i0 * k1) % N]);
        }
        cluster.sync();
        // (III) T1[(v*A + i0)*LPT + l] = T0 of block (i0 mod P) at row (i0/P)*B + k1, k1 = r + P*v.
        // All of a thread's remote loads are issued before any local store.
        {
            constexpr int PER = BP * A * LPT / THREADS;
            static_assert(PER * THREADS == BP * A * LPT, "exchange divides evenly");
            float2 stage[PER];
#pragma unroll
            for (int k = 0; k < PER; ++k) {
                const int e = tid + k * THREADS;
                const int row = e / LPT, v = row / A, i0 = row - v * A;
                const int owner = i0 % P, k1 = r + P * v;
                const float2 *src = cluster.map_shared_rank(T0, owner);
                stage[k] = src[((i0 / P) * B + k1) * LPT + l];
            }
#pragma unroll
            for (int k = 0; k < PER; ++k)
                T1[tid + k * THREADS] = stage[k];
        }
        cluster.sync();
        { // (IV) DFT_A on sub-lines (v, l)
            const int sub = tid / LPT, v = sub / TA, t = sub % TA;
            SmemCol<LPT> sl{T1 + v * A * LPT + l};
            EngineFixed<A, TA, 1, RadA>::template run<false, true>(t, sl, sl, sl, twA);
        }
        __syncthreads();
        float2 *ob = a.out + id.c0 + l + id.a * a.g.oa + id.b * a.g.ob;
#pragma unroll 4
        for (int e = tid; e < BP * A * LPT; e += THREADS) {
            const int row = e / LPT, v = row / A, k0 = row - v * A;
            const int64_t k = r + P * v + (int64_t)B * k0;
            if (valid) {
                const float2 y = T1[e];
                ob[k * a.g.ok] = conj ? cconj(y) : y;
            }
        }
    }
}

#define FFT3_VOLC_ROW(N, A, B, P, LPT, TA, RA, TB, RB)                                                     \
    {N, A, B, P, LPT, LPT *(A / P) * TB, TA, TB, {RA}, {RB},                                               \
     (const void *)&k_volc<N, A, B, P, LPT, TA, Radices<RA>, TB, Radices<RB>>},

static const VolcKernel g_volc_kernels[] = {FFT3_VOLC_LIST(FFT3_VOLC_ROW)};

const VolcKernel *volc_kernels(int *count)
{
    *count = (int)(sizeof(g_volc_kernels) / sizeof(g_volc_kernels[0]));
    return g_volc_kernels;
}

} // namespace fft3
