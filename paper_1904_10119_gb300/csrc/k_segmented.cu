// k_segmented.cu -- batched uneven 3D DFTs as three segmented passes: all x
// lines of every problem, then all y lines, then all z lines (the
// pencil-pencil-pencil definition of Section 2.3 applied to each problem).
// A launch covers the lines of one length along one dimension of every
// problem that has that length there; each tile is LPT lines of one problem,
// found through a per-tile table.  The line transforms are the compile-time
// Stockham engine of the single-array passes (fft_engine.cuh), so the
// per-value instruction count stays that of k_pass_j / k_pass_c.
//
// Line c of a problem (n0, n1, n2) in pass d, with element stride es:
//   d = 0: c < n1*n2, first element c*n0, es = 1       (rows, contiguous)
//   d = 1: c < n0*n2, first element (c / n0)*n0*n1 + c % n0, es = n0
//   d = 2: c < n0*n1, first element c, es = n0*n1
// so consecutive lines of a strided tile are adjacent columns (a y tile may
// run across the end of one slab into the next).  The first stage reads its
// inputs straight from global memory and the last stage writes its outputs
// there (threads of a line adjacent for x lines, of a row of columns for y and
// z lines).  Pass 0 reads `in` and writes `out`; passes 1 and 2 work in place
// on `out`.
#include "batched.h"
#include "pass_kernels.cuh"
#include "seg_plans.h"

namespace fft3 {

template <int N, int T, class Rad, int LPT, bool CONTIG>
__global__ void __launch_bounds__(T *LPT) k_seg(SegArgs a)
{
    extern __shared__ float2 smem[];
    constexpr int S = line_pitch(N);
    float2 *tw = smem;
    float2 *buf = smem + tw_slots(a.tw_len);
    load_twiddles(tw, a.tw, a.tw_len);
    const int t = CONTIG ? (int)threadIdx.x % T : (int)threadIdx.x / LPT;
    const int l = CONTIG ? (int)threadIdx.x / T : (int)threadIdx.x % LPT;
    const bool conj = a.conj != 0;
    for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        __syncthreads();
        const int slot = a.tcube[tile];
        const BatchCube &cb = a.cubes[a.list[slot]];
        const int64_t n0 = cb.n0, n1 = cb.n1, n2 = cb.n2;
        const int64_t c = (tile - a.tstart[slot]) * LPT + l;
        int64_t lines, first, es;
        if (a.dim == 0) {
            lines = n1 * n2; first = c * n0; es = 1;
        } else if (a.dim == 1) {
            lines = n0 * n2; first = (c / n0) * n0 * n1 + c % n0; es = n0;
        } else {
            lines = n0 * n1; first = c; es = n0 * n1;
        }
        const bool valid = c < lines;
        const float2 *ip = a.src + cb.off + (valid ? first : 0);
        float2 *op = a.out + cb.off + (valid ? first : 0);
        if constexpr (CONTIG) {
            GLoad1 src{ip, valid, conj};
            GStore1 dst{op, valid, conj};
            SmemLine<S> sm{buf + l * S};
            EngineFixed<N, T, 1, Rad>::template run<true, false>(t, src, sm, dst, tw);
        } else {
            GLoad src{ip, es, valid, conj};
            GStore dst{op, es, valid, conj};
            SmemCol<LPT> sm{buf + l};
            EngineFixed<N, T, 1, Rad>::template run<true, false>(t, src, sm, dst, tw);
        }
    }
}

#define FFT3_SEG_ROW_C(N, T, L, ...)                                                                      \
    {N, T, L, Radices<__VA_ARGS__>::count, {__VA_ARGS__}, (const void *)&k_seg<N, T, Radices<__VA_ARGS__>, L, true>},
#define FFT3_SEG_ROW_S(N, T, L, ...)                                                                      \
    {N, T, L, Radices<__VA_ARGS__>::count, {__VA_ARGS__}, (const void *)&k_seg<N, T, Radices<__VA_ARGS__>, L, false>},

static const SegKernel g_seg_contig[] = {FFT3_SEG_PLANS_CONTIG(FFT3_SEG_ROW_C)};
static const SegKernel g_seg_strided[] = {FFT3_SEG_PLANS_STRIDED(FFT3_SEG_ROW_S)};

const SegKernel *seg_kernels(bool contiguous, int *count)
{
    if (contiguous) {
        *count = (int)(sizeof(g_seg_contig) / sizeof(g_seg_contig[0]));
        return g_seg_contig;
    }
    *count = (int)(sizeof(g_seg_strided) / sizeof(g_seg_strided[0]));
    return g_seg_strided;
}

} // namespace fft3
