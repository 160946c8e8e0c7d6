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
#include "warp_fft.cuh"

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

// x lines by the warp-shuffle line transform: L / 2 lanes per line, 512 / L
// lines per 256-thread tile, every line in registers (no shared memory, no
// block barrier); the lanes' twiddles are read once from the table w_N^m.
template <int N, int R, int L>
__global__ void __launch_bounds__(256) k_segw(SegArgs a)
{
    using WL = WarpLine<N, R, L>;
    constexpr int LPT = 256 / WL::W;
    const int u = (int)threadIdx.x % WL::W, l = (int)threadIdx.x / WL::W;
    typename WL::Tw tw;
    WL::load_tw(tw, a.tw, u);
    const bool conj = a.conj != 0;
    for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        const int slot = a.tcube[tile];
        const BatchCube &cb = a.cubes[a.list[slot]];
        const int64_t c = (tile - a.tstart[slot]) * LPT + l;
        const bool valid = c < (int64_t)cb.n1 * cb.n2;
        const float2 *ip = a.src + cb.off + (valid ? c * N : 0);
        float2 *op = a.out + cb.off + (valid ? c * N : 0);
        float2 v[2][R];
        WL::load(v, ip, u, valid, conj);
        WL::run(v, tw, u);
        WL::store(v, op, u, valid, conj);
    }
}

// y and z lines (columns) by the same transform: lane group l of a tile is
// column c0 + l, the L / 2 lanes of a column on different rows of it.
template <int N, int R, int L>
__global__ void __launch_bounds__(256) k_segw_s(SegArgs a)
{
    using WL = WarpLine<N, R, L>;
    constexpr int LPT = 256 / WL::W;
    const int u = (int)threadIdx.x % WL::W, l = (int)threadIdx.x / WL::W;
    typename WL::Tw tw;
    WL::load_tw(tw, a.tw, u);
    const bool conj = a.conj != 0;
    for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        const int slot = a.tcube[tile];
        const BatchCube &cb = a.cubes[a.list[slot]];
        const int64_t n0 = cb.n0, n1 = cb.n1, n2 = cb.n2;
        const int64_t c = (tile - a.tstart[slot]) * LPT + l;
        int64_t lines, first, es;
        if (a.dim == 1) {
            lines = n0 * n2; first = (c / n0) * n0 * n1 + c % n0; es = n0;
        } else {
            lines = n0 * n1; first = c; es = n0 * n1;
        }
        const bool valid = c < lines;
        const float2 *ip = a.src + cb.off + (valid ? first : 0);
        float2 *op = a.out + cb.off + (valid ? first : 0);
        float2 v[2][R];
        WL::load_strided(v, ip, es, u, valid, conj);
        WL::run(v, tw, u);
        WL::store_strided(v, op, es, u, valid, conj);
    }
}

#define FFT3_SEGW_ROW(N, R, L, D) {N, L / 2, 512 / L, 2, {R, L}, (const void *)&k_segw<N, R, L>, 1, D},
#define FFT3_SEGW_ROW_S(N, R, L, D) {N, L / 2, 512 / L, 2, {R, L}, (const void *)&k_segw_s<N, R, L>, 1, D},
static const SegKernel g_segw[] = {FFT3_SEGW_PLANS(FFT3_SEGW_ROW)};
static const SegKernel g_segw_s[] = {FFT3_SEGW_PLANS_STRIDED(FFT3_SEGW_ROW_S)};

const SegKernel *segw_kernels(int *count, bool contiguous)
{
    if (!contiguous) {
        *count = (int)(sizeof(g_segw_s) / sizeof(g_segw_s[0]));
        return g_segw_s;
    }
    *count = (int)(sizeof(g_segw) / sizeof(g_segw[0]));
    return g_segw;
}

// ---------------------------------------------------------------------------
// The whole batch in one persistent cooperative launch (k_seg_all): the same
// line kernels, 256-thread blocks (lines per tile 256 / T; the few threads
// left over work on a scratch line and store nothing), every step's tiles
// dealt out over the grid, steps separated by grid barriers with bounded
// waits.  A step holds the x, y or z lines of a wave of problems; with several
// waves the x lines of wave w, the y lines of wave w-1 and the z lines of wave
// w-2 share a step, so a wave's intermediate is re-read while it is in L2.

template <int N, int T, class Rad, bool CONTIG>
__device__ __noinline__ void seg_all_tile(const SegAllArgs &a, const SegAllSeg &sg, int64_t ltile, float2 *buf,
                                             const float2 *tw)
{
    constexpr int L = kSegAllThreads / T;                // lines (columns) per tile
    constexpr bool SPARE = L * T < kSegAllThreads;      // threads left over: one scratch line
    constexpr int LS = L + (SPARE ? 1 : 0);              // lines held in shared memory
    constexpr int S = line_pitch(N);
    const int tid = threadIdx.x;
    const int t = CONTIG ? (tid < L * T ? tid % T : tid - L * T) : (tid < L * T ? tid / L : tid - L * T);
    const int l = tid < L * T ? (CONTIG ? tid / T : tid % L) : L;
    const bool conj = a.conj != 0;
    const int slot = a.tcube[sg.tcube_off + ltile];
    const BatchCube &cb = a.cubes[a.list[sg.list_off + slot]];
    const int64_t n0 = cb.n0, n1 = cb.n1, n2 = cb.n2;
    const int64_t c = (ltile - a.tstart[sg.tstart_off + slot]) * L + l;
    int64_t lines, first, es;
    if (sg.dim == 0) {
        lines = n1 * n2; first = c * n0; es = 1;
    } else if (sg.dim == 1) {
        lines = n0 * n2; first = (c / n0) * n0 * n1 + c % n0; es = n0;
    } else {
        lines = n0 * n1; first = c; es = n0 * n1;
    }
    const bool valid = l < L && c < lines;
    const float2 *ip = (sg.dim == 0 ? a.in : a.out) + cb.off + (valid ? first : 0);
    float2 *op = a.out + cb.off + (valid ? first : 0);
    const float2 *twl = tw + sg.tw_off;
    if constexpr (CONTIG) {
        GLoad1 src{ip, valid, conj};
        GStore1 dst{op, valid, conj};
        SmemLine<S> sm{buf + l * S};
        EngineFixed<N, T, 1, Rad>::template run<true, false>(t, src, sm, dst, twl);
    } else {
        GLoad src{ip, es, valid, conj};
        GStore dst{op, es, valid, conj};
        SmemCol<LS> sm{buf + l};
        EngineFixed<N, T, 1, Rad>::template run<true, false>(t, src, sm, dst, twl);
    }
}

// Shared-memory values of one tile of a line kernel.
template <int N, int T, bool CONTIG>
constexpr int seg_all_buf()
{
    constexpr int L = kSegAllThreads / T;
    constexpr int LS = L + (L * T < kSegAllThreads ? 1 : 0);
    return CONTIG ? LS * line_pitch(N) : LS * N;
}

#define FFT3_SEGALL_BUF_C(N, T, L, ...) m = seg_all_buf<N, T, true>() > m ? seg_all_buf<N, T, true>() : m;
#define FFT3_SEGALL_BUF_S(N, T, L, ...) m = seg_all_buf<N, T, false>() > m ? seg_all_buf<N, T, false>() : m;

constexpr int seg_all_buf_max()
{
    int m = 0;
    FFT3_SEG_PLANS_CONTIG(FFT3_SEGALL_BUF_C)
    FFT3_SEG_PLANS_STRIDED(FFT3_SEGALL_BUF_S)
    return m;
}

__device__ __forceinline__ void seg_all_run(int kidx, const SegAllArgs &a, const SegAllSeg &sg, int64_t lt,
                                            float2 *buf, const float2 *tw)
{
    int k = 0;
#define FFT3_SEGALL_IF_C(N, T, L, ...)                                                       \
    if (kidx == k++) {                                                                       \
        seg_all_tile<N, T, Radices<__VA_ARGS__>, true>(a, sg, lt, buf, tw);                 \
        return;                                                                              \
    }
#define FFT3_SEGALL_IF_S(N, T, L, ...)                                                       \
    if (kidx == k++) {                                                                       \
        seg_all_tile<N, T, Radices<__VA_ARGS__>, false>(a, sg, lt, buf, tw);                \
        return;                                                                              \
    }
    FFT3_SEG_PLANS_CONTIG(FFT3_SEGALL_IF_C)
    FFT3_SEG_PLANS_STRIDED(FFT3_SEGALL_IF_S)
}

__device__ __forceinline__ int ld_acquire_seg(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__global__ void __launch_bounds__(kSegAllThreads, 4) k_seg_all(SegAllArgs a)
{
    extern __shared__ float2 smem[];
    float2 *tw = smem;
    float2 *buf = smem + tw_slots(a.tw_len);
    for (int i = threadIdx.x; i < a.tw_len; i += blockDim.x)
        tw[i] = a.tw[i];
    bool late = false;
    for (int s = 0; s < a.nsteps; ++s) {
        const int s0 = a.seg0[s], s1 = a.seg0[s + 1];
        int cur = s0;
        for (int64_t tile = blockIdx.x; tile < a.ntiles[s]; tile += gridDim.x) {
            while (cur + 1 < s1 && a.segs[cur + 1].tile0 <= tile)
                ++cur;
            const SegAllSeg sg = a.segs[cur];
            __syncthreads(); // the previous tile's shared buffer (and, first, the twiddles)
            seg_all_run(sg.kidx, a, sg, tile - sg.tile0, buf, tw);
        }
        if (s + 1 == a.nsteps)
            break;
        // grid barrier: every block's stores of step s before any block's loads of step s + 1
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(a.barrier, 1);
            const int want = (s + 1) * (int)gridDim.x;
            const long long t0 = clock64();
            while (ld_acquire_seg(a.barrier) < want) {
                if (clock64() - t0 > a.wait_budget) {
                    late = true;
                    break;
                }
                __nanosleep(100);
            }
        }
        __syncthreads();
    }
    if (late)
        atomicOr(a.err, kErrWaitTimeout);
}

int seg_all_smem_bytes(int tw_len) { return (tw_slots(tw_len) + seg_all_buf_max()) * (int)sizeof(float2); }

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
