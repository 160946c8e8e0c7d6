// k_slabz.cu -- batched uneven 3D DFTs in one persistent launch, slab by slab
// (the slab-pencil decomposition of Section 2.3 applied to every problem):
//   slab items: a few n0 x n1 slabs of a problem, stacked in shared memory:
//               their x lines (rows) are read from global memory, transformed
//               and written into the buffer, then their y lines (columns) are
//               transformed in place in the buffer, and the stack is copied to
//               global memory with contiguous stores: one read and one write
//               per value for the 2D stage;
//   z items:    tiles of adjacent columns of a problem's n0*n1 plane, their z
//               lines read through L2 (the slabs were written earlier in the
//               launch), transformed and written back in place.
// Rows and columns are warp-shuffle line transforms (warp_fft.cuh; a line in
// the registers of a few lanes, no barrier within a transform), the z tiles
// the compile-time Stockham engines of FFT3_SLABZ_Z_PLANS (seg_plans.h).
// Work items come from a ticket counter in the order the host gives them
// (problems in groups, the z items of a group after the slab items of the
// next group, so a problem's slabs are still in L2 when its z items read
// them); a z item first waits until every slab item of its problem has
// finished.  Those slab items hold smaller tickets, so they were claimed by
// blocks that are already running and never wait: every wait ends.  Each wait
// is still bounded (about two seconds of clock cycles); on expiry the kernel
// records kErrWaitTimeout and carries on.  A block claims its next ticket
// while it runs the current item and, for a slab item, prefetches that item's
// input into L2.
#include "batched.h"
#include "pass_kernels.cuh"
#include "seg_plans.h"
#include "warp_fft.cuh"

namespace fft3 {

namespace {

constexpr int kSzThreads = 256;

// Column l of the z tile buffer (element j at p[j * LPT]), with a validity
// flag: an invalid line reads zeros and stores nothing, so every thread of the
// block can run every barrier of the engine whatever the number of lines.
template <int LPT>
struct SzTile {
    float2 *p;
    bool valid;
    __device__ __forceinline__ float2 operator()(int j) const { return valid ? p[j * LPT] : make_float2(0.f, 0.f); }
    __device__ __forceinline__ void operator()(int k, float2 v) const
    {
        if (valid)
            p[k * LPT] = v;
    }
};
// Strided global line read through L2 (written earlier in this launch by
// other blocks) / written back.
struct SzGLoad {
    const float2 *p;
    int64_t s;
    bool valid, conj;
    __device__ __forceinline__ float2 operator()(int j) const
    {
        const float2 v = valid ? __ldcg(p + (int64_t)j * s) : make_float2(0.f, 0.f);
        return conj ? cconj(v) : v;
    }
};

// Rows of the stacked slabs (x lines) straight from global memory into the
// shared buffer (rows `pitch` values apart, pitch odd): a row in the
// registers of L/2 lanes (warp_fft.cuh), 512 / L rows per round, no barrier;
// `w` is the table w_N^m (m < N).
template <int N, int R, int L>
__device__ __noinline__ void sz_rows_warp(const float2 *src, float2 *A, int pitch, int rows, const float2 *w,
                                          bool conj)
{
    using WL = WarpLine<N, R, L>;
    constexpr int RPR = kSzThreads / WL::W; // rows per round
    const int u = threadIdx.x % WL::W, l = threadIdx.x / WL::W;
    typename WL::Tw tw;
    WL::load_tw(tw, w, u);
    for (int r0 = 0; r0 < rows; r0 += RPR) {
        const int row = r0 + l;
        const bool valid = row < rows;
        float2 v[2][R];
        WL::load(v, src + (int64_t)(valid ? row : 0) * N, u, valid, conj);
        WL::run(v, tw, u);
        if (valid) {
            float2 *ar = A + row * pitch;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int k0 = R * WL::rev(2 * u + e);
#pragma unroll
                for (int k = 0; k < R; ++k)
                    ar[k0 + k] = v[e][k];
            }
        }
    }
}

// Columns of the stacked slabs (y lines) in the registers of L/2 lanes
// (warp_fft.cuh): the lanes of a column read different rows of the buffer
// (pitch odd: conflict free), adjacent lane groups take adjacent columns, and
// each group writes its column's outputs back in place (a group owns its
// column: no barrier).
template <int N, int R, int L>
__device__ __noinline__ void sz_cols_warp(float2 *A, int pitch, int cols, int w, int slab_stride, const float2 *tw_w)
{
    using WL = WarpLine<N, R, L>;
    constexpr int CPR = kSzThreads / WL::W; // columns per round
    const int u = threadIdx.x % WL::W, l = threadIdx.x / WL::W;
    typename WL::Tw tw;
    WL::load_tw(tw, tw_w, u);
    for (int c0 = 0; c0 < cols; c0 += CPR) {
        const int c = c0 + l;
        const bool valid = c < cols;
        const int cs = valid ? c / w : 0, cc = valid ? c - cs * w : 0;
        float2 *p = A + cs * slab_stride + cc;
        float2 v[2][R];
        WL::load_strided(v, p, pitch, u, valid, false);
        WL::run(v, tw, u);
        WL::store_strided(v, p, pitch, u, valid, false);
    }
}

// The stacked slabs (rows of n0 values, n0 even, `pitch` apart) to dst, where
// they are contiguous: each thread moves pairs of values of a row, 16-byte
// stores when dst is 16-byte aligned; conjugated for the inverse.
__device__ __noinline__ void sz_copy_out(const float2 *A, int pitch, int n0, int rows, float2 *dst, bool conj)
{
    const int half = n0 >> 1, rpp = kSzThreads / half; // rows per pass
    const int rr = threadIdx.x / half, x = 2 * (threadIdx.x - rr * half);
    if (rr >= rpp)
        return;
    const bool v4 = (reinterpret_cast<uintptr_t>(dst) & 15) == 0;
    for (int r = rr; r < rows; r += rpp) {
        float2 a = A[r * pitch + x], b = A[r * pitch + x + 1];
        if (conj) {
            a = cconj(a);
            b = cconj(b);
        }
        float2 *q = dst + (int64_t)r * n0 + x;
        if (v4) {
            *reinterpret_cast<float4 *>(q) = make_float4(a.x, a.y, b.x, b.y);
        } else {
            q[0] = a;
            q[1] = b;
        }
    }
}

// Tiles [t0, t1) of LPT adjacent columns of the n0*n1 plane (z lines, element
// stride es), in place through the shared tile buffers: 256 / (T LPT) tiles
// at a time, one per thread group.
template <int N, int T, class Rad, int LPT>
__device__ __noinline__ void sz_ztiles(float2 *base, int64_t t0, int64_t t1, int64_t ncols, int64_t es, float2 *buf,
                                       const float2 *tw, bool conj)
{
    constexpr int GT = T * LPT, G = kSzThreads / GT;
    const int tid = threadIdx.x, g = tid / GT, gl = tid % GT;
    const int l = gl % LPT, t = gl / LPT;
    for (int64_t tile0 = t0; tile0 < t1; tile0 += G) {
        if (tile0 > t0)
            __syncthreads(); // the tile buffers are free
        const int64_t tile = tile0 + g, c = tile * LPT + l;
        const bool valid = g < G && tile < t1 && c < ncols;
        float2 *p = base + (valid ? c : 0);
        SzGLoad src{p, es, valid, conj};
        GStore dst{p, es, valid, conj};
        SzTile<LPT> sm{buf + (g < G ? g : 0) * (LPT * N) + l, valid};
        EngineFixed<N, T, 1, Rad>::template run<true, false>(t, src, sm, dst, tw);
    }
}

__device__ __forceinline__ void sz_run_rows_warp(int n0, const float2 *src, float2 *A, int pitch, int rows,
                                                 const float2 *tw, const int *off, bool conj)
{
    int k = 0;
#define FFT3_SZ_WROW(N, R, L)                                                        \
    if (n0 == N) {                                                                   \
        sz_rows_warp<N, R, L>(src, A, pitch, rows, tw + off[k], conj);              \
        return;                                                                      \
    }                                                                                \
    ++k;
    FFT3_SLABZ_WARP_PLANS(FFT3_SZ_WROW)
#undef FFT3_SZ_WROW
}

__device__ __forceinline__ void sz_run_cols_warp(int n1, float2 *A, int pitch, int cols, int w, int slab_stride,
                                                 const float2 *tw, const int *off)
{
    int k = 0;
#define FFT3_SZ_WCOL(N, R, L)                                                        \
    if (n1 == N) {                                                                   \
        sz_cols_warp<N, R, L>(A, pitch, cols, w, slab_stride, tw + off[k]);          \
        return;                                                                      \
    }                                                                                \
    ++k;
    FFT3_SLABZ_WARP_PLANS(FFT3_SZ_WCOL)
#undef FFT3_SZ_WCOL
}

__device__ __forceinline__ void sz_run_ztiles(int n2, float2 *base, int64_t t0, int64_t t1, int64_t ncols,
                                              int64_t es, float2 *buf, const float2 *tw, const int *off, bool conj)
{
    int k = 0;
#define FFT3_SZ_Z(N, T, L, ...)                                                                      \
    if (n2 == N) {                                                                                   \
        sz_ztiles<N, T, Radices<__VA_ARGS__>, L>(base, t0, t1, ncols, es, buf, tw + off[k], conj);   \
        return;                                                                                      \
    }                                                                                                \
    ++k;
    FFT3_SLABZ_Z_PLANS(FFT3_SZ_Z)
#undef FFT3_SZ_Z
}

__device__ __forceinline__ int ld_acquire_sz(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

} // namespace

__global__ void __launch_bounds__(kSzThreads, 3) k_slabz(SlabZArgs z)
{
    extern __shared__ __align__(16) float2 smem[];
    const BatchArgs &a = z.b;
    const float2 *tw = z.tw; // read through L1: the shared memory holds the slabs
    float2 *A = smem;
    __shared__ int s_next[2]; // tickets of the current and the next item, alternating slots
    const bool conj = a.conj != 0;
    if (threadIdx.x == 0)
        s_next[0] = atomicAdd(a.counters, 1);
    for (int slot = 0;; slot ^= 1) {
        __syncthreads(); // the previous item is done (buffer free, counter published); s_next[slot] written
        const int q = s_next[slot];
        if (q >= a.nitems)
            break;
        if (threadIdx.x == 0) { // the next item, claimed while this one runs; the other slot was
            const int qn = atomicAdd(a.counters, 1); // read before the barrier above
            s_next[slot ^ 1] = qn;
            if (qn < a.nitems && a.items[qn].phase == 0) {
                // a slab item: its input (contiguous slabs) is fetched into L2
                // now, so its row loads find it there; only the 16-byte-aligned
                // interior of the range, in pieces of at most 32 KB
                const BatchItem nt = a.items[qn];
                const BatchCube &nc = a.cubes[nt.cube];
                const int s0 = nt.index * nc.spi, ns = min(nc.n2, s0 + nc.spi) - s0;
                const float2 *p = a.in + nc.off + (int64_t)s0 * nc.n0 * nc.n1;
                uintptr_t b = ((uintptr_t)p + 15) & ~(uintptr_t)15;
                const uintptr_t e = (uintptr_t)(p + (int64_t)ns * nc.n0 * nc.n1) & ~(uintptr_t)15;
                for (; b < e; b += 32768) {
                    const unsigned len = (unsigned)min((uintptr_t)32768, e - b);
                    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(b), "r"(len) : "memory");
                }
            }
        }
        const BatchItem it = a.items[q];
        const BatchCube &cb = a.cubes[it.cube];
        const int n0 = cb.n0, n1 = cb.n1, n2 = cb.n2;
        if (it.phase == 0) {
            // slabs [index * spi, ...) stacked in shared memory: all their rows,
            // then all their columns
            const int s0 = it.index * cb.spi, ns = min(n2, s0 + cb.spi) - s0;
            const int P = n0 | 1;
            const float2 *src = a.in + cb.off + (int64_t)s0 * n0 * n1;
            float2 *dst = a.out + cb.off + (int64_t)s0 * n0 * n1;
            sz_run_rows_warp(n0, src, A, P, n1 * ns, tw, z.tw_w, conj);
            __syncthreads();
            sz_run_cols_warp(n1, A, P, n0 * ns, n0, n1 * P, tw, z.tw_w);
            __syncthreads();
            sz_copy_out(A, P, n0, n1 * ns, dst, conj);
        } else {
            if (threadIdx.x == 0) {
                const int *done = a.counters + 1 + 3 * it.cube;
                const long long t0 = clock64();
                while (ld_acquire_sz(done) < cb.items[0]) {
                    if (clock64() - t0 > a.wait_budget) {
                        atomicOr(a.err, kErrWaitTimeout);
                        break;
                    }
                    __nanosleep(32);
                }
            }
            __syncthreads();
            const int64_t plane = (int64_t)n0 * n1, ntiles = (plane + cb.lpt - 1) / cb.lpt;
            const int64_t t0 = (int64_t)it.index * cb.zpi, t1 = min(ntiles, t0 + cb.zpi);
            sz_run_ztiles(n2, a.out + cb.off, t0, t1, plane, plane, A, tw, z.tw_z, conj);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(a.counters + 1 + 3 * it.cube + it.phase, 1);
        }
    }
}

// Shared memory of one block: the larger of the stacked slabs of an item and
// its z tiles.
int slabz_smem_bytes(int buf_elems) { return buf_elems * (int)sizeof(float2); }

} // namespace fft3
