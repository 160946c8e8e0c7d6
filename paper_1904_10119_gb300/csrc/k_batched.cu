// k_batched.cu -- thousands of independent, unevenly sized 3D DFTs in one
// persistent launch.
//
// Every problem is split into phases (slab-pencil: 2D slabs, then z lines;
// pencil-pencil-pencil: x, y, z lines) and every phase into work items (a few
// slabs, a few rows, or a tile of adjacent columns).  The host orders the
// items so that a problem's later phase follows its earlier phase by one
// group of problems, which keeps a problem's intermediate result in L2
// between its phases.  Blocks take items from a ticket counter; an item of
// phase p > 0 first waits until every item of phase p-1 of its problem has
// finished.  Those items hold smaller tickets, so they were claimed by blocks
// that are already running and never wait on later tickets: every wait ends.
// Each wait is still bounded; on expiry the kernel records kErrWaitTimeout
// and goes on.
#include "batch_stages.cuh"
#include "batched.h"
#include "pass_kernels.cuh"

namespace fft3 {

__device__ __forceinline__ int ld_acquire_b(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// nl lines of length L.n (N when it is a compile-time constant, else 0):
// line l starts at src + l*ls, element j at j*es.  Contiguous lines (es == 1)
// are moved with j fastest across threads, strided ones with l fastest.
// Loads from data written earlier in this launch go through L2 only.
template <int N>
__device__ __forceinline__ void batch_lines(const float2 *src, float2 *dst, bool l2_only, const LineRt &L, const float2 *tw,
                            int nl, int64_t ls, int64_t es, float2 *A, float2 *B, bool conj)
{
    const int n = N > 0 ? N : L.n, P = line_pitch(n);
    const bool contig = es == 1;
    // strided: l = e mod lp, j = e / lp with lp the power of two >= nl
    int sh = 0;
    while ((1 << sh) < nl)
        ++sh;
    const int lp = 1 << sh;
    const int tot = contig ? nl * n : lp * n;
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
        int l, j;
        if (contig) { l = e / n; j = e - l * n; }
        else { l = e & (lp - 1); j = e >> sh; }
        if (l < nl) {
            const float2 *p = src + l * ls + (int64_t)j * es;
            const float2 v = l2_only ? __ldcg(p) : *p;
            A[l * P + padpos(j)] = conj ? cconj(v) : v;
        }
    }
    __syncthreads();
    const float2 *r = batch_stages<false>(L, nl, P, A, B, tw + L.tw_off);
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
        int l, j;
        if (contig) { l = e / n; j = e - l * n; }
        else { l = e & (lp - 1); j = e >> sh; }
        if (l < nl) {
            const float2 v = r[l * P + padpos(j)];
            dst[l * ls + (int64_t)j * es] = conj ? cconj(v) : v;
        }
    }
}

// One n0 x n1 slab (N0 = n0 when compile-time, else 0): x lines then y lines
// in shared memory.
template <int N0>
__device__ __forceinline__ void batch_slab(const float2 *src, float2 *dst, const LineRt &X, const LineRt &Y, const float2 *tw,
                           float2 *A, float2 *B, bool conj)
{
    const int n0 = N0 > 0 ? N0 : X.n, n1 = Y.n, P = line_pitch(n0), nel = n0 * n1;
    for (int e = threadIdx.x; e < nel; e += blockDim.x) {
        const int row = e / n0, col = e - row * n0;
        const float2 v = src[e];
        A[row * P + padpos(col)] = conj ? cconj(v) : v;
    }
    __syncthreads();
    float2 *r1 = batch_stages<false>(X, n1, P, A, B, tw + X.tw_off);
    float2 *o1 = (r1 == A) ? B : A;
    float2 *r2 = batch_stages<true>(Y, n0, P, r1, o1, tw + Y.tw_off);
    for (int e = threadIdx.x; e < nel; e += blockDim.x) {
        const int row = e / n0, col = e - row * n0;
        const float2 v = r2[row * P + padpos(col)];
        dst[e] = conj ? cconj(v) : v;
    }
}

// Compile-time line lengths for the index arithmetic of the loads and stores.
#define FFT3_BATCH_LENGTHS(X) X(16) X(24) X(32) X(40) X(48) X(64) X(80) X(96) X(128)

__device__ __forceinline__ void batch_lines_any(const float2 *src, float2 *dst, bool l2_only, const LineRt &L, const float2 *tw,
                                int nl, int64_t ls, int64_t es, float2 *A, float2 *B, bool conj)
{
    switch (es == 1 ? L.n : 0) {
#define FFT3_BATCH_CASE(N) \
    case N: batch_lines<N>(src, dst, l2_only, L, tw, nl, ls, es, A, B, conj); return;
        FFT3_BATCH_LENGTHS(FFT3_BATCH_CASE)
#undef FFT3_BATCH_CASE
    default: batch_lines<0>(src, dst, l2_only, L, tw, nl, ls, es, A, B, conj); return;
    }
}

__device__ __forceinline__ void batch_slab_any(const float2 *src, float2 *dst, const LineRt &X, const LineRt &Y, const float2 *tw,
                               float2 *A, float2 *B, bool conj)
{
    switch (X.n) {
#define FFT3_BATCH_CASE(N) \
    case N: batch_slab<N>(src, dst, X, Y, tw, A, B, conj); return;
        FFT3_BATCH_LENGTHS(FFT3_BATCH_CASE)
#undef FFT3_BATCH_CASE
    default: batch_slab<0>(src, dst, X, Y, tw, A, B, conj); return;
    }
}

__global__ void __launch_bounds__(256, 3) k_batched(BatchArgs a)
{
    extern __shared__ float2 smem[];
    float2 *A = smem, *B = smem + a.buf_elems;
    __shared__ int s_item;
    const bool conj = a.conj != 0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0)
            s_item = atomicAdd(a.counters, 1);
        __syncthreads();
        const int q = s_item;
        if (q >= a.nitems)
            break;
        const BatchItem it = a.items[q];
        const BatchCube cb = a.cubes[it.cube];
        int *done = a.counters + 1 + 3 * it.cube;
        if (it.phase > 0) {
            if (threadIdx.x == 0) {
                const long long t0 = clock64();
                while (ld_acquire_b(done + it.phase - 1) < cb.items[it.phase - 1]) {
                    if (clock64() - t0 > a.wait_budget) {
                        atomicOr(a.err, kErrWaitTimeout);
                        break;
                    }
                    __nanosleep(32);
                }
            }
            __syncthreads();
        }
        const bool first = it.phase == 0;
        const float2 *src = (first ? a.in : a.out) + cb.off;
        float2 *dst = a.out + cb.off;
        const int64_t n0 = cb.n0, n1 = cb.n1, n2 = cb.n2;
        const int dim = cb.decomp == BD_SLAB ? (first ? 3 : 2) : it.phase;
        if (dim == 3) { // slabs [index*spi, ...)
            const int s0 = it.index * cb.spi;
            const int s1 = min((int)n2, s0 + cb.spi);
            for (int s = s0; s < s1; ++s) {
                batch_slab_any(src + s * n0 * n1, dst + s * n0 * n1, a.lines[cb.lx], a.lines[cb.ly], a.tw, A, B,
                               conj);
                __syncthreads();
            }
        } else {
            int64_t base, ls, es;
            int nl, li;
            if (dim == 0) { // rows of length n0
                const int64_t r0 = (int64_t)it.index * cb.spi;
                nl = (int)min((int64_t)cb.spi, n1 * n2 - r0);
                base = r0 * n0; ls = n0; es = 1; li = cb.lx;
            } else if (dim == 1) { // columns x in slab z, element stride n0
                const int per = (int)((n0 + cb.lpty - 1) / cb.lpty);
                const int64_t z = it.index / per, c0 = (int64_t)(it.index % per) * cb.lpty;
                nl = (int)min((int64_t)cb.lpty, n0 - c0);
                base = z * n0 * n1 + c0; ls = 1; es = n0; li = cb.ly;
            } else { // columns c of the n0*n1 plane, element stride n0*n1
                const int64_t c0 = (int64_t)it.index * cb.lpt;
                nl = (int)min((int64_t)cb.lpt, n0 * n1 - c0);
                base = c0; ls = 1; es = n0 * n1; li = cb.lz;
            }
            batch_lines_any(src + base, dst + base, !first, a.lines[li], a.tw, nl, ls, es, A, B, conj);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(done + it.phase, 1);
        }
    }
}

} // namespace fft3
