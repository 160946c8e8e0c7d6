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

// An item, decoded from its ticket: a tile of nl lines of length L (line l at
// base + l*ls, element j at j*es) or the slabs [s0, s1) of a slab-pencil cube.
struct ItemView {
    int cube, phase, dim; // dim 0/1/2: lines along that dimension; 3: slabs
    const float2 *src;    // cube base (input of this phase)
    float2 *dst;          // cube base (output)
    int64_t base, ls, es;
    int nl, li;
    int s0, s1;
};

__device__ __forceinline__ ItemView view_item(const BatchArgs &a, int q)
{
    const BatchItem it = a.items[q];
    const BatchCube &cb = a.cubes[it.cube];
    ItemView v;
    v.cube = it.cube;
    v.phase = it.phase;
    const bool first = it.phase == 0;
    v.src = (first ? a.in : a.out) + cb.off;
    v.dst = a.out + cb.off;
    v.dim = cb.decomp == BD_SLAB ? (first ? 3 : 2) : it.phase;
    const int64_t n0 = cb.n0, n1 = cb.n1, n2 = cb.n2;
    v.s0 = v.s1 = 0;
    v.base = 0; v.ls = 1; v.es = 1; v.nl = 0; v.li = cb.lx;
    if (v.dim == 3) { // slabs [index*spi, ...)
        v.s0 = it.index * cb.spi;
        v.s1 = min((int)n2, v.s0 + cb.spi);
        v.nl = (int)n1; // rows of a slab
    } else if (v.dim == 0) { // rows of length n0
        const int64_t r0 = (int64_t)it.index * cb.spi;
        v.nl = (int)min((int64_t)cb.spi, n1 * n2 - r0);
        v.base = r0 * n0; v.ls = n0; v.es = 1; v.li = cb.lx;
    } else if (v.dim == 1) { // columns x in slab z, element stride n0
        const int per = (int)((n0 + cb.lpty - 1) / cb.lpty);
        const int64_t z = it.index / per, c0 = (int64_t)(it.index % per) * cb.lpty;
        v.nl = (int)min((int64_t)cb.lpty, n0 - c0);
        v.base = z * n0 * n1 + c0; v.ls = 1; v.es = n0; v.li = cb.ly;
    } else { // columns c of the n0*n1 plane, element stride n0*n1
        const int64_t c0 = (int64_t)it.index * cb.lpt;
        v.nl = (int)min((int64_t)cb.lpt, n0 * n1 - c0);
        v.base = c0; v.ls = 1; v.es = n0 * n1; v.li = cb.lz;
    }
    return v;
}

// ------------------------------------------------------------ prefetch --- //
// The first tile of the next item is copied raw into the staging buffer S by
// cp.async (16 bytes, L2 only: the data may have been written earlier in this
// launch by another SM) while the current item computes.  Raw layouts:
//   contiguous lines: S[l*n + j];  strided lines: S[j*nl + l];  slab: S[row*n0 + col].
// An item qualifies when every 16-byte copy holds two elements of the same
// line (or row) and starts 16-byte aligned.
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
                 "l"(gsrc)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ bool prefetchable(const BatchArgs &a, const ItemView &v)
{
    const BatchCube &cb = a.cubes[v.cube];
    const float2 *p = v.src + v.base + (v.dim == 3 ? (int64_t)v.s0 * cb.n0 * cb.n1 : 0);
    if (((uintptr_t)p & 15) != 0)
        return false;
    if (v.dim == 3)
        return ((cb.n0 * cb.n1) & 1) == 0;
    const int n = a.lines[v.li].n;
    if (v.es == 1)
        return (n & 1) == 0 && (v.ls & 1) == 0;
    return (v.nl & 1) == 0 && (v.es & 1) == 0;
}

__device__ __forceinline__ void issue_prefetch(const BatchArgs &a, const ItemView &v, float2 *S)
{
    const BatchCube &cb = a.cubes[v.cube];
    if (v.dim == 3) {
        const int nel = cb.n0 * cb.n1;
        const float2 *p = v.src + (int64_t)v.s0 * nel;
        for (int e = 2 * threadIdx.x; e < nel; e += 2 * blockDim.x)
            cp_async16(S + e, p + e);
    } else {
        const int n = a.lines[v.li].n, tot = v.nl * n;
        const float2 *p = v.src + v.base;
        for (int e = 2 * threadIdx.x; e < tot; e += 2 * blockDim.x) {
            int l, j;
            if (v.es == 1) { l = e / n; j = e - l * n; }
            else { j = e / v.nl; l = e - j * v.nl; }
            cp_async16(S + e, p + l * v.ls + (int64_t)j * v.es);
        }
    }
    cp_async_commit();
}

// ---------------------------------------------------------------- lines --- //
// nl lines of length L.n (N when it is a compile-time constant, else 0) into
// the padded line-major buffer A, from global memory or from the raw staging
// buffer S.  Global loads of data written earlier in this launch go through
// L2 only.
template <int N>
__device__ __forceinline__ void lines_load(const ItemView &v, const LineRt &L, const float2 *S, float2 *A, bool conj)
{
    const int n = N > 0 ? N : L.n, P = line_pitch(n), nl = v.nl;
    const bool contig = v.es == 1;
    if (S) {
        for (int e = threadIdx.x; e < nl * n; e += blockDim.x) {
            int l, j;
            if (contig) { l = e / n; j = e - l * n; }
            else { j = e / nl; l = e - j * nl; }
            const float2 x = S[e];
            A[l * P + padpos(j)] = conj ? cconj(x) : x;
        }
        return;
    }
    const float2 *src = v.src + v.base;
    const bool l2_only = v.phase > 0;
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
            const float2 *p = src + l * v.ls + (int64_t)j * v.es;
            const float2 x = l2_only ? __ldcg(p) : *p;
            A[l * P + padpos(j)] = conj ? cconj(x) : x;
        }
    }
}

// Stages of the lines in A (ping-pong with B) and the store to global memory.
template <int N>
__device__ __forceinline__ void lines_finish(const ItemView &v, const LineRt &L, const float2 *tw, float2 *A,
                                             float2 *B, bool conj)
{
    const int n = N > 0 ? N : L.n, P = line_pitch(n), nl = v.nl;
    const bool contig = v.es == 1;
    const float2 *r = batch_stages<false, N>(L, nl, P, A, B, tw + L.tw_off);
    float2 *dst = v.dst + v.base;
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
            const float2 x = r[l * P + padpos(j)];
            dst[l * v.ls + (int64_t)j * v.es] = conj ? cconj(x) : x;
        }
    }
}

// ----------------------------------------------------------------- slabs -- //
// One n0 x n1 slab (N0 = n0 when compile-time, else 0) into A, from global
// memory or from the raw staging buffer S.
template <int N0>
__device__ __forceinline__ void slab_load(const float2 *src, const float2 *S, int n1, float2 *A, int n0rt, bool conj)
{
    const int n0 = N0 > 0 ? N0 : n0rt, P = line_pitch(n0), nel = n0 * n1;
    for (int e = threadIdx.x; e < nel; e += blockDim.x) {
        const int row = e / n0, col = e - row * n0;
        const float2 x = S ? S[e] : src[e];
        A[row * P + padpos(col)] = conj ? cconj(x) : x;
    }
}

// x lines then y lines of the slab in A, and the store.
template <int N0>
__device__ __forceinline__ void slab_finish(float2 *dst, const LineRt &X, const LineRt &Y, const float2 *tw, float2 *A,
                                            float2 *B, bool conj)
{
    const int n0 = N0 > 0 ? N0 : X.n, n1 = Y.n, P = line_pitch(n0), nel = n0 * n1;
    float2 *r1 = batch_stages<false, N0>(X, n1, P, A, B, tw + X.tw_off);
    float2 *o1 = (r1 == A) ? B : A;
    float2 *r2 = batch_stages<true, 0>(Y, n0, P, r1, o1, tw + Y.tw_off);
    for (int e = threadIdx.x; e < nel; e += blockDim.x) {
        const int row = e / n0, col = e - row * n0;
        const float2 x = r2[row * P + padpos(col)];
        dst[e] = conj ? cconj(x) : x;
    }
}

// Compile-time line lengths for the index arithmetic of the loads and stores.
#define FFT3_BATCH_LENGTHS(X) X(16) X(24) X(32) X(40) X(48) X(64) X(80) X(96) X(128)

// First tile of an item (its lines, or its first slab) into A.
__device__ __forceinline__ void item_load(const BatchArgs &a, const ItemView &v, const float2 *S, float2 *A, bool conj)
{
    if (v.dim == 3) {
        const BatchCube &cb = a.cubes[v.cube];
        const float2 *src = v.src + (int64_t)v.s0 * cb.n0 * cb.n1;
        switch (cb.n0) {
#define FFT3_BATCH_CASE(N) \
    case N: slab_load<N>(src, S, cb.n1, A, cb.n0, conj); return;
            FFT3_BATCH_LENGTHS(FFT3_BATCH_CASE)
#undef FFT3_BATCH_CASE
        default: slab_load<0>(src, S, cb.n1, A, cb.n0, conj); return;
        }
    }
    const LineRt &L = a.lines[v.li];
    switch (v.es == 1 ? L.n : 0) {
#define FFT3_BATCH_CASE(N) \
    case N: lines_load<N>(v, L, S, A, conj); return;
        FFT3_BATCH_LENGTHS(FFT3_BATCH_CASE)
#undef FFT3_BATCH_CASE
    default: lines_load<0>(v, L, S, A, conj); return;
    }
}

// The rest of an item once its first tile is in A: transform and store it,
// then (slab items) load, transform and store the following slabs.
__device__ __forceinline__ void item_finish(const BatchArgs &a, const ItemView &v, float2 *A, float2 *B, bool conj)
{
    if (v.dim == 3) {
        const BatchCube &cb = a.cubes[v.cube];
        const LineRt &X = a.lines[cb.lx], &Y = a.lines[cb.ly];
        const int64_t nel = (int64_t)cb.n0 * cb.n1;
        for (int s = v.s0; s < v.s1; ++s) {
            if (s > v.s0) {
                __syncthreads();
                switch (cb.n0) {
#define FFT3_BATCH_CASE(N) \
    case N: slab_load<N>(v.src + s * nel, nullptr, cb.n1, A, cb.n0, conj); break;
                    FFT3_BATCH_LENGTHS(FFT3_BATCH_CASE)
#undef FFT3_BATCH_CASE
                default: slab_load<0>(v.src + s * nel, nullptr, cb.n1, A, cb.n0, conj); break;
                }
                __syncthreads();
            }
            switch (cb.n0) {
#define FFT3_BATCH_CASE(N) \
    case N: slab_finish<N>(v.dst + s * nel, X, Y, a.tw, A, B, conj); break;
                FFT3_BATCH_LENGTHS(FFT3_BATCH_CASE)
#undef FFT3_BATCH_CASE
            default: slab_finish<0>(v.dst + s * nel, X, Y, a.tw, A, B, conj); break;
            }
        }
        return;
    }
    const LineRt &L = a.lines[v.li];
    switch (v.es == 1 ? L.n : 0) {
#define FFT3_BATCH_CASE(N) \
    case N: lines_finish<N>(v, L, a.tw, A, B, conj); return;
        FFT3_BATCH_LENGTHS(FFT3_BATCH_CASE)
#undef FFT3_BATCH_CASE
    default: lines_finish<0>(v, L, a.tw, A, B, conj); return;
    }
}

// Whether every item of the previous phase of v's problem has finished.
__device__ __forceinline__ bool deps_done(const BatchArgs &a, const ItemView &v)
{
    if (v.phase == 0)
        return true;
    const int *done = a.counters + 1 + 3 * v.cube;
    return ld_acquire_b(done + v.phase - 1) >= a.cubes[v.cube].items[v.phase - 1];
}

__global__ void __launch_bounds__(256, 3) k_batched(BatchArgs a)
{
    extern __shared__ __align__(16) float2 smem[];
    float2 *A = smem, *B = smem + a.buf_elems;
    float2 *S = a.prefetch ? smem + 2 * a.buf_elems : nullptr; // raw staging of the next item's first tile
    __shared__ int s_q, s_ok;
    const bool conj = a.conj != 0;
    if (threadIdx.x == 0)
        s_q = atomicAdd(a.counters, 1);
    __syncthreads();
    int q = s_q;
    bool pre = false; // S holds item q's first tile (uniform over the block)
    while (q < a.nitems) {
        const ItemView v = view_item(a, q);
        if (!pre && v.phase > 0) {
            if (threadIdx.x == 0) {
                const long long t0 = clock64();
                while (!deps_done(a, v)) {
                    if (clock64() - t0 > a.wait_budget) {
                        atomicOr(a.err, kErrWaitTimeout);
                        break;
                    }
                    __nanosleep(32);
                }
            }
        }
        if (pre)
            cp_async_wait_all();
        __syncthreads(); // dependencies met; this thread's staged copies landed
        if (threadIdx.x == 0)
            s_q = atomicAdd(a.counters, 1); // the next item, claimed now so its data can be staged
        item_load(a, v, pre ? S : nullptr, A, conj);
        __syncthreads(); // A complete, S free, s_q visible
        const int qn = s_q;
        bool pn = false;
        if (S && qn < a.nitems) {
            const ItemView w = view_item(a, qn);
            if (threadIdx.x == 0)
                s_ok = deps_done(a, w) && prefetchable(a, w);
            __syncthreads();
            if (s_ok) {
                issue_prefetch(a, w, S);
                pn = true;
            }
        }
        item_finish(a, v, A, B, conj);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(a.counters + 1 + 3 * v.cube + v.phase, 1);
        }
        q = qn;
        pre = pn;
    }
}

} // namespace fft3
