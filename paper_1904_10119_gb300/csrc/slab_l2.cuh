// slab_l2.cuh -- slab stage of the slab-pencil decomposition (Section 2.3,
// Fig. 3ddftopt a: a 2D DFT on each n0 x n1 slab) for slabs too large for one
// block: x-line tiles and y-column tiles of the same slab run in one
// persistent launch, so a slab's x-stage output is read back by its y tiles
// from L2 rather than from HBM.
//
// Work is handed out by a ticket counter in this order (D = lag in slabs):
//   x tiles of slab 0 .. D-1, then for every later slab s: the x tiles of s
//   followed by the y tiles of s - D, then the y tiles of the last D slabs.
// A y tile waits until all x tiles of its slab have finished.  Those tiles
// hold smaller tickets, so they were claimed by blocks that are already
// running and never wait themselves: the waits always end, whatever the
// number of resident blocks.  Each wait is still bounded (about two seconds
// of clock cycles); on expiry the kernel records kErrWaitTimeout in the
// plan's error word and carries on, and fft3_plan_check reports
// FFT3_ERR_TIMEOUT.
#pragma once

#include "pass_kernels.cuh"
#include "tma.cuh"

namespace fft3 {

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

struct GLoadCG { // strided, L2-only loads (data written earlier in this launch)
    const float2 *p;
    int64_t s;
    bool conj;
    __device__ __forceinline__ float2 operator()(int j) const
    {
        float2 v = __ldcg(p + (int64_t)j * s);
        return conj ? cconj(v) : v;
    }
};

// Column layout with padded positions: element j of column l at
// p[padpos(j)*LPT + l] (conflict free also for narrow tiles).
template <int LPT>
struct SmemColPad {
    float2 *p; // buf + l
    __device__ __forceinline__ float2 operator()(int j) const { return p[padpos(j) * LPT]; }
    __device__ __forceinline__ void operator()(int k, float2 v) const { p[padpos(k) * LPT] = v; }
};

struct SlabTicket {
    int64_t slab;
    int tile;
    bool is_y;
};

__device__ __forceinline__ SlabTicket decode_slab_ticket(int64_t q, int64_t nslabs, int64_t tps, int64_t D)
{
    SlabTicket t;
    if (q < D * tps) {
        t.slab = q / tps;
        t.tile = (int)(q % tps);
        t.is_y = false;
        return t;
    }
    q -= D * tps;
    const int64_t mid = (nslabs - D) * 2 * tps;
    if (q < mid) {
        const int64_t ph = q / (2 * tps), w = q % (2 * tps);
        if (w < tps) {
            t.slab = D + ph;
            t.tile = (int)w;
            t.is_y = false;
        } else {
            t.slab = ph;
            t.tile = (int)(w - tps);
            t.is_y = true;
        }
        return t;
    }
    q -= mid;
    t.slab = (nslabs - D) + q / tps;
    t.tile = (int)(q % tps);
    t.is_y = true;
    return t;
}

constexpr long long kWaitBudgetCycles = 4000000000LL; // about two seconds

// N x N slabs, fixed plan (N, T, Rad), LPT rows (x tiles) or columns (y
// tiles) per tile, blockDim = LPT*T.  Small tiles let several blocks share an
// SM; the y tiles read L2-resident data, where narrow rows cost little.
// counters[0] = ticket, counters[1 + s] = finished x tiles of slab s.
template <int N, int T, class Rad, int LPT>
__global__ void __launch_bounds__(T *LPT) k_slab_l2(PassArgs a)
{
    constexpr int S = line_pitch(N);
    constexpr int TPS = N / LPT;
    extern __shared__ float2 smem[];
    float2 *tw = smem;
    float2 *buf = smem + tw_slots(a.tw_len);
    __shared__ int64_t s_ticket;
    load_twiddles(tw, a.tw, a.tw_len);
    const bool conj = a.conj != 0;
    const int64_t nslabs = a.g.A * a.g.B;
    const int64_t D = nslabs < 2 ? nslabs : 2;
    const int64_t total = 2 * (int64_t)TPS * nslabs;
    int *ticket = a.counters;
    int *done = a.counters + 1;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0)
            s_ticket = atomicAdd(ticket, 1);
        __syncthreads();
        const int64_t q = s_ticket;
        if (q >= total)
            break;
        const SlabTicket tk = decode_slab_ticket(q, nslabs, TPS, D);
        const int64_t sa = tk.slab % a.g.A, sb = tk.slab / a.g.A;
        const int64_t slab_off = sa * a.g.ia + sb * a.g.ib;
        if (!tk.is_y) {
            // x lines: rows tile*16 + l of the slab, contiguous, thread t of line l
            const int t = threadIdx.x % T, l = threadIdx.x / T;
            const int64_t row = (int64_t)tk.tile * LPT + l;
            GLoad1 src{a.in + slab_off + row * a.g.ic, true, conj};
            GStore1 dst{a.out + slab_off + row * a.g.oc, true, conj};
            SmemLine<S> sm{buf + l * S};
            EngineFixed<N, T, 1, Rad>::template run<true, false>(t, src, sm, dst, tw);
            __syncthreads();
            if (threadIdx.x == 0 && tk.slab != a.nosignal_slab) {
                __threadfence();
                atomicAdd(done + tk.slab, 1);
            }
        } else {
            if (threadIdx.x == 0) {
                const long long t0 = clock64();
                while (ld_acquire(done + tk.slab) < TPS) {
                    if (clock64() - t0 > a.wait_budget) {
                        atomicOr(a.err, kErrWaitTimeout);
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __syncthreads();
            // y lines: columns tile*16 + l, element stride n0, c fastest
            const int l = threadIdx.x % LPT, t = threadIdx.x / LPT;
            const int64_t col = (int64_t)tk.tile * LPT + l;
            GLoadCG src{a.out + slab_off + col, a.g.ic, conj};
            GStore dst{a.out + slab_off + col, a.g.oc, true, conj};
            SmemColPad<LPT> sm{buf + l};
            EngineFixed<N, T, 1, Rad>::template run<true, false>(t, src, sm, dst, tw);
        }
    }
}

// Accessors of the blocked layout: rows of 16 columns, 16 complex values
// apart (a compile-time stride, so one base register serves a whole line).
struct GStoreBlk { // element k of an x line at p[(k/16)*s + k%16]
    float2 *p;
    int64_t s;
    bool conj;
    __device__ __forceinline__ void operator()(int k, float2 v) const
    {
        p[(int64_t)(k >> 4) * s + (k & 15)] = conj ? cconj(v) : v;
    }
};
struct GCol16 { // element j of a column of a block at p[16 j]; stores are marked
                // evict-first (the final values leave L2 first)
    float2 *p;
    bool conj;
    __device__ __forceinline__ void operator()(int k, float2 v) const { __stcs(p + 16 * k, conj ? cconj(v) : v); }
};

// Readers of a landing buffer filled by TMA (dense, no padding), with the
// conjugation of the inverse transform.
struct LandRow { // element j of this thread's row at p[j]
    const float2 *p;
    bool conj;
    __device__ __forceinline__ float2 operator()(int j) const { return conj ? cconj(p[j]) : p[j]; }
};
template <int LPT>
struct LandCol { // element j of column l at p[j*LPT] (p = buffer + l)
    const float2 *p;
    bool conj;
    __device__ __forceinline__ float2 operator()(int j) const
    {
        const float2 v = p[j * LPT];
        return conj ? cconj(v) : v;
    }
};

// Slab stage fused with the slab-to-pencil redistribution (Section 2.3): the
// 2D DFT of every N x N slab z, its output laid out as the z pencils
// [x/16][z][y][x%16] the last pass reads, in one persistent launch whose
// intermediate stays in L2 (one HBM sweep for the x and y stages).
//
// Tiles are handed out in the ticket order of k_slab_l2 (x tiles of slab s,
// then y tiles of slab s - D).  An x tile is LPT consecutive rows of `in`
// (one contiguous bulk copy); its transformed rows are stored into the
// blocked layout.  A y tile is LPT of the 16 columns of one block [x/16][z]
// (N rows 128 bytes apart, loaded as 2D TMA boxes of the blocked layout once
// every x tile of the slab has signalled); it is transformed in place.
//
// Warp roles: warps 0 .. T*LPT/32-1 transform (named barrier 1); lane 0 of
// the last warp is the producer: it claims tickets, waits (bounded) for the
// x tiles a y tile needs, and issues the loads into a ring of NBUF landing
// buffers (full / empty mbarriers), so loads run NBUF-1 tiles ahead of the
// arithmetic.  The first stage moves a landing buffer into the padded work
// buffer, after which the buffer is handed back.
//
// Deadlock freedom: tickets are claimed in increasing order, an x tile is
// loaded as soon as it is claimed, and a block's transforming warps depend
// only on their own loads; so every claimed x tile finishes, and a y tile
// waits only for x tiles with smaller tickets.  Every wait is bounded: on
// expiry the kernel records kErrWaitTimeout and carries on (or, for a load
// that never lands, stops), and fft3_plan_check reports FFT3_ERR_TIMEOUT.
//
// The input is read with an evict-first L2 policy and the final values are
// stored evict-first, so the slabs' intermediate values are what L2 keeps.
// Geometry: in row stride g.ic (== N), slab stride g.ia; blocked output slab
// stride g.oa = 16 N, block stride g.ob = 16 N n2; `tws` maps the workspace
// as rows of 16 values, boxes of LPT x min(N, 256).
template <int N, int T, class Rad, int LPT, int NBUF>
__global__ void __launch_bounds__(T *LPT + 32, LPT >= 8 ? 1 : 2) k_slab_tma(PassArgs a, const __grid_constant__ CUtensorMap tws)
{
    constexpr int S = line_pitch(N);
    constexpr int TPS = N / LPT;
    constexpr int NC = T * LPT; // transforming threads
    constexpr int BOX = N < 256 ? N : 256;
    constexpr uint32_t TILE_BYTES = (uint32_t)LPT * N * 8u;
    static_assert(NC % 32 == 0 && N % BOX == 0 && (LPT * 8) % 16 == 0 && 16 % LPT == 0, "tile shape");
    extern __shared__ __align__(128) float2 smem[];
    __shared__ __align__(8) uint64_t full[NBUF], empty[NBUF];
    __shared__ int64_t s_tk[NBUF];
    float2 *tw = smem;
    float2 *work = smem + tw_slots(a.tw_len);
    float2 *land = work + round_up(LPT * S, 16);
    load_twiddles(tw, a.tw, a.tw_len);
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int b = 0; b < NBUF; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], 1);
        }
        fence_mbar_init();
    }
    __syncthreads();
    const bool conj = a.conj != 0;
    const int64_t nslabs = a.g.A * a.g.B;
    const int64_t D = nslabs < 3 ? nslabs : 3;
    const int64_t total = 2 * (int64_t)TPS * nslabs;
    if (tid >= NC) {
        // ---------------------------------------------------------- producer
        if (tid != NC)
            return;
        int *ticket = a.counters;
        const int *done = a.counters + 1;
        const uint64_t pol = l2_evict_first_policy();
        int64_t armed[NBUF]; // last ring position loaded into each buffer (-1: none)
#pragma unroll
        for (int b = 0; b < NBUF; ++b)
            armed[b] = -1;
        for (int64_t i = 0;; ++i) {
            const int b = (int)(i % NBUF);
            if (i >= NBUF && !mbar_wait(&empty[b], (uint32_t)((i / NBUF - 1) & 1), 2 * a.wait_budget)) {
                atomicOr(a.err, kErrWaitTimeout); // the transforming warps stopped
                break;
            }
            const int64_t q = atomicAdd(ticket, 1);
            s_tk[b] = q;
            if (q >= total) {
                mbar_arrive(&full[b]); // end of work: no bytes to wait for
                armed[b] = i;
                break;
            }
            const SlabTicket tk = decode_slab_ticket(q, nslabs, TPS, D);
            float2 *dst = land + (int64_t)b * LPT * N;
            if (!tk.is_y) {
                mbar_expect_tx(&full[b], TILE_BYTES);
                bulk_load(dst, a.in + tk.slab * a.g.ia + (int64_t)tk.tile * LPT * a.g.ic, TILE_BYTES, &full[b], pol);
            } else {
                const long long t0 = clock64();
                while (ld_acquire(done + tk.slab) < TPS) {
                    if (clock64() - t0 > a.wait_budget) { // carry on; the plan reports the timeout
                        atomicOr(a.err, kErrWaitTimeout);
                        break;
                    }
                    __nanosleep(64);
                }
                fence_proxy_async_global(); // the x tiles' stores, seen through the acquire, before the TMA reads
                mbar_expect_tx(&full[b], TILE_BYTES);
                const int col = tk.tile * LPT;
                const int64_t row0 = (int64_t)(col >> 4) * (a.g.ob / 16) + tk.slab * N;
#pragma unroll 1
                for (int k = 0; k < N / BOX; ++k)
                    tma_load_2d(dst + k * BOX * LPT, &tws, col & 15, (int)(row0 + k * BOX), &full[b]);
            }
            armed[b] = i;
        }
        // the block's shared memory must outlive every copy issued into it
#pragma unroll
        for (int b = 0; b < NBUF; ++b)
            if (armed[b] >= 0 && !mbar_wait(&full[b], (uint32_t)((armed[b] / NBUF) & 1), a.wait_budget))
                atomicOr(a.err, kErrWaitTimeout);
        return;
    }
    // --------------------------------------------------- transforming warps
    int *done = a.counters + 1;
    for (int64_t i = 0;; ++i) {
        const int b = (int)(i % NBUF);
        // twice the producer's budget: a y tile whose slab never completes is
        // loaded (and flagged) once the producer's own wait has run out
        bool late = !mbar_wait(&full[b], (uint32_t)((i / NBUF) & 1), 2 * a.wait_budget);
        uint32_t any;
        asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, 1, %2, p;\n\t"
                     "selp.u32 %0, 1, 0, q;\n\t}"
                     : "=r"(any)
                     : "r"(late ? 1u : 0u), "n"(NC)
                     : "memory");
        if (any) { // a load never landed: stop (the producer's waits expire too)
            if (tid == 0)
                atomicOr(a.err, kErrWaitTimeout);
            break;
        }
        const int64_t q = s_tk[b];
        if (q >= total)
            break;
        const SlabTicket tk = decode_slab_ticket(q, nslabs, TPS, D);
        const float2 *lb = land + (int64_t)b * LPT * N;
        auto release = [&]() {
            if (tid == 0)
                mbar_arrive(&empty[b]);
        };
        if (!tk.is_y) {
            const int t = tid % T, l = tid / T;
            const int64_t row = (int64_t)tk.tile * LPT + l;
            LandRow src{lb + l * N, conj};
            GStoreBlk dst{a.out + tk.slab * a.g.oa + row * 16, a.g.ob, conj};
            SmemLine<S> sm{work + l * S};
            EngineSplitFirst<N, T, Rad, 1, NC>::run(t, src, sm, dst, tw, release);
            fence_proxy_async_global(); // this thread's stores, before the release below
            lines_sync<1, NC>();
            if (tid == 0 && tk.slab != a.nosignal_slab) {
                __threadfence();
                atomicAdd(done + tk.slab, 1);
            }
        } else {
            const int l = tid % LPT, t = tid / LPT;
            const int col = tk.tile * LPT + l;
            LandCol<LPT> src{lb + l, conj};
            GCol16 dst{a.out + (col >> 4) * a.g.ob + tk.slab * a.g.oa + (col & 15), conj};
            SmemColPad<LPT> sm{work + l};
            EngineSplitFirst<N, T, Rad, 1, NC>::run(t, src, sm, dst, tw, release);
            lines_sync<1, NC>(); // the work buffer is read out before the next tile's first stage
        }
    }
}

} // namespace fft3
