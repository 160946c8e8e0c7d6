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

} // namespace fft3
