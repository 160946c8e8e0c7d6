// k_cstream.cu -- streamed strided-line pass (y or z lines, tiles of LPT
// adjacent columns) whose loads overlap its arithmetic.
//
// A tile of LPT columns of N points (128 KB for N = 1024, LPT = 16) is too
// large for two copies to sit in one SM's shared memory, so a whole tile can
// not be double-buffered.  Instead the Cooley-Tukey split of Section 2.1
// (Eq. ct with n0 = Q, n1 = M) is taken in decimation-in-time order:
//   (I)   each decimated sub-line x_q[j'] = x[Q*j' + q] (q < Q) is loaded by
//         TMA as one box (LPT columns x M rows at row stride Q*ij) and gets
//         its M-point DFT, M = R1*R2, as two Stockham stages into slot q of
//         the tile's result buffer,
//   (II)  twiddle w_N^{q k'},
//   (IV)  one radix-Q butterfly per (k', column): y[k' + M*s], s < Q, stored
//         straight to global memory (LPT*8 contiguous bytes per row).
// The threads form G groups; group g transforms the sub-lines q = g, g+G, ...
// through its own ring of S staging buffers.  A staging buffer is refilled as
// soon as the group has read its first-stage inputs out of it, so nearly the
// whole ring (G*S sub-lines, across tile boundaries) is in flight while the
// groups compute and while the block stores the previous tile.
//
// With P = 2 a cluster of two blocks shares a tile twice as wide (LPT = 32
// columns, 256-byte rows): block r loads and transforms the sub-lines
// q in [r*Q/2, (r+1)*Q/2) into its own slots, and in the final stage computes
// the outputs k' in [r*M/2, (r+1)*M/2) of all LPT columns, reading the other
// block's slots through distributed shared memory.  Rows of 256 bytes are what
// lines strided by whole planes (z lines) need to reach full DRAM throughput;
// a single block can not hold a 32-column tile's result.
//
// Twiddles: the stage-major table of the radix list (R1, R2, Q) for length
// N.  Its first M-1 entries are the M-point table of (R1, R2) (an entry
// w_N^{r k N/(NS R)} depends on NS*R only) and the last (Q-1)*M entries are
// w_N^{r k'}, the twiddles (II) of the final stage.
#include <cooperative_groups.h>

#include "pass_tc.cuh"
#include "pass_tma.cuh"
#include "plans.h"

namespace cg = cooperative_groups;

namespace fft3 {

// Barrier of thread group g (named barriers 1..G; 0 is __syncthreads), with
// an OR-reduction of a predicate.  The ids are compile-time constants so the
// kernel reserves only G + 1 barriers.
template <int ID, int NT>
__device__ __forceinline__ bool named_sync_or(bool pred)
{
    uint32_t out;
    asm volatile("{\n\t.reg .pred p, q;\n\t"
                 "setp.ne.u32 p, %1, 0;\n\t"
                 "bar.red.or.pred q, %2, %3, p;\n\t"
                 "selp.u32 %0, 1, 0, q;\n\t}"
                 : "=r"(out)
                 : "r"(pred ? 1u : 0u), "n"(ID), "n"(NT)
                 : "memory");
    return out != 0;
}

template <int G, int NT>
__device__ __forceinline__ bool group_sync_or(int g, bool pred)
{
    static_assert(G <= 4, "at most four groups");
    if constexpr (G == 1) {
        return __syncthreads_or(pred) != 0;
    } else {
        switch (g) {
        case 0: return named_sync_or<1, NT>(pred);
        case 1: return named_sync_or<2, NT>(pred);
        case 2: return named_sync_or<3, NT>(pred);
        default: return named_sync_or<4, NT>(pred);
        }
    }
}

template <int G, int NT>
__device__ __forceinline__ void group_sync(int g)
{
    if constexpr (G == 1) {
        __syncthreads();
    } else {
        switch (g) {
        case 0: asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory"); break;
        case 1: asm volatile("bar.sync 2, %0;" ::"n"(NT) : "memory"); break;
        case 2: asm volatile("bar.sync 3, %0;" ::"n"(NT) : "memory"); break;
        default: asm volatile("bar.sync 4, %0;" ::"n"(NT) : "memory"); break;
        }
    }
}

// Block barrier (P = 1) or cluster barrier (P = 2, with the release /
// acquire ordering that makes the slots visible to the other block).
template <int P>
__device__ __forceinline__ void tile_sync()
{
    if constexpr (P == 1)
        __syncthreads();
    else
        cg::this_cluster().sync();
}

// The two halves of a cluster barrier (P = 2): every thread of both blocks
// arrives after its last read of the tile's slots, and waits before its first
// write of the next tile's slots, so the barrier's latency overlaps the next
// tile's first load.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

// Staging buffer as a tile accessor (line = column, position = row of the
// sub-line), conjugating on load for the inverse transform.
template <int LPT>
struct StageTile {
    const float2 *p;
    bool conj;
    __device__ __forceinline__ float2 operator()(int l, int j) const
    {
        const float2 v = p[j * LPT + l];
        return conj ? cconj(v) : v;
    }
};

// TC = 0: FP32 sub-line stages.  TC = 1: the first 16-point stage of every
// sub-line on the tensor cores in split BF16 (tc_stage.cuh); TC = 2: both.
template <int N, int Q, int R1, int R2, int G, int S, int LPT, int P, int TC>
__global__ void __launch_bounds__(G *LPT *R2, cstream_min_blocks(cstream_smem_p(N, Q, Q / P, LPT, G *S), G *LPT *R2))
    k_cstream(PassArgs a, const __grid_constant__ CUtensorMap tin)
{
    static_assert(TC == 0 || (R1 == 16 && R2 == 16 && P == 1), "tensor-core sub-lines are 16 x 16");
    constexpr int M = R1 * R2;
    constexpr int T1 = M / R1;          // threads per column in a group (= first-stage butterflies)
    constexpr int GT = LPT * T1;        // threads per group
    constexpr int THREADS = G * GT;
    constexpr int QP = Q / P;           // sub-lines (slots) per block
    constexpr int W = QP / G;           // sub-lines per group per tile
    constexpr int MP = M / P;           // final-stage outputs k' per block
    constexpr int NB2 = M / R2;         // second-stage butterflies per column
    constexpr int BPT2 = (NB2 + T1 - 1) / T1;
    constexpr int TF = THREADS / LPT;   // threads per column in the final stage
    constexpr uint32_t SUB_BYTES = (uint32_t)M * LPT * 8u;
    static_assert(M * Q == N && Q % P == 0 && QP % G == 0 && M % P == 0 && GT % 32 == 0,
                  "N = M * Q, whole sub-lines per block and group, whole warps per group");
    static_assert(M <= 256 && LPT <= 256 && (LPT * 8) % 16 == 0, "a sub-line is one TMA box");
    static_assert(P == 1 || P == 2, "one block or a pair");
    extern __shared__ __align__(128) float2 smem[];
    __shared__ __align__(8) uint64_t bars[G * S];
    float2 *tw = smem;
    float2 *res = smem + tw_slots(a.tw_len); // QP slots of M x LPT, slot s at s*M*LPT
    float2 *stg = res + QP * M * LPT;        // G*S staging buffers of M x LPT; group g owns g*S .. g*S+S-1
    load_twiddles(tw, a.tw, a.tw_len);
    const int tid = threadIdx.x, g = tid / GT, gtid = tid % GT;
    const int l = gtid % LPT, t1 = gtid / LPT;
    const bool conj = a.conj != 0;
    int r = 0;
    const float2 *peer = res; // the other block's slots (P = 2)
    if constexpr (P > 1) {
        cg::cluster_group cluster = cg::this_cluster();
        r = (int)cluster.block_rank();
        peer = cluster.map_shared_rank(res, r ^ 1);
    }
    const int64_t cid = blockIdx.x / P, ncl = gridDim.x / P;
    TcW wtc;
    if constexpr (TC > 0) {
        __syncthreads(); // twiddles, including w_16^m at tw_split_off
        tc_build_w(wtc, tw + a.tw_split_off);
    }
    if (tid == 0) {
        for (int b = 0; b < G * S; ++b)
            mbar_init(&bars[b], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // The k-th sub-line of group g: tile cid + (k / W) * ncl, local slot g + G*(k % W)
    // (sub-line q = r*QP + slot), staging buffer g*S + k % S, mbarrier phase (k / S) & 1.
    auto tile_of = [&](int64_t k) { return cid + (k / W) * ncl; };
    const bool prefetch_l2 = a.g.ij * 8 <= (1 << 20);
    auto issue = [&](int64_t k) {
        const int64_t tile = tile_of(k);
        if (tile >= a.ntiles)
            return;
        const TileId id = decode_tile(tile, a.tiles_c, a.g.A, LPT);
        const int b = g * S + (int)(k % S);
        mbar_expect_tx(&bars[b], SUB_BYTES);
        tma_load_5d(stg + b * M * LPT, &tin, (int)id.c0, r * QP + g + G * (int)(k % W), 0, (int)id.a,
                    (int)id.b, &bars[b]);
        // the group's following sub-line goes to L2 now, so its load into the
        // staging buffer (issued once the buffer is free) finds it there; not
        // for rows megabytes apart (every row its own page: measured slower)
        const int64_t kp = k + S;
        const int64_t tp = tile_of(kp);
        if (prefetch_l2 && tp < a.ntiles) {
            const TileId ip = decode_tile(tp, a.tiles_c, a.g.A, LPT);
            tma_prefetch_5d(&tin, (int)ip.c0, r * QP + g + G * (int)(kp % W), 0, (int)ip.a, (int)ip.b);
        }
    };
    if (gtid == 0) {
        for (int k = 0; k < S; ++k)
            issue(k);
    }
    // With one second-stage butterfly per thread (q2 = t1) its twiddles
    // w^{r (q2 mod R1)} are the same for every sub-line and tile: kept in registers.
    float2 w2[R2];
    if constexpr (BPT2 == 1) {
        __syncthreads(); // twiddles in shared memory
#pragma unroll
        for (int r = 1; r < R2; ++r)
            w2[r] = t1 < NB2 ? tw[(R1 - 1) + (r - 1) * R1 + t1 % R1] : make_float2(1.f, 0.f);
    }
    // A wait that runs out of budget marks the group failed: it stops waiting
    // and loading but keeps every barrier (the other groups and the block
    // barriers stay matched), and at the end waits, bounded, for the copies it
    // still has in flight.
    bool failed = false;
    int64_t k_fail = 0;
    int64_t k = 0;
    bool armed = false; // P = 2: this thread arrived after the previous tile's final stage
    for (int64_t tile = cid; tile < a.ntiles; tile += ncl) {
        const TileId id = decode_tile(tile, a.tiles_c, a.g.A, LPT);
#pragma unroll 1
        for (int w = 0; w < W; ++w, ++k) {
            const int q = g + G * w; // local slot
            const int b = g * S + (int)(k % S);
            const bool late = !failed && !mbar_wait(&bars[b], (uint32_t)((k / S) & 1), a.wait_budget);
            const float2 *sb = stg + b * M * LPT;
            float2 *slot = res + q * M * LPT;
            if constexpr (TC > 0) {
                // (I) first 16-point stage on the tensor cores: staging buffer -> slot q
                tc_stage16<M, 1, LPT, true>(StageTile<LPT>{sb, conj}, TileColSmem<LPT>{slot}, tw, wtc,
                                            gtid >> 5, GT / 32);
                if (group_sync_or<G, GT>(g, late) && !failed) {
                    failed = true;
                    k_fail = k;
                }
                if (gtid == 0 && !failed)
                    issue(k + S); // the staging buffer is read out: refill it
            } else {
                // (I) first stage, radix R1, NS = 1: inputs x_q[t1 + r*T1] of column l
                float2 x[R1];
#pragma unroll
                for (int r = 0; r < R1; ++r) {
                    const float2 e = sb[(t1 + r * T1) * LPT + l];
                    x[r] = conj ? cconj(e) : e;
                }
                if (group_sync_or<G, GT>(g, late) && !failed) {
                    failed = true;
                    k_fail = k;
                }
                if (gtid == 0 && !failed)
                    issue(k + S); // the staging buffer is read out: refill it
                Bfly<R1>::run(x);
                if constexpr (P > 1) {
                    if (armed) { // both blocks are done reading the previous tile's slots
                        cluster_wait();
                        armed = false;
                    }
                }
#pragma unroll
                for (int r = 0; r < R1; ++r)
                    slot[(t1 * R1 + r) * LPT + l] = x[r];
                group_sync<G, GT>(g);
            }
            if constexpr (TC == 2) {
                // (I) second 16-point stage on the tensor cores, in place in slot q: with
                // NS = 16 and M = 256 the outputs of a butterfly are its own inputs'
                // positions, and a warp reads all its inputs before its MMAs
                tc_stage16<M, R1, LPT, true>(TileColSmem<LPT>{slot}, TileColSmem<LPT>{slot}, tw + (R1 - 1), wtc,
                                             gtid >> 5, GT / 32);
                continue;
            }
            // (I) second stage, radix R2, NS = R1, in place in slot q
            float2 y[BPT2][R2];
#pragma unroll
            for (int bb = 0; bb < BPT2; ++bb) {
                const int q2 = t1 + bb * T1;
                if (q2 < NB2) {
#pragma unroll
                    for (int r = 0; r < R2; ++r)
                        y[bb][r] = slot[(q2 + r * NB2) * LPT + l];
                }
            }
            group_sync<G, GT>(g);
            const float2 *tw2 = tw + (R1 - 1);
#pragma unroll
            for (int bb = 0; bb < BPT2; ++bb) {
                const int q2 = t1 + bb * T1;
                if (q2 < NB2) {
                    const int kk = q2 % R1;
#pragma unroll
                    for (int r = 1; r < R2; ++r)
                        y[bb][r] = cmul(y[bb][r], BPT2 == 1 ? w2[r] : tw2[(r - 1) * R1 + kk]);
                    Bfly<R2>::run(y[bb]);
                    const int base = (q2 / R1) * M + kk;
#pragma unroll
                    for (int r = 0; r < R2; ++r)
                        slot[(base + r * R1) * LPT + l] = y[bb][r];
                }
            }
        }
        tile_sync<P>(); // every slot of the tile (of both blocks) is complete
        // (II)+(IV): radix-Q stage with NS = M over the Q slots, stored to global
        {
            const int lf = tid % LPT, tf = tid / LPT;
            const int64_t c = id.c0 + lf;
            const bool valid = c < a.g.C;
            float2 *op = a.out + c * a.g.oc + id.a * a.g.oa + id.b * a.g.ob;
            const float2 *twf = tw + (M - 1);
#pragma unroll 2
            for (int kk = r * MP + tf; kk < (r + 1) * MP; kk += TF) {
                float2 z[Q];
#pragma unroll
                for (int s = 0; s < Q; ++s) {
                    const float2 *src = (s / QP == r) ? res : peer;
                    z[s] = src[((s % QP) * M + kk) * LPT + lf];
                }
#pragma unroll
                for (int s = 1; s < Q; ++s)
                    z[s] = cmul(z[s], twf[(s - 1) * M + kk]);
                Bfly<Q>::run(z);
                if (valid) {
#pragma unroll
                    for (int s = 0; s < Q; ++s)
                        op[(int64_t)(kk + s * M) * a.g.ok] = conj ? cconj(z[s]) : z[s];
                }
            }
        }
        if constexpr (P > 1) {
            cluster_arrive(); // waited for before this thread's next slot write
            armed = true;
        } else {
            __syncthreads(); // the next tile's first stages overwrite the slots
        }
    }
    if constexpr (P > 1) {
        if (armed)
            cluster_wait(); // the other block has finished reading this block's slots
    }
    if (failed && gtid == 0) {
        atomicOr(a.err, kErrWaitTimeout);
        for (int64_t v = k_fail; v < k_fail + S; ++v)
            if (tile_of(v) < a.ntiles)
                mbar_wait(&bars[g * S + (int)(v % S)], (uint32_t)((v / S) & 1), a.wait_budget);
    }
}

template <int N, int Q, int R1, int R2, int G, int S, int LPT, int P, int TC>
constexpr const void *cstream_tc_ptr()
{
    if constexpr (R1 == 16 && R2 == 16 && P == 1)
        return (const void *)&k_cstream<N, Q, R1, R2, G, S, LPT, P, TC>;
    else
        return nullptr;
}

#define FFT3_CSTREAM_ROW(N, Q, R1, R2, G, S, LPT, P)                                      \
    {N, Q, R1, R2, G, S, LPT, P, G * LPT * R2, (const void *)&k_cstream<N, Q, R1, R2, G, S, LPT, P, 0>, \
     {cstream_tc_ptr<N, Q, R1, R2, G, S, LPT, P, 1>(), cstream_tc_ptr<N, Q, R1, R2, G, S, LPT, P, 2>()}},

static const CStreamKernel g_cstream_kernels[] = {FFT3_CSTREAM_LIST(FFT3_CSTREAM_ROW)};

const CStreamKernel *cstream_kernels(int *count)
{
    *count = (int)(sizeof(g_cstream_kernels) / sizeof(g_cstream_kernels[0]));
    return g_cstream_kernels;
}

} // namespace fft3
