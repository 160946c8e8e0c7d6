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
// Twiddles: the stage-major table of the radix list (R1, R2, Q) for length
// N.  Its first M-1 entries are the M-point table of (R1, R2) (an entry
// w_N^{r k N/(NS R)} depends on NS*R only) and the last (Q-1)*M entries are
// w_N^{r k'}, the twiddles (II) of the final stage.
#include "pass_tma.cuh"
#include "plans.h"

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

template <int N, int Q, int R1, int R2, int G, int S, int LPT>
__global__ void __launch_bounds__(G *LPT *R2, cstream_min_blocks(N, Q, LPT, G *S, G *LPT *R2))
    k_cstream(PassArgs a, const __grid_constant__ CUtensorMap tin)
{
    constexpr int M = R1 * R2;
    constexpr int T1 = M / R1;          // threads per column in a group (= first-stage butterflies)
    constexpr int GT = LPT * T1;        // threads per group
    constexpr int THREADS = G * GT;
    constexpr int W = Q / G;            // sub-lines per group per tile
    constexpr int NB2 = M / R2;         // second-stage butterflies per column
    constexpr int BPT2 = (NB2 + T1 - 1) / T1;
    constexpr int TF = THREADS / LPT;   // threads per column in the final stage
    constexpr uint32_t SUB_BYTES = (uint32_t)M * LPT * 8u;
    static_assert(M * Q == N && Q % G == 0 && GT % 32 == 0, "N = M * Q, whole warps per group");
    static_assert(M <= 256 && (LPT * 8) % 16 == 0, "a sub-line is one TMA box");
    extern __shared__ __align__(128) float2 smem[];
    __shared__ __align__(8) uint64_t bars[G * S];
    float2 *tw = smem;
    float2 *res = smem + tw_slots(a.tw_len); // Q slots of M x LPT, slot q at q*M*LPT
    float2 *stg = res + N * LPT;             // G*S staging buffers of M x LPT; group g owns g*S .. g*S+S-1
    load_twiddles(tw, a.tw, a.tw_len);
    const int tid = threadIdx.x, g = tid / GT, gtid = tid % GT;
    const int l = gtid % LPT, t1 = gtid / LPT;
    const bool conj = a.conj != 0;
    if (tid == 0) {
        for (int b = 0; b < G * S; ++b)
            mbar_init(&bars[b], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // The k-th sub-line of group g: tile blockIdx.x + (k / W) * gridDim.x, q = g + G*(k % W),
    // staging buffer g*S + k % S, mbarrier phase (k / S) & 1.
    auto tile_of = [&](int64_t k) { return (int64_t)blockIdx.x + (k / W) * (int64_t)gridDim.x; };
    auto issue = [&](int64_t k) {
        const int64_t tile = tile_of(k);
        if (tile >= a.ntiles)
            return;
        const TileId id = decode_tile(tile, a.tiles_c, a.g.A, LPT);
        const int b = g * S + (int)(k % S);
        mbar_expect_tx(&bars[b], SUB_BYTES);
        tma_load_5d(stg + b * M * LPT, &tin, (int)id.c0, g + G * (int)(k % W), 0, (int)id.a, (int)id.b,
                    &bars[b]);
    };
    if (gtid == 0) {
        for (int k = 0; k < S; ++k)
            issue(k);
    }
    // A wait that runs out of budget marks the group failed: it stops waiting
    // and loading but keeps every barrier (the other groups and the block
    // barriers stay matched), and at the end waits, bounded, for the copies it
    // still has in flight.
    bool failed = false;
    int64_t k_fail = 0;
    int64_t k = 0;
    for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        const TileId id = decode_tile(tile, a.tiles_c, a.g.A, LPT);
#pragma unroll 1
        for (int w = 0; w < W; ++w, ++k) {
            const int q = g + G * w;
            const int b = g * S + (int)(k % S);
            const bool late = !failed && !mbar_wait(&bars[b], (uint32_t)((k / S) & 1), a.wait_budget);
            // (I) first stage, radix R1, NS = 1: inputs x_q[t1 + r*T1] of column l
            float2 x[R1];
            const float2 *sb = stg + b * M * LPT;
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
            float2 *slot = res + q * M * LPT;
#pragma unroll
            for (int r = 0; r < R1; ++r)
                slot[(t1 * R1 + r) * LPT + l] = x[r];
            group_sync<G, GT>(g);
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
                        y[bb][r] = cmul(y[bb][r], tw2[(r - 1) * R1 + kk]);
                    Bfly<R2>::run(y[bb]);
                    const int base = (q2 / R1) * M + kk;
#pragma unroll
                    for (int r = 0; r < R2; ++r)
                        slot[(base + r * R1) * LPT + l] = y[bb][r];
                }
            }
        }
        __syncthreads(); // every slot of the tile is complete
        // (II)+(IV): radix-Q stage with NS = M over the Q slots, stored to global
        {
            const int lf = tid % LPT, tf = tid / LPT;
            const int64_t c = id.c0 + lf;
            const bool valid = c < a.g.C;
            float2 *op = a.out + c * a.g.oc + id.a * a.g.oa + id.b * a.g.ob;
            const float2 *twf = tw + (M - 1);
#pragma unroll 2
            for (int kk = tf; kk < M; kk += TF) {
                float2 z[Q];
#pragma unroll
                for (int r = 0; r < Q; ++r)
                    z[r] = res[(kk + r * M) * LPT + lf];
#pragma unroll
                for (int r = 1; r < Q; ++r)
                    z[r] = cmul(z[r], twf[(r - 1) * M + kk]);
                Bfly<Q>::run(z);
                if (valid) {
#pragma unroll
                    for (int r = 0; r < Q; ++r)
                        op[(int64_t)(kk + r * M) * a.g.ok] = conj ? cconj(z[r]) : z[r];
                }
            }
        }
        __syncthreads(); // the next tile's first stages overwrite the slots
    }
    if (failed && gtid == 0) {
        atomicOr(a.err, kErrWaitTimeout);
        for (int64_t v = k_fail; v < k_fail + S; ++v)
            if (tile_of(v) < a.ntiles)
                mbar_wait(&bars[g * S + (int)(v % S)], (uint32_t)((v / S) & 1), a.wait_budget);
    }
}

#define FFT3_CSTREAM_ROW(N, Q, R1, R2, G, S, LPT) \
    {N, Q, R1, R2, G, S, LPT, G * LPT * R2, (const void *)&k_cstream<N, Q, R1, R2, G, S, LPT>},

static const CStreamKernel g_cstream_kernels[] = {FFT3_CSTREAM_LIST(FFT3_CSTREAM_ROW)};

const CStreamKernel *cstream_kernels(int *count)
{
    *count = (int)(sizeof(g_cstream_kernels) / sizeof(g_cstream_kernels[0]));
    return g_cstream_kernels;
}

} // namespace fft3
