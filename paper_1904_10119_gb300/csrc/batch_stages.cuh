// batch_stages.cuh -- compile-time line transforms for the batched executor.
//
// The lines of one work item sit in shared memory in one of two layouts:
//   lines:   line i at buf + i*pitch, element j at padpos(j)
//   columns: column i at buf + padpos(i), element j at j*pitch
// A stage of radix R (Stockham, as in fft_engine.cuh) is flattened over all
// butterflies of all lines of the item, so every thread of the block works
// whatever the line length, and the stages ping-pong between two buffers
// with one block barrier each.  Line length and radix list are template
// parameters, so all index arithmetic is by constants; a line plan whose
// radix list matches no compiled sequence runs through runtime_stages.cuh.
#pragma once

#include "runtime_stages.cuh"

namespace fft3 {

template <int N, int R, int NS, bool COLS>
__device__ __forceinline__ void flat_stage(int nl, int pitch, const float2 *src, float2 *dst, const float2 *tw)
{
    constexpr int NB = N / R;
    const int total = nl * NB;
    for (int b = threadIdx.x; b < total; b += blockDim.x) {
        int line, q;
        if constexpr (COLS) { // consecutive threads take consecutive columns
            q = b / nl;
            line = b - q * nl;
        } else {
            line = b / NB;
            q = b - line * NB;
        }
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int j = q + r * NB;
            v[r] = COLS ? src[j * pitch + padpos(line)] : src[line * pitch + padpos(j)];
        }
        const int k = NS == 1 ? 0 : q % NS;
        if constexpr (NS > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r)
                v[r] = cmul(v[r], tw[(r - 1) * NS + k]);
        }
        Bfly<R>::run(v);
        const int base = NS == 1 ? q * R : (q / NS) * NS * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int j = base + r * NS;
            if (COLS)
                dst[j * pitch + padpos(line)] = v[r];
            else
                dst[line * pitch + padpos(j)] = v[r];
        }
    }
}

template <int N, bool COLS, int NS, int... Rs>
struct FlatStages;

template <int N, bool COLS, int NS>
struct FlatStages<N, COLS, NS> {
    __device__ __forceinline__ static float2 *run(int, int, float2 *cur, float2 *, const float2 *) { return cur; }
};

template <int N, bool COLS, int NS, int R, int... Rest>
struct FlatStages<N, COLS, NS, R, Rest...> {
    __device__ __forceinline__ static float2 *run(int nl, int pitch, float2 *cur, float2 *nxt, const float2 *tw)
    {
        flat_stage<N, R, NS, COLS>(nl, pitch, cur, nxt, tw);
        __syncthreads();
        return FlatStages<N, COLS, NS * R, Rest...>::run(nl, pitch, nxt, cur, tw + (R - 1) * NS);
    }
};

template <int N, int... Rs>
struct FlatPlan {
    __device__ __forceinline__ static bool match(const LineRt &L)
    {
        constexpr int rad[] = {Rs...};
        if (L.n != N || L.nst != (int)sizeof...(Rs))
            return false;
#pragma unroll
        for (int s = 0; s < (int)sizeof...(Rs); ++s)
            if (L.rad[s] != rad[s])
                return false;
        return true;
    }
    template <bool COLS>
    __device__ __forceinline__ static float2 *run(int nl, int pitch, float2 *A, float2 *B, const float2 *tw)
    {
        return FlatStages<N, COLS, 1, Rs...>::run(nl, pitch, A, B, tw);
    }
};

// The radix lists the planner picks by default for the lengths of the batched
// workloads (2, 3 and 5 factors up to 128).
#define FFT3_FLAT_PLANS(X)                                                                              \
    X(16, 16) X(24, 8, 3) X(32, 16, 2) X(40, 8, 5) X(48, 16, 3) X(64, 16, 4) X(80, 16, 5) X(96, 16, 2, 3) \
    X(128, 16, 8) X(20, 4, 5) X(60, 4, 5, 3) X(120, 8, 5, 3) X(8, 8) X(12, 4, 3) X(4, 4)

// Transforms nl lines (COLS = false) or columns (COLS = true) of length L.n
// held in A; returns the buffer (A or B) holding the result.  Every compiled
// sequence is tried (one out-of-line copy per layout).
template <bool COLS>
__device__ __noinline__ float2 *batch_stages_all(const LineRt &L, int nl, int pitch, float2 *A, float2 *B,
                                                 const float2 *tw)
{
#define FFT3_FLAT_TRY(N, ...)                                                    \
    if (FlatPlan<N, __VA_ARGS__>::match(L))                                      \
        return FlatPlan<N, __VA_ARGS__>::template run<COLS>(nl, pitch, A, B, tw);
    FFT3_FLAT_PLANS(FFT3_FLAT_TRY)
#undef FFT3_FLAT_TRY
    return COLS ? run_stages_cols(L, nl, pitch, A, B, tw) : run_stages_lines(L, nl, pitch, A, B, tw);
}

// The same when the line length is known at compile time (NF > 0): only the
// sequences of that length are tried inline; NF = 0 calls batch_stages_all.
template <bool COLS, int NF>
__device__ __forceinline__ float2 *batch_stages(const LineRt &L, int nl, int pitch, float2 *A, float2 *B,
                                                const float2 *tw)
{
    if constexpr (NF == 0) {
        return batch_stages_all<COLS>(L, nl, pitch, A, B, tw);
    } else {
#define FFT3_FLAT_TRY(N, ...)                                                    \
        if constexpr (N == NF) {                                                 \
            if (FlatPlan<N, __VA_ARGS__>::match(L))                              \
                return FlatPlan<N, __VA_ARGS__>::template run<COLS>(nl, pitch, A, B, tw); \
        }
        FFT3_FLAT_PLANS(FFT3_FLAT_TRY)
#undef FFT3_FLAT_TRY
        return batch_stages_all<COLS>(L, nl, pitch, A, B, tw);
    }
}

} // namespace fft3
