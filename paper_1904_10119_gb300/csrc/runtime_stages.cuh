// runtime_stages.cuh -- runs a runtime radix list (LineRt) on lines held in
// shared memory, ping-ponging between two buffers with a block barrier after
// every stage.  Teams of T threads take one line each; lines beyond the number
// of teams are taken in further rounds.
#pragma once

#include "fft_engine.cuh"
#include "geom.h"

namespace fft3 {

template <class C>
struct SmemLineRtAccT { // line-major, padded positions
    C *p;
    __device__ __forceinline__ C operator()(int j) const { return p[padpos(j)]; }
    __device__ __forceinline__ void operator()(int k, C v) const { p[padpos(k)] = v; }
};
using SmemLineRtAcc = SmemLineRtAccT<float2>;

template <class C>
struct SmemStrideAccT { // element j at p[j * s]
    C *p;
    int s;
    __device__ __forceinline__ C operator()(int j) const { return p[j * s]; }
    __device__ __forceinline__ void operator()(int k, C v) const { p[k * s] = v; }
};
using SmemStrideAcc = SmemStrideAccT<float2>;

// Lines: line i starts at buf + i*pitch, element j at padpos(j).  C is float2
// (FP32) or double2 (the complex128 path).
template <class C>
__device__ __forceinline__ C *run_stages_lines(const LineRt &L, int nlines, int pitch, C *A, C *B, const C *tw)
{
    const int T = L.T;
    const int nteams = blockDim.x / T;
    const int team = threadIdx.x / T, t = threadIdx.x - team * T;
    C *cur = A, *nxt = B;
    int NS = 1, off = 0;
    for (int s = 0; s < L.nst; ++s) {
        const int R = L.rad[s];
        if (team < nteams)
            for (int line = team; line < nlines; line += nteams)
                stage_rt_dispatch(R, L.n, T, NS, t, SmemLineRtAccT<C>{cur + line * pitch},
                                  SmemLineRtAccT<C>{nxt + line * pitch}, tw + off, true);
        __syncthreads();
        off += (R - 1) * NS;
        NS *= R;
        C *x = cur;
        cur = nxt;
        nxt = x;
    }
    return cur;
}

// Columns of a row-major padded matrix: column i (i < ncols) has element j at
// buf + j*pitch + padpos(i).
template <class C>
__device__ __forceinline__ C *run_stages_cols(const LineRt &L, int ncols, int pitch, C *A, C *B, const C *tw)
{
    const int T = L.T;
    const int nteams = blockDim.x / T;
    const int team = threadIdx.x / T, t = threadIdx.x - team * T;
    C *cur = A, *nxt = B;
    int NS = 1, off = 0;
    for (int s = 0; s < L.nst; ++s) {
        const int R = L.rad[s];
        if (team < nteams)
            for (int col = team; col < ncols; col += nteams)
                stage_rt_dispatch(R, L.n, T, NS, t, SmemStrideAccT<C>{cur + padpos(col), pitch},
                                  SmemStrideAccT<C>{nxt + padpos(col), pitch}, tw + off, true);
        __syncthreads();
        off += (R - 1) * NS;
        NS *= R;
        C *x = cur;
        cur = nxt;
        nxt = x;
    }
    return cur;
}

} // namespace fft3
