// runtime_stages.cuh -- runs a runtime radix list (LineRt) on lines held in
// shared memory, ping-ponging between two buffers with a block barrier after
// every stage.  Teams of T threads take one line each; lines beyond the number
// of teams are taken in further rounds.
#pragma once

#include "fft_engine.cuh"
#include "geom.h"

namespace fft3 {

struct SmemLineRtAcc { // line-major, padded positions
    float2 *p;
    __device__ __forceinline__ float2 operator()(int j) const { return p[padpos(j)]; }
    __device__ __forceinline__ void operator()(int k, float2 v) const { p[padpos(k)] = v; }
};

struct SmemStrideAcc { // element j at p[j * s]
    float2 *p;
    int s;
    __device__ __forceinline__ float2 operator()(int j) const { return p[j * s]; }
    __device__ __forceinline__ void operator()(int k, float2 v) const { p[k * s] = v; }
};

// Lines: line i starts at buf + i*pitch, element j at padpos(j).
__device__ __forceinline__ float2 *run_stages_lines(const LineRt &L, int nlines, int pitch, float2 *A,
                                                    float2 *B, const float2 *tw)
{
    const int T = L.T;
    const int nteams = blockDim.x / T;
    const int team = threadIdx.x / T, t = threadIdx.x - team * T;
    float2 *cur = A, *nxt = B;
    int NS = 1, off = 0;
    for (int s = 0; s < L.nst; ++s) {
        const int R = L.rad[s];
        if (team < nteams)
            for (int line = team; line < nlines; line += nteams)
                stage_rt_dispatch(R, L.n, T, NS, t, SmemLineRtAcc{cur + line * pitch},
                                  SmemLineRtAcc{nxt + line * pitch}, tw + off, true);
        __syncthreads();
        off += (R - 1) * NS;
        NS *= R;
        float2 *x = cur;
        cur = nxt;
        nxt = x;
    }
    return cur;
}

// Columns of a row-major padded matrix: column i (i < ncols) has element j at
// buf + j*pitch + padpos(i).
__device__ __forceinline__ float2 *run_stages_cols(const LineRt &L, int ncols, int pitch, float2 *A,
                                                   float2 *B, const float2 *tw)
{
    const int T = L.T;
    const int nteams = blockDim.x / T;
    const int team = threadIdx.x / T, t = threadIdx.x - team * T;
    float2 *cur = A, *nxt = B;
    int NS = 1, off = 0;
    for (int s = 0; s < L.nst; ++s) {
        const int R = L.rad[s];
        if (team < nteams)
            for (int col = team; col < ncols; col += nteams)
                stage_rt_dispatch(R, L.n, T, NS, t, SmemStrideAcc{cur + padpos(col), pitch},
                                  SmemStrideAcc{nxt + padpos(col), pitch}, tw + off, true);
        __syncthreads();
        off += (R - 1) * NS;
        NS *= R;
        float2 *x = cur;
        cur = nxt;
        nxt = x;
    }
    return cur;
}

} // namespace fft3
