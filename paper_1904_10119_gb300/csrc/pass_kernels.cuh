// pass_kernels.cuh -- one pass of batched 1D DFTs over a 3D (or 4D with batch)
// array, with the redistribution of the pass fused into its loads and stores.
//
// Geometry of a pass (all strides in complex elements):
//   lines are indexed by (c, a, b), c in [0,C) fastest, a in [0,A), b in [0,B);
//   input  element j of line (c,a,b) is at in [j*ij + c*ic + a*ia + b*ib],
//   output element k of line (c,a,b) is at out[k*ok + c*oc + a*oa + b*ob].
// A tile is `LPT` consecutive c at fixed (a, b).  The pencil passes of
// Section 2.3 and the data rotations xyz -> yzx -> zxy of Section 2.4 are all
// instances of this geometry; only the strides differ.
//
// Kernels (one thread block per tile, grid-stride over tiles):
//   k_pass_j   contiguous lines (ij == 1).  Threads of a line are adjacent
//              (t fastest), so the first stage's loads are coalesced along
//              the line.  ROT = false: last stage stores directly (ok == 1).
//              ROT = true: last stage writes shared memory and the tile is
//              stored transposed, c fastest (oc == 1) -- the fused rotation.
//   k_pass_c   strided lines (ic == 1, oc == 1): the LPT lines of a tile are
//              adjacent columns, threads of one butterfly index are adjacent
//              (c fastest), so every load and store moves LPT*8 contiguous
//              bytes.  Shared layout [position][column] is conflict free.
//   k_pass_g   runtime radix list (any 2*3*5-smooth n up to 4096): the tile is
//              staged through shared memory with whichever mapping keeps the
//              global accesses coalesced, and the stages ping-pong between two
//              shared buffers.
#pragma once

#include "fft_engine.cuh"
#include "geom.h"

namespace fft3 {

__host__ __device__ constexpr int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Shared memory: twiddles first (rounded to 16 entries), then the data.
__host__ __device__ constexpr int tw_slots(int tw_len) { return round_up(tw_len > 0 ? tw_len : 1, 16); }

__device__ __forceinline__ void load_twiddles(float2 *tw_s, const float2 *tw_g, int len)
{
    for (int i = threadIdx.x; i < len; i += blockDim.x)
        tw_s[i] = tw_g[i];
}

struct TileId {
    int64_t c0, a, b;
};

__device__ __forceinline__ TileId decode_tile(int64_t tile, int64_t tiles_c, int64_t A, int lpt)
{
    TileId id;
    int64_t tc = tile % tiles_c;
    int64_t rest = tile / tiles_c;
    id.c0 = tc * lpt;
    id.a = rest % A;
    id.b = rest / A;
    return id;
}

// ---------------------------------------------------------- accessors ---- //
// Global line reader with optional conjugation; elements past the ragged
// edge of a tile read as zero.
struct GLoad {
    const float2 *p;
    int64_t s;
    bool valid, conj;
    __device__ __forceinline__ float2 operator()(int j) const
    {
        float2 v = valid ? p[(int64_t)j * s] : make_float2(0.f, 0.f);
        return conj ? cconj(v) : v;
    }
};
struct GLoad1 { // unit stride
    const float2 *p;
    bool valid, conj;
    __device__ __forceinline__ float2 operator()(int j) const
    {
        float2 v = valid ? p[j] : make_float2(0.f, 0.f);
        return conj ? cconj(v) : v;
    }
};
struct GStore {
    float2 *p;
    int64_t s;
    bool valid, conj;
    __device__ __forceinline__ void operator()(int k, float2 v) const
    {
        if (valid)
            p[(int64_t)k * s] = conj ? cconj(v) : v;
    }
};
struct GStore1 {
    float2 *p;
    bool valid, conj;
    __device__ __forceinline__ void operator()(int k, float2 v) const
    {
        if (valid)
            p[k] = conj ? cconj(v) : v;
    }
};
// Line-major shared layout with padding (one line of the tile).
template <int S>
struct SmemLine {
    float2 *p; // start of this line
    __device__ __forceinline__ float2 operator()(int j) const { return p[padpos(j)]; }
    __device__ __forceinline__ void operator()(int k, float2 v) const { p[padpos(k)] = v; }
};
// Position-major shared layout: element j of column l at p[j*LPT + l].
template <int LPT>
struct SmemCol {
    float2 *p; // buf + l
    __device__ __forceinline__ float2 operator()(int j) const { return p[j * LPT]; }
    __device__ __forceinline__ void operator()(int k, float2 v) const { p[k * LPT] = v; }
};

// --------------------------------------------------------- k_pass_j ----- //
template <int N, int T, class Rad, int LPT, bool ROT>
__global__ void __launch_bounds__(T *LPT) k_pass_j(PassArgs a)
{
    extern __shared__ float2 smem[];
    constexpr int S = line_pitch(N);
    float2 *tw = smem;
    float2 *buf = smem + tw_slots(a.tw_len);
    load_twiddles(tw, a.tw, a.tw_len);
    const int t = threadIdx.x % T, l = threadIdx.x / T;
    const bool conj = a.conj != 0;
    for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        __syncthreads();
        const TileId id = decode_tile(tile, a.tiles_c, a.g.A, LPT);
        const int64_t c = id.c0 + l;
        const bool valid = c < a.g.C;
        GLoad1 src{a.in + c * a.g.ic + id.a * a.g.ia + id.b * a.g.ib, valid, conj};
        SmemLine<S> sm{buf + l * S};
        if constexpr (!ROT) {
            GStore1 dst{a.out + c * a.g.oc + id.a * a.g.oa + id.b * a.g.ob, valid, conj};
            EngineFixed<N, T, 1, Rad>::template run<true, false>(t, src, sm, dst, tw);
        } else {
            EngineFixed<N, T, 1, Rad>::template run<true, true>(t, src, sm, sm, tw);
            __syncthreads();
            // transposed store: c fastest across threads
            float2 *ob = a.out + id.a * a.g.oa + id.b * a.g.ob;
            const int64_t nval = min((int64_t)LPT, a.g.C - id.c0);
            for (int e = threadIdx.x; e < LPT * N; e += T * LPT) {
                const int ll = e % LPT, k = e / LPT;
                if (ll < nval) {
                    float2 v = buf[ll * S + padpos(k)];
                    ob[(id.c0 + ll) * a.g.oc + (int64_t)k * a.g.ok] = conj ? cconj(v) : v;
                }
            }
        }
    }
}

// --------------------------------------------------------- k_pass_c ----- //
template <int N, int T, class Rad, int LPT>
__global__ void __launch_bounds__(T *LPT) k_pass_c(PassArgs a)
{
    extern __shared__ float2 smem[];
    float2 *tw = smem;
    float2 *buf = smem + tw_slots(a.tw_len);
    load_twiddles(tw, a.tw, a.tw_len);
    const int l = threadIdx.x % LPT, t = threadIdx.x / LPT;
    const bool conj = a.conj != 0;
    for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        __syncthreads();
        const TileId id = decode_tile(tile, a.tiles_c, a.g.A, LPT);
        const int64_t c = id.c0 + l;
        const bool valid = c < a.g.C;
        GLoad src{a.in + c * a.g.ic + id.a * a.g.ia + id.b * a.g.ib, a.g.ij, valid, conj};
        GStore dst{a.out + c * a.g.oc + id.a * a.g.oa + id.b * a.g.ob, a.g.ok, valid, conj};
        SmemCol<LPT> sm{buf + l};
        EngineFixed<N, T, 1, Rad>::template run<true, false>(t, src, sm, dst, tw);
    }
}

// --------------------------------------------------------- k_pass_g ----- //
// Shared layout: line-major with padded positions, pitch P (odd).
struct SmemLineRt {
    float2 *p;
    __device__ __forceinline__ float2 operator()(int j) const { return p[padpos(j)]; }
    __device__ __forceinline__ void operator()(int k, float2 v) const { p[padpos(k)] = v; }
};

__host__ __device__ inline int generic_pitch(int n) { return line_pitch(n); }

__global__ void k_pass_g(PassArgs a);
__global__ void k_pass_g64(PassArgs a); // the same in FP64 on complex128 arrays

// Identity probe of a pass geometry: out[k*ok...] = in[k*ij...] for every
// element (used to check the fused redistributions bit-exactly).
__global__ void k_probe_pass(PassArgs a);

} // namespace fft3
