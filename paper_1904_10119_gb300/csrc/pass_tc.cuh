// pass_tc.cuh -- line passes whose radix-16 stages run on the tensor cores in
// split BF16 (tc_stage.cuh); the other stages, the twiddles and all data
// movement are those of the FP32 kernels (pass_kernels.cuh).
#pragma once

#include "pass_kernels.cuh"
#include "tc_stage.cuh"

namespace fft3 {

// Tile accessors: (line, position) -> element, and bind(line) -> the
// single-line accessor the FP32 stages use.
template <int LPT>
struct TileColSmem { // [position][line]
    float2 *p;
    __device__ __forceinline__ float2 operator()(int l, int j) const { return p[j * LPT + l]; }
    __device__ __forceinline__ void operator()(int l, int k, float2 v) const { p[k * LPT + l] = v; }
    __device__ __forceinline__ SmemCol<LPT> bind(int l) const { return SmemCol<LPT>{p + l}; }
};
template <int S>
struct TileLineSmem { // line-major, padded positions
    float2 *p;
    __device__ __forceinline__ float2 operator()(int l, int j) const { return p[l * S + padpos(j)]; }
    __device__ __forceinline__ void operator()(int l, int k, float2 v) const { p[l * S + padpos(k)] = v; }
    __device__ __forceinline__ SmemLine<S> bind(int l) const { return SmemLine<S>{p + l * S}; }
};
// Global tile: line l starts at p + l*ls, element j at j*es; lines >= nval
// read as zero and are not stored.
struct TileGlobal {
    const float2 *pin;
    float2 *pout;
    int64_t ls, es;
    int nval;
    bool conj;
    __device__ __forceinline__ float2 operator()(int l, int j) const
    {
        float2 v = l < nval ? pin[l * ls + (int64_t)j * es] : make_float2(0.f, 0.f);
        return conj ? cconj(v) : v;
    }
    __device__ __forceinline__ void operator()(int l, int k, float2 v) const
    {
        if (l < nval)
            pout[l * ls + (int64_t)k * es] = conj ? cconj(v) : v;
    }
    __device__ __forceinline__ GLoad bind_load(int l) const { return GLoad{pin + l * ls, es, l < nval, conj}; }
    __device__ __forceinline__ GStore bind_store(int l) const { return GStore{pout + l * ls, es, l < nval, conj}; }
    // stage_fixed needs a source and a sink functor; a global tile is only
    // ever the source of the first stage or the sink of the last
    struct Both {
        GLoad ld;
        GStore st;
        __device__ __forceinline__ float2 operator()(int j) const { return ld(j); }
        __device__ __forceinline__ void operator()(int k, float2 v) const { st(k, v); }
    };
    __device__ __forceinline__ Both bind(int l) const { return Both{bind_load(l), bind_store(l)}; }
};

// Stages ping-pong between two shared buffers (A: even stages' outputs, B:
// odd), one block barrier per stage; the first stage reads `src` (global),
// the last writes `dst` (global).
template <int N, int T, int LPT, bool GL, int TCMASK, int S, int NS, class Rad>
struct EngineTC;

template <int N, int T, int LPT, bool GL, int TCMASK, int S, int NS, int R>
struct EngineTC<N, T, LPT, GL, TCMASK, S, NS, Radices<R>> {
    template <class Src, class Buf, class Dst>
    __device__ __forceinline__ static void run(int t, int l, const Src &src, const Buf &, const Buf &, const Dst &dst,
                                               const float2 *tw, const TcW &w)
    {
        if constexpr (R == 16 && ((TCMASK >> S) & 1))
            tc_stage16<N, NS, LPT, GL>(src, dst, tw, w);
        else
            stage_fixed<N, T, R, NS, false>(t, src.bind(l), dst.bind(l), tw);
    }
};

template <int N, int T, int LPT, bool GL, int TCMASK, int S, int NS, int R, int R2, int... Rest>
struct EngineTC<N, T, LPT, GL, TCMASK, S, NS, Radices<R, R2, Rest...>> {
    template <class Src, class Buf, class Dst>
    __device__ __forceinline__ static void run(int t, int l, const Src &src, const Buf &a, const Buf &b,
                                               const Dst &dst, const float2 *tw, const TcW &w)
    {
        if constexpr (R == 16 && ((TCMASK >> S) & 1))
            tc_stage16<N, NS, LPT, GL>(src, a, tw, w);
        else
            stage_fixed<N, T, R, NS, false>(t, src.bind(l), a.bind(l), tw);
        __syncthreads();
        EngineTC<N, T, LPT, GL, TCMASK, S + 1, NS * R, Radices<R2, Rest...>>::run(t, l, a, b, a, dst,
                                                                                  tw + (R - 1) * NS, w);
    }
};

// Contiguous lines (ij == 1, ok == 1), groups of 8 butterflies along a line.
// Shared memory: twiddles (including w_16^m at tw_split_off) + 2 line buffers.
template <int N, int T, class Rad, int LPT, int TCMASK>
__global__ void __launch_bounds__(T *LPT) k_pass_j_tc(PassArgs a)
{
    extern __shared__ float2 smem[];
    constexpr int S = line_pitch(N);
    float2 *tw = smem;
    float2 *b0 = smem + tw_slots(a.tw_len);
    float2 *b1 = b0 + LPT * S;
    load_twiddles(tw, a.tw, a.tw_len);
    __syncthreads();
    TcW w;
    tc_build_w(w, tw + a.tw_split_off);
    const int t = threadIdx.x % T, l = threadIdx.x / T;
    const bool conj = a.conj != 0;
    for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        __syncthreads();
        const TileId id = decode_tile(tile, a.tiles_c, a.g.A, LPT);
        const int nval = (int)min((int64_t)LPT, a.g.C - id.c0);
        TileGlobal in{a.in + id.c0 * a.g.ic + id.a * a.g.ia + id.b * a.g.ib, nullptr, a.g.ic, 1, nval, conj};
        TileGlobal out{nullptr, a.out + id.c0 * a.g.oc + id.a * a.g.oa + id.b * a.g.ob, a.g.oc, 1, nval, conj};
        EngineTC<N, T, LPT, false, TCMASK, 0, 1, Rad>::run(t, l, in, TileLineSmem<S>{b0}, TileLineSmem<S>{b1}, out,
                                                           tw, w);
    }
}

// Strided lines (ic == 1, oc == 1), groups of 8 butterflies across 8 lines.
template <int N, int T, class Rad, int LPT, int TCMASK>
__global__ void __launch_bounds__(T *LPT) k_pass_c_tc(PassArgs a)
{
    extern __shared__ float2 smem[];
    float2 *tw = smem;
    float2 *b0 = smem + tw_slots(a.tw_len);
    float2 *b1 = b0 + LPT * N;
    load_twiddles(tw, a.tw, a.tw_len);
    __syncthreads();
    TcW w;
    tc_build_w(w, tw + a.tw_split_off);
    const int l = threadIdx.x % LPT, t = threadIdx.x / LPT;
    const bool conj = a.conj != 0;
    for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        __syncthreads();
        const TileId id = decode_tile(tile, a.tiles_c, a.g.A, LPT);
        const int nval = (int)min((int64_t)LPT, a.g.C - id.c0);
        TileGlobal in{a.in + id.c0 + id.a * a.g.ia + id.b * a.g.ib, nullptr, 1, a.g.ij, nval, conj};
        TileGlobal out{nullptr, a.out + id.c0 + id.a * a.g.oa + id.b * a.g.ob, 1, a.g.ok, nval, conj};
        EngineTC<N, T, LPT, true, TCMASK, 0, 1, Rad>::run(t, l, in, TileColSmem<LPT>{b0}, TileColSmem<LPT>{b1}, out,
                                                          tw, w);
    }
}

// Stage mask of the radix-16 stages of a radix list (all of them, or the first).
template <int... Rs>
__host__ __device__ constexpr int tc_mask_all(Radices<Rs...>)
{
    int m = 0, s = 0;
    ((m |= (Rs == 16 ? 1 : 0) << s++), ...);
    return m;
}
template <int... Rs>
__host__ __device__ constexpr int tc_mask_first(Radices<Rs...> r)
{
    const int all = tc_mask_all(r);
    return all & (-all);
}
// The radix-16 stages whose operands are both in shared memory (neither the
// first stage, which reads global memory, nor the last, which writes it).
template <int... Rs>
__host__ __device__ constexpr int tc_mask_inner(Radices<Rs...> r)
{
    return tc_mask_all(r) & ~1 & ~(1 << ((int)sizeof...(Rs) - 1));
}
// tc_stages option: 0 = the first radix-16 stage with both operands in shared
// memory, 1 = every radix-16 stage with both operands in shared memory, 2 =
// every radix-16 stage.
template <class Rad>
__host__ __device__ constexpr int tc_mask_mode(int mode)
{
    return mode == 0 ? (tc_mask_inner(Rad{}) & -tc_mask_inner(Rad{})) : mode == 1 ? tc_mask_inner(Rad{})
                                                                                  : tc_mask_all(Rad{});
}

} // namespace fft3
