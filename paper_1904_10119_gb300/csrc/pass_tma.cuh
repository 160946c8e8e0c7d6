// pass_tma.cuh -- strided-line pass (y or z lines, tiles of LPT adjacent
// columns) with its tiles moved by the tensor memory accelerator.
//
// One persistent block per SM double-buffers tiles in shared memory: while
// the block transforms tile i in place (Stockham stages exchanging through
// the same buffer), TMA loads tile i+1 into the other buffer, and the result
// of tile i leaves through a TMA store.  The array is described to TMA as a
// 4D tensor {C columns (contiguous), n line elements, A, B}; a tile is LPT
// columns x n elements, moved as n/256 boxes of LPT x 256.  The shared
// layout TMA produces, [element][column], is the conflict-free column layout
// of k_pass_c.
#pragma once

#include "pass_kernels.cuh"
#include "tma.cuh"

namespace fft3 {

// Position-major column accessor that conjugates on load and store (first
// and last stage of an inverse transform).
template <int LPT>
struct SmemColIO {
    float2 *p;
    bool conj;
    __device__ __forceinline__ float2 operator()(int j) const
    {
        float2 v = p[j * LPT];
        return conj ? cconj(v) : v;
    }
    __device__ __forceinline__ void operator()(int k, float2 v) const { p[k * LPT] = conj ? cconj(v) : v; }
};

template <int N, int LPT>
struct TmaTile {
    static constexpr int BR = N < 256 ? N : 256; // box rows
    static constexpr int NBOX = N / BR;
    static constexpr uint32_t BYTES = (uint32_t)N * LPT * 8u;
};

template <int N, int T, class Rad, int LPT>
__global__ void __launch_bounds__(T *LPT) k_pass_c_tma(PassArgs a, const __grid_constant__ CUtensorMap tin,
                                                       const __grid_constant__ CUtensorMap tout)
{
    using TT = TmaTile<N, LPT>;
    extern __shared__ __align__(128) float2 smem[];
    __shared__ __align__(8) uint64_t bars[2];
    float2 *tw = smem;
    float2 *buf0 = smem + tw_slots(a.tw_len);
    float2 *buf1 = buf0 + N * LPT;
    load_twiddles(tw, a.tw, a.tw_len);
    const int l = threadIdx.x % LPT, t = threadIdx.x / LPT;
    const bool conj = a.conj != 0;
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue_load = [&](int64_t tl, int s) {
        const TileId id = decode_tile(tl, a.tiles_c, a.g.A, LPT);
        float2 *dst = s ? buf1 : buf0;
        mbar_expect_tx(&bars[s], TT::BYTES);
#pragma unroll
        for (int k = 0; k < TT::NBOX; ++k)
            tma_load_4d(dst + k * TT::BR * LPT, &tin, (int)id.c0, k * TT::BR, (int)id.a, (int)id.b, &bars[s]);
    };
    int64_t tile = blockIdx.x;
    if (threadIdx.x == 0 && tile < a.ntiles)
        issue_load(tile, 0);
    for (int i = 0; tile < a.ntiles; tile += gridDim.x, ++i) {
        const int s = i & 1;
        float2 *cur = s ? buf1 : buf0;
        const int64_t next = tile + gridDim.x;
        if (threadIdx.x == 0 && next < a.ntiles) {
            bulk_wait_read0(); // the store from the other buffer has finished reading it
            issue_load(next, s ^ 1);
        }
        if (!mbar_wait(&bars[s], (uint32_t)((i >> 1) & 1), a.wait_budget))
            atomicOr(a.err, kErrWaitTimeout);
        SmemColIO<LPT> io{cur + l, conj};
        SmemCol<LPT> sm{cur + l};
        EngineFixed<N, T, 1, Rad>::template run<false, true>(t, io, sm, io, tw);
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            const TileId id = decode_tile(tile, a.tiles_c, a.g.A, LPT);
#pragma unroll
            for (int k = 0; k < TT::NBOX; ++k)
                tma_store_4d(&tout, (int)id.c0, k * TT::BR, (int)id.a, (int)id.b, cur + k * TT::BR * LPT);
            bulk_commit();
        }
    }
    if (threadIdx.x == 0)
        bulk_wait0();
}

} // namespace fft3
