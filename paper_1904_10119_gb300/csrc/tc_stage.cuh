// tc_stage.cuh -- a radix-16 Stockham stage computed on the tensor cores in
// split BF16.
//
// The 16-point DFT of a butterfly is a dense product y = W x with
// W[k][r] = w_16^{kr}.  In real arithmetic, with x = (xr, xi) and
// W = Wr + i Wi, the outputs are yr = Wr xr - Wi xi and yi = Wi xr + Wr xi:
// one 32 x 32 real matrix applied to 32-element columns.  Eight butterflies
// form the N = 8 columns of an m16n8k16 BF16 MMA with FP32 accumulation; the
// 32 x 32 matrix is 2 x 2 blocks of 16 x 16 (rows: yr | yi, columns: xr | xi).
// Both operands are split into a high and a low BF16 part, v = v_hi + v_lo
// with v_hi = bf16(v) and v_lo = bf16(v - v_hi), and three products are
// accumulated: W_hi x_hi + W_hi x_lo + W_lo x_hi (W_lo x_lo is dropped).
// Twiddles are applied to x in FP32 before the split.
//
// Fragment layouts of mma.sync.m16n8k16 (g = lane / 4, t = lane % 4):
//   A (16 x 16, row-major): {a0,a1} = (g, 2t..2t+1), {a2,a3} = (g+8, 2t..),
//                           {a4,a5} = (g, 2t+8..), {a6,a7} = (g+8, 2t+8..)
//   B (16 x 8, column):     {b0,b1} = (2t..2t+1, g), {b2,b3} = (2t+8.., g)
//   C (16 x 8):             {c0,c1} = (g, 2t..2t+1), {c2,c3} = (g+8, 2t..)
// so thread (g, t) supplies inputs r in {2t, 2t+1, 2t+8, 2t+9} of butterfly
// g of its group and receives outputs k in {g, g+8} of butterflies 2t, 2t+1.
#pragma once

#include <cuda_bf16.h>

#include "fft_engine.cuh"

namespace fft3 {

__device__ __forceinline__ uint32_t bf16x2_bits(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// (x0, x1) -> packed high parts and packed low parts.
__device__ __forceinline__ void split_pair(float x0, float x1, uint32_t &hi, uint32_t &lo)
{
    const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
    const __nv_bfloat16 l0 = __float2bfloat16_rn(x0 - __bfloat162float(h0));
    const __nv_bfloat16 l1 = __float2bfloat16_rn(x1 - __bfloat162float(h1));
    hi = bf16x2_bits(h0, h1);
    lo = bf16x2_bits(l0, l1);
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// The real-ified DFT_16 as split-BF16 A fragments of this lane.
struct TcW {
    uint32_t hi[2][2][4], lo[2][2][4]; // [row block: yr|yi][column block: xr|xi][register]
};

// w16[m] = w_16^m (float32, from the FP64 generator).
__device__ __forceinline__ void tc_build_w(TcW &w, const float2 *w16)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mb = 0; mb < 2; ++mb)
#pragma unroll
        for (int kb = 0; kb < 2; ++kb)
#pragma unroll
            for (int reg = 0; reg < 4; ++reg) {
                const int i = g + ((reg & 1) ? 8 : 0);
                const int j0 = 2 * t + ((reg & 2) ? 8 : 0);
                float v[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const float2 c = w16[(i * (j0 + e)) & 15];
                    // blocks: (yr,xr) = Wr, (yr,xi) = -Wi, (yi,xr) = Wi, (yi,xi) = Wr
                    v[e] = (mb == kb) ? c.x : (mb == 0 ? -c.y : c.y);
                }
                split_pair(v[0], v[1], w.hi[mb][kb][reg], w.lo[mb][kb][reg]);
            }
}

// Butterfly (line, q) of group `grp`, lane group g (GROUP_LINES: a group is
// 8 adjacent lines at one q; otherwise 8 adjacent q of one line).
template <int NB, int LPT, bool GROUP_LINES>
__device__ __forceinline__ void tc_butterfly(int grp, int n, int &line, int &q)
{
    if constexpr (GROUP_LINES) {
        q = grp / (LPT / 8);
        line = (grp % (LPT / 8)) * 8 + n;
    } else {
        line = grp / (NB / 8);
        q = (grp % (NB / 8)) * 8 + n;
    }
}

// One radix-16 stage of lines of N points on the tensor cores: the NB*LPT
// butterflies (line, q) of a tile, in groups of 8, each warp taking every
// nwarps-th group.  Src and Dst are tile accessors acc(line, pos) and must not
// alias (the stage streams group by group; the caller ping-pongs buffers).
// `warp` / `nwarps`: this warp's index among the warps sharing the stage (by
// default every warp of the block).
template <int N, int NS, int LPT, bool GROUP_LINES, class Src, class Dst>
__device__ __forceinline__ void tc_stage16(const Src &src, const Dst &dst, const float2 *tw, const TcW &w,
                                           int warp = -1, int nwarps = 0)
{
    constexpr int NB = N / 16;
    constexpr int NGROUPS = NB * LPT / 8;
    const int lane = threadIdx.x & 31;
    if (warp < 0) {
        warp = threadIdx.x >> 5;
        nwarps = blockDim.x >> 5;
    }
    const int g = lane >> 2, t = lane & 3;
    for (int grp = warp; grp < NGROUPS; grp += nwarps) {
        int line, q;
        tc_butterfly<NB, LPT, GROUP_LINES>(grp, g, line, q);
        float2 v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int r = 2 * t + (e & 1) + ((e & 2) ? 8 : 0);
            float2 x = src(line, q + r * NB);
            if constexpr (NS > 1) {
                if (r > 0)
                    x = cmul(x, tw[(r - 1) * NS + (q % NS)]);
            }
            v[e] = x;
        }
        uint32_t bh[2][2], bl[2][2]; // [xr|xi][register]
        split_pair(v[0].x, v[1].x, bh[0][0], bl[0][0]);
        split_pair(v[2].x, v[3].x, bh[0][1], bl[0][1]);
        split_pair(v[0].y, v[1].y, bh[1][0], bl[1][0]);
        split_pair(v[2].y, v[3].y, bh[1][1], bl[1][1]);
        float d[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
        for (int mb = 0; mb < 2; ++mb)
#pragma unroll
            for (int kb = 0; kb < 2; ++kb) {
                // small products first, the hi x hi product last
                mma_bf16_16816(d[mb], w.lo[mb][kb], bh[kb][0], bh[kb][1]);
                mma_bf16_16816(d[mb], w.hi[mb][kb], bl[kb][0], bl[kb][1]);
                mma_bf16_16816(d[mb], w.hi[mb][kb], bh[kb][0], bh[kb][1]);
            }
        // this lane holds outputs k in {g, g+8} of butterflies n in {2t, 2t+1}
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int k = g + ((e & 2) ? 8 : 0);
            int ol, oq;
            tc_butterfly<NB, LPT, GROUP_LINES>(grp, 2 * t + (e & 1), ol, oq);
            const int base = (NS == 1) ? oq * 16 : (oq / NS) * NS * 16 + (oq % NS);
            dst(ol, base + k * NS, make_float2(d[0][e], d[1][e]));
        }
    }
}

} // namespace fft3
