// warp_fft.cuh -- line transforms held in the registers of a group of lanes
// of one warp: the exchanges between lanes are warp shuffles and global memory
// moves in 128-bit pieces (two complex values), so a line needs neither shared
// memory nor a block barrier.
//
// A line of N = R * L points (L a power of two) is held by W = L / 2 adjacent
// lanes.  With the Cooley-Tukey split j = t + L i, k = k' + R k'' (t, k'' < L;
// i, k' < R; Section 2.1, Eq. ct), lane u of the group holds the two
// sub-sequences t = 2u and t = 2u + 1, R points each:
//   load      x[t + L i] for both t: one 16-byte load per i (positions 2u, 2u+1);
//   (I)       DFT_R over i in registers, for each t                 (Bfly<R>);
//   (II)      twiddle w_N^{t k'};
//   (IV)      DFT_L over t for each k': radix-2 decimation-in-frequency steps,
//             the steps of half-size h = L/2 .. 2 across lanes (partner lane
//             u xor h/2, __shfl_xor_sync), the step h = 1 (between t = 2u and
//             2u + 1) in registers; position t ends with frequency rev_L(t),
//             the bit reversal of t over log2(L) bits;
//   store     X[k' + R rev_L(t)] for k' < R: R consecutive outputs per
//             sub-sequence, 16 bytes per store.
// A decimation-in-frequency step of half-size h maps the pair (a, b) at
// positions (t, t + h), t mod 2h < h, to (a + b, (a - b) w_{2h}^{t mod h}).
// Every lane of a warp takes part in every shuffle: lanes of lines past the
// end transform zeros and store nothing.
#pragma once

#include "fft_engine.cuh"

namespace fft3 {

template <int N, int R, int L>
struct WarpLine {
    static_assert(N == R * L && L >= 2 && (L & (L - 1)) == 0 && L <= 64, "N = R * L, L a power of two");
    static constexpr int W = L / 2; // lanes per line
    static constexpr int LOGL = L == 2 ? 1 : L == 4 ? 2 : L == 8 ? 3 : L == 16 ? 4 : L == 32 ? 5 : 6;
    static constexpr int NET = LOGL - 1; // steps across lanes

    // Per-lane twiddles, from the table w_N^m (m < N) of the line length.
    struct Tw {
        float2 in[2][R];              // w_N^{t k'}, t = 2u + e
        float2 net[NET > 0 ? NET : 1][2]; // step s (h = L >> (s + 1)): w_{2h}^{t mod h} on the upper
                                          // position of a pair, 1 on the lower one
    };

    __device__ __forceinline__ static int rev(int t) { return (int)(__brev((unsigned)t) >> (32 - LOGL)); }

    __device__ __forceinline__ static void load_tw(Tw &tw, const float2 *table, int u)
    {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int t = 2 * u + e;
#pragma unroll
            for (int k = 0; k < R; ++k)
                tw.in[e][k] = table[(t * k) % N];
#pragma unroll
            for (int s = 0; s < NET; ++s) {
                const int h = L >> (s + 1);
                tw.net[s][e] = (t & h) ? table[(t % h) * (N / (2 * h))] : make_float2(1.f, 0.f);
            }
        }
    }

    // Strided lines (element j at p[j * es]): the lanes of a line sit on
    // different rows, adjacent lines (columns) in adjacent lane groups, so a
    // warp's access covers one run of adjacent columns per row.
    __device__ __forceinline__ static void load_strided(float2 (&v)[2][R], const float2 *p, int64_t es, int u,
                                                        bool valid, bool conj)
    {
#pragma unroll
        for (int i = 0; i < R; ++i) {
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float2 x = valid ? p[(int64_t)(2 * u + e + L * i) * es] : make_float2(0.f, 0.f);
                v[e][i] = conj ? cconj(x) : x;
            }
        }
    }

    __device__ __forceinline__ static void store_strided(float2 (&v)[2][R], float2 *p, int64_t es, int u,
                                                         bool valid, bool conj)
    {
        if (!valid)
            return;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int64_t r0 = (int64_t)R * rev(2 * u + e);
#pragma unroll
            for (int k = 0; k < R; ++k)
                p[(r0 + k) * es] = conj ? cconj(v[e][k]) : v[e][k];
        }
    }

    // v[e][i] = x[2u + e + L i] (conjugated for the inverse); zeros when !valid.
    // Streaming loads (evict first from L1): each value is read once, and L1
    // keeps what is read again (twiddle tables).
    __device__ __forceinline__ static void load(float2 (&v)[2][R], const float2 *p, int u, bool valid, bool conj)
    {
        if (valid && ((reinterpret_cast<uintptr_t>(p) & 15) == 0)) {
#pragma unroll
            for (int i = 0; i < R; ++i) {
                const float4 q = __ldcs(reinterpret_cast<const float4 *>(p + 2 * u + L * i));
                v[0][i] = make_float2(q.x, q.y);
                v[1][i] = make_float2(q.z, q.w);
            }
        } else {
#pragma unroll
            for (int i = 0; i < R; ++i) {
                v[0][i] = valid ? __ldcs(p + 2 * u + L * i) : make_float2(0.f, 0.f);
                v[1][i] = valid ? __ldcs(p + 2 * u + 1 + L * i) : make_float2(0.f, 0.f);
            }
        }
        if (conj) {
#pragma unroll
            for (int i = 0; i < R; ++i) {
                v[0][i] = cconj(v[0][i]);
                v[1][i] = cconj(v[1][i]);
            }
        }
    }

    __device__ __forceinline__ static void run(float2 (&v)[2][R], const Tw &tw, int u)
    {
        // (I), (II)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            Bfly<R>::run(v[e]);
#pragma unroll
            for (int k = 1; k < R; ++k)
                v[e][k] = cmul(v[e][k], tw.in[e][k]);
        }
        // (IV) across lanes: the lower position keeps a + b, the upper takes
        // (a - b) w = (-b + a) w, with its own value b and the partner's a
#pragma unroll
        for (int s = 0; s < NET; ++s) {
            const int m = W >> (s + 1); // lane mask of half-size h = 2m
            const float sg = (u & m) ? -1.f : 1.f;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const float px = __shfl_xor_sync(0xffffffffu, v[e][k].x, m);
                    const float py = __shfl_xor_sync(0xffffffffu, v[e][k].y, m);
                    const float2 d = make_float2(fmaf(sg, v[e][k].x, px), fmaf(sg, v[e][k].y, py));
                    v[e][k] = cmul(d, tw.net[s][e]);
                }
            }
        }
        // (IV) last step, h = 1, in registers
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const float2 a = v[0][k], b = v[1][k];
            v[0][k] = cadd(a, b);
            v[1][k] = csub(a, b);
        }
    }

    // X[k' + R rev(2u + e)] = v[e][k'] (conjugated for the inverse).
    __device__ __forceinline__ static void store(float2 (&v)[2][R], float2 *p, int u, bool valid, bool conj)
    {
        if (!valid)
            return;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            float2 *q = p + R * rev(2 * u + e);
            if constexpr (R % 2 == 0) {
                if ((reinterpret_cast<uintptr_t>(p) & 15) == 0) {
#pragma unroll
                    for (int k = 0; k < R; k += 2) {
                        const float2 a = conj ? cconj(v[e][k]) : v[e][k];
                        const float2 b = conj ? cconj(v[e][k + 1]) : v[e][k + 1];
                        *reinterpret_cast<float4 *>(q + k) = make_float4(a.x, a.y, b.x, b.y);
                    }
                    continue;
                }
            }
#pragma unroll
            for (int k = 0; k < R; ++k)
                q[k] = conj ? cconj(v[e][k]) : v[e][k];
        }
    }
};

} // namespace fft3
