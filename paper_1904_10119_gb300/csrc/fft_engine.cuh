// fft_engine.cuh -- device-side building blocks of the line transforms.
//
// A line of n complex values is transformed by a sequence of Stockham
// radix-R stages (the Cooley-Tukey split n = n0*n1 of Section 2.1, Eq. ct,
// applied repeatedly with the transposition (III) folded into the index
// map of every stage so the result comes out in natural order):
//
//   stage with radix R, NS = product of the radices of the earlier stages,
//   butterfly q in [0, n/R):
//     v[r]  = src[q + r*n/R]                                   r < R
//     v[r] *= w_{NS*R}^{r*(q mod NS)}                           twiddle (II)
//     v     = DFT_R v                                           butterfly (I/IV)
//     dst[(q div NS)*NS*R + (q mod NS) + r*NS] = v[r]
//
// The twiddles of all stages sit in one stage-major table:
//   table[off_s + (r-1)*NS_s + k] = w_n^{r*k*n/(NS_s*R_s)},  r in [1,R), k < NS_s,
// off_s = sum over earlier stages of (R-1)*NS, which is at most n-1 entries.
// The table is produced in FP64 on the GPU and rounded to float32
// (twiddle.cu).  The butterflies below are the forward transform; the
// inverse is computed as conj(DFT(conj(x))) by conjugating on load and store.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "geom.h"

namespace fft3 {

// ------------------------------------------------------------ complex ---- //
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); } // a * (-i)
__device__ __forceinline__ float2 mul_pi(float2 a) { return make_float2(-a.y, a.x); } // a * (+i)
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// The same operations in FP64 (complex128 path).
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 mul_mi(double2 a) { return make_double2(a.y, -a.x); }
__device__ __forceinline__ double2 mul_pi(double2 a) { return make_double2(-a.y, a.x); }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

// Scalar type of a complex type, and construction / fused multiply-add in it.
template <class C>
struct Cx;
template <>
struct Cx<float2> {
    using S = float;
    __device__ __forceinline__ static float2 make(float r, float i) { return make_float2(r, i); }
    __device__ __forceinline__ static float fma_(float a, float b, float c) { return fmaf(a, b, c); }
};
template <>
struct Cx<double2> {
    using S = double;
    __device__ __forceinline__ static double2 make(double r, double i) { return make_double2(r, i); }
    __device__ __forceinline__ static double fma_(double a, double b, double c) { return fma(a, b, c); }
};

// cos(2 pi m / 16) and sin(2 pi m / 16) from the first-octant values.
constexpr double kC16 = 0.923879532511286756128183189396788933; // cos(pi/8)
constexpr double kS16 = 0.382683432365089771728459984030398866; // sin(pi/8)
constexpr double kH = 0.707106781186547524400844362104849039;   // sqrt(1/2)

__host__ __device__ constexpr double cos16(int m)
{
    m &= 15;
    return m == 0 ? 1.0 : m == 1 ? kC16 : m == 2 ? kH : m == 3 ? kS16 : m == 4 ? 0.0
         : m == 5 ? -kS16 : m == 6 ? -kH : m == 7 ? -kC16 : m == 8 ? -1.0 : m == 9 ? -kC16
         : m == 10 ? -kH : m == 11 ? -kS16 : m == 12 ? 0.0 : m == 13 ? kS16 : m == 14 ? kH : kC16;
}
__host__ __device__ constexpr double sin16(int m) { return cos16(m - 4); }

// a * w_R^M with w_R = exp(-2 pi i / R), R in {2, 4, 8, 16}, M known at compile time.
template <int R, int M, class C>
__device__ __forceinline__ C mul_w(C a)
{
    using X = Cx<C>;
    using S = typename X::S;
    constexpr int m16 = ((M % R) + R) % R * (16 / R);
    if constexpr (m16 == 0) {
        return a;
    } else if constexpr (m16 == 4) {
        return mul_mi(a);
    } else if constexpr (m16 == 8) {
        return X::make(-a.x, -a.y);
    } else if constexpr (m16 == 12) {
        return mul_pi(a);
    } else if constexpr (m16 == 2 || m16 == 6 || m16 == 10 || m16 == 14) {
        // (c - i s) with |c| = |s| = sqrt(1/2)
        constexpr S c = (S)cos16(m16), s = (S)sin16(m16);
        return X::make((a.x * c + a.y * s), (a.y * c - a.x * s));
    } else {
        constexpr S c = (S)cos16(m16), s = (S)sin16(m16);
        return X::make(X::fma_(a.x, c, a.y * s), X::fma_(a.y, c, -a.x * s));
    }
}

// ---------------------------------------------------------- butterflies -- //
// In-register forward DFT_R of v[0..R) in natural order (Section 2.1 definition).
template <int R>
struct Bfly;

template <>
struct Bfly<2> {
    template <class C>
    __device__ __forceinline__ static void run(C *v)
    {
        C a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <>
struct Bfly<4> {
    template <class C>
    __device__ __forceinline__ static void run(C *v)
    {
        C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        C t2 = cadd(v[1], v[3]), t3 = mul_mi(csub(v[1], v[3]));
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    }
};

// 8 = 2 * 4 (Eq. ct with n0 = 2, n1 = 4): DFT_4 on x[i0 + 2 i1], twiddle
// w_8^{i0 k1}, DFT_2 across i0, output y[k1 + 4 k0].
template <>
struct Bfly<8> {
    template <class C>
    __device__ __forceinline__ static void run(C *v)
    {
        C e[4] = {v[0], v[2], v[4], v[6]};
        C o[4] = {v[1], v[3], v[5], v[7]};
        Bfly<4>::run(e);
        Bfly<4>::run(o);
        o[1] = mul_w<8, 1>(o[1]);
        o[2] = mul_w<8, 2>(o[2]);
        o[3] = mul_w<8, 3>(o[3]);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = cadd(e[k], o[k]);
            v[k + 4] = csub(e[k], o[k]);
        }
    }
};

// 16 = 4 * 4 (Eq. ct with n0 = n1 = 4).
template <>
struct Bfly<16> {
    template <class C>
    __device__ __forceinline__ static void run(C *v)
    {
        C t[4][4];
#pragma unroll
        for (int i0 = 0; i0 < 4; ++i0) {
#pragma unroll
            for (int i1 = 0; i1 < 4; ++i1)
                t[i0][i1] = v[i0 + 4 * i1];
            Bfly<4>::run(t[i0]);
        }
        t[1][1] = mul_w<16, 1>(t[1][1]);
        t[1][2] = mul_w<16, 2>(t[1][2]);
        t[1][3] = mul_w<16, 3>(t[1][3]);
        t[2][1] = mul_w<16, 2>(t[2][1]);
        t[2][2] = mul_w<16, 4>(t[2][2]);
        t[2][3] = mul_w<16, 6>(t[2][3]);
        t[3][1] = mul_w<16, 3>(t[3][1]);
        t[3][2] = mul_w<16, 6>(t[3][2]);
        t[3][3] = mul_w<16, 9>(t[3][3]);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            C c[4] = {t[0][k1], t[1][k1], t[2][k1], t[3][k1]};
            Bfly<4>::run(c);
#pragma unroll
            for (int k0 = 0; k0 < 4; ++k0)
                v[k1 + 4 * k0] = c[k0];
        }
    }
};

// cos(pi m / 16) and sin(pi m / 16) for m in 0..7, from which every power of
// w_32 follows by symmetry.
constexpr double kC32[8] = {1.0,
                            0.980785280403230449126182236134239037,
                            0.923879532511286756128183189396788933,
                            0.831469612302545237078788377617905756,
                            0.707106781186547524400844362104849039,
                            0.555570233019602224742830813948532874,
                            0.382683432365089771728459984030398866,
                            0.195090322016128267848284868477022240};
__host__ __device__ constexpr double cos32(int m)
{
    m &= 31;
    return m <= 8 ? (m == 8 ? 0.0 : kC32[m]) : m < 16 ? -cos32(16 - m) : m < 24 ? -cos32(m - 16) : cos32(32 - m);
}
__host__ __device__ constexpr double sin32(int m) { return cos32(m - 8); }

// a * w_32^M, M known at compile time (the exact cases of mul_w where M is a
// multiple of 2, the general complex product otherwise).
template <int M, class C>
__device__ __forceinline__ C mul_w32(C a)
{
    if constexpr ((M & 1) == 0) {
        return mul_w<16, M / 2>(a);
    } else {
        using X = Cx<C>;
        using S = typename X::S;
        constexpr S c = (S)cos32(M), s = (S)sin32(M);
        return X::make(X::fma_(a.x, c, a.y * s), X::fma_(a.y, c, -a.x * s));
    }
}

// A constant in the scalar type: the float literal for FP32 (as written), the
// double literal for FP64.
template <class S>
__host__ __device__ constexpr S kpick(float f, double d)
{
    if constexpr (sizeof(S) == 4)
        return f;
    else
        return (S)d;
}

// 32 = 2 * 16 (Eq. ct with n0 = 2, n1 = 16): DFT_16 on x[i0 + 2 i1], twiddle
// w_32^{i0 k1}, DFT_2 across i0, output y[k1 + 16 k0].  Every value stays in
// registers: one thread transforms a whole 32-point sub-line.
template <int K>
struct Tw32Step {
    template <class C>
    __device__ __forceinline__ static void run(C *o)
    {
        o[K] = mul_w32<K>(o[K]);
        if constexpr (K + 1 < 16)
            Tw32Step<K + 1>::run(o);
    }
};

template <>
struct Bfly<32> {
    template <class C>
    __device__ __forceinline__ static void run(C *v)
    {
        C e[16], o[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            e[i] = v[2 * i];
            o[i] = v[2 * i + 1];
        }
        Bfly<16>::run(e);
        Bfly<16>::run(o);
        Tw32Step<1>::run(o);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            v[k] = cadd(e[k], o[k]);
            v[k + 16] = csub(e[k], o[k]);
        }
    }
};

// DFT_3: w_3 = -1/2 - i sqrt(3)/2.
template <>
struct Bfly<3> {
    template <class C>
    __device__ __forceinline__ static void run(C *v)
    {
        using X = Cx<C>;
        using S = typename X::S;
        constexpr S s3 = kpick<S>(0.866025403784438646763723170752936183f,
                                  0.866025403784438646763723170752936183); // sin(2 pi / 3)
        C s = cadd(v[1], v[2]), d = csub(v[1], v[2]);
        C a = X::make(X::fma_((S)-0.5, s.x, v[0].x), X::fma_((S)-0.5, s.y, v[0].y));
        C b = X::make(d.x * s3, d.y * s3);
        v[0] = cadd(v[0], s);
        v[1] = X::make(a.x + b.y, a.y - b.x); // a - i b
        v[2] = X::make(a.x - b.y, a.y + b.x); // a + i b
    }
};

// DFT_5 with the conjugate-pair form: y_1,4 = a1 -/+ i b1, y_2,3 = a2 -/+ i b2.
template <>
struct Bfly<5> {
    template <class C>
    __device__ __forceinline__ static void run(C *v)
    {
        using X = Cx<C>;
        using S = typename X::S;
        constexpr S c1 = kpick<S>(0.309016994374947424102293417182819059f,
                                  0.309016994374947424102293417182819059);  // cos(2 pi/5)
        constexpr S c2 = kpick<S>(-0.809016994374947424102293417182819059f,
                                  -0.809016994374947424102293417182819059); // cos(4 pi/5)
        constexpr S s1 = kpick<S>(0.951056516295153572116439333379382143f,
                                  0.951056516295153572116439333379382143);  // sin(2 pi/5)
        constexpr S s2 = kpick<S>(0.587785252292473129168705954639072769f,
                                  0.587785252292473129168705954639072769);  // sin(4 pi/5)
        C x0 = v[0];
        C sa = cadd(v[1], v[4]), da = csub(v[1], v[4]);
        C sb = cadd(v[2], v[3]), db = csub(v[2], v[3]);
        C a1 = X::make(x0.x + c1 * sa.x + c2 * sb.x, x0.y + c1 * sa.y + c2 * sb.y);
        C a2 = X::make(x0.x + c2 * sa.x + c1 * sb.x, x0.y + c2 * sa.y + c1 * sb.y);
        C b1 = X::make(s1 * da.x + s2 * db.x, s1 * da.y + s2 * db.y);
        C b2 = X::make(s2 * da.x - s1 * db.x, s2 * da.y - s1 * db.y);
        v[0] = X::make(x0.x + sa.x + sb.x, x0.y + sa.y + sb.y);
        v[1] = X::make(a1.x + b1.y, a1.y - b1.x);
        v[4] = X::make(a1.x - b1.y, a1.y + b1.x);
        v[2] = X::make(a2.x + b2.y, a2.y - b2.x);
        v[3] = X::make(a2.x - b2.y, a2.y + b2.x);
    }
};

// cos and sin of 2 pi m / 12 (multiples of 30 degrees) and of 2 pi m / 10
// (multiples of 36 degrees): the twiddles of the composite butterflies below.
constexpr double kS3 = 0.866025403784438646763723170752936183;  // cos(pi/6)
constexpr double kC36 = 0.809016994374947424102293417182819059; // cos(pi/5)
constexpr double kS36 = 0.587785252292473129168705954639072769; // sin(pi/5)
constexpr double kC72 = 0.309016994374947424102293417182819059; // cos(2 pi/5)
constexpr double kS72 = 0.951056516295153572116439333379382143; // sin(2 pi/5)

__host__ __device__ constexpr double cos12(int m)
{
    m = ((m % 12) + 12) % 12;
    return m == 0 ? 1.0 : m == 1 ? kS3 : m == 2 ? 0.5 : m == 3 ? 0.0 : m == 4 ? -0.5 : m == 5 ? -kS3
         : m == 6 ? -1.0 : m == 7 ? -kS3 : m == 8 ? -0.5 : m == 9 ? 0.0 : m == 10 ? 0.5 : kS3;
}
__host__ __device__ constexpr double sin12(int m) { return cos12(m - 3); }
__host__ __device__ constexpr double cos10(int m)
{
    m = ((m % 10) + 10) % 10;
    return m == 0 ? 1.0 : m == 1 ? kC36 : m == 2 ? kC72 : m == 3 ? -kC72 : m == 4 ? -kC36 : m == 5 ? -1.0
         : m == 6 ? -kC36 : m == 7 ? -kC72 : m == 8 ? kC72 : kC36;
}
__host__ __device__ constexpr double sin10(int m)
{
    m = ((m % 10) + 10) % 10;
    return m == 0 || m == 5 ? 0.0 : m == 1 || m == 4 ? kS36 : m == 2 || m == 3 ? kS72 : m == 6 || m == 9 ? -kS36
                                                                                        : -kS72;
}

// a * w_N^M for N in {6, 10, 12} (and the powers of two of mul_w), M known at
// compile time.
template <int N, int M, class C>
__device__ __forceinline__ C mul_wn(C a)
{
    if constexpr (16 % N == 0) {
        return mul_w<N, M>(a);
    } else {
        static_assert(N == 6 || N == 10 || N == 12, "composite twiddles exist for 6, 10 and 12 points");
        using X = Cx<C>;
        using S = typename X::S;
        constexpr int m = ((M % N) + N) % N;
        if constexpr (m == 0) {
            return a;
        } else if constexpr (N != 10 && (m * (12 / N)) % 3 == 0) {
            return mul_w<4, (m * (12 / N)) / 3>(a); // multiples of 90 degrees
        } else {
            constexpr S c = (S)(N == 10 ? cos10(m) : cos12(m * (12 / N)));
            constexpr S s = (S)(N == 10 ? sin10(m) : sin12(m * (12 / N)));
            return X::make(X::fma_(a.x, c, a.y * s), X::fma_(a.y, c, -a.x * s));
        }
    }
}

// DFT_{A B} in registers by Eq. ct with n0 = A, n1 = B: DFT_B on x[i0 + A i1]
// for each i0, twiddle w_{AB}^{i0 k1}, DFT_A across i0, output y[k1 + B k0].
template <int A, int B, int I>
struct CtTwiddle {
    template <class C>
    __device__ __forceinline__ static void run(C (*t)[B])
    {
        if constexpr (I < A * B) {
            constexpr int i0 = I / B, k1 = I % B;
            if constexpr (i0 > 0 && k1 > 0)
                t[i0][k1] = mul_wn<A * B, i0 * k1>(t[i0][k1]);
            CtTwiddle<A, B, I + 1>::run(t);
        }
    }
};

template <int A, int B>
struct BflyCt {
    template <class C>
    __device__ __forceinline__ static void run(C *v)
    {
        C t[A][B];
#pragma unroll
        for (int i0 = 0; i0 < A; ++i0) {
#pragma unroll
            for (int i1 = 0; i1 < B; ++i1)
                t[i0][i1] = v[i0 + A * i1];
            Bfly<B>::run(t[i0]);
        }
        CtTwiddle<A, B, 0>::run(t);
#pragma unroll
        for (int k1 = 0; k1 < B; ++k1) {
            C c[A];
#pragma unroll
            for (int i0 = 0; i0 < A; ++i0)
                c[i0] = t[i0][k1];
            Bfly<A>::run(c);
#pragma unroll
            for (int k0 = 0; k0 < A; ++k0)
                v[k1 + B * k0] = c[k0];
        }
    }
};

template <>
struct Bfly<6> : BflyCt<2, 3> {};
template <>
struct Bfly<10> : BflyCt<2, 5> {};
template <>
struct Bfly<12> : BflyCt<4, 3> {};

// ------------------------------------------------------ stage indexing -- //
// Shared-memory position of intra-line index `pos` for the line-major layout:
// one padding slot per 16 keeps the first stages' strided writes free of
// bank conflicts.
__host__ __device__ __forceinline__ constexpr int padpos(int pos) { return pos + (pos >> 4); }

// Line pitch (complex elements) of the padded line-major layout; odd so that
// reading one position of 16 consecutive lines is conflict free too.
__host__ __device__ constexpr int line_pitch(int n) { return (padpos(n - 1) + 1) | 1; }

// Barrier of the threads running the line transforms: the whole block
// (BAR = 0), or the NT threads of named barrier BAR when other warps of the
// block do other work.
template <int BAR, int NT>
__device__ __forceinline__ void lines_sync()
{
    if constexpr (BAR == 0)
        __syncthreads();
    else
        asm volatile("bar.sync %0, %1;" ::"n"(BAR), "n"(NT) : "memory");
}

// One compile-time Stockham stage (see the file header).  `src(j)` returns
// element j of this thread's line, `dst(k, v)` stores element k.  When the
// source and destination alias, SYNC_MID places a barrier between reading
// every input and writing any output.
template <int N, int T, int R, int NS, bool SYNC_MID, int BAR = 0, int NT = 0, class Src, class Dst, class C>
__device__ __forceinline__ void stage_fixed(int t, const Src &src, const Dst &dst, const C *tw)
{
    constexpr int NB = N / R;
    constexpr int BPT = (NB + T - 1) / T;
    constexpr bool FULL = (NB % T) == 0;
    C v[BPT][R];
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int q = t + b * T;
        if (FULL || q < NB) {
#pragma unroll
            for (int r = 0; r < R; ++r)
                v[b][r] = src(q + r * NB);
        }
    }
    if constexpr (SYNC_MID)
        lines_sync<BAR, NT>();
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int q = t + b * T;
        if (FULL || q < NB) {
            const int k = (NS == 1) ? 0 : q % NS;
            if constexpr (NS > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r)
                    v[b][r] = cmul(v[b][r], tw[(r - 1) * NS + k]);
            }
            Bfly<R>::run(v[b]);
            const int base = (NS == 1) ? q * R : (q / NS) * NS * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r)
                dst(base + r * NS, v[b][r]);
        }
    }
}

// Compile-time radix list.
template <int... Rs>
struct Radices {
    static constexpr int count = sizeof...(Rs);
};

// BAR, NT: the barrier of the transforming threads (lines_sync).
template <int N, int T, int NS, class Rad, int BAR = 0, int NT = 0>
struct EngineFixed;

// Last stage: source is shared memory (or global for a single-stage line),
// destination is the caller's sink.
template <int N, int T, int NS, int R, int BAR, int NT>
struct EngineFixed<N, T, NS, Radices<R>, BAR, NT> {
    template <bool FIRST, bool SINK_ALIASES, class Src, class Smem, class Dst, class C>
    __device__ __forceinline__ static void run(int t, const Src &src, const Smem &, const Dst &dst, const C *tw)
    {
        stage_fixed<N, T, R, NS, SINK_ALIASES, BAR, NT>(t, src, dst, tw);
    }
};

template <int N, int T, int NS, int R, int R2, int... Rest, int BAR, int NT>
struct EngineFixed<N, T, NS, Radices<R, R2, Rest...>, BAR, NT> {
    template <bool FIRST, bool SINK_ALIASES, class Src, class Smem, class Dst, class C>
    __device__ __forceinline__ static void run(int t, const Src &src, const Smem &sm, const Dst &dst, const C *tw)
    {
        // The first stage reads its own source; later stages read the shared
        // buffer they also write, so they need the mid-stage barrier.
        stage_fixed<N, T, R, NS, !FIRST, BAR, NT>(t, src, sm, tw);
        lines_sync<BAR, NT>();
        EngineFixed<N, T, NS * R, Radices<R2, Rest...>, BAR, NT>::template run<false, SINK_ALIASES>(
            t, sm, sm, dst, tw + (R - 1) * NS);
    }
};

// The first stage (source -> shared buffer), then `between()` after the
// barrier that ends it (the source has been read by every thread), then the
// remaining stages (shared buffer -> sink).
template <int N, int T, class Rad, int BAR, int NT>
struct EngineSplitFirst;

template <int N, int T, int R, int... Rest, int BAR, int NT>
struct EngineSplitFirst<N, T, Radices<R, Rest...>, BAR, NT> {
    static_assert(sizeof...(Rest) > 0, "at least two stages");
    template <class Src, class Smem, class Dst, class Between>
    __device__ __forceinline__ static void run(int t, const Src &src, const Smem &sm, const Dst &dst,
                                               const float2 *tw, const Between &between)
    {
        stage_fixed<N, T, R, 1, false, BAR, NT>(t, src, sm, tw);
        lines_sync<BAR, NT>();
        between();
        EngineFixed<N, T, R, Radices<Rest...>, BAR, NT>::template run<false, false>(t, sm, sm, dst,
                                                                                  tw + (R - 1));
    }
};

// --------------------------------------------------- runtime stage path -- //
// Same stage with R known at compile time but n, T, NS at run time; used by
// the generic kernels whose radix list is data (any 2*3*5-smooth length).
template <int R, class Src, class Dst, class C>
__device__ __forceinline__ void stage_rt(int n, int T, int NS, int t, const Src &src, const Dst &dst,
                                         const C *tw, bool active)
{
    const int NB = n / R;
    if (!active)
        return;
    for (int q = t; q < NB; q += T) {
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r)
            v[r] = src(q + r * NB);
        const int k = q % NS;
        if (NS > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r)
                v[r] = cmul(v[r], tw[(r - 1) * NS + k]);
        }
        Bfly<R>::run(v);
        const int base = (q / NS) * NS * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r)
            dst(base + r * NS, v[r]);
    }
}

template <class Src, class Dst, class C>
__device__ __forceinline__ void stage_rt_dispatch(int R, int n, int T, int NS, int t, const Src &src,
                                                  const Dst &dst, const C *tw, bool active)
{
    switch (R) {
    case 2: stage_rt<2>(n, T, NS, t, src, dst, tw, active); break;
    case 3: stage_rt<3>(n, T, NS, t, src, dst, tw, active); break;
    case 4: stage_rt<4>(n, T, NS, t, src, dst, tw, active); break;
    case 5: stage_rt<5>(n, T, NS, t, src, dst, tw, active); break;
    case 8: stage_rt<8>(n, T, NS, t, src, dst, tw, active); break;
    case 16: stage_rt<16>(n, T, NS, t, src, dst, tw, active); break;
    default: break;
    }
}

} // namespace fft3
