/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the 3D complex DFT.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load it (through oracle/__init__.py).  It
 * shares no code, header, table or constant with the CUDA path.
 *
 * Conventions (paper: Popovici, Schatz, Franchetti, Low, "A Flexible
 * Framework for Parallel Multi-Dimensional DFTs"):
 *   - Section 2.1: y = DFT_n x with DFT_n = [w_n^{lk}], w_n the n-th root of
 *     unity.  The printed exponent is garbled; it is read here as
 *     w_n = exp(sign * 2*pi*i / n) with sign = -1 for the forward transform
 *     and +1 for the (unnormalised) inverse.
 *   - Section 2.3: a 3D array of n0 x n1 x n2 complex values is stored column
 *     major, n0 fastest: element (j0, j1, j2) of batch b sits at flat index
 *     j0 + n0*(j1 + n1*(j2 + n2*b)).
 *   - Complex values are interleaved (re, im) doubles.
 *
 * Every root of unity is formed from an exactly reduced integer exponent
 * m = (j*k) mod n, then cos/sin of 2*pi*m/n in long double, rounded once to
 * double.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double re, im;
} cplx;

static const long double TWO_PI_L =
    6.283185307179586476925286766559005768394338798750211641949889L;

static inline cplx cmul(cplx a, cplx b)
{
    cplx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
    return r;
}

static inline cplx cadd(cplx a, cplx b)
{
    cplx r = {a.re + b.re, a.im + b.im};
    return r;
}

/* w_n^m = exp(sign * 2 pi i m / n), m reduced mod n in integers first
 * (Section 2.1, definition of DFT_n and of the twiddle matrix). */
static cplx root_of_unity(int64_t n, int64_t m, int sign)
{
    m %= n;
    if (m < 0)
        m += n;
    long double a = TWO_PI_L * (long double)m / (long double)n;
    cplx w = {(double)cosl(a), (double)((long double)sign * sinl(a))};
    return w;
}

/* Table of w_n^m for m in [0, n). */
static cplx *root_table(int64_t n, int sign)
{
    cplx *t = (cplx *)malloc((size_t)n * sizeof(cplx));
    if (!t)
        return NULL;
    for (int64_t m = 0; m < n; ++m)
        t[m] = root_of_unity(n, m, sign);
    return t;
}

int oracle_version(void) { return 3; }

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int t)
{
#ifdef _OPENMP
    if (t > 0)
        omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* Exported for the twiddle pin: w_n^{m_i} for a list of exponents. */
void oracle_roots(int64_t n, const int64_t *m, int64_t count, int sign, double *out)
{
    for (int64_t i = 0; i < count; ++i) {
        cplx w = root_of_unity(n, m[i], sign);
        out[2 * i] = w.re;
        out[2 * i + 1] = w.im;
    }
}

/* ------------------------------------------------------------------------ */
/* 1D DFT as the dense matrix-vector product of Section 2.1:                 */
/*   y[k] = sum_j x[j] * w_n^{j k}                                           */
/* x is read at stride xs (complex elements), y written at stride ys.        */
/* W is the table of w_n^m, m in [0, n).                                     */
/* ------------------------------------------------------------------------ */
static void dft1_direct_tab(const cplx *x, int64_t xs, cplx *y, int64_t ys, int64_t n,
                            const cplx *W)
{
    for (int64_t k = 0; k < n; ++k) {
        cplx acc = {0.0, 0.0};
        for (int64_t j = 0; j < n; ++j) {
            int64_t m = (j * k) % n;
            acc = cadd(acc, cmul(x[j * xs], W[m]));
        }
        y[k * ys] = acc;
    }
}

void oracle_dft1_direct(const double *x, double *y, int64_t n, int sign)
{
    cplx *W = root_table(n, sign);
    if (!W)
        return;
    dft1_direct_tab((const cplx *)x, 1, (cplx *)y, 1, n, W);
    free(W);
}

/* ------------------------------------------------------------------------ */
/* Recursive Cooley-Tukey FFT, Section 2.1 (Eq. ct):                          */
/*   n = n0 * n1, x~[i0, i1] = x[i0 + n0*i1] (n0 x n1, column major),        */
/*   (I)  DFT_{n1} on every row i0 of x~  (elements at stride n0),           */
/*   (II) point-wise product with Twid[i0, k1] = w_n^{i0 k1},                */
/*   (III) transpose,                                                         */
/*   (IV) DFT_{n0} on every column k1, giving y[k1 + n1*k0].                  */
/* Here n0 is the smallest prime factor p of n; a prime n is the leaf and is */
/* transformed by the direct sum above.                                       */
/*                                                                            */
/* x: input at stride xs; y: contiguous output of length n; tmp: n elements  */
/* of scratch for this level plus what deeper levels need (2n in total).     */
/* Wn: table of w_N^m for the top-level length N; the roots for a sub-length */
/* n | N are w_n^m = w_N^{m N / n}.                                           */
/* ------------------------------------------------------------------------ */
static int64_t smallest_prime_factor(int64_t n)
{
    if (n % 2 == 0)
        return 2;
    for (int64_t p = 3; p * p <= n; p += 2)
        if (n % p == 0)
            return p;
    return n;
}

static void fft1_rec(const cplx *x, int64_t xs, cplx *y, int64_t n, const cplx *WN, int64_t N,
                     cplx *tmp)
{
    int64_t scale = N / n; /* w_n^m = w_N^{m*scale} */
    if (n == 1) {
        y[0] = x[0];
        return;
    }
    int64_t p = smallest_prime_factor(n);
    if (p == n) {
        /* leaf: direct DFT_n */
        for (int64_t k = 0; k < n; ++k) {
            cplx acc = {0.0, 0.0};
            for (int64_t j = 0; j < n; ++j)
                acc = cadd(acc, cmul(x[j * xs], WN[((j * k) % n) * scale]));
            y[k] = acc;
        }
        return;
    }
    int64_t n0 = p, n1 = n / p;
    cplx *t = tmp;         /* t[i0*n1 + k1], n elements */
    cplx *deeper = tmp + n;
    /* (I) DFT_{n1} on row i0 of x~: elements x[i0 + n0*i1], i.e. stride n0*xs */
    for (int64_t i0 = 0; i0 < n0; ++i0)
        fft1_rec(x + i0 * xs, xs * n0, t + i0 * n1, n1, WN, N, deeper);
    /* (II) twiddle w_n^{i0 k1}; (III) transpose and (IV) DFT_{n0} per column k1 */
    for (int64_t k1 = 0; k1 < n1; ++k1) {
        for (int64_t i0 = 0; i0 < n0; ++i0)
            t[i0 * n1 + k1] = cmul(t[i0 * n1 + k1], WN[((i0 * k1) % n) * scale]);
        for (int64_t k0 = 0; k0 < n0; ++k0) {
            cplx acc = {0.0, 0.0};
            for (int64_t i0 = 0; i0 < n0; ++i0)
                acc = cadd(acc, cmul(t[i0 * n1 + k1], WN[((i0 * k0) % n0) * (N / n0)]));
            y[k1 + n1 * k0] = acc;
        }
    }
}

void oracle_fft1_rec(const double *x, double *y, int64_t n, int sign)
{
    cplx *W = root_table(n, sign);
    cplx *tmp = (cplx *)malloc((size_t)(2 * n + 2) * sizeof(cplx));
    if (W && tmp)
        fft1_rec((const cplx *)x, 1, (cplx *)y, n, W, n, tmp);
    free(W);
    free(tmp);
}

/* ------------------------------------------------------------------------ */
/* Batched 1D transforms along one dimension of a 3D array (Section 2.3).    */
/* data: batch * n0*n1*n2 complex values, n0 fastest; transformed in place.  */
/* dim: 0, 1 or 2.  method: 0 = direct sum, 1 = recursive FFT,               */
/* 2 = direct for n <= 64, recursive above.                                  */
/* ------------------------------------------------------------------------ */
static void lines_along(cplx *data, int64_t n0, int64_t n1, int64_t n2, int64_t batch, int dim,
                        int sign, int method)
{
    int64_t n = dim == 0 ? n0 : (dim == 1 ? n1 : n2);
    int64_t es = dim == 0 ? 1 : (dim == 1 ? n0 : n0 * n1); /* element stride */
    int64_t N3 = n0 * n1 * n2;
    int64_t lines = batch * N3 / n;
    int use_direct = (method == 0) || (method == 2 && n <= 64);
    cplx *W = root_table(n, sign);
    if (!W)
        return;
#pragma omp parallel
    {
        cplx *line = (cplx *)malloc((size_t)n * sizeof(cplx));
        cplx *res = (cplx *)malloc((size_t)n * sizeof(cplx));
        cplx *tmp = (cplx *)malloc((size_t)(2 * n + 2) * sizeof(cplx));
#pragma omp for schedule(static)
        for (int64_t l = 0; l < lines; ++l) {
            /* line l -> base offset of its first element */
            int64_t base;
            if (dim == 0) {
                base = l * n0;
            } else if (dim == 1) {
                int64_t i0 = l % n0, rest = l / n0; /* rest = b*n2 + i2 */
                base = rest * n0 * n1 + i0;
            } else {
                int64_t i01 = l % (n0 * n1), b = l / (n0 * n1);
                base = b * N3 + i01;
            }
            for (int64_t j = 0; j < n; ++j)
                line[j] = data[base + j * es];
            if (use_direct)
                dft1_direct_tab(line, 1, res, 1, n, W);
            else
                fft1_rec(line, 1, res, n, W, n, tmp);
            for (int64_t k = 0; k < n; ++k)
                data[base + k * es] = res[k];
        }
        free(line);
        free(res);
        free(tmp);
    }
    free(W);
}

/* 3D DFT by the pencil-pencil-pencil definition of Section 2.3: DFT_{n0}
 * along the fastest dimension, then DFT_{n1}, then DFT_{n2}.  Only the
 * dimensions whose bit is set in dim_mask are transformed, so single passes
 * can be checked on their own. */
void oracle_fft3_dims(const double *x, double *y, int64_t n0, int64_t n1, int64_t n2,
                      int64_t batch, int sign, int method, int dim_mask)
{
    int64_t total = batch * n0 * n1 * n2;
    if (x != y)
        memcpy(y, x, (size_t)total * sizeof(cplx));
    for (int d = 0; d < 3; ++d)
        if (dim_mask & (1 << d))
            lines_along((cplx *)y, n0, n1, n2, batch, d, sign, method);
}

void oracle_fft3(const double *x, double *y, int64_t n0, int64_t n1, int64_t n2, int64_t batch,
                 int sign, int method)
{
    oracle_fft3_dims(x, y, n0, n1, n2, batch, sign, method, 7);
}

/* Batched 1D transforms of `lines` lines of length n, line l at x + l*ls,
 * element stride es (complex units), in place.  Used by the CPU baseline to
 * time a bounded sample of the lines of a large transform. */
void oracle_fft1_lines(double *data, int64_t n, int64_t lines, int64_t ls, int64_t es, int sign,
                       int method)
{
    cplx *d = (cplx *)data;
    int use_direct = (method == 0) || (method == 2 && n <= 64);
    cplx *W = root_table(n, sign);
    if (!W)
        return;
#pragma omp parallel
    {
        cplx *line = (cplx *)malloc((size_t)n * sizeof(cplx));
        cplx *res = (cplx *)malloc((size_t)n * sizeof(cplx));
        cplx *tmp = (cplx *)malloc((size_t)(2 * n + 2) * sizeof(cplx));
#pragma omp for schedule(static)
        for (int64_t l = 0; l < lines; ++l) {
            for (int64_t j = 0; j < n; ++j)
                line[j] = d[l * ls + j * es];
            if (use_direct)
                dft1_direct_tab(line, 1, res, 1, n, W);
            else
                fft1_rec(line, 1, res, n, W, n, tmp);
            for (int64_t k = 0; k < n; ++k)
                d[l * ls + k * es] = res[k];
        }
        free(line);
        free(res);
        free(tmp);
    }
    free(W);
}

/* ------------------------------------------------------------------------ */
/* Brute force 3D DFT: every output is the full N-term sum                    */
/*   X[k0,k1,k2] = sum_j x[j0,j1,j2] w_{n0}^{j0k0} w_{n1}^{j1k1} w_{n2}^{j2k2} */
/* with the three phases combined into one exact integer exponent over       */
/* L = n0*n1*n2:  m = j0k0*(L/n0) + j1k1*(L/n1) + j2k2*(L/n2)  (mod L).       */
/* O(N^2): for the smallest shapes only.                                      */
/* ------------------------------------------------------------------------ */
void oracle_bruteforce3(const double *x, double *y, int64_t n0, int64_t n1, int64_t n2, int sign)
{
    const cplx *xc = (const cplx *)x;
    cplx *yc = (cplx *)y;
    int64_t L = n0 * n1 * n2;
    for (int64_t k2 = 0; k2 < n2; ++k2)
        for (int64_t k1 = 0; k1 < n1; ++k1)
            for (int64_t k0 = 0; k0 < n0; ++k0) {
                long double sr = 0.0L, si = 0.0L;
                for (int64_t j2 = 0; j2 < n2; ++j2)
                    for (int64_t j1 = 0; j1 < n1; ++j1)
                        for (int64_t j0 = 0; j0 < n0; ++j0) {
                            int64_t m = ((j0 * k0) % n0) * (L / n0) + ((j1 * k1) % n1) * (L / n1) +
                                        ((j2 * k2) % n2) * (L / n2);
                            m %= L;
                            long double a = TWO_PI_L * (long double)m / (long double)L;
                            long double c = cosl(a), s = (long double)sign * sinl(a);
                            cplx v = xc[j0 + n0 * (j1 + n1 * j2)];
                            sr += (long double)v.re * c - (long double)v.im * s;
                            si += (long double)v.re * s + (long double)v.im * c;
                        }
                yc[k0 + n0 * (k1 + n1 * k2)].re = (double)sr;
                yc[k0 + n0 * (k1 + n1 * k2)].im = (double)si;
            }
}
