// plans.h -- the line-transform plans compiled ahead of time.
//
// Each row: id, line length N, threads per line T, radix list (first stage
// first).  The same list drives the device template instantiations
// (k_fixed.cu) and the host planner's metadata (planner.cpp), so the two can
// not disagree on a radix order.  Lengths without a row run through the
// runtime-radix kernel (any 2*3*5-smooth length up to 4096).
//
// Candidates for one length are listed best-first by default; the planner's
// `radix_order` option (and the autotuner) picks among them (ids follow the
// table order: a new candidate goes to the end, after the existing ids).
#pragma once

#define FFT3_FIXED_PLANS_A(X)          \
    X(0, 1024, 64, 16, 16, 4)          \
    X(1, 1024, 64, 4, 16, 16)          \
    X(2, 1024, 32, 16, 16, 4)          \
    X(3, 1024, 64, 8, 8, 16)           \
    X(4, 512, 32, 16, 8, 4)            \
    X(5, 512, 64, 8, 8, 8)             \
    X(6, 512, 32, 4, 8, 16)

#define FFT3_FIXED_PLANS_B(X)          \
    X(7, 256, 16, 16, 16)              \
    X(8, 256, 32, 8, 8, 4)             \
    X(9, 256, 16, 4, 4, 16)            \
    X(10, 128, 8, 16, 8)               \
    X(11, 128, 16, 8, 16)              \
    X(12, 64, 4, 16, 4)                \
    X(13, 64, 8, 8, 8)                 \
    X(14, 64, 16, 4, 4, 4)             \
    X(15, 32, 4, 8, 4)                 \
    X(16, 32, 2, 16, 2)                \
    X(17, 16, 1, 16)                   \
    X(18, 16, 4, 4, 4)                 \
    X(19, 8, 1, 8)                     \
    X(20, 4, 1, 4)                     \
    X(21, 2, 1, 2)                     \
    X(22, 1024, 32, 32, 32)

#define FFT3_FIXED_PLANS(X) FFT3_FIXED_PLANS_A(X) FFT3_FIXED_PLANS_B(X)

// Compile-time volumetric splits of strided lines (k_volc.cu): line length N =
// A * B over a cluster of P blocks, LPT columns per tile, sub-line plans
// (TA threads, radix list RA) for DFT_A and (TB, RB) for DFT_B.
#define FFT3_COMMA ,
#define FFT3_VOLC_LIST(X)                                              \
    X(1024, 32, 32, 4, 16, 2, 16 FFT3_COMMA 2, 2, 16 FFT3_COMMA 2)      \
    X(1024, 32, 32, 2, 16, 2, 16 FFT3_COMMA 2, 2, 16 FFT3_COMMA 2)      \
    X(1024, 32, 32, 8, 16, 2, 16 FFT3_COMMA 2, 2, 16 FFT3_COMMA 2)      \
    X(1024, 32, 32, 8, 32, 2, 16 FFT3_COMMA 2, 2, 16 FFT3_COMMA 2)      \
    X(1024, 32, 32, 4, 32, 2, 16 FFT3_COMMA 2, 2, 16 FFT3_COMMA 2)      \
    X(1024, 32, 32, 8, 64, 2, 16 FFT3_COMMA 2, 2, 16 FFT3_COMMA 2)      \
    X(512, 16, 32, 4, 16, 1, 16, 2, 16 FFT3_COMMA 2)                    \
    X(512, 16, 32, 2, 16, 1, 16, 2, 16 FFT3_COMMA 2)                    \
    X(256, 16, 16, 4, 16, 1, 16, 1, 16)                                 \
    X(256, 16, 16, 2, 16, 1, 16, 1, 16)

// Streamed strided passes (k_cstream.cu).  A line of N = M * Q points is
// taken as Q decimated sub-lines x[Q*j' + q] (Eq. ct with n0 = Q); per tile of
// LPT adjacent columns, G thread groups transform the sub-lines (M = R1 * R2,
// two Stockham stages), each through its own ring of S TMA staging buffers
// refilled as soon as they are read, then one radix-Q stage with twiddles
// w_N^{q k'} stores the lines.  With P = 2 a cluster of two blocks shares a
// tile of LPT = 32 columns, each block holding half of the sub-lines.  The
// line's twiddle table is the stage-major table of (R1, R2, Q).
// Row: N, Q, R1, R2, G, S, LPT, P.
#define FFT3_CSTREAM_LIST(X)             \
    X(1024, 4, 16, 16, 2, 1, 16, 1)      \
    X(1024, 8, 16, 8, 2, 1, 32, 2)       \
    X(1024, 4, 16, 16, 1, 2, 16, 1)      \
    X(1024, 8, 16, 8, 4, 1, 16, 1)       \
    X(1024, 8, 16, 8, 2, 2, 16, 1)       \
    X(1024, 8, 8, 16, 2, 2, 16, 1)       \
    X(512, 4, 16, 8, 2, 1, 16, 1)        \
    X(512, 2, 16, 16, 1, 2, 16, 1)       \
    X(512, 2, 16, 16, 2, 1, 16, 1)       \
    X(512, 4, 16, 8, 2, 1, 32, 2)

namespace fft3 {

struct CStreamKernel {
    int n, q, r1, r2, groups, stages, lpt, pair, threads;
    const void *func;      // nullptr in the host-only metadata
    const void *func_tc[2]; // split-BF16 tensor-core sub-line stages: [0] the first, [1] both (R1 = R2 = 16)
                            // (tc_stages 0 takes [0]; 1 and 2 take [1]: both stages work in shared memory,
                            // the staging buffer and the result slot)
};
// Compiled list (device translation unit) and the host-only metadata.
const CStreamKernel *cstream_kernels(int *count);
const CStreamKernel *cstream_meta(int *count);
// Dynamic shared memory of one block of a streamed pass: twiddles (N-1
// entries rounded to 16), its qp slots of the tile's result (M x LPT each)
// and `bufs` staging buffers (M x LPT); M = n / q.
constexpr int cstream_smem_p(int n, int q, int qp, int lpt, int bufs)
{
    return ((n - 1 + 15) / 16 * 16 + (qp + bufs) * (n / q) * lpt) * 8;
}
constexpr int cstream_smem(int n, int q, int lpt, int bufs) { return cstream_smem_p(n, q, q, lpt, bufs); }
// Blocks per SM the launch bounds ask for: two when two copies of the
// shared memory fit.
constexpr int cstream_min_blocks(int smem_bytes, int threads)
{
    return (2 * (smem_bytes + 1024) <= 228 * 1024 && threads <= 512) ? 2 : 1;
}

// Split-BF16 tcgen05 passes of 1024-point lines (k_tc32.cu): one block of
// four 128-thread groups per SM, tiles of 4 lines, one landing buffer of 34816
// bytes per group (the 32 KB tile, then its padded transposition), the DFT_32
// operand (16 KB), the w_1024 twiddle table (8 KB) and 1 KB of alignment slack.
constexpr int kTc32Groups = 4;
constexpr int kTc32Threads = 128 * kTc32Groups;
constexpr int kTc32Lpt = 4;
constexpr int kTc32LandBytes = kTc32Lpt * 32 * 34 * 8;
constexpr int kTc32SmemBytes = 2 * 64 * 128 + 1024 * 8 + kTc32Groups * kTc32LandBytes + 1024;
// Strided columns (k_tc32s): tiles of 16 columns, six rotating quarter
// buffers of 4096 values (16 columns x 8 x 32 decimated values).
constexpr int kTcsLpt = 16;
constexpr int kTcsQuarters = 6;
constexpr int kTcsQuarterBytes = 4096 * 8;
constexpr int kTcsSmemBytes = 2 * 64 * 128 + 1024 * 8 + kTcsQuarters * kTcsQuarterBytes + 1024;
// mode 0: contiguous lines (bulk copies), 1: strided columns (4D tensor map)
const void *tc32_kernel(int mode);

struct VolcKernel {
    int n, a, b, p, lpt, threads, ta, tb;
    int ra[4], rb[4];
    const void *func; // nullptr in the host-only metadata
};
// Compiled list (device translation unit) and its size.
const VolcKernel *volc_kernels(int *count);
// Host-only metadata: the same list without kernel pointers.
const VolcKernel *volc_meta(int *count);

struct FixedPlanMeta {
    int id, n, T, nrad;
    int rad[8];
};

// Host copy of the list above.
int fixed_plan_count();
const FixedPlanMeta &fixed_plan_meta(int id);

// Device entry points compiled for one fixed plan (nullptr = not compiled).
struct FixedKernels {
    int id;
    const void *j;    // k_pass_j, direct store
    const void *jrot; // k_pass_j, rotated store
    const void *c16;  // k_pass_c, 16 lines per tile
    const void *c8;   // k_pass_c, 8 lines per tile
    const void *l2;   // k_slab_l2 (square slabs), 0 if not compiled
    const void *l2blk[2]; // k_slab_tma (square slabs, blocked output), 4 and 8 lines per tile
    const void *ctma; // k_pass_c_tma (TMA-pipelined strided lines), 0 if not compiled
    // split-BF16 tensor-core variants by tc_stages mode: [0] the first radix-16 stage
    // with both operands in shared memory, [1] every such stage, [2] every radix-16 stage
    const void *j_tc[3]; // contiguous lines, lpt_j(T) lines per tile
    const void *c_tc[3]; // strided lines, 8 lines per tile
};
const FixedKernels *fixed_kernels(int id);

// complex128 passes of a fixed plan (k_pass64.cu): contiguous lines, lpt_j(T)
// lines per tile; strided lines, kLpt64Strided columns per tile (0 if not compiled)
constexpr int kLpt64Strided = 8;
struct Fixed64Kernels {
    int id;
    const void *j;
    const void *c;
};
const Fixed64Kernels *fixed64_kernels(int id);

// Lines per tile of each compiled kernel kind for a plan with T threads per
// line (0 = not compiled).
// rows (x tiles) and columns (y tiles) per tile of the L2-resident slab kernel
constexpr int kSlabL2Lpt = 4;
// landing buffers of the fused slab kernel (k_slab_tma) and its dynamic
// shared memory: twiddles (n-1 rounded to 16), the padded work buffer, the
// ring of landing buffers
constexpr int kSlabTmaBufs = 2;
constexpr int slab_tma_smem(int n, int lpt)
{
    return ((n - 1 + 15) / 16 * 16 + (lpt * ((n - 1 + (n - 1) / 16 + 1) | 1) + 15) / 16 * 16 +
            kSlabTmaBufs * lpt * n) * 8;
}
constexpr int lpt_j(int T) { return T >= 256 ? 1 : 256 / T; }
constexpr int lpt_rot(int T) { return T >= 64 ? 8 : (128 / T > 16 ? 128 / T : 16); }
constexpr int lpt_c(int T, int want) { return T * want <= 1024 ? want : 0; }
// Split-BF16 tensor-core variants exist for plans with a radix-16 stage and
// N >= 128, with at most 512 threads per block (k_fixed.cuh instantiates the
// same conditions).
constexpr int lpt_c_tc() { return 8; }
constexpr bool tc_j_ok(int N, int T, bool has16) { return has16 && N >= 128 && T * lpt_j(T) <= 512 && (T * lpt_j(T)) % 32 == 0; }
constexpr bool tc_c_ok(int N, int T, bool has16) { return has16 && N >= 128 && T * lpt_c_tc() <= 512; }
// Host copy of the stage mask of a radix list for a tc_stages mode (0: the
// first radix-16 stage that is neither the first nor the last stage, 1: every
// such stage, 2: all radix-16 stages).
inline int tc_mask_host(const int *rad, int nrad, int mode)
{
    int all = 0;
    for (int s = 0; s < nrad; ++s)
        all |= (rad[s] == 16 ? 1 : 0) << s;
    const int inner = all & ~1 & ~(1 << (nrad - 1));
    if (mode == 0)
        return inner & (-inner);
    if (mode == 1)
        return inner;
    return all;
}

// TMA-pipelined strided pass: two tiles of N x LPT complex values in flight.
constexpr int lpt_tma(int N, int T) { return (N >= 1024 ? 8 : 16) * T <= 1024 && N >= 16 ? (N >= 1024 ? 8 : 16) : 0; }

} // namespace fft3
