/*
 * fft3.h -- C ABI of libfft3: batched forward and inverse 3D complex DFTs on
 * one GB300 (sm_103a), computed as passes of batched 1D DFTs along each
 * dimension with the data redistributions between passes fused into the
 * passes' loads and stores.
 *
 * The operations follow Popovici, Schatz, Franchetti, Low, "A Flexible
 * Framework for Parallel Multi-Dimensional DFTs":
 *   - Section 2.1: y = DFT_n x with DFT_n = [w_n^{lk}], w_n = exp(-2 pi i / n)
 *     for the forward transform (the printed exponent is garbled and is read
 *     with the imaginary unit); the inverse uses exp(+2 pi i / n) and is
 *     unnormalised, so inverse(forward(x)) = n0*n1*n2 * x.
 *   - Section 2.3: an n0 x n1 x n2 array is stored column major with n0
 *     fastest; element (j0, j1, j2) of batch entry b is at complex offset
 *     j0 + n0*(j1 + n1*(j2 + n2*b)).  In PyTorch terms a contiguous complex64
 *     tensor of shape (batch, n2, n1, n0).
 *   - Sections 2.3 and 2.4: the slab-pencil and pencil-pencil-pencil
 *     decompositions; Section 3.2 and Fig. cuboid: the volumetric
 *     decomposition, where each 1D DFT is itself split Cooley-Tukey style
 *     (n = a*b, Eq. ct) over a group of p cooperating thread blocks holding the
 *     line in elemental-cyclic order.
 *
 * Data: complex64, interleaved (re, im) float32, 8 bytes per element.
 * Device pointers must be 16-byte aligned (cudaMalloc / torch allocations are).
 *
 * Errors: every entry point returns FFT3_OK (0) or a negative FFT3_ERR_*
 * code; fft3_last_error() then holds a message for the calling thread.  The
 * library never aborts or exits the process.
 *
 * Threading: plans are independent objects; one plan must not execute on two
 * streams at once (its workspace and counters are shared).
 */
#ifndef FFT3_H
#define FFT3_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fft3_plan_s *fft3_plan; /* opaque; owned by the library */

/* arithmetic of the line transforms; storage is complex64 except for FFT3_C128_FP64 */
enum fft3_dtype {
    FFT3_C64_FP32 = 0,         /* FP32 CUDA-core butterflies */
    FFT3_C64_SPLITBF16_TC = 1, /* radix-32 / radix-16 sub-DFTs as split-BF16 tensor-core GEMMs (hi + lo
                                  BF16 parts, three products), FP32 accumulation (options.tc_stages) */
    FFT3_C128_FP64 = 2         /* complex128 arrays (interleaved FP64 re, im; 16 bytes per element),
                                  FP64 butterflies and FP64 twiddles: the paper's own precision
                                  (Section 4).  Natural pencil-pencil-pencil schedule of runtime-radix
                                  passes (slab-pencil and FFT3_AUTO lower to it; volumetric, rotated,
                                  blocked and permuted layouts are refused).  Buffers hold
                                  n0*n1*n2*batch complex128 values */
};

enum fft3_decomp {
    FFT3_SLAB_PENCIL = 0, /* 2D DFT on n0 x n1 slabs, then DFT_{n2} (Section 2.3, Fig. 3ddftopt a) */
    FFT3_PENCIL3 = 1,     /* DFT_{n0}, DFT_{n1}, DFT_{n2} (Section 2.3, Fig. 3ddftopt b) */
    FFT3_VOLUMETRIC = 2,  /* every 1D DFT split over p cooperating blocks (Section 3.2) */
    FFT3_AUTO = 3         /* the planner's fixed rule: slab-pencil when a slab fits one block's shared
                             memory, else pencil-pencil-pencil with the blocked intermediate where it
                             applies; fft3_autotune and the learned chooser pick by measurement */
};

enum fft3_direction { FFT3_FORWARD = -1, FFT3_INVERSE = +1 }; /* sign of the exponent */

enum fft3_status {
    FFT3_OK = 0,
    FFT3_ERR_INVALID_ARG = -1,         /* null pointer, non-positive size, bad enum */
    FFT3_ERR_UNSUPPORTED_SIZE = -2,    /* prime factor > 5, line too long, infeasible split */
    FFT3_ERR_OOM = -3,                 /* device or host allocation failed */
    FFT3_ERR_CUDA = -4,                /* CUDA runtime error; message in fft3_last_error() */
    FFT3_ERR_TIMEOUT = -5,             /* a bounded device-side wait expired */
    FFT3_ERR_INPLACE_UNSUPPORTED = -6, /* in == out */
    FFT3_ERR_NO_DEVICE = -7            /* no CUDA device visible */
};

/* Pencil-pencil-pencil variants (options.variant). */
enum fft3_ppp_variant {
    FFT3_PPP_NATURAL = 0, /* x pass out-of-place, y and z passes in place on strided lines */
    FFT3_PPP_ROTATE = 1,  /* each pass stores its result rotated xyz -> yzx -> zxy -> xyz (Section 2.4) */
    FFT3_PPP_BLOCKED = 2  /* the y pass stores into a workspace blocked as [x/16][z][y][x%16], so each
                             16-column tile of the y pass is one contiguous block and the z pass reads
                             rows 16*n1 values apart instead of n0*n1; the z pass restores natural order.
                             Needs n0 % 16 == 0, batch 1 and streamed kernels for n1 and n2; otherwise the
                             natural variant is used */
};

/* Layout of the spectrum (options.layout): where a forward plan writes X[k0,k1,k2]
 * of batch b and where an inverse plan reads it.  Section 2.4: applications that
 * only need the spectrum in some known order (convolutions, PDE solvers) can skip
 * the last redistribution and keep the data shuffled.  fft3_layout_positions
 * gives the position of every element, N = n0*n1*n2:
 *   NATURAL  k0 + n0*(k1 + n1*k2) + N*b;
 *   ROTATED  the paper's shuffled order after the rotations xyz -> yzx -> zxy with
 *            the final rotation back to xyz dropped: k2 + n2*(k0 + n0*k1) + N*b;
 *   PENCILS  z pencils blocked by 16 columns of x, [k0/16][k2][k1][k0%16]:
 *            (k0/16)*16*n1*n2 + k2*16*n1 + k1*16 + k0%16 (batch 1, n0 % 16 == 0);
 *            the layout the default schedule's z pass reads, so a forward plan
 *            saves that pass's redistribution and an inverse plan starts from it.
 * Permuted layouts need every dimension > 1 and a slab-pencil, pencil-pencil-pencil
 * or automatic decomposition (FFT3_LAYOUT_PENCILS also with the split-BF16 dtype). */
enum fft3_layout { FFT3_LAYOUT_NATURAL = 0, FFT3_LAYOUT_ROTATED = 1, FFT3_LAYOUT_PENCILS = 2 };

/* Volumetric variants (options.variant with FFT3_VOLUMETRIC). */
enum fft3_vol_variant {
    FFT3_VOL_CYCLIC = 0,           /* elemental-cyclic ownership of every split line: one exchange
                                      (Section 3.2, needs p | a and p | b) */
    FFT3_VOL_BLOCKED_SIX_STEP = 1  /* blocked ownership (block r owns elements [r n/p, (r+1) n/p) of a
                                      line): the six-step algorithm of Section 2.2, Eq. ctparallel,
                                      with three exchanges; a comparison schedule for what the cyclic
                                      distribution saves (runtime-radix cluster kernel) */
};

/* Optional planner controls.  Zero-initialise and set what you need. */
typedef struct fft3_options {
    int variant;      /* fft3_ppp_variant for FFT3_PENCIL3, fft3_vol_variant for FFT3_VOLUMETRIC */
    int radix_order;  /* index into the candidate radix orders of each line length (0 = default) */
    int tile_lines;   /* strided passes: 0 = default (the streamed kernel where one is
                         compiled for the line length, else 16 lines per tile);
                         8 or 16 = lines per tile of the plain strided kernel;
                         1 = tiles moved by TMA, double-buffered (8 or 16 lines by length);
                         2 = the streamed kernel: decimated sub-lines loaded by TMA
                             while earlier ones are transformed (512 and 1024 points) */
    int mesh[3];      /* volumetric: blocks cooperating on one line of dim d, 1/2/4/8 (0 = auto) */
    int slab_mode;    /* slab-pencil: 0 = auto, 1 = one block per slab in shared memory,
                         2 = L2-resident x/y stages in one persistent launch,
                         3 = x and y passes as two launches,
                         4 = x and y passes pipelined over chunks of slabs on two
                             streams: the y lines of a chunk run on the plan's side
                             stream while the x lines of the next chunk run on the
                             caller's stream, so the y pass reads what the x pass
                             has just left in L2; the side stream joins the caller's
                             stream before the z pass,
                         5 = x and y tiles of every slab in one persistent launch that
                             stores the slabs as z pencils ([x/16][z][y][x%16] in the
                             workspace) with the intermediate kept in L2 (one HBM
                             sweep for the 2D slab stage; tiles loaded by TMA), then
                             the z pass back to natural order.  Square 256, 512 or
                             1024 slabs, batch 1, n2 > 1; the workspace is array-sized */
    int tc_stages;    /* FFT3_C64_SPLITBF16_TC: which sub-DFTs run on the tensor cores:
                         0 = 1024-point lines as two radix-32 stages, both split-BF16 GEMMs on
                             the tcgen05 tensor cores (M = 128 rows of 4 lines, N = K = 64), other
                             lengths as mode 3 (the default),
                         1 = every radix-16 stage whose operands are both in shared memory
                             (mma.sync m16n8k16),
                         2 = every radix-16 stage (mma.sync m16n8k16),
                         3 = per line, the first radix-16 stage whose operands are both in
                             shared memory (mma.sync m16n8k16; lines without one stay FP32) */
    int slab_chunk;   /* slab_mode 4: slabs per chunk (0 = about 32 MiB of slabs) */
    int slab_lines;   /* slab_mode 5: rows per x tile and columns per y tile, 4 or 8 (0 = 4) */
    int layout;       /* fft3_layout of the forward output / inverse input (0 = natural) */
    int dist_ranks;   /* > 1: a rank-local plan of the slab-pencil decomposition distributed over
                         dist_ranks processes (Section 2.4, a 1D grid of P processes; FFT3_SLAB_PENCIL,
                         batch 1, complex64 or complex128).  Rank r owns the slabs z in
                         [r n2/P, (r+1) n2/P) of the input and the x range [r n0/P, (r+1) n0/P) of
                         the spectrum.  dist_stage selects the plan:
                         1 = the 2D DFT of the rank's slabs: create with (n0, n1, n2/P); `in` holds the
                             rank's slabs [z_local][y][x]; `out` receives them packed for the all-to-all
                             as [dest][z_local][y][x_local] (the y pass stores there directly), so block
                             `dest` of n0 n1 n2 / P^2 values goes to rank dest (needs P | n0);
                         2 = the DFTs along z of the rank's pencils: create with (n0/P, n1, n2); `in` is
                             the all-to-all's receive buffer, [src][z_local][y][x_local] = the natural
                             layout [z][y][x_local] of the rank's x range; `out` the same layout.
                         3 = the local side of the second exchange, which returns the spectrum to
                             slabs (Fig. 3dslabpencil; optional, as the paper allows leaving the
                             spectrum in pencils): create with (n0, n1, n2/P); forward: `in` is that
                             exchange's receive buffer [src][z_local][y][x_local], `out` the natural
                             slabs [z_local][y][x]; inverse: the reverse, packing natural spectrum
                             slabs for the first exchange.
                         Forward: stage 1, exchange, stage 2 (then exchange, stage 3); inverse: (stage 3,
                         exchange,) stage 2, exchange, stage 1.  The exchanges (all-to-alls of P equal
                         blocks of n0 n1 n2 / P^2 values) belong to the caller's communication library.
                         Rejected with FFT3_ERR_INVALID_ARG: dist_ranks < 0, a stage outside 0..3, a
                         stage without dist_ranks > 1 or dist_ranks > 1 without a stage;
                         FFT3_ERR_UNSUPPORTED_SIZE: another decomposition than FFT3_SLAB_PENCIL or
                         FFT3_AUTO, the split-BF16 dtype, batch > 1, a permuted layout, and for
                         stages 1 and 3 a rank count that does not divide n0 */
    int dist_stage;   /* see dist_ranks */
    int dist_ranks2;  /* FFT3_PENCIL3 with dist_stage 1..3: a rank-local plan of the pencil-pencil-pencil
                         decomposition on a Py x Pz grid of processes (Section 2.4), Py = dist_ranks >= 1,
                         Pz = dist_ranks2 >= 1 (0 = 1), Py Pz > 1.  Rank (p, q) holds at first the x lines
                         of y in [p n1/Py, (p+1) n1/Py) and z in [q n2/Pz, (q+1) n2/Pz); after the first
                         all-to-all (among the Py ranks of its row q) the y lines of x in
                         [p n0/Py, (p+1) n0/Py), z as before; after the second (among the Pz ranks of its
                         column p) the z lines of that x range and of y in [q n1/Pz, (q+1) n1/Pz), its brick
                         of the spectrum (the last redistribution left out).  Forward stages:
                         1 = x lines: create with (n0, n1/Py, n2/Pz); `in` natural [z][y][x]; `out` packed
                             for the row exchange as [dest][x_local][z][y] (the rotated store of the pass);
                         2 = y lines: create with (n0/Py, n1, n2/Pz); `in` the row exchange's receive
                             buffer [src][x][z][y_local] (each line read in its Py runs); `out` packed for
                             the column exchange as [dest][y_local][z][x];
                         3 = z lines: create with (n0/Py, n1/Pz, n2); `in` the column exchange's receive
                             buffer [src][y][z_local][x]; `out` the brick in natural order [z][y][x].
                         The inverse takes the same plans in the order 3, 2, 1 (each storing what the
                         previous forward stage read).  Needs Py | n0, Py | n1, Pz | n1, Pz | n2
                         (FFT3_ERR_UNSUPPORTED_SIZE otherwise); these stages run the runtime-radix kernels
                         where a line is split over exchange blocks */
    int reserved[8];  /* test hooks of the failure-detection tests, 0 in normal use:
                         [0] = s + 1 makes the x tiles of slab s never signal their
                         completion, so the waits of its y tiles expire;
                         [1] = bound of each device-side wait, in thousands of clock
                         cycles (0 = about two seconds) */
} fft3_options;

/* Create a plan for `batch` transforms of n0 x n1 x n2 (n0 fastest).
 * dtype: fft3_dtype; decomposition: fft3_decomp; direction: fft3_direction.
 * Allocates the plan's device twiddle tables (computed in FP64 on the GPU,
 * rounded to float32) and any workspace on the current device.
 * Returns FFT3_ERR_UNSUPPORTED_SIZE for sizes with a prime factor > 5 or
 * line lengths above 4096, and for volumetric meshes that do not divide the
 * Cooley-Tukey split (p | a and p | b, Section 3.2). */
int fft3_plan_create(fft3_plan *out, int n0, int n1, int n2, int batch, int dtype,
                     int decomposition, int direction);

/* As fft3_plan_create, with planner controls (opts may be NULL). */
int fft3_plan_create_ex(fft3_plan *out, int n0, int n1, int n2, int batch, int dtype,
                        int decomposition, int direction, const fft3_options *opts);

/* Batched uneven transforms: `count` independent 3D DFTs (Section 2.3 for
 * each), problem i of size dims[3i] x dims[3i+1] x dims[3i+2] (first fastest)
 * starting at complex offset offsets[i] of both the input and the output
 * buffer (the problems' extents must not overlap).  Three execution modes,
 * each captured once in a CUDA graph (re-captured when the buffers change):
 *   slab executor: one persistent launch of work items from a ticket counter,
 *              the slab-pencil definition of Section 2.3 per problem: an item
 *              is a few n0 x n1 slabs of a problem (x lines read from global
 *              memory into a shared-memory stack, y lines from the stack
 *              written to global memory: one read and one write for the 2D
 *              stage) or a group of z-line tiles of a problem (read through L2
 *              once every slab of the problem is done; bounded waits).  The x
 *              and y lines run in the registers of a few lanes of a warp (warp
 *              shuffles, no block barrier), the z tiles through shared memory;
 *              line lengths 8, 16, 24, 32, 40, 48, 64, 80, 96, 128;
 *   segmented: three passes over the whole batch (all x lines, all y lines,
 *              all z lines of every problem, one compile-time line kernel per
 *              line length, the same lengths), the pencil-pencil-pencil
 *              definition of Section 2.3 per problem.  The x lines of most
 *              lengths run in the registers of a few lanes of a warp (16-byte
 *              loads and stores where a problem starts 16-byte aligned); in
 *              this mode the radix_order field picks the x-line kernel of each
 *              length: 0 = the length's default, r + 1 = candidate r (the
 *              shared-memory kernel, then the warp-shuffle kernels), modulo
 *              their number;
 *   executor:  one persistent launch with its counter reset; work items of
 *              every problem's phases (runtime radix lists) in waves that keep
 *              a problem's intermediate in L2.
 * FFT3_AUTO with tuning == NULL on a batch of at least 4 Mi values takes the
 * slab executor when every length is one of its lengths and every slab fits
 * one item (n1 * (n0 | 1) <= 96 * 97), else the segmented passes when every
 * line length has a compiled plan; other batches take the executor.  With
 * tuning codes: FFT3_TUNE_SLABZ on every code asks for the slab executor,
 * decomposition field 3 on every code for the segmented passes, anything
 * else for the executor.
 * Dimensions: 2*3*5-smooth, <= 128.
 * decomposition: FFT3_SLAB_PENCIL, FFT3_PENCIL3 or FFT3_AUTO (per problem).
 * dtype: FFT3_C64_FP32.  `tuning` may be NULL or point to `count` tuning
 * codes built with FFT3_TUNE (0 = defaults); fft3_autotune_many writes them. */
#define FFT3_TUNE(decomp, radix_order, tile_code, items_code)                        \
    ((decomp) | (((radix_order) + 1) << 2) | ((tile_code) << 5) | ((items_code) << 8))
/* decomp: 1 = slab-pencil, 2 = pencil-pencil-pencil, 3 = the segmented passes
 * (whole batch: every code must ask for it); tile_code: columns per
 * tile of the strided phases, 1 -> 4, 2 -> 8, 3 -> 16, 4 -> 32; items_code
 * (4 bits, 0..15): slabs (slab-pencil) or rows (pencil) per first-phase work
 * item, k -> 2^(k-1), or with decomp 3 the segmented passes in one
 * cooperative launch in 2^(k-1) waves (k <= 11).
 * FFT3_TUNE_SLABZ or'ed into every code: the slab executor whatever the
 * batch size (FFT3_ERR_UNSUPPORTED_SIZE when a length is not one of its
 * lengths); the other fields are ignored. */
#define FFT3_TUNE_SLABZ (1 << 12)
int fft3_plan_create_many(fft3_plan *out, int count, const int *dims, const int64_t *offsets,
                          int dtype, int decomposition, int direction, const int *tuning);

/* Host-only planning of a batched plan, no device needed: the JSON description
 * fft3_plan_create_many's plan would give (mode, kernel launches, problems,
 * work items, line plans, size classes with their tuning codes), without the
 * launch grid.  Same arguments as fft3_plan_create_many; returns the length
 * needed (excluding the terminator) or a negative FFT3_ERR_* code. */
int fft3_plan_schedule_many(int count, const int *dims, const int64_t *offsets, int dtype, int decomposition,
                            int direction, const int *tuning, char *buf, size_t len);

/* Computes the plan's transform: for every batch entry b,
 *   X[k0,k1,k2] = sum_{j0,j1,j2} x[j0,j1,j2] w_n0^{j0 k0} w_n1^{j1 k1} w_n2^{j2 k2}
 * (Section 2.1: DFT_n = [w_n^{lk}], w_n = exp(-2 pi i / n) forward, read with
 * the imaginary unit the printed exponent lacks; exp(+2 pi i / n) for the
 * inverse, unnormalised, so inverse(forward(x)) = n0*n1*n2 * x), as the
 * plan's passes of batched 1D DFTs (Section 2.3: slab-pencil and
 * pencil-pencil-pencil; Section 3.2: volumetric).
 * in, out: device pointers to batch*n0*n1*n2 complex64 values (complex128
 * for FFT3_C128_FP64), or the extent covered by the offsets of a batched
 * plan; element (j0, j1, j2) of entry b at j0 + n0*(j1 + n1*(j2 + n2*b))
 * (Section 2.3: column major, n0 fastest); the output in the same order
 * unless options.layout asks for a permuted spectrum.  `in` is not modified;
 * both buffers stay owned by the caller and must be 16-byte aligned.
 * stream: a cudaStream_t (NULL = legacy default stream); asynchronous and
 * stream ordered.  Errors: FFT3_ERR_INVALID_ARG (null plan or buffer),
 * FFT3_ERR_INPLACE_UNSUPPORTED (in == out), FFT3_ERR_CUDA (launch failure,
 * message in fft3_last_error). */
int fft3_plan_execute(fft3_plan p, const void *in, void *out, void *stream);

/* The transform of fft3_plan_execute (Section 2.1 definition, Section 2.3
 * layout) from and to HOST memory (batch*n0*n1*n2 values each, caller-owned),
 * then synchronises `stream`.  Two ways, picked per call:
 *   direct: when h_in is host memory the device can address (pinned or
 *           registered with CUDA) and the plan's first pass reads its input
 *           with plain loads (the default complex64 and complex128 schedules;
 *           not batched plans, not the tensor-core x pass, which loads by
 *           TMA), the first pass reads h_in in place over the host link (on a
 *           Grace host, the chip-to-chip link): no input copy; the result,
 *           left in a plan-owned device array, is copied to h_out;
 *   staged: otherwise h_in is copied to a plan-owned device array, the plan
 *           runs device to device, and the result is copied to h_out.
 * The device arrays are allocated on the first call that needs them and kept
 * by the plan (FFT3_ERR_OOM if that fails).  The paper's arrays live in the
 * nodes' memory; this entry point is the end-to-end form for callers whose
 * data live on the host. */
int fft3_plan_execute_host(fft3_plan p, const void *h_in, void *h_out, void *stream);

/* `count` transforms from and to HOST memory, pipelined: transform i reads
 * h_in[i] and writes h_out[i] (arrays of `count` host pointers, each to one
 * plan-sized complex64 array; h_out[i] must not overlap any h_in[j]).  Two
 * sets of plan-owned device staging buffers alternate, so the host-to-device
 * copy of transform i+1, the transform of i and the device-to-host copy of
 * i-1 run at the same time on three plan-owned streams.  Returns after every
 * h_out[i] is complete; `stream` is ordered before the first copy.  The
 * staging buffers are allocated on the first call that needs them and kept by
 * the plan.  The paper has no host-memory interface; this is the end-to-end
 * form of the transform for callers whose data live in host memory. */
int fft3_plan_execute_host_pipelined(fft3_plan p, const void *const *h_in, void *const *h_out, int count,
                                     void *stream);

/* Reads and clears the plan's device error flag (set when a bounded wait in a
 * persistent kernel expired).  Synchronises the plan's last stream. */
int fft3_plan_check(fft3_plan p);

/* Frees a plan and everything it owns (twiddle tables, workspace, staging
 * buffers, streams, graphs).  The plan must not be executing.  Planning and
 * plan objects have no counterpart in the paper (its local DFTs are FFTW
 * plans, Section 4.1).  Returns FFT3_ERR_INVALID_ARG for a null plan. */
int fft3_plan_destroy(fft3_plan p);

/* Device bytes the plan owns besides its twiddle tables: the array-sized
 * workspace of schedules that redistribute into a second buffer (the blocked
 * and rotated intermediates of Section 2.4) and the counters of persistent
 * kernels; 0 for a null plan.  No counterpart in the paper, whose
 * redistributions go through MPI buffers (Section 4.1). */
size_t fft3_plan_workspace_bytes(fft3_plan p);

/* Number of passes of the schedule: the valid indices of fft3_plan_execute_pass.
 * Without pipelined pairs (slab_mode 4) it is also the number of kernel
 * launches one fft3_plan_execute issues; a batched plan counts as one (its
 * CUDA graph). */
int fft3_plan_launches(fft3_plan p);

/* Number of kernel launches one fft3_plan_execute issues (a pipelined pair
 * of passes launches each of its two kernels once per chunk; a batched plan's
 * graph holds one launch in executor mode, one per line length and dimension
 * in segmented mode). */
int fft3_plan_kernel_launches(fft3_plan p);

/* JSON description of the pass schedule (decomposition, passes, kernels,
 * line lengths, radix lists, layouts, bytes moved).  Returns the length
 * needed (excluding the terminator), or a negative error. */
int fft3_plan_describe(fft3_plan p, char *buf, size_t len);

/* Host-only planning, no device needed: the JSON schedule that
 * fft3_plan_create_ex would build.  Same return convention as describe. */
int fft3_plan_schedule(int n0, int n1, int n2, int batch, int dtype, int decomposition,
                       int direction, const fft3_options *opts, char *buf, size_t len);

/* Host-only: positions of spectrum elements in a permuted layout (fft3_layout,
 * Section 2.4).  For each natural flat index idx[i] = k0 + n0*(k1 + n1*k2) + N*b
 * (0 <= idx[i] < N*batch) writes pos[i], its offset in complex elements in the
 * buffer a forward plan with that layout writes (and an inverse plan reads).
 * idx and pos are host arrays of `count` entries owned by the caller.  Returns
 * FFT3_OK, FFT3_ERR_INVALID_ARG (null pointer, bad layout, index out of range) or
 * FFT3_ERR_UNSUPPORTED_SIZE (the layout does not exist for these sizes). */
int fft3_layout_positions(int layout, int n0, int n1, int n2, int batch, const int64_t *idx, int64_t *pos,
                          int64_t count);

/* Host-only: the radix list the planner uses for a line of length n under
 * radix_order `order`; returns the number of stages (<= cap) or a negative
 * error (FFT3_ERR_UNSUPPORTED_SIZE for a prime factor > 5). */
int fft3_factorize(int n, int order, int *radices, int cap);

/* FP64 GPU twiddle generator (Section 2.1, twiddle matrix w_n^{kl}): for each
 * of `count` integer exponents m[i] (device int64 array) writes
 * w_n^{m[i]} = exp(sign*2 pi i m[i]/n), with m reduced mod n in integers, as
 * doubles to d_out64 (2*count, may be NULL) and rounded to float32 to
 * d_out32 (2*count, may be NULL).  Device pointers; asynchronous on stream. */
int fft3_twiddles(int n, int sign, const int64_t *d_m, int64_t count, double *d_out64,
                  float *d_out32, void *stream);

/* Layout probe: runs the first `npasses` passes of the plan's schedule (all of
 * them when npasses < 0) with every line transform replaced by the identity,
 * so the composed load/store maps (the redistributions) can be compared
 * bit-exactly with their definitions.  Carry integer source indices in the
 * float32 pairs.  The result always lands in `out` (a pass that ends in the
 * plan's workspace is followed by a copy to `out`). */
int fft3_plan_probe_layout(fft3_plan p, const void *in, void *out, int npasses, void *stream);

/* Executes pass `k` (0-based) of the schedule alone, on the same buffers as
 * fft3_plan_execute: used to time passes one by one with events.  The
 * transform is only complete after passes 0 .. launches-1 ran in order. */
int fft3_plan_execute_pass(fft3_plan p, int k, const void *in, void *out, void *stream);

/* Split-BF16 helper used by the tensor-core path, exposed for tests:
 * hi[i] = bf16(x[i]), lo[i] = bf16(x[i] - hi[i]) (round to nearest even),
 * written as raw uint16 bit patterns.  Device pointers. */
int fft3_split_bf16(const float *d_x, int64_t count, uint16_t *d_hi, uint16_t *d_lo,
                    void *stream);

/* ---- allocation-free transform (no counterpart in the paper) --------------
 * For callers that must not allocate device memory: code embedded in a host
 * application or framework that owns every device allocation and only hands
 * out buffers, and latency-critical loops that cannot afford cudaMalloc and
 * cudaFree, which may synchronise the whole device and can fail once memory is
 * fragmented.  fft3_execute_noalloc computes the same transform as a
 * pencil-pencil-pencil plan with FFT3_PPP_ROTATE, but its workspace and its
 * twiddle tables live in fixed arrays inside the library (16 MiB + 128 KiB of
 * device memory, reserved on a GPU when the library's device code is first
 * loaded there -- with CUDA's default lazy loading, at the first use of the
 * library on that GPU -- and held until the process exits) and it calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *   - in, out: device pointers to batch*n0*n1*n2 complex64 values (n0 fastest);
 *     in is not modified; in == out returns FFT3_ERR_INPLACE_UNSUPPORTED.
 *   - batch*n0*n1*n2 must not exceed FFT3_NOALLOC_MAX_ELEMENTS, otherwise the
 *     call returns FFT3_ERR_UNSUPPORTED_SIZE and does nothing.  The twiddle
 *     tables take at most n0 + n1 + n2 + 48 entries, which always fits
 *     FFT3_NOALLOC_MAX_TWIDDLES because no line may exceed 4096 points (a
 *     longer line, e.g. 8192 x 2 x 1, is FFT3_ERR_UNSUPPORTED_SIZE as for
 *     fft3_plan_create).
 *   - The first call on a device looks up the arrays' device addresses on the
 *     current device (cudaGetSymbolAddress); make that first call before any
 *     stream capture.
 *   - Every call shares the arrays: calls that overlap on the GPU (other
 *     streams, other threads) race and corrupt each other's results; order
 *     them on one stream or synchronise between them.
 *   - Asynchronous on `stream` like fft3_plan_execute. */
#define FFT3_NOALLOC_MAX_ELEMENTS (1 << 21)
#define FFT3_NOALLOC_MAX_TWIDDLES (1 << 14)
int fft3_execute_noalloc(int n0, int n1, int n2, int batch, int direction, const void *in, void *out,
                         void *stream);

/* ---- measured plan selection (no counterpart in the paper, which leaves the
 * choice of decomposition to the user; Section 4.3 shows no single one wins) */

/* Times one plan: creates it, allocates two scratch arrays of the problem's
 * size, runs two untimed executions and `reps` timed ones (CUDA events on the
 * legacy default stream), destroys everything, and writes the mean ms of one
 * execution to *ms. */
int fft3_time_plan(int n0, int n1, int n2, int batch, int dtype, int decomposition, int direction,
                   const fft3_options *opts, int reps, float *ms);

/* Times `count` candidate plans of one shape (decompositions[i], opts[i]) on
 * shared scratch arrays, as fft3_time_plan does for one; ms_out[i] = -1 for a
 * candidate the planner rejects. */
int fft3_time_candidates(int n0, int n1, int n2, int batch, int dtype, int direction, int reps, int count,
                         const int *decompositions, const fft3_options *opts, float *ms_out);

/* Exhaustive autotuning of one shape over the candidate decompositions,
 * pencil variants, slab modes, strided tiles, the 2x2x2 volumetric mesh and
 * radix orders 0..3; infeasible candidates are skipped.  Writes the fastest
 * plan's options, decomposition and mean ms.  Allocates scratch arrays. */
int fft3_autotune(int n0, int n1, int n2, int batch, int dtype, int direction, int reps,
                  fft3_options *best, int *best_decomposition, float *best_ms);

/* Autotuning of a batched plan: times the whole batch (packed into scratch
 * arrays) under the default codes and under each candidate FFT3_TUNE code
 * (both decompositions, radix orders 0..3, tiles of 8/16/32 columns) applied
 * to every problem whose shared-buffer need stays within the default
 * buffers; then, for three size classes (thirds of the batch by problem
 * volume) in turn, the code that makes the whole batch fastest (kept when it
 * gains at least 1%); finally the segmented passes (code 3 for every problem)
 * and the slab executor (FFT3_TUNE_SLABZ on every code), each taken when
 * faster.  Writes the assignment to tuning_out.  The batch is
 * timed as a whole because the executor's buffers, blocks per SM and item
 * order depend on all its problems (per-shape timings in isolation chose
 * codes that made the mixed batch slower).  `offsets` and `max_per_class`
 * are unused and may be NULL / 0. */
int fft3_autotune_many(int count, const int *dims, const int64_t *offsets, int direction, int reps,
                       int max_per_class, int *tuning_out);

/* ---- learned plan cost model (no counterpart in the paper): a perceptron
 * F -> H -> H -> 1 with exact GELU, 0.5 x (1 + erf(x / sqrt 2)), trained on
 * measured plan timings (target: log run time) with the MSE loss and Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8), forward and backward computed by the
 * library's own kernels in FP32.  Parameters form one flat float array
 * [W1 (H x F), b1 (H), W2 (H x H), b2 (H), W3 (1 x H), b3 (1)], row-major;
 * samples are rows of a row-major (n x F) float matrix. */
typedef struct fft3_mlp_s *fft3_mlp;

/* Allocates the model on the current device; weights ~ N(0, 2/fan_in) from a
 * seeded generator, biases 0, Adam moments 0. */
int fft3_mlp_create(fft3_mlp *out, int n_features, int hidden, unsigned long long seed);
int fft3_mlp_destroy(fft3_mlp m);
int fft3_mlp_num_params(fft3_mlp m);
/* Host copies of the flat parameter array (setting also clears Adam's state). */
int fft3_mlp_set_params(fft3_mlp m, const float *h_params);
int fft3_mlp_get_params(fft3_mlp m, float *h_params);
/* Device pointers: d_X (B x F), d_pred (B); asynchronous on stream. */
int fft3_mlp_forward(fft3_mlp m, const float *d_X, int B, float *d_pred, void *stream);
/* Loss (mean squared error against d_y) and its gradient with respect to the
 * flat parameters (written to d_grad, may be NULL; d_loss may be NULL). */
int fft3_mlp_grad(fft3_mlp m, const float *d_X, const float *d_y, int B, float *d_grad, float *d_loss,
                  void *stream);
/* One Adam update with the given gradient (NULL: the last fft3_mlp_grad). */
int fft3_mlp_adam_step(fft3_mlp m, const float *d_grad, float lr, void *stream);
/* Training loop on host arrays: `epochs` passes over a seeded shuffle in
 * minibatches of `batch`; h_loss_curve (epochs floats, may be NULL) receives
 * the full-data loss after every epoch.  Synchronous. */
int fft3_mlp_train(fft3_mlp m, const float *h_X, const float *h_y, int n, int epochs, int batch, float lr,
                   unsigned long long seed, float *h_loss_curve);
/* Predictions for n host samples into h_pred.  Synchronous. */
int fft3_mlp_predict(fft3_mlp m, const float *h_X, int n, float *h_pred);

/* Message of the last failed call on the calling thread (thread-local,
 * owned by the library, valid until that thread's next failing call).  No
 * counterpart in the paper. */
const char *fft3_last_error(void);
/* Version number of the library, increased whenever the C ABI changes. */
int fft3_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FFT3_H */
