// planner.h -- host-side lowering of a 3D DFT decomposition to a schedule of
// passes with fused load/store maps (no CUDA calls; testable without a GPU).
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fft3.h"
#include "geom.h"

namespace fft3 {

enum PassKind {
    PK_J = 0,      // fixed plan, contiguous lines, direct store
    PK_JROT = 1,   // fixed plan, contiguous lines, rotated (transposed) store
    PK_C = 2,      // fixed plan, strided columns
    PK_G = 3,      // runtime radix list, staged through shared memory
    PK_SLAB = 4,   // 2D DFT of whole n0 x n1 slabs in one block's shared memory
    PK_SLABL2 = 5, // 2D slab DFT: x and y tiles in one persistent launch, slab kept in L2
    PK_VOL = 6,    // 1D DFT split n = a*b over a cluster of p blocks (DSMEM exchange)
    PK_COPY = 7,   // all dimensions of length 1: plain copy
    PK_CTMA = 9,   // fixed plan, strided columns, TMA double-buffered tiles
    PK_JTC = 10,   // split-BF16 tensor-core radix-16 stages, contiguous lines
    PK_CTC = 11,   // split-BF16 tensor-core radix-16 stages, strided columns
    PK_VOLC = 12,  // compile-time volumetric split of strided lines (k_volc.cu)
    PK_CSTREAM = 13, // strided lines, decimated sub-lines streamed by TMA (k_cstream.cu)
    PK_SLABBLK = 14, // 2D slab DFT in one persistent launch, stored as blocked z pencils (k_slab_tma)
    PK_G64 = 15,     // complex128: runtime radix list in FP64 (k_pass_g64)
    PK_J64 = 16,     // complex128: fixed plan, contiguous lines (k_pass_j64)
    PK_C64 = 17,     // complex128: fixed plan, strided columns (k_pass_c64)
    PK_TCX = 18,     // split-BF16 radix-32 tcgen05 GEMM stages, contiguous 1024-point lines (k_tc32.cu)
    PK_TCS = 19,     // split-BF16 radix-32 tcgen05 GEMM stages, strided 1024-point columns (k_tc32.cu)
};

enum BufId { BUF_IN = 0, BUF_OUT = 1, BUF_WS = 2 };

struct LineChoice {
    int n = 1;
    int fixed = -1; // fixed plan id, -1 = runtime radix list
    int T = 1;      // threads per line
    int nst = 0;
    int rad[kMaxStages] = {0};
};

// Twiddle segment: w_n^{m} for the listed exponents, in order.
struct TwSeg {
    int n;
    std::vector<int64_t> m;
    int64_t off = 0; // element offset in the plan's device table
};

struct PassPlan {
    int kind = PK_G;
    int dim = 0; // 0/1/2 transformed dimension; 3 = slab (0 and 1)
    LineChoice line; // 1D passes; slab: x lines
    LineChoice line2; // slab: y lines; volumetric: the a-length sub-lines
    PassGeom g{};
    int src = BUF_IN, dst = BUF_OUT;
    int lpt = 1;
    int tw_seg[3] = {-1, -1, -1}; // segments used (line, line2, split twiddle)
    // volumetric split
    int p = 1, split_a = 1, split_b = 1;
    int threads = 0;     // block size
    int smem_bytes = 0;  // dynamic shared memory per block
    int64_t ntiles = 0, tiles_c = 0;
    int tc_mode = -1;           // split-BF16 tensor-core stages (tc_stages option); -1 = FP32 pass
    int volc = -1;              // PK_VOLC: index into the compiled volumetric list
    int cstream = -1;           // PK_CSTREAM: index into the compiled streamed-pass list
    int chunk = 0;              // slabs per chunk of a two-stream pipelined slab stage (0 = one launch)
    bool pair_next = false;     // this pass and the next run chunk-interleaved on two streams
    bool six_step = false;      // PK_VOL: blocked ownership, three exchanges (Section 2.2)
};

struct Schedule {
    int n0 = 1, n1 = 1, n2 = 1, batch = 1;
    int dtype = FFT3_C64_FP32, decomp = FFT3_PENCIL3, direction = FFT3_FORWARD;
    fft3_options opts{};
    std::vector<PassPlan> passes;
    std::vector<TwSeg> tw;
    int64_t tw_total = 0;
    bool need_ws = false;
    std::string json() const;
};

// Radix list for a line of length n under radix order `order` (runtime path).
int factorize(int n, int order, int *rad, int cap);

// Returns FFT3_OK or an FFT3_ERR_* code (message in *err).
int build_schedule(int n0, int n1, int n2, int batch, int dtype, int decomp, int direction,
                   const fft3_options *opts, Schedule *out, std::string *err);

// Position of natural flat index idx in a permuted layout (fft3_layout).
int layout_position(int layout, int64_t n0, int64_t n1, int64_t n2, int64_t batch, int64_t idx, int64_t *pos);

// Runtime radix list for a line of length n (radix order `order`) and its
// stage-major twiddle exponents.
int choose_runtime_line(int n, int order, LineChoice *lc, std::string *err);
void line_twiddle_exponents(const LineChoice &lc, std::vector<int64_t> *m);

// Lines per tile and shared memory of the runtime-radix kernel for a pass.
void generic_launch_shape(int n, int T, bool strided, int tw_len, int *lpt, int *threads,
                          int *smem);
// The same for elements of esize bytes (16 for complex128).
void generic_launch_shape_elem(int n, int T, bool strided, int tw_len, int esize, int *lpt, int *threads,
                               int *smem);

constexpr int kMaxLine = 4096;
constexpr int kTileTma = 1; // fft3_options.tile_lines value selecting the TMA strided kernel
constexpr int kTileStream = 2; // fft3_options.tile_lines value selecting the streamed strided kernel
constexpr int kSmemLimit = 227 * 1024;

} // namespace fft3
