// batched_host.cu -- fft3_plan_create_many: planning and graph-captured
// execution of a batch of independent, unevenly sized 3D DFTs in one
// persistent launch (k_batched.cu).
//
// Per problem, a tuning code (fft3.h, FFT3_TUNE_*) selects the decomposition
// (slab-pencil or pencil-pencil-pencil), the radix order of its line plans,
// the columns per tile of its strided phases and the slabs/rows per item of
// its first phase; zero picks the defaults below.  Problems are grouped
// (largest first) into groups of about 16 MB and the work items are emitted
// in waves: wave w holds phase p of group w - p, so a problem's next phase
// runs one group later, while its intermediate result is still in L2.
#include <string.h>

#include <algorithm>
#include <map>
#include <numeric>
#include <sstream>

#include "capi_internal.h"
#include "seg_plans.h"

#include <type_traits>

namespace fft3 {

__global__ void k_batched(BatchArgs a);
__global__ void k_roots(int n, int sign, const int64_t *m, int64_t count, double *o64, float2 *o32);

// One launch of the segmented mode: lines of length n along dimension dim.
struct SegLaunch {
    int dim, n, kernel, lpt, threads, smem;
    const void *func;  // the line kernel (k_seg, or k_segw for warp-shuffle x lines)
    int warp, R, L;    // k_segw: N = R * L, L / 2 lanes per line
    int64_t ntiles;
    int64_t list_off, tstart_off, tcube_off; // offsets into the concatenated device tables
    int64_t tw_off, tw_len;
    dim3 grid;
};

struct BatchState {
    int seg = 0; // 1: three segmented passes (k_segmented.cu) instead of the persistent executor
    std::vector<SegLaunch> seg_launches;
    // the segmented passes as one cooperative launch (k_seg_all): waves of
    // problems, steps of segments, and their tables
    int seg1 = 0;
    // the slab-by-slab executor (k_slabz): tuning codes with FFT3_TUNE_SLABZ
    int slabz = 0;
    int sz_tw_z[16] = {}, sz_tw_w[16] = {};
    int sz_smem = 0;
    dim3 sz_grid;
    int waves = 1;
    std::vector<SegAllSeg> sa_segs;
    std::vector<int> sa_seg0, sa_list, sa_tcube;
    std::vector<int64_t> sa_ntiles, sa_tstart;
    int64_t sa_tw_off = 0;
    int sa_tw_len = 0;
    SegAllSeg *d_sa_segs = nullptr;
    int *d_sa_seg0 = nullptr, *d_sa_list = nullptr, *d_sa_tcube = nullptr, *d_sa_barrier = nullptr;
    int64_t *d_sa_ntiles = nullptr, *d_sa_tstart = nullptr;
    int sa_smem = 0;
    dim3 sa_grid;
    // host tables built by the planning: twiddle segments (offset, count), their
    // exponents and line lengths; the segmented passes' problem lists, first
    // tiles and per-tile slots
    std::vector<std::pair<int64_t, int64_t>> h_segs;
    std::vector<std::vector<int64_t>> h_exps;
    std::vector<int> h_exp_n;
    std::vector<int> h_seg_list, h_seg_tcube;
    std::vector<int64_t> h_seg_tstart;
    int *d_seg_list = nullptr, *d_seg_tcube = nullptr;
    int64_t *d_seg_tstart = nullptr;
    std::vector<BatchCube> cubes;
    std::vector<BatchItem> items;
    std::vector<LineRt> lines;
    std::vector<LineChoice> line_choice;
    std::vector<int> tuning; // effective tuning code per problem
    BatchCube *d_cubes = nullptr;
    BatchItem *d_items = nullptr;
    LineRt *d_lines = nullptr;
    float2 *d_tw = nullptr;
    int *d_counters = nullptr;
    unsigned *d_err = nullptr;
    size_t counters_bytes = 0;
    int64_t tw_total = 0;
    int buf_elems = 0;
    int prefetch = 0;
    int smem = 0;
    int threads = 256;
    dim3 grid;
    int conj = 0;
    int64_t extent = 0;
    // CUDA graph of [counter reset, k_batched], re-captured when the buffers change
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap_stream = nullptr;
    const void *g_in = nullptr;
    void *g_out = nullptr;
    int groups = 0;
};

static inline int pitch_b(int n) { return ((n - 1) + ((n - 1) >> 4) + 1) | 1; }
static bool smooth_b(int n)
{
    if (n < 1)
        return false;
    for (int p : {2, 3, 5})
        while (n % p == 0)
            n /= p;
    return n == 1;
}

void batch_free(BatchState *b)
{
    if (!b)
        return;
    if (b->exec)
        cudaGraphExecDestroy(b->exec);
    if (b->graph)
        cudaGraphDestroy(b->graph);
    if (b->cap_stream)
        cudaStreamDestroy(b->cap_stream);
    cudaFree(b->d_seg_list);
    cudaFree(b->d_seg_tcube);
    cudaFree(b->d_seg_tstart);
    cudaFree(b->d_sa_segs);
    cudaFree(b->d_sa_seg0);
    cudaFree(b->d_sa_list);
    cudaFree(b->d_sa_tcube);
    cudaFree(b->d_sa_barrier);
    cudaFree(b->d_sa_ntiles);
    cudaFree(b->d_sa_tstart);
    cudaFree(b->d_cubes);
    cudaFree(b->d_items);
    cudaFree(b->d_lines);
    cudaFree(b->d_tw);
    cudaFree(b->d_counters);
    cudaFree(b->d_err);
    delete b;
}

static int line_index(BatchState *b, std::map<std::pair<int, int>, int> &idx, int n, int order, std::string *err)
{
    auto key = std::make_pair(n, order);
    auto it = idx.find(key);
    if (it != idx.end())
        return it->second;
    LineChoice lc;
    int rc = choose_runtime_line(n, order, &lc, err);
    if (rc)
        return rc;
    int id = (int)b->line_choice.size();
    b->line_choice.push_back(lc);
    idx[key] = id;
    return id;
}

// Elements per shared buffer that keep four blocks of 256 threads on an SM.
constexpr int kBatchBufTarget = 3072;

// Shared-memory values the slab executor gives a work item's stacked slabs:
// one 96 x 96 slab with its rows 97 values apart.
constexpr int kSlabzRoom = 96 * 97;

// The z-tile plans of the slab executor (FFT3_SLABZ_Z_PLANS): length,
// threads per line, columns per tile and radix list.
struct SlabZPlan {
    int n, T, lpt, nrad, rad[4];
};
template <int... R>
constexpr SlabZPlan slabz_plan(int n, int T, int lpt)
{
    return {n, T, lpt, (int)sizeof...(R), {R...}};
}
#define FFT3_SZ_ZPLAN(N, T, LPT, ...) slabz_plan<__VA_ARGS__>(N, T, LPT),
constexpr SlabZPlan kSlabZPlans[] = {FFT3_SLABZ_Z_PLANS(FFT3_SZ_ZPLAN)};
#undef FFT3_SZ_ZPLAN

// FFT3_AUTO without tuning codes runs the segmented passes from this many
// values on (every line length compiled in seg_plans.h).
constexpr int64_t kSegMinElems = 1ll << 22;

// The compiled kernels for lines of length n in the segmented mode (x lines:
// contiguous; y and z lines: strided), in the
// order the radix_order field of a tuning code selects them (field value
// r + 1 -> entry r mod count): the shared-memory Stockham kernel, then the
// warp-shuffle kernels in table order.  Field value 0 takes the length's
// default: its warp-shuffle kernel marked default, else the shared-memory one.
static std::vector<const SegKernel *> seg_line_candidates(int n, bool contiguous, const SegKernel **dflt)
{
    std::vector<const SegKernel *> c;
    int cnt = 0;
    const SegKernel *k = seg_kernels(contiguous, &cnt);
    for (int i = 0; i < cnt; ++i)
        if (k[i].n == n)
            c.push_back(&k[i]);
    *dflt = c.empty() ? nullptr : c[0];
    k = segw_kernels(&cnt, contiguous);
    for (int i = 0; i < cnt; ++i)
        if (k[i].n == n) {
            c.push_back(&k[i]);
            if (k[i].dflt)
                *dflt = &k[i];
        }
    return c;
}

// Decodes a tuning code (0 = defaults): items of roughly 2-4 thousand
// elements, buffers of at most kBatchBufTarget elements unless a slab needs more.
static void decode_tuning(int code, int n0, int n1, int n2, int *decomp, int *order, int *lpt, int *lpty,
                          int *spi)
{
    const int d = code & 3, o = (code >> 2) & 7, l = (code >> 5) & 7, s = (code >> 8) & 7;
    // slab-pencil keeps the whole slab in shared memory; prefer it for small slabs
    *decomp = d == 1 ? BD_SLAB : d == 2 ? BD_PPP : (n1 * pitch_b(n0) <= kBatchBufTarget ? BD_SLAB : BD_PPP);
    if (*decomp == BD_SLAB && 2 * n1 * pitch_b(n0) * 8 > 200 * 1024)
        *decomp = BD_PPP;
    *order = o ? o - 1 : 0;
    if (l) {
        *lpt = 2 << l; // 1 -> 4, 2 -> 8, 3 -> 16, 4 -> 32, 5 -> 64, 6 -> 128
        *lpty = std::min(n0, *lpt);
    } else {
        *lpt = std::max(16, std::min(4096 / n2, kBatchBufTarget / pitch_b(n2)) / 16 * 16);
        *lpty = std::max(1, std::min(n0, kBatchBufTarget / pitch_b(n1)));
    }
    if (s) {
        *spi = 1 << (s - 1);
    } else if (*decomp == BD_SLAB) {
        *spi = std::max(1, 4096 / (n0 * n1));
    } else {
        *spi = std::max(1, kBatchBufTarget / pitch_b(n0));
    }
}

// Shared-buffer elements one problem needs under a tuning code (the batch's
// buffers are sized by the largest need over its problems).
int batch_buffer_need(int n0, int n1, int n2, int code)
{
    int decomp, order, lpt, lpty, spi;
    decode_tuning(code, n0, n1, n2, &decomp, &order, &lpt, &lpty, &spi);
    if (decomp == BD_SLAB)
        return std::max(n1 * pitch_b(n0), lpt * pitch_b(n2));
    spi = std::max(1, std::min(spi, n1 * n2));
    return std::max(spi * pitch_b(n0), std::max(lpty * pitch_b(n1), lpt * pitch_b(n2)));
}

int batch_kernel_launches(const BatchState *b) { return b->seg && !b->seg1 ? (int)b->seg_launches.size() : 1; }

int batch_describe(const BatchState *b, std::string *json)
{
    std::ostringstream o;
    std::map<std::tuple<int, int, int>, std::pair<int, int>> cls; // shape -> (count, tuning)
    for (size_t i = 0; i < b->cubes.size(); ++i) {
        const BatchCube &c = b->cubes[i];
        auto &e = cls[std::make_tuple(c.n0, c.n1, c.n2)];
        e.first++;
        e.second = b->tuning[i];
    }
    o << "{\"batched\":true,\"mode\":\""
      << (b->seg1 ? "segmented_one_launch" : b->seg ? "segmented" : b->slabz ? "slab_executor" : "executor")
      << "\",\"kernel_launches\":"
      << batch_kernel_launches(b) << ",\"problems\":" << b->cubes.size() << ",\"items\":" << b->items.size()
      << ",\"groups\":" << b->groups << ",\"line_plans\":" << b->lines.size() << ",\"grid\":" << b->grid.x
      << ",\"block\":" << b->threads << ",\"smem\":" << b->smem << ",\"prefetch\":" << b->prefetch << ",\"twiddle_entries\":" << b->tw_total
      << ",\"extent\":" << b->extent;
    if (b->slabz)
        o << ",\"slab_executor_grid\":" << b->sz_grid.x << ",\"slab_executor_smem\":" << b->sz_smem;
    if (b->seg1)
        o << ",\"waves\":" << b->waves << ",\"steps\":" << b->sa_ntiles.size() << ",\"segments\":" << b->sa_segs.size()
          << ",\"one_launch_grid\":" << b->sa_grid.x << ",\"one_launch_smem\":" << b->sa_smem;
    o << ",\"segmented_launches\":[";
    for (size_t k = 0; k < b->seg_launches.size(); ++k) {
        const SegLaunch &L = b->seg_launches[k];
        const int64_t nprob = (k + 1 < b->seg_launches.size() ? b->seg_launches[k + 1].list_off
                                                              : (int64_t)b->h_seg_list.size()) - L.list_off;
        o << (k ? "," : "") << "{\"dim\":" << L.dim << ",\"n\":" << L.n << ",\"lines_per_tile\":" << L.lpt
          << ",\"tiles\":" << L.ntiles << ",\"problems\":" << nprob << ",\"threads\":" << L.threads
          << ",\"smem\":" << L.smem;
        if (L.warp)
            o << ",\"kernel\":\"warp_shuffle\",\"R\":" << L.R << ",\"L\":" << L.L;
        else
            o << ",\"kernel\":\"shared_memory\"";
        o << "}";
    }
    o << "],\"classes\":[";
    bool first = true;
    for (auto &kv : cls) {
        o << (first ? "" : ",") << "{\"dims\":[" << std::get<0>(kv.first) << "," << std::get<1>(kv.first) << ","
          << std::get<2>(kv.first) << "],\"count\":" << kv.second.first << ",\"tuning\":" << kv.second.second << "}";
        first = false;
    }
    o << "]}";
    *json = o.str();
    return FFT3_OK;
}

static int capture(fft3_plan_s *P, const void *in, void *out)
{
    BatchState *b = P->batch;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    BatchArgs a{};
    a.in = (const float2 *)in;
    a.out = (float2 *)out;
    a.cubes = b->d_cubes;
    a.items = b->d_items;
    a.nitems = (int)b->items.size();
    a.lines = b->d_lines;
    a.tw = b->d_tw;
    a.counters = b->d_counters;
    a.err = b->d_err;
    a.wait_budget = 4000000000LL;
    a.conj = b->conj;
    a.buf_elems = b->buf_elems;
    a.prefetch = b->prefetch;
    CUDA_TRY(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    if (b->seg1) {
        SegAllArgs s{};
        s.in = (const float2 *)in;
        s.out = (float2 *)out;
        s.cubes = b->d_cubes;
        s.list = b->d_sa_list;
        s.tstart = b->d_sa_tstart;
        s.tcube = b->d_sa_tcube;
        s.segs = b->d_sa_segs;
        s.seg0 = b->d_sa_seg0;
        s.ntiles = b->d_sa_ntiles;
        s.nsteps = (int)b->sa_ntiles.size();
        s.tw = b->d_tw + b->sa_tw_off;
        s.tw_len = b->sa_tw_len;
        s.barrier = b->d_sa_barrier;
        s.err = b->d_err;
        s.wait_budget = 4000000000LL;
        s.conj = b->conj;
        e = cudaMemsetAsync(b->d_sa_barrier, 0, sizeof(int), b->cap_stream);
        if (e == cudaSuccess) {
            // cooperative: every block resident at once, so the grid barriers end
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeCooperative;
            attr[0].val.cooperative = 1;
            cfg.gridDim = b->sa_grid;
            cfg.blockDim = dim3(kSegAllThreads);
            cfg.dynamicSmemBytes = b->sa_smem;
            cfg.stream = b->cap_stream;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            void *params[1] = {&s};
            e = cudaLaunchKernelExC(&cfg, (const void *)&k_seg_all, params);
        }
    } else if (b->seg) {
        for (const SegLaunch &L : b->seg_launches) {
            SegArgs s{};
            s.src = L.dim == 0 ? (const float2 *)in : (const float2 *)out;
            s.out = (float2 *)out;
            s.cubes = b->d_cubes;
            s.list = b->d_seg_list + L.list_off;
            s.tstart = b->d_seg_tstart + L.tstart_off;
            s.tcube = b->d_seg_tcube + L.tcube_off;
            s.ntiles = L.ntiles;
            s.dim = L.dim;
            s.tw = b->d_tw + L.tw_off;
            s.tw_len = (int)L.tw_len;
            s.conj = b->conj;
            void *params[1] = {&s};
            e = cudaLaunchKernel(L.func, L.grid, dim3(L.threads), params, L.smem, b->cap_stream);
            if (e != cudaSuccess)
                break;
        }
    } else if (b->slabz) {
        SlabZArgs z{};
        z.b = a;
        z.tw = b->d_tw + b->sa_tw_off;
        z.tw_len = b->sa_tw_len;
        for (int k = 0; k < 16; ++k) {
            z.tw_z[k] = b->sz_tw_z[k];
            z.tw_w[k] = b->sz_tw_w[k];
        }
        e = cudaMemsetAsync(b->d_counters, 0, b->counters_bytes, b->cap_stream);
        if (e == cudaSuccess) {
            void *params[1] = {&z};
            e = cudaLaunchKernel((const void *)&k_slabz, b->sz_grid, dim3(256), params, b->sz_smem, b->cap_stream);
        }
    } else {
        e = cudaMemsetAsync(b->d_counters, 0, b->counters_bytes, b->cap_stream);
        if (e == cudaSuccess) {
            void *params[1] = {&a};
            e = cudaLaunchKernel((const void *)&k_batched, b->grid, dim3(b->threads), params, b->smem,
                                 b->cap_stream);
        }
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g)
            cudaGraphDestroy(g);
        cudaGetLastError();
        return fail(FFT3_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    b->graph = g;
    CUDA_TRY(cudaGraphInstantiate(&b->exec, b->graph, 0));
    b->g_in = in;
    b->g_out = out;
    return FFT3_OK;
}

int batch_execute(fft3_plan p, const void *in, void *out, cudaStream_t st)
{
    BatchState *b = p->batch;
    if (!b->exec || b->g_in != in || b->g_out != out) {
        int rc = capture(p, in, out);
        if (rc)
            return rc;
    }
    CUDA_TRY(cudaGraphLaunch(b->exec, st));
    return FFT3_OK;
}

} // namespace fft3

using namespace fft3;

// Host planning of a batched plan (no device calls): problems, line plans and
// their twiddle exponents, work items of the executor, and the launches and
// tables of the segmented passes.  Errors return an FFT3_ERR_* code (message
// in fft3_last_error); the caller frees `b`.
static int batch_plan_host(BatchState *b, int count, const int *dims, const int64_t *offsets, int dtype,
                           int decomposition, int direction, const int *tuning)
{
    auto &segs = b->h_segs;
    auto &exps = b->h_exps;
    auto &exp_n = b->h_exp_n;
    auto &seg_list = b->h_seg_list;
    auto &seg_tcube = b->h_seg_tcube;
    auto &seg_tstart = b->h_seg_tstart;
    if (count < 1 || !dims || !offsets)
        return fail(FFT3_ERR_INVALID_ARG, "count must be positive and dims/offsets non-null");
    if (direction != FFT3_FORWARD && direction != FFT3_INVERSE)
        return fail(FFT3_ERR_INVALID_ARG, "direction must be FFT3_FORWARD or FFT3_INVERSE");
    if (dtype != FFT3_C64_FP32)
        return fail(FFT3_ERR_UNSUPPORTED_SIZE, "batched plans compute in FP32 only");
    if (decomposition != FFT3_AUTO && decomposition != FFT3_SLAB_PENCIL && decomposition != FFT3_PENCIL3)
        return fail(FFT3_ERR_INVALID_ARG, "batched plans support slab-pencil, pencil-pencil-pencil or auto");
    std::string err;
    std::map<std::pair<int, int>, int> lidx;
    b->conj = direction == FFT3_INVERSE ? 1 : 0;
    b->cubes.resize(count);
    b->tuning.resize(count);
    int64_t extent = 0;
    int bufmax = 1;
    // FFT3_TUNE_SLABZ on every code: the slab-by-slab executor
    int slabz = tuning ? 1 : 0;
    for (int i = 0; slabz && i < count; ++i)
        slabz = (tuning[i] & FFT3_TUNE_SLABZ) ? 1 : 0;
    // FFT3_AUTO without tuning codes takes it from kSegMinElems values on
    // when every length has its line variants and every slab fits the room of
    // an item (three blocks per SM); otherwise the segmented rule below
    if (!tuning && decomposition == FFT3_AUTO) {
#define FFT3_SZ_LEN(N, R, L) N,
        const int wl[] = {FFT3_SLABZ_WARP_PLANS(FFT3_SZ_LEN)};
#undef FFT3_SZ_LEN
        auto has = [&](int n, bool z) {
            bool f = false;
            if (z)
                for (const SlabZPlan &q : kSlabZPlans)
                    f = f || q.n == n;
            else
                for (int m : wl)
                    f = f || m == n;
            return f;
        };
        bool fit = true;
        int64_t values = 0;
        for (int i = 0; fit && i < count; ++i) {
            const int n0 = dims[3 * i], n1 = dims[3 * i + 1], n2 = dims[3 * i + 2];
            fit = has(n0, false) && has(n1, false) && has(n2, true) && n1 * (n0 | 1) <= kSlabzRoom;
            values += (int64_t)n0 * n1 * n2;
        }
        slabz = fit && values >= kSegMinElems ? 1 : 0;
    }
    b->slabz = slabz;
    for (int i = 0; i < count; ++i) {
        const int n0 = dims[3 * i], n1 = dims[3 * i + 1], n2 = dims[3 * i + 2];
        if (n0 < 1 || n1 < 1 || n2 < 1 || n0 > kBatchMaxLine || n1 > kBatchMaxLine || n2 > kBatchMaxLine ||
            !smooth_b(n0) || !smooth_b(n1) || !smooth_b(n2) || offsets[i] < 0) {
            return fail(FFT3_ERR_UNSUPPORTED_SIZE, "problem " + std::to_string(i) +
                                                       ": dimensions must be 2*3*5-smooth and at most " +
                                                       std::to_string(kBatchMaxLine) + ", offsets non-negative");
        }
        int code = tuning ? tuning[i] : 0;
        if (slabz)
            code = (code & ~3) | 1;
        if (decomposition == FFT3_SLAB_PENCIL && (code & 3) == 0)
            code |= 1;
        if (decomposition == FFT3_PENCIL3 && (code & 3) == 0)
            code |= 2;
        int decomp, order, lpt, lpty, spi;
        decode_tuning(code, n0, n1, n2, &decomp, &order, &lpt, &lpty, &spi);
        BatchCube &c = b->cubes[i];
        c.off = offsets[i];
        c.n0 = n0; c.n1 = n1; c.n2 = n2;
        c.decomp = decomp;
        c.lpt = lpt;
        c.lpty = lpty;
        int lx = line_index(b, lidx, n0, order, &err), ly = line_index(b, lidx, n1, order, &err),
            lz = line_index(b, lidx, n2, order, &err);
        if (lx < 0 || ly < 0 || lz < 0) {
            return fail(FFT3_ERR_UNSUPPORTED_SIZE, err);
        }
        c.lx = lx; c.ly = ly; c.lz = lz;
        if (slabz) {
            // z tiles of the FFT3_SLABZ_Z_PLANS plan of n2
            const SlabZPlan *zp = nullptr;
            for (const SlabZPlan &q : kSlabZPlans)
                zp = q.n == n2 ? &q : zp;
            if (!zp)
                return fail(FFT3_ERR_UNSUPPORTED_SIZE, "the slab executor has no compiled line kernel for length " +
                                                           std::to_string(n2));
            // items of about 8 Ki values: several small slabs stacked in the
            // buffer (at most the room of one 96 x 96 slab), several z tiles
            // (as many at a time as 256 threads hold groups of the line plan)
            const int zl = zp->lpt, zg = std::max(1, 256 / (zp->T * zp->lpt));
            decomp = BD_SLAB;
            c.decomp = BD_SLAB;
            c.lpt = lpt = zl;
            c.spi = std::max(1, std::min({n2, 8192 / (n0 * n1), kSlabzRoom / (n1 * (n0 | 1))}));
            c.zpi = std::max(zg, 8192 / (zl * n2) / zg * zg);
            c.nph = 2;
            c.items[0] = (n2 + c.spi - 1) / c.spi;
            c.items[1] = ((n0 * n1 + zl - 1) / zl + c.zpi - 1) / c.zpi;
            c.items[2] = 0;
            bufmax = std::max(bufmax, std::max(c.spi * n1 * (n0 | 1), zg * zl * n2));
        } else if (decomp == BD_SLAB) {
            c.spi = std::max(1, std::min(spi, n2));
            c.nph = 2;
            c.items[0] = (n2 + c.spi - 1) / c.spi;
            c.items[1] = (n0 * n1 + lpt - 1) / lpt;
            c.items[2] = 0;
            bufmax = std::max(bufmax, std::max(n1 * pitch_b(n0), lpt * pitch_b(n2)));
        } else {
            c.spi = std::max(1, std::min(spi, n1 * n2));
            c.nph = 3;
            c.items[0] = (n1 * n2 + c.spi - 1) / c.spi;
            c.items[1] = n2 * ((n0 + lpty - 1) / lpty);
            c.items[2] = (n0 * n1 + lpt - 1) / lpt;
            bufmax = std::max(bufmax, std::max(c.spi * pitch_b(n0), std::max(lpty * pitch_b(n1), lpt * pitch_b(n2))));
        }
        b->tuning[i] = (decomp == BD_SLAB ? 1 : 2) | ((order + 1) << 2) |
                       ((lpt == 4 ? 1 : lpt == 8 ? 2 : lpt == 16 ? 3 : 4) << 5);
        extent = std::max(extent, offsets[i] + (int64_t)n0 * n1 * n2);
    }
    b->extent = extent;
    if (slabz) {
        // rows and columns by the warp-shuffle variants (the z length was
        // checked against the z-tile plans above)
#define FFT3_SZ_LEN(N, R, L) N,
        const int wl[] = {FFT3_SLABZ_WARP_PLANS(FFT3_SZ_LEN)};
#undef FFT3_SZ_LEN
        for (int i = 0; i < count; ++i) {
            bool x = false, y = false;
            for (int n : wl) {
                x = x || n == dims[3 * i];
                y = y || n == dims[3 * i + 1];
            }
            if (!x || !y)
                return fail(FFT3_ERR_UNSUPPORTED_SIZE, "the slab executor has no compiled line kernel for a length "
                                                       "of problem " + std::to_string(i));
        }
    }
    // segmented mode: every line length compiled, and every tuning code asks
    // for it (decomposition field 3), or FFT3_AUTO without tuning codes (a
    // null array; an array of zeros keeps the executor) on a large enough batch
    int ccnt = 0, scnt = 0;
    const SegKernel *skc = seg_kernels(true, &ccnt), *sks = seg_kernels(false, &scnt);
    auto seg_find = [&](bool contiguous, int n) {
        const SegKernel *k = contiguous ? skc : sks;
        const int cnt = contiguous ? ccnt : scnt;
        for (int i = 0; i < cnt; ++i)
            if (k[i].n == n)
                return i;
        return -1;
    };
    auto seg_index = [&](int n) { return std::min(seg_find(true, n), seg_find(false, n)); };
    {
        bool ok = true, all3 = tuning != nullptr;
        int64_t values = 0;
        for (int i = 0; i < count; ++i) {
            for (int k = 0; k < 3; ++k)
                ok = ok && seg_index(dims[3 * i + k]) >= 0;
            if (tuning)
                all3 = all3 && (tuning[i] & 3) == 3;
            values += (int64_t)dims[3 * i] * dims[3 * i + 1] * dims[3 * i + 2];
        }
        if (all3 && !ok) {
            return fail(FFT3_ERR_UNSUPPORTED_SIZE, "the segmented passes have no compiled plan for a line length "
                                                   "of this batch");
        }
        b->seg = ok && !slabz && (all3 || (decomposition == FFT3_AUTO && !tuning && values >= kSegMinElems)) ? 1 : 0;
        // decomposition field 3 with the items field k >= 1 on every code: the
        // segmented passes in one cooperative launch, in 2^(k-1) waves
        int items = all3 ? (tuning[0] >> 8) & 15 : 0;
        for (int i = 0; all3 && i < count; ++i)
            items = ((tuning[i] >> 8) & 15) == items ? items : -1;
        if (b->seg && items > 0) {
            if (items > 11)
                return fail(FFT3_ERR_INVALID_ARG, "at most 1024 waves");
            b->seg1 = 1;
            b->waves = std::min(count, 1 << (items - 1));
        }
        if (b->seg)
            for (int i = 0; i < count; ++i)
                b->tuning[i] = 3 | (tuning ? tuning[i] & (7 << 2) : 0) | (b->seg1 ? items << 8 : 0);
    }
    b->buf_elems = (bufmax + 31) / 32 * 32;
    if (!slabz) {
        // the item executor's two buffers, and a third that stages the next
        // item's first tile when it still fits (the slab executor has one
        // stack, sized below)
        b->prefetch = 3 * b->buf_elems * (int)sizeof(float2) <= 200 * 1024 ? 1 : 0;
        b->smem = (2 + b->prefetch) * b->buf_elems * (int)sizeof(float2);
        if (b->smem > 227 * 1024) {
            return fail(FFT3_ERR_UNSUPPORTED_SIZE,
                        "a work item of this batch needs more shared memory than a block has");
        }
    }
    // line plans and their twiddle tables
    std::vector<int64_t> m;
    int64_t tw_total = 0;
    for (const LineChoice &lc : b->line_choice) {
        std::vector<int64_t> e;
        line_twiddle_exponents(lc, &e);
        if (e.empty())
            e.push_back(0);
        LineRt r{};
        r.n = lc.n;
        r.T = lc.T;
        r.nst = lc.nst;
        r.tw_off = (int)tw_total;
        for (int k = 0; k < kMaxStages; ++k)
            r.rad[k] = lc.rad[k];
        b->lines.push_back(r);
        segs.push_back({tw_total, (int64_t)e.size()});
        tw_total += ((int64_t)e.size() + 15) / 16 * 16;
        exps.push_back(std::move(e));
        exp_n.push_back(lc.n);
    }
    // segmented passes: per dimension and line length, the listed problems,
    // the first tile of each and the problem slot of every tile
    if (b->seg) {
        for (int d = 0; d < 3; ++d) {
            std::map<int, std::vector<int>> byn;
            for (int i = 0; i < count; ++i)
                byn[dims[3 * i + d]].push_back(i);
            for (auto &kv : byn) {
                // the radix_order field of the first problem's code picks among the
                // shared-memory kernel and the warp-shuffle kernels of this length
                // and direction (0 = the length's default, seg_line_candidates)
                const int ord = tuning ? (tuning[kv.second[0]] >> 2) & 7 : 0;
                int kidx = seg_find(d == 0, kv.first);
                const SegKernel *dk = nullptr;
                std::vector<const SegKernel *> cand = seg_line_candidates(kv.first, d == 0, &dk);
                const SegKernel &K = ord ? *cand[(size_t)(ord - 1) % cand.size()] : *dk;
                kidx = K.warp ? -1 : kidx;
                SegLaunch L{};
                L.dim = d;
                L.n = kv.first;
                L.kernel = kidx;
                L.func = K.func;
                L.warp = K.warp;
                L.R = K.warp ? K.rad[0] : 0;
                L.L = K.warp ? K.rad[1] : 0;
                L.lpt = K.lpt;
                L.threads = K.T * L.lpt;
                L.list_off = (int64_t)seg_list.size();
                L.tstart_off = (int64_t)seg_tstart.size();
                L.tcube_off = (int64_t)seg_tcube.size();
                int64_t tiles = 0;
                for (size_t s = 0; s < kv.second.size(); ++s) {
                    const int i = kv.second[s];
                    const int64_t n0 = dims[3 * i], n1 = dims[3 * i + 1], n2 = dims[3 * i + 2];
                    const int64_t lines = d == 0 ? n1 * n2 : d == 1 ? n0 * n2 : n0 * n1;
                    const int64_t nt = (lines + L.lpt - 1) / L.lpt;
                    seg_list.push_back(i);
                    seg_tstart.push_back(tiles);
                    seg_tcube.insert(seg_tcube.end(), (size_t)nt, (int)s);
                    tiles += nt;
                }
                seg_tstart.push_back(tiles);
                L.ntiles = tiles;
                LineChoice lc{};
                lc.n = K.n;
                lc.fixed = -1;
                lc.T = K.T;
                lc.nst = K.nrad;
                for (int r = 0; r < K.nrad; ++r)
                    lc.rad[r] = K.rad[r];
                std::vector<int64_t> e;
                if (K.warp) {
                    // the warp-shuffle kernels read w_n^m, m < n, and keep their lanes' twiddles in registers
                    for (int m = 0; m < K.n; ++m)
                        e.push_back(m);
                } else {
                    line_twiddle_exponents(lc, &e);
                }
                if (e.empty())
                    e.push_back(0);
                L.tw_off = tw_total;
                L.tw_len = ((int64_t)e.size() + 15) / 16 * 16;
                segs.push_back({tw_total, (int64_t)e.size()});
                tw_total += L.tw_len;
                exps.push_back(std::move(e));
                exp_n.push_back(K.n);
                L.smem = K.warp ? 0
                                : (int)(L.tw_len + (d == 0 ? L.lpt * pitch_b(K.n) : L.lpt * K.n)) * (int)sizeof(float2);
                b->seg_launches.push_back(L);
            }
        }
    }
    std::vector<int> kt(ccnt + scnt);
    if (b->seg1 || b->slabz) {
        // the line kernels' twiddle tables, one after the other (the
        // segmented kernels' copied to shared memory by every block of the
        // one-launch segmented executor; the slab executor's read through L1)
        b->sa_tw_off = tw_total;
        int64_t local = 0;
        for (int k = 0; k < (b->seg1 ? ccnt + scnt : 0); ++k) {
            const SegKernel &K = k < ccnt ? skc[k] : sks[k - ccnt];
            LineChoice lc{};
            lc.n = K.n;
            lc.fixed = -1;
            lc.T = K.T;
            lc.nst = K.nrad;
            for (int r = 0; r < K.nrad; ++r)
                lc.rad[r] = K.rad[r];
            std::vector<int64_t> e;
            line_twiddle_exponents(lc, &e);
            if (e.empty())
                e.push_back(0);
            kt[k] = (int)local;
            segs.push_back({tw_total + local, (int64_t)e.size()});
            local += ((int64_t)e.size() + 15) / 16 * 16;
            exps.push_back(std::move(e));
            exp_n.push_back(K.n);
        }
        if (b->slabz) {
            // the z-tile plans' stage twiddles
            for (int k = 0; k < (int)(sizeof(kSlabZPlans) / sizeof(kSlabZPlans[0])) && k < 16; ++k) {
                const SlabZPlan &q = kSlabZPlans[k];
                LineChoice lc{};
                lc.n = q.n;
                lc.fixed = -1;
                lc.T = q.T;
                lc.nst = q.nrad;
                for (int r = 0; r < q.nrad; ++r)
                    lc.rad[r] = q.rad[r];
                std::vector<int64_t> e;
                line_twiddle_exponents(lc, &e);
                if (e.empty())
                    e.push_back(0);
                b->sz_tw_z[k] = (int)local;
                segs.push_back({tw_total + local, (int64_t)e.size()});
                local += ((int64_t)e.size() + 15) / 16 * 16;
                exps.push_back(std::move(e));
                exp_n.push_back(q.n);
            }
            // w_N^m, m < N, for the warp-shuffle rows and columns
#define FFT3_SZ_LEN(N, R, L) N,
            const int wl[] = {FFT3_SLABZ_WARP_PLANS(FFT3_SZ_LEN)};
#undef FFT3_SZ_LEN
            for (int k = 0; k < (int)(sizeof(wl) / sizeof(wl[0])); ++k) {
                std::vector<int64_t> e(wl[k]);
                for (int m = 0; m < wl[k]; ++m)
                    e[m] = m;
                b->sz_tw_w[k] = (int)local;
                segs.push_back({tw_total + local, (int64_t)e.size()});
                local += ((int64_t)e.size() + 15) / 16 * 16;
                exps.push_back(std::move(e));
                exp_n.push_back(wl[k]);
            }
        }
        b->sa_tw_len = (int)local;
        tw_total += local;
        b->sz_smem = slabz_smem_bytes((bufmax + 31) / 32 * 32);
        if (b->sz_smem > 227 * 1024)
            return fail(FFT3_ERR_UNSUPPORTED_SIZE, "a slab of this batch needs more shared memory than a block has");
    }
    if (b->seg1) {
        // waves: consecutive problems of about equal volume
        std::vector<int> wave_of(count);
        {
            int64_t total = 0, acc = 0;
            for (int i = 0; i < count; ++i)
                total += (int64_t)dims[3 * i] * dims[3 * i + 1] * dims[3 * i + 2];
            for (int i = 0; i < count; ++i) {
                wave_of[i] = (int)std::min<int64_t>(b->waves - 1, acc * b->waves / std::max<int64_t>(1, total));
                acc += (int64_t)dims[3 * i] * dims[3 * i + 1] * dims[3 * i + 2];
            }
        }
        // steps: with one wave the x, y and z lines; with W waves, step k holds the
        // x lines of wave k, the y lines of wave k-1 and the z lines of wave k-2
        const int W = b->waves;
        const int nsteps = W == 1 ? 3 : W + 2;
        for (int st = 0; st < nsteps; ++st) {
            b->sa_seg0.push_back((int)b->sa_segs.size());
            int64_t tiles = 0;
            for (int d = 0; d < 3; ++d) {
                const int w = W == 1 ? (st == d ? 0 : -1) : st - d;
                if (w < 0 || w >= W)
                    continue;
                std::map<int, std::vector<int>> byn;
                for (int i = 0; i < count; ++i)
                    if (wave_of[i] == w)
                        byn[dims[3 * i + d]].push_back(i);
                for (auto &kv : byn) {
                    const int kidx = d == 0 ? seg_find(true, kv.first) : ccnt + seg_find(false, kv.first);
                    const int T = kidx < ccnt ? skc[kidx].T : sks[kidx - ccnt].T;
                    const int L = kSegAllThreads / T;
                    SegAllSeg sg{};
                    sg.tile0 = tiles;
                    sg.list_off = (int64_t)b->sa_list.size();
                    sg.tstart_off = (int64_t)b->sa_tstart.size();
                    sg.tcube_off = (int64_t)b->sa_tcube.size();
                    sg.kidx = kidx;
                    sg.dim = d;
                    sg.tw_off = kt[kidx];
                    int64_t t = 0;
                    for (size_t q = 0; q < kv.second.size(); ++q) {
                        const int i = kv.second[q];
                        const int64_t n0 = dims[3 * i], n1 = dims[3 * i + 1], n2 = dims[3 * i + 2];
                        const int64_t lines = d == 0 ? n1 * n2 : d == 1 ? n0 * n2 : n0 * n1;
                        const int64_t nt = (lines + L - 1) / L;
                        b->sa_list.push_back(i);
                        b->sa_tstart.push_back(t);
                        b->sa_tcube.insert(b->sa_tcube.end(), (size_t)nt, (int)q);
                        t += nt;
                    }
                    b->sa_tstart.push_back(t);
                    tiles += t;
                    b->sa_segs.push_back(sg);
                }
            }
            b->sa_ntiles.push_back(tiles);
        }
        b->sa_seg0.push_back((int)b->sa_segs.size());
        b->sa_smem = seg_all_smem_bytes(b->sa_tw_len);
    }
    b->tw_total = tw_total;
    // work items in waves over groups of problems (largest first)
    std::vector<int> order_idx(count);
    std::iota(order_idx.begin(), order_idx.end(), 0);
    std::stable_sort(order_idx.begin(), order_idx.end(), [&](int x, int y) {
        const BatchCube &a = b->cubes[x], &c = b->cubes[y];
        return (int64_t)a.n0 * a.n1 * a.n2 > (int64_t)c.n0 * c.n1 * c.n2;
    });
    std::vector<std::vector<int>> groups;
    int64_t acc = 0;
    const int64_t group_bytes = 16ll << 20;
    for (int i : order_idx) {
        const BatchCube &c = b->cubes[i];
        const int64_t bytes = (int64_t)c.n0 * c.n1 * c.n2 * 8;
        if (groups.empty() || acc + bytes > group_bytes) {
            groups.emplace_back();
            acc = 0;
        }
        groups.back().push_back(i);
        acc += bytes;
    }
    b->groups = (int)groups.size();
    const int G = (int)groups.size();
    for (int w = 0; w < G + 3; ++w)
        for (int p = 0; p < 3; ++p) {
            const int g = w - p;
            if (g < 0 || g >= G)
                continue;
            for (int ci : groups[g]) {
                const BatchCube &c = b->cubes[ci];
                if (p >= c.nph)
                    continue;
                for (int k = 0; k < c.items[p]; ++k)
                    b->items.push_back(BatchItem{ci, p, k, 0});
            }
        }
    if (b->items.size() >= (size_t)0x7fffffff) {
        return fail(FFT3_ERR_UNSUPPORTED_SIZE, "too many work items");
    }
    return FFT3_OK;
}

extern "C" int fft3_plan_create_many(fft3_plan *out, int count, const int *dims, const int64_t *offsets, int dtype,
                                     int decomposition, int direction, const int *tuning)
{
    if (!out)
        return fail(FFT3_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    auto *b = new (std::nothrow) BatchState();
    if (!b)
        return fail(FFT3_ERR_OOM, "host allocation failed");
    int rc = batch_plan_host(b, count, dims, offsets, dtype, decomposition, direction, tuning);
    if (rc) {
        batch_free(b);
        return rc;
    }
    const auto &segs = b->h_segs;
    const auto &exps = b->h_exps;
    const auto &exp_n = b->h_exp_n;
    const auto &seg_list = b->h_seg_list;
    const auto &seg_tcube = b->h_seg_tcube;
    const auto &seg_tstart = b->h_seg_tstart;
    const int64_t extent = b->extent, tw_total = b->tw_total;
    int ccnt = 0, scnt = 0;
    const SegKernel *skc = seg_kernels(true, &ccnt), *sks = seg_kernels(false, &scnt);
    // device state
    int dev = 0;
    rc = check_device(&dev);
    if (rc) {
        batch_free(b);
        return rc;
    }
    auto *P = new (std::nothrow) fft3_plan_s();
    if (!P) {
        batch_free(b);
        return fail(FFT3_ERR_OOM, "host allocation failed");
    }
    P->device = dev;
    P->elems = extent;
    P->batch = b;
    auto bail = [&](int code) {
        cudaGetLastError();
        fft3_plan_destroy(P);
        return code;
    };
    b->counters_bytes = (size_t)(1 + 3 * count) * sizeof(int);
    if (cudaMalloc(&b->d_cubes, b->cubes.size() * sizeof(BatchCube)) != cudaSuccess ||
        cudaMalloc(&b->d_items, b->items.size() * sizeof(BatchItem)) != cudaSuccess ||
        cudaMalloc(&b->d_lines, b->lines.size() * sizeof(LineRt)) != cudaSuccess ||
        cudaMalloc(&b->d_tw, std::max<int64_t>(16, tw_total) * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&b->d_counters, b->counters_bytes) != cudaSuccess ||
        cudaMalloc(&b->d_err, sizeof(unsigned)) != cudaSuccess)
        return bail(fail(FFT3_ERR_OOM, "device allocation for the batched plan failed"));
    if (cudaMemcpy(b->d_cubes, b->cubes.data(), b->cubes.size() * sizeof(BatchCube), cudaMemcpyHostToDevice) ||
        cudaMemcpy(b->d_items, b->items.data(), b->items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice) ||
        cudaMemcpy(b->d_lines, b->lines.data(), b->lines.size() * sizeof(LineRt), cudaMemcpyHostToDevice) ||
        cudaMemset(b->d_err, 0, sizeof(unsigned)) || cudaMemset(b->d_tw, 0, std::max<int64_t>(16, tw_total) * 8))
        return bail(fail(FFT3_ERR_CUDA, "uploading the batched plan failed"));
    P->d_err = b->d_err;
    {
        size_t maxm = 1;
        for (auto &e : exps)
            maxm = std::max(maxm, e.size());
        int64_t *d_m = nullptr;
        if (cudaMalloc(&d_m, maxm * sizeof(int64_t)) != cudaSuccess)
            return bail(fail(FFT3_ERR_OOM, "twiddle scratch allocation failed"));
        for (size_t i = 0; i < exps.size(); ++i) {
            cudaMemcpy(d_m, exps[i].data(), exps[i].size() * sizeof(int64_t), cudaMemcpyHostToDevice);
            int blocks = (int)std::max<int64_t>(1, ((int64_t)exps[i].size() + 255) / 256);
            k_roots<<<blocks, 256>>>(exp_n[i], FFT3_FORWARD, d_m, (int64_t)exps[i].size(), nullptr,
                                     b->d_tw + segs[i].first);
        }
        cudaError_t e = cudaDeviceSynchronize();
        cudaFree(d_m);
        if (e != cudaSuccess)
            return bail(fail(FFT3_ERR_CUDA, std::string("twiddle generation: ") + cudaGetErrorString(e)));
    }
    if (!b->slabz) {
        rc = prepare_func((const void *)&k_batched, b->smem);
        if (!rc)
            rc = occupancy_grid((const void *)&k_batched, b->threads, b->smem, 0, dev, &b->grid);
        if (rc)
            return bail(rc);
    }
    if (b->seg) {
        if (cudaMalloc(&b->d_seg_list, std::max<size_t>(1, seg_list.size()) * sizeof(int)) != cudaSuccess ||
            cudaMalloc(&b->d_seg_tcube, std::max<size_t>(1, seg_tcube.size()) * sizeof(int)) != cudaSuccess ||
            cudaMalloc(&b->d_seg_tstart, std::max<size_t>(1, seg_tstart.size()) * sizeof(int64_t)) != cudaSuccess)
            return bail(fail(FFT3_ERR_OOM, "device allocation for the segmented passes failed"));
        if (cudaMemcpy(b->d_seg_list, seg_list.data(), seg_list.size() * sizeof(int), cudaMemcpyHostToDevice) ||
            cudaMemcpy(b->d_seg_tcube, seg_tcube.data(), seg_tcube.size() * sizeof(int), cudaMemcpyHostToDevice) ||
            cudaMemcpy(b->d_seg_tstart, seg_tstart.data(), seg_tstart.size() * sizeof(int64_t),
                       cudaMemcpyHostToDevice))
            return bail(fail(FFT3_ERR_CUDA, "uploading the segmented pass tables failed"));
        for (SegLaunch &L : b->seg_launches) {
            const void *f = L.func;
            rc = prepare_func(f, L.smem);
            if (!rc)
                rc = occupancy_grid(f, L.threads, L.smem, L.ntiles, dev, &L.grid);
            if (rc)
                return bail(rc);
        }
    }
    if (b->seg1) {
        auto up = [&](auto **d, const auto &v) -> bool {
            using T = typename std::remove_reference<decltype(v)>::type::value_type;
            if (cudaMalloc((void **)d, std::max<size_t>(1, v.size()) * sizeof(T)) != cudaSuccess)
                return false;
            return v.empty() || cudaMemcpy(*d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) == cudaSuccess;
        };
        if (!up(&b->d_sa_segs, b->sa_segs) || !up(&b->d_sa_seg0, b->sa_seg0) || !up(&b->d_sa_list, b->sa_list) ||
            !up(&b->d_sa_tcube, b->sa_tcube) || !up(&b->d_sa_ntiles, b->sa_ntiles) ||
            !up(&b->d_sa_tstart, b->sa_tstart) || cudaMalloc(&b->d_sa_barrier, sizeof(int)) != cudaSuccess)
            return bail(fail(FFT3_ERR_OOM, "device tables of the one-launch executor"));
        rc = prepare_func((const void *)&k_seg_all, b->sa_smem);
        if (!rc)
            rc = occupancy_grid((const void *)&k_seg_all, kSegAllThreads, b->sa_smem, 0, dev, &b->sa_grid);
        if (rc)
            return bail(rc);
    }
    if (b->slabz) {
        if (b->sz_smem > 227 * 1024)
            return bail(fail(FFT3_ERR_UNSUPPORTED_SIZE, "a slab of this batch needs more shared memory than a block has"));
        rc = prepare_func((const void *)&k_slabz, b->sz_smem);
        if (!rc)
            rc = occupancy_grid((const void *)&k_slabz, 256, b->sz_smem, 0, dev, &b->sz_grid);
        if (rc)
            return bail(rc);
    }
    if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(FFT3_ERR_CUDA, "stream creation failed"));
    *out = P;
    return FFT3_OK;
}

extern "C" int fft3_plan_schedule_many(int count, const int *dims, const int64_t *offsets, int dtype,
                                       int decomposition, int direction, const int *tuning, char *buf, size_t len)
{
    auto *b = new (std::nothrow) BatchState();
    if (!b)
        return fail(FFT3_ERR_OOM, "host allocation failed");
    int rc = batch_plan_host(b, count, dims, offsets, dtype, decomposition, direction, tuning);
    std::string j;
    if (!rc)
        batch_describe(b, &j);
    batch_free(b);
    if (rc)
        return rc;
    if (buf && len > 0) {
        const size_t c = std::min(len - 1, j.size());
        memcpy(buf, j.data(), c);
        buf[c] = 0;
    }
    return (int)j.size();
}
