// capi.cu -- the C ABI of libfft3 (include/fft3.h): plan objects, twiddle
// generation at plan time, and the launch of each pass of a schedule.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "capi_internal.h"
#include "roots.cuh"

namespace fft3 {
__global__ void k_pass_g(PassArgs a);
__global__ void k_pass_g64(PassArgs a);
__global__ void k_slab(PassArgs a);
__global__ void k_vol(PassArgs a);
__global__ void k_probe_pass(PassArgs a);
__global__ void k_copy(const float2 *in, float2 *out, int64_t total);
__global__ void k_roots(int n, int sign, const int64_t *m, int64_t count, double *o64, float2 *o32);
__global__ void k_split_bf16(const float *x, int64_t count, uint16_t *hi, uint16_t *lo);
extern const FixedKernels g_fixed_kernels_a[];
extern const int g_fixed_kernels_a_count;
extern const FixedKernels g_fixed_kernels_b[];
extern const int g_fixed_kernels_b_count;

const FixedKernels *fixed_kernels(int id)
{
    for (int i = 0; i < g_fixed_kernels_a_count; ++i)
        if (g_fixed_kernels_a[i].id == id)
            return &g_fixed_kernels_a[i];
    for (int i = 0; i < g_fixed_kernels_b_count; ++i)
        if (g_fixed_kernels_b[i].id == id)
            return &g_fixed_kernels_b[i];
    return nullptr;
}
} // namespace fft3

using namespace fft3;

// ------------------------------------------------------------- errors ---- //
static thread_local std::string g_err;

int fft3::fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

int fft3::device_sms(int dev)
{
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
}

// Raise the dynamic shared-memory cap of a kernel to the device's opt-in
// maximum (the cap is per function, so it is never lowered by a later plan).
int fft3::prepare_func(const void *func, int smem, bool max_shared)
{
    if (smem > 0) {
        int dev = 0, optin = 0;
        CUDA_TRY(cudaGetDevice(&dev));
        CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        cudaFuncAttributes fa;
        CUDA_TRY(cudaFuncGetAttributes(&fa, func));
        const int cap = optin - (int)fa.sharedSizeBytes; // static shared memory counts against the opt-in
        if (smem > cap)
            return fail(FFT3_ERR_UNSUPPORTED_SIZE, "pass needs more shared memory than the device offers");
        if (smem + (int)fa.sharedSizeBytes > 48 * 1024)
            CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
        // the largest shared-memory carveout (least L1), on request
        if (max_shared)
            CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          cudaSharedmemCarveoutMaxShared));
    }
    return FFT3_OK;
}

// ------------------------------------------------------- tensor maps ----- //
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        else
            cudaGetLastError();
    }
    return fn;
}

// The array seen by a strided pass as the 4D tensor {C, n, A, B} of 8-byte
// elements; boxes of lpt columns x min(n, 256) line elements.
static int encode_pass_map(CUtensorMap *m, const void *base, const PassGeom &g, int n, int lpt, bool output)
{
    auto fn = encode_fn();
    if (!fn)
        return fail(FFT3_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    if ((uintptr_t)base & 15)
        return fail(FFT3_ERR_INVALID_ARG, "this plan moves tiles with TMA: buffers must be 16-byte aligned");
    const int64_t sj = output ? g.ok : g.ij, sa = output ? g.oa : g.ia, sb = output ? g.ob : g.ib;
    cuuint64_t dims[4] = {(cuuint64_t)g.C, (cuuint64_t)n, (cuuint64_t)g.A, (cuuint64_t)g.B};
    cuuint64_t strides[3] = {(cuuint64_t)sj * 8, (cuuint64_t)sa * 8,
                             (cuuint64_t)(g.B > 1 ? sb : sa * g.A) * 8};
    cuuint32_t box[4] = {(cuuint32_t)lpt, (cuuint32_t)(n < 256 ? n : 256), 1, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, const_cast<void *>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(FFT3_ERR_CUDA, "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
    return FFT3_OK;
}

// The blocked workspace of the fused slab stage as rows of 16 values; boxes of
// lpt columns x min(n, 256) rows.
static int encode_blocked_map(CUtensorMap *m, const void *base, int64_t elems, int n, int lpt)
{
    auto fn = encode_fn();
    if (!fn)
        return fail(FFT3_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    if ((uintptr_t)base & 15)
        return fail(FFT3_ERR_INVALID_ARG, "this plan moves tiles with TMA: buffers must be 16-byte aligned");
    cuuint64_t dims[2] = {16, (cuuint64_t)(elems / 16)};
    cuuint64_t strides[1] = {16 * 8};
    cuuint32_t box[2] = {(cuuint32_t)lpt, (cuuint32_t)(n < 256 ? n : 256)};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<void *>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(FFT3_ERR_CUDA, "cuTensorMapEncodeTiled (blocked workspace) failed with code " +
                                       std::to_string((int)r));
    return FFT3_OK;
}

// Input map of a streamed strided pass: the array as {C, Q, M, A, B} with
// line element j = Q*j' + q, so one box {LPT, QBOX, M, 1, 1} holds QBOX
// consecutive decimated sub-lines q of a tile.
static int encode_stream_map(CUtensorMap *m, const void *base, const PassGeom &g, int n, int q, int lpt,
                             int qbox = 1)
{
    auto fn = encode_fn();
    if (!fn)
        return fail(FFT3_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    if ((uintptr_t)base & 15)
        return fail(FFT3_ERR_INVALID_ARG, "this plan moves tiles with TMA: buffers must be 16-byte aligned");
    const int mm = n / q;
    cuuint64_t dims[5] = {(cuuint64_t)g.C, (cuuint64_t)q, (cuuint64_t)mm, (cuuint64_t)g.A, (cuuint64_t)g.B};
    cuuint64_t strides[4] = {(cuuint64_t)g.ij * 8, (cuuint64_t)g.ij * q * 8, (cuuint64_t)g.ia * 8,
                             (cuuint64_t)(g.B > 1 ? g.ib : g.ia * g.A) * 8};
    cuuint32_t box[5] = {(cuuint32_t)lpt, (cuuint32_t)qbox, (cuuint32_t)mm, 1, 1};
    cuuint32_t es[5] = {1, 1, 1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 5, const_cast<void *>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(FFT3_ERR_CUDA, "cuTensorMapEncodeTiled (streamed pass) failed with code " + std::to_string((int)r));
    return FFT3_OK;
}

int fft3::occupancy_grid(const void *func, int threads, int smem, int64_t ntiles, int dev, dim3 *grid)
{
    int nb = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, func, threads, smem));
    if (nb < 1)
        return fail(FFT3_ERR_UNSUPPORTED_SIZE, "kernel does not fit on an SM with this launch shape");
    int64_t g = (int64_t)nb * device_sms(dev);
    if (ntiles > 0)
        g = std::min<int64_t>(g, ntiles);
    grid->x = (unsigned)std::max<int64_t>(1, g);
    grid->y = grid->z = 1;
    return FFT3_OK;
}

static LineRt to_rt(const LineChoice &l, int tw_off)
{
    LineRt r{};
    r.n = l.n;
    r.T = l.T;
    r.nst = l.nst;
    r.tw_off = tw_off;
    for (int i = 0; i < kMaxStages; ++i)
        r.rad[i] = l.rad[i];
    return r;
}

static PassGeom natural_x(const Schedule &s)
{
    PassGeom g{};
    int64_t N = (int64_t)s.n0 * s.n1 * s.n2;
    g.C = s.n1; g.A = s.n2; g.B = s.batch;
    g.ij = 1; g.ic = s.n0; g.ia = (int64_t)s.n0 * s.n1; g.ib = N;
    g.ok = g.ij; g.oc = g.ic; g.oa = g.ia; g.ob = g.ib;
    return g;
}

static int build_launches(fft3_plan_s *P)
{
    const Schedule &s = P->sched;
    const int conj = s.direction == FFT3_INVERSE ? 1 : 0;
    for (const PassPlan &p : s.passes) {
        Launch L;
        L.kind = p.kind;
        L.src = p.src;
        L.dst = p.dst;
        PassArgs &a = L.args;
        a.g = p.g;
        a.conj = conj;
        a.ntiles = p.ntiles;
        a.tiles_c = p.tiles_c;
        a.lpt = p.lpt;
        a.err = P->d_err;
        // test hooks (options.reserved[0] = slab whose x tiles never signal, plus one;
        // options.reserved[1] = wait budget in thousands of cycles)
        a.nosignal_slab = s.opts.reserved[0] > 0 ? (int64_t)s.opts.reserved[0] - 1 : -1;
        a.wait_budget = s.opts.reserved[1] > 0 ? (long long)s.opts.reserved[1] * 1000LL : 4000000000LL;
        int64_t base = -1, end = 0;
        for (int k = 0; k < 3; ++k) {
            if (p.tw_seg[k] < 0)
                continue;
            const TwSeg &sg = s.tw[p.tw_seg[k]];
            if (base < 0)
                base = sg.off;
            end = sg.off + ((int64_t)sg.m.size() + 15) / 16 * 16;
        }
        if (base < 0)
            base = 0;
        a.tw = P->esize == 16 ? (const float2 *)((const double2 *)P->d_tw + base) : P->d_tw + base;
        a.tw_len = (int)(end - base);
        if (p.tw_seg[0] >= 0)
            a.L[0] = to_rt(p.line, (int)(s.tw[p.tw_seg[0]].off - base));
        if (p.tw_seg[1] >= 0)
            a.L[1] = to_rt(p.line2, (int)(s.tw[p.tw_seg[1]].off - base));
        if (p.tw_seg[2] >= 0)
            a.tw_split_off = (int)(s.tw[p.tw_seg[2]].off - base);
        a.p = p.p;
        a.six_step = p.six_step ? 1 : 0;
        a.split_a = p.split_a;
        a.split_b = p.split_b;
        L.probe_g = p.g;
        L.probe_n = p.line.n;
        L.smem = p.smem_bytes;
        L.chunk = p.chunk;
        L.pair_next = p.pair_next;
        L.block = dim3(std::max(1, p.threads));
        const FixedKernels *fk = p.line.fixed >= 0 ? fixed_kernels(p.line.fixed) : nullptr;
        switch (p.kind) {
        case PK_J: L.func = fk ? fk->j : nullptr; break;
        case PK_JROT: L.func = fk ? fk->jrot : nullptr; break;
        case PK_C: L.func = fk ? (p.lpt == 16 ? fk->c16 : fk->c8) : nullptr; break;
        case PK_CTMA:
            L.func = fk ? fk->ctma : nullptr;
            L.tma = true;
            break;
        case PK_G: L.func = (const void *)&k_pass_g; break;
        case PK_G64: L.func = (const void *)&k_pass_g64; break;
        case PK_J64:
        case PK_C64: {
            const Fixed64Kernels *k64 = p.line.fixed >= 0 ? fixed64_kernels(p.line.fixed) : nullptr;
            L.func = k64 ? (p.kind == PK_J64 ? k64->j : k64->c) : nullptr;
            break;
        }
        case PK_SLAB:
            L.func = (const void *)&k_slab;
            L.probe_g = natural_x(s);
            L.probe_n = s.n0;
            break;
        case PK_SLABL2:
            L.func = fk ? fk->l2 : nullptr;
            L.reset_counters = true;
            L.probe_g = natural_x(s);
            L.probe_n = s.n0;
            break;
        case PK_SLABBLK:
            L.func = fk ? fk->l2blk[p.lpt == 8 ? 1 : 0] : nullptr;
            L.reset_counters = true;
            L.slab_map = true;
            L.probe_g = natural_x(s);
            L.probe_n = s.n0;
            break;
        case PK_VOL:
            L.func = (const void *)&k_vol;
            L.cluster = p.p;
            L.probe_n = p.split_a * p.split_b;
            break;
        case PK_VOLC: {
            int cnt = 0;
            const VolcKernel *vk = volc_kernels(&cnt);
            L.func = (p.volc >= 0 && p.volc < cnt) ? vk[p.volc].func : nullptr;
            L.cluster = p.p;
            L.probe_n = p.split_a * p.split_b;
            break;
        }
        case PK_CSTREAM: {
            int cnt = 0;
            const CStreamKernel *ck = cstream_kernels(&cnt);
            L.func = (p.cstream >= 0 && p.cstream < cnt)
                         ? (p.tc_mode < 0 ? ck[p.cstream].func : ck[p.cstream].func_tc[p.tc_mode == 0 ? 0 : 1])
                         : nullptr;
            L.stream_q = L.func ? ck[p.cstream].q : 0;
            L.cluster = p.p;
            break;
        }
        case PK_TCX:
        case PK_TCS:
            L.func = tc32_kernel(p.kind == PK_TCX ? 0 : 1);
            L.tc32 = p.kind == PK_TCS ? 2 : 1;
            break;
        case PK_JTC:
            L.func = fk && p.tc_mode >= 0 ? fk->j_tc[p.tc_mode] : nullptr;
            break;
        case PK_CTC:
            L.func = fk && p.tc_mode >= 0 ? fk->c_tc[p.tc_mode] : nullptr;
            break;
        case PK_COPY:
            L.func = (const void *)&k_copy;
            L.probe_n = 1;
            break;
        default: break;
        }
        if (!L.func)
            return fail(FFT3_ERR_UNSUPPORTED_SIZE, "no compiled kernel for this pass");
        int rc = prepare_func(L.func, L.smem, L.tc32 != 0);
        if (rc)
            return rc;
        if (p.kind == PK_VOL || p.kind == PK_VOLC || (p.kind == PK_CSTREAM && p.p > 1)) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = p.p;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(p.p * 4);
            cfg.blockDim = L.block;
            cfg.dynamicSmemBytes = L.smem;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int ncl = 0;
            CUDA_TRY(cudaOccupancyMaxActiveClusters(&ncl, L.func, &cfg));
            if (ncl < 1)
                return fail(FFT3_ERR_UNSUPPORTED_SIZE, "volumetric cluster does not fit on the GPU");
            int64_t g = std::min<int64_t>(ncl, p.ntiles);
            L.grid = dim3((unsigned)(std::max<int64_t>(1, g) * p.p));
        } else if (p.kind == PK_COPY) {
            L.grid = dim3((unsigned)std::min<int64_t>(4096, (P->elems * (P->esize / 8) + 255) / 256 + 1));
            L.block = dim3(256);
        } else if (p.kind == PK_SLABL2 || p.kind == PK_SLABBLK) {
            rc = occupancy_grid(L.func, L.block.x, L.smem, 0, P->device, &L.grid);
            if (rc)
                return rc;
            P->counters_bytes = std::max(P->counters_bytes,
                                         (size_t)(1 + p.g.A * p.g.B) * sizeof(int));
        } else if (L.tc32) {
            // one block per SM (contiguous lines: each running kTc32Groups streams of tiles)
            rc = occupancy_grid(L.func, L.block.x, L.smem,
                                p.kind == PK_TCX ? (p.ntiles + kTc32Groups - 1) / kTc32Groups : p.ntiles,
                                P->device, &L.grid);
            if (rc)
                return rc;
        } else {
            rc = occupancy_grid(L.func, L.block.x, L.smem, p.ntiles, P->device, &L.grid);
            if (rc)
                return rc;
        }
        P->launches.push_back(L);
    }
    bool pair = false;
    for (size_t i = 0; i + 1 < P->launches.size(); ++i)
        pair = pair || (P->launches[i].pair_next && P->launches[i].chunk > 0);
    if (pair) {
        CUDA_TRY(cudaStreamCreateWithFlags(&P->side, cudaStreamNonBlocking));
        CUDA_TRY(cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming));
        CUDA_TRY(cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming));
    }
    return FFT3_OK;
}

static void free_plan(fft3_plan_s *P)
{
    if (!P)
        return;
    cudaFree(P->d_tw);
    cudaFree(P->d_ws);
    cudaFree(P->d_counters);
    if (!P->batch) // a batched plan's error word belongs to its batch state
        cudaFree(P->d_err);
    cudaFree(P->d_stage_in);
    cudaFree(P->d_stage_out);
    cudaFree(P->d_stage_in2);
    cudaFree(P->d_stage_out2);
    for (int i = 0; i < 3; ++i)
        if (P->pipe_st[i])
            cudaStreamDestroy(P->pipe_st[i]);
    for (int b = 0; b < 2; ++b)
        for (int e = 0; e < 3; ++e)
            if (P->pipe_ev[b][e])
                cudaEventDestroy(P->pipe_ev[b][e]);
    if (P->side)
        cudaStreamDestroy(P->side);
    if (P->ev_fork)
        cudaEventDestroy(P->ev_fork);
    if (P->ev_join)
        cudaEventDestroy(P->ev_join);
    batch_free(P->batch);
    delete P;
}

static int generate_twiddles(fft3_plan_s *P)
{
    const Schedule &s = P->sched;
    int64_t total = std::max<int64_t>(16, s.tw_total);
    const bool fp64 = P->esize == 16; // complex128: the FP64 values are the table
    CUDA_TRY(cudaMalloc(&P->d_tw, total * P->esize));
    CUDA_TRY(cudaMemset(P->d_tw, 0, total * P->esize));
    size_t maxm = 1;
    for (const TwSeg &sg : s.tw)
        maxm = std::max(maxm, sg.m.size());
    int64_t *d_m = nullptr;
    CUDA_TRY(cudaMalloc(&d_m, maxm * sizeof(int64_t)));
    for (const TwSeg &sg : s.tw) {
        cudaError_t e = cudaMemcpy(d_m, sg.m.data(), sg.m.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            int blocks = (int)std::min<int64_t>(1024, ((int64_t)sg.m.size() + 255) / 256);
            k_roots<<<std::max(1, blocks), 256>>>(sg.n, FFT3_FORWARD, d_m, (int64_t)sg.m.size(),
                                                  fp64 ? (double *)P->d_tw + 2 * sg.off : nullptr,
                                                  fp64 ? nullptr : P->d_tw + sg.off);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) {
            cudaFree(d_m);
            return fail(FFT3_ERR_CUDA, std::string("twiddle generation: ") + cudaGetErrorString(e));
        }
    }
    cudaError_t e = cudaDeviceSynchronize();
    cudaFree(d_m);
    if (e != cudaSuccess)
        return fail(FFT3_ERR_CUDA, std::string("twiddle generation: ") + cudaGetErrorString(e));
    return FFT3_OK;
}

int fft3::check_device(int *dev)
{
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || count == 0) {
        cudaGetLastError();
        return fail(FFT3_ERR_NO_DEVICE, "no CUDA device visible");
    }
    CUDA_TRY(cudaGetDevice(dev));
    return FFT3_OK;
}

extern "C" {

const char *fft3_last_error(void) { return g_err.c_str(); }

int fft3_version(void) { return 1; }

int fft3_factorize(int n, int order, int *radices, int cap)
{
    if (!radices || cap < 1 || n < 1 || order < 0)
        return fail(FFT3_ERR_INVALID_ARG, "bad argument to fft3_factorize");
    int r = factorize(n, order, radices, cap);
    if (r < 0)
        return fail(r, "length has a prime factor other than 2, 3, 5 or too many stages");
    return r;
}

int fft3_layout_positions(int layout, int n0, int n1, int n2, int batch, const int64_t *idx, int64_t *pos,
                          int64_t count)
{
    if (!idx || !pos || count < 0 || n0 < 1 || n1 < 1 || n2 < 1 || batch < 1)
        return fail(FFT3_ERR_INVALID_ARG, "bad argument to fft3_layout_positions");
    if (layout < FFT3_LAYOUT_NATURAL || layout > FFT3_LAYOUT_PENCILS)
        return fail(FFT3_ERR_INVALID_ARG, "unknown layout");
    for (int64_t i = 0; i < count; ++i) {
        int rc = layout_position(layout, n0, n1, n2, batch, idx[i], &pos[i]);
        if (rc == FFT3_ERR_UNSUPPORTED_SIZE)
            return fail(rc, "the pencils layout needs batch 1 and n0 % 16 == 0");
        if (rc)
            return fail(rc, "index " + std::to_string(idx[i]) + " outside the array");
    }
    return FFT3_OK;
}

int fft3_plan_schedule(int n0, int n1, int n2, int batch, int dtype, int decomposition, int direction,
                       const fft3_options *opts, char *buf, size_t len)
{
    Schedule s;
    std::string err;
    int rc = build_schedule(n0, n1, n2, batch, dtype, decomposition, direction, opts, &s, &err);
    if (rc)
        return fail(rc, err);
    std::string j = s.json();
    if (buf && len > 0) {
        size_t c = std::min(len - 1, j.size());
        memcpy(buf, j.data(), c);
        buf[c] = 0;
    }
    return (int)j.size();
}

int fft3_plan_create_ex(fft3_plan *out, int n0, int n1, int n2, int batch, int dtype,
                        int decomposition, int direction, const fft3_options *opts)
{
    if (!out)
        return fail(FFT3_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    auto *P = new (std::nothrow) fft3_plan_s();
    if (!P)
        return fail(FFT3_ERR_OOM, "host allocation failed");
    std::string err;
    int rc = build_schedule(n0, n1, n2, batch, dtype, decomposition, direction, opts, &P->sched, &err);
    if (rc) {
        delete P;
        return fail(rc, err);
    }
    rc = check_device(&P->device);
    if (rc) {
        delete P;
        return rc;
    }
    P->elems = (int64_t)n0 * n1 * n2 * batch;
    P->esize = dtype == FFT3_C128_FP64 ? 16 : 8;
    cudaError_t e = cudaMalloc(&P->d_err, sizeof(unsigned));
    if (e == cudaSuccess)
        e = cudaMemset(P->d_err, 0, sizeof(unsigned));
    if (e != cudaSuccess) {
        free_plan(P);
        return fail(FFT3_ERR_CUDA, std::string("plan allocation: ") + cudaGetErrorString(e));
    }
    rc = generate_twiddles(P);
    if (!rc)
        rc = build_launches(P);
    if (!rc && P->sched.need_ws) {
        P->ws_bytes = (size_t)P->elems * P->esize;
        e = cudaMalloc(&P->d_ws, P->ws_bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = fail(FFT3_ERR_OOM, "workspace allocation failed");
        }
    }
    if (!rc && P->counters_bytes) {
        e = cudaMalloc(&P->d_counters, P->counters_bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = fail(FFT3_ERR_OOM, "counter allocation failed");
        }
        for (Launch &L : P->launches)
            L.args.counters = P->d_counters;
    }
    if (rc) {
        free_plan(P);
        return rc;
    }
    *out = P;
    return FFT3_OK;
}

int fft3_plan_create(fft3_plan *out, int n0, int n1, int n2, int batch, int dtype, int decomposition,
                     int direction)
{
    return fft3_plan_create_ex(out, n0, n1, n2, batch, dtype, decomposition, direction, nullptr);
}

static int launch_one(fft3_plan_s *P, const Launch &L, const void *func, PassArgs a, cudaStream_t st)
{
    if (L.reset_counters)
        CUDA_TRY(cudaMemsetAsync(P->d_counters, 0, P->counters_bytes, st));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = L.grid;
    cfg.blockDim = L.block;
    cfg.dynamicSmemBytes = L.smem;
    cfg.stream = st;
    if (L.cluster > 1) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = L.cluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    if (L.stream_q > 0) {
        CUtensorMap tin;
        int rc = encode_stream_map(&tin, a.in, a.g, L.probe_n, L.stream_q, a.lpt);
        if (rc)
            return rc;
        void *params[2] = {&a, &tin};
        CUDA_TRY(cudaLaunchKernelExC(&cfg, func, params));
        return FFT3_OK;
    }
    if (L.tc32) {
        if ((uintptr_t)a.in & 15)
            return fail(FFT3_ERR_INVALID_ARG, "this plan moves tiles with TMA: buffers must be 16-byte aligned");
        CUtensorMap tin;
        void *params[2] = {&a, &tin};
        if (L.tc32 == 2) { // 16 columns x 8 decimated sub-sequences x 32 values per box
            int rc = encode_stream_map(&tin, a.in, a.g, L.probe_n, 32, kTcsLpt, 8);
            if (rc)
                return rc;
        }
        CUDA_TRY(cudaLaunchKernelExC(&cfg, func, params)); // the contiguous-line kernel takes only `a`
        return FFT3_OK;
    }
    if (L.slab_map) {
        if ((uintptr_t)a.in & 15)
            return fail(FFT3_ERR_INVALID_ARG, "this plan moves tiles with TMA: buffers must be 16-byte aligned");
        CUtensorMap tws;
        int rc = encode_blocked_map(&tws, a.out, P->elems, L.probe_n, a.lpt);
        if (rc)
            return rc;
        void *params[2] = {&a, &tws};
        CUDA_TRY(cudaLaunchKernelExC(&cfg, func, params));
        return FFT3_OK;
    }
    if (L.tma) {
        CUtensorMap tin, tout;
        int rc = encode_pass_map(&tin, a.in, a.g, L.probe_n, a.lpt, false);
        if (!rc)
            rc = encode_pass_map(&tout, a.out, a.g, L.probe_n, a.lpt, true);
        if (rc)
            return rc;
        void *params[3] = {&a, &tin, &tout};
        CUDA_TRY(cudaLaunchKernelExC(&cfg, func, params));
        return FFT3_OK;
    }
    void *params[1] = {&a};
    CUDA_TRY(cudaLaunchKernelExC(&cfg, func, params));
    return FFT3_OK;
}

static float2 *buf_ptr(fft3_plan_s *P, int id, const void *in, void *out)
{
    return id == BUF_IN ? (float2 *)in : (id == BUF_OUT ? (float2 *)out : P->d_ws);
}

static bool pair_head(const fft3_plan_s *P, size_t k)
{
    return k + 1 < P->launches.size() && P->launches[k].pair_next && P->launches[k].chunk > 0;
}

// Two passes over the same slabs, pipelined in chunks of `chunk` values of a:
// chunk c of the first pass runs on the caller's stream, chunk c of the second
// on the plan's side stream once the first has finished it, so the second
// pass reads a chunk the first has just written (still in L2) while the first
// moves on to chunk c+1.  The side stream joins the caller's stream at the end.
static int run_pair(fft3_plan_s *P, size_t k, const void *in, void *out, cudaStream_t st)
{
    const Launch &X = P->launches[k], &Y = P->launches[k + 1];
    const int64_t na_total = X.args.g.A, K = X.chunk;
    for (int64_t a0 = 0; a0 < na_total; a0 += K) {
        const int64_t na = std::min(K, na_total - a0);
        for (int w = 0; w < 2; ++w) {
            const Launch &L = w ? Y : X;
            PassArgs a = L.args;
            a.in = buf_ptr(P, L.src, in, out) + a0 * a.g.ia;
            a.out = buf_ptr(P, L.dst, in, out) + a0 * a.g.oa;
            a.g.A = na;
            a.ntiles = a.tiles_c * na * a.g.B;
            int rc = launch_one(P, L, L.func, a, w ? P->side : st);
            if (rc)
                return rc;
            if (!w) {
                CUDA_TRY(cudaEventRecord(P->ev_fork, st));
                CUDA_TRY(cudaStreamWaitEvent(P->side, P->ev_fork, 0));
            }
        }
    }
    CUDA_TRY(cudaEventRecord(P->ev_join, P->side));
    CUDA_TRY(cudaStreamWaitEvent(st, P->ev_join, 0));
    return FFT3_OK;
}

int fft3_plan_execute(fft3_plan p, const void *in, void *out, void *stream)
{
    if (!p || !in || !out)
        return fail(FFT3_ERR_INVALID_ARG, "null plan or buffer");
    if (in == out)
        return fail(FFT3_ERR_INPLACE_UNSUPPORTED, "in-place execution is not supported (in == out)");
    if (((uintptr_t)in | (uintptr_t)out) & 7)
        return fail(FFT3_ERR_INVALID_ARG, "buffers must be 8-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    p->last_stream = st;
    if (p->batch)
        return batch_execute(p, in, out, st);
    for (size_t k = 0; k < p->launches.size(); ++k) {
        const Launch &L = p->launches[k];
        if (pair_head(p, k)) {
            int rc = run_pair(p, k, in, out, st);
            if (rc)
                return rc;
            ++k;
            continue;
        }
        PassArgs a = L.args;
        a.in = buf_ptr(p, L.src, in, out);
        a.out = buf_ptr(p, L.dst, in, out);
        if (L.kind == PK_COPY) {
            k_copy<<<L.grid, L.block, 0, st>>>(a.in, a.out, p->elems * (p->esize / 8));
            CUDA_TRY(cudaGetLastError());
            continue;
        }
        int rc = launch_one(p, L, L.func, a, st);
        if (rc)
            return rc;
    }
    return FFT3_OK;
}

int fft3_plan_probe_layout(fft3_plan p, const void *in, void *out, int npasses, void *stream)
{
    if (!p || !in || !out || in == out)
        return fail(FFT3_ERR_INVALID_ARG, "null plan or buffer, or in == out");
    if (p->esize != 8)
        return fail(FFT3_ERR_INVALID_ARG, "the layout probe moves complex64 elements");
    cudaStream_t st = (cudaStream_t)stream;
    int count = (int)p->launches.size();
    if (npasses >= 0 && npasses < count)
        count = npasses;
    int last_dst = BUF_IN;
    for (int i = 0; i < count; ++i) {
        const Launch &L = p->launches[i];
        PassArgs a = L.args;
        a.in = buf_ptr(p, L.src, in, out);
        a.out = buf_ptr(p, L.dst, in, out);
        last_dst = L.dst;
        if (L.kind == PK_COPY || a.in == a.out) {
            if (a.in != a.out) {
                k_copy<<<L.grid, L.block, 0, st>>>(a.in, a.out, p->elems * (p->esize / 8));
                CUDA_TRY(cudaGetLastError());
            }
            continue; // an in-place pass moves nothing
        }
        a.g = L.probe_g;
        a.L[0].n = L.probe_n;
        int64_t total = (int64_t)L.probe_n * a.g.C * a.g.A * a.g.B;
        int blocks = (int)std::min<int64_t>(8192, (total + 255) / 256);
        k_probe_pass<<<std::max(1, blocks), 256, 0, st>>>(a);
        CUDA_TRY(cudaGetLastError());
    }
    if (last_dst == BUF_WS) {
        k_copy<<<4096, 256, 0, st>>>(p->d_ws, (float2 *)out, p->elems);
        CUDA_TRY(cudaGetLastError());
    } else if (last_dst == BUF_IN) {
        k_copy<<<4096, 256, 0, st>>>((const float2 *)in, (float2 *)out, p->elems);
        CUDA_TRY(cudaGetLastError());
    }
    return FFT3_OK;
}

int fft3_plan_execute_pass(fft3_plan p, int k, const void *in, void *out, void *stream)
{
    if (!p || !in || !out)
        return fail(FFT3_ERR_INVALID_ARG, "null plan or buffer");
    if (in == out)
        return fail(FFT3_ERR_INPLACE_UNSUPPORTED, "in-place execution is not supported (in == out)");
    if (k < 0 || k >= (int)p->launches.size())
        return fail(FFT3_ERR_INVALID_ARG, "pass index out of range");
    cudaStream_t st = (cudaStream_t)stream;
    p->last_stream = st;
    if (pair_head(p, (size_t)k))
        return run_pair(p, (size_t)k, in, out, st);
    if (k > 0 && pair_head(p, (size_t)k - 1))
        return FFT3_OK; // ran with the pass before it
    const Launch &L = p->launches[k];
    PassArgs a = L.args;
    a.in = buf_ptr(p, L.src, in, out);
    a.out = buf_ptr(p, L.dst, in, out);
    if (L.kind == PK_COPY) {
        k_copy<<<L.grid, L.block, 0, st>>>(a.in, a.out, p->elems * (p->esize / 8));
        CUDA_TRY(cudaGetLastError());
        return FFT3_OK;
    }
    return launch_one(p, L, L.func, a, st);
}

// The address kernels use for host memory the device can reach (pinned or
// registered with CUDA), or null for other memory.
static void *host_device_ptr(const void *h)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, h) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// Whether the schedule can read its input from host memory in its first pass:
// the input is read only by the first pass, with plain loads (not by TMA), the
// result ends in the output array, and there is no two-stream pair.
static bool host_direct_ok(const fft3_plan_s *p)
{
    const size_t n = p->launches.size();
    if (p->batch || n == 0 || p->launches[n - 1].dst != BUF_OUT)
        return false;
    for (size_t k = 0; k < n; ++k) {
        const Launch &L = p->launches[k];
        if (pair_head(p, k) || L.dst == BUF_IN || (L.src == BUF_IN && k != 0))
            return false;
        if (L.src == BUF_IN && (L.stream_q > 0 || L.tc32 || L.slab_map || L.tma))
            return false;
    }
    return true;
}

// The schedule with the first pass reading the host input `hin` and the
// output array in device memory (`mid`, the workspace `ws`).  No kernel
// stores to host memory: with the last pass of one transform storing to host
// memory while the first pass of another read host memory on a second
// stream, one of five transforms came out wrong in a reproducible way (the
// same sequence with the result moved by a copy was right every time), so
// results leave the device by copies.
static int execute_host_direct(fft3_plan_s *p, const void *hin, float2 *mid, float2 *ws, cudaStream_t st)
{
    const size_t n = p->launches.size();
    for (size_t k = 0; k < n; ++k) {
        const Launch &L = p->launches[k];
        PassArgs a = L.args;
        a.in = L.src == BUF_IN ? (const float2 *)hin : L.src == BUF_OUT ? mid : ws;
        a.out = L.dst == BUF_OUT ? mid : ws;
        if (L.kind == PK_COPY) {
            k_copy<<<L.grid, L.block, 0, st>>>(a.in, a.out, p->elems * (p->esize / 8));
            CUDA_TRY(cudaGetLastError());
            continue;
        }
        int rc = launch_one(p, L, L.func, a, st);
        if (rc)
            return rc;
    }
    return FFT3_OK;
}

int fft3_plan_execute_host(fft3_plan p, const void *h_in, void *h_out, void *stream)
{
    if (!p || !h_in || !h_out)
        return fail(FFT3_ERR_INVALID_ARG, "null plan or buffer");
    size_t bytes = (size_t)p->elems * p->esize;
    void *hin = host_device_ptr(h_in);
    if (hin && host_direct_ok(p)) {
        if (!p->d_stage_out)
            CUDA_TRY(cudaMalloc(&p->d_stage_out, bytes));
        cudaStream_t st = (cudaStream_t)stream;
        p->last_stream = st;
        int rc = execute_host_direct(p, hin, p->d_stage_out, p->d_ws, st);
        if (rc)
            return rc;
        CUDA_TRY(cudaMemcpyAsync(h_out, p->d_stage_out, bytes, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        return FFT3_OK;
    }
    if (!p->d_stage_in)
        CUDA_TRY(cudaMalloc(&p->d_stage_in, bytes));
    if (!p->d_stage_out)
        CUDA_TRY(cudaMalloc(&p->d_stage_out, bytes));
    cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(cudaMemcpyAsync(p->d_stage_in, h_in, bytes, cudaMemcpyHostToDevice, st));
    int rc = fft3_plan_execute(p, p->d_stage_in, p->d_stage_out, stream);
    if (rc)
        return rc;
    CUDA_TRY(cudaMemcpyAsync(h_out, p->d_stage_out, bytes, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return FFT3_OK;
}

int fft3_plan_execute_host_pipelined(fft3_plan p, const void *const *h_in, void *const *h_out, int count,
                                     void *stream)
{
    if (!p || !h_in || !h_out || count < 0)
        return fail(FFT3_ERR_INVALID_ARG, "null plan or pointer arrays, or negative count");
    for (int i = 0; i < count; ++i)
        if (!h_in[i] || !h_out[i])
            return fail(FFT3_ERR_INVALID_ARG, "null host buffer in the pointer arrays");
    if (count == 0)
        return FFT3_OK;
    const size_t bytes = (size_t)p->elems * p->esize;
    if (!p->d_stage_in)
        CUDA_TRY(cudaMalloc(&p->d_stage_in, bytes));
    if (!p->d_stage_out)
        CUDA_TRY(cudaMalloc(&p->d_stage_out, bytes));
    if (!p->d_stage_in2)
        CUDA_TRY(cudaMalloc(&p->d_stage_in2, bytes));
    if (!p->d_stage_out2)
        CUDA_TRY(cudaMalloc(&p->d_stage_out2, bytes));
    for (int i = 0; i < 3; ++i)
        if (!p->pipe_st[i])
            CUDA_TRY(cudaStreamCreateWithFlags(&p->pipe_st[i], cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b)
        for (int e = 0; e < 3; ++e)
            if (!p->pipe_ev[b][e])
                CUDA_TRY(cudaEventCreateWithFlags(&p->pipe_ev[b][e], cudaEventDisableTiming));
    cudaStream_t user = (cudaStream_t)stream;
    cudaStream_t h2d = p->pipe_st[0], comp = p->pipe_st[1], d2h = p->pipe_st[2];
    float2 *din[2] = {p->d_stage_in, p->d_stage_in2}, *dout[2] = {p->d_stage_out, p->d_stage_out2};
    // everything the caller queued on `stream` comes first
    CUDA_TRY(cudaEventRecord(p->pipe_ev[0][0], user));
    for (int i = 0; i < 3; ++i)
        CUDA_TRY(cudaStreamWaitEvent(p->pipe_st[i], p->pipe_ev[0][0], 0));
    for (int i = 0; i < count; ++i) {
        const int b = i & 1;
        cudaEvent_t *ev = p->pipe_ev[b];
        if (i >= 2) // the transform of i-2 has read din[b]
            CUDA_TRY(cudaStreamWaitEvent(h2d, ev[1], 0));
        CUDA_TRY(cudaMemcpyAsync(din[b], h_in[i], bytes, cudaMemcpyHostToDevice, h2d));
        CUDA_TRY(cudaEventRecord(ev[0], h2d));
        CUDA_TRY(cudaStreamWaitEvent(comp, ev[0], 0));
        if (i >= 2) // the copy-out of i-2 has drained dout[b]
            CUDA_TRY(cudaStreamWaitEvent(comp, ev[2], 0));
        int rc = fft3_plan_execute(p, din[b], dout[b], comp);
        if (rc)
            return rc;
        CUDA_TRY(cudaEventRecord(ev[1], comp)); // din[b] read, dout[b] written
        CUDA_TRY(cudaStreamWaitEvent(d2h, ev[1], 0));
        CUDA_TRY(cudaMemcpyAsync(h_out[i], dout[b], bytes, cudaMemcpyDeviceToHost, d2h));
        CUDA_TRY(cudaEventRecord(ev[2], d2h));
    }
    CUDA_TRY(cudaStreamSynchronize(d2h));
    p->last_stream = comp;
    return FFT3_OK;
}

int fft3_plan_check(fft3_plan p)
{
    if (!p)
        return fail(FFT3_ERR_INVALID_ARG, "null plan");
    CUDA_TRY(cudaStreamSynchronize(p->last_stream));
    unsigned flags = 0;
    CUDA_TRY(cudaMemcpy(&flags, p->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (flags) {
        CUDA_TRY(cudaMemset(p->d_err, 0, sizeof(unsigned)));
        if (flags & kErrWaitTimeout)
            return fail(FFT3_ERR_TIMEOUT, "a bounded device-side wait expired");
        return fail(FFT3_ERR_CUDA, "device error flags set: " + std::to_string(flags));
    }
    return FFT3_OK;
}

int fft3_plan_destroy(fft3_plan p)
{
    if (!p)
        return fail(FFT3_ERR_INVALID_ARG, "null plan");
    free_plan(p);
    return FFT3_OK;
}

size_t fft3_plan_workspace_bytes(fft3_plan p) { return p ? p->ws_bytes : 0; }

int fft3_plan_launches(fft3_plan p)
{
    if (!p)
        return fail(FFT3_ERR_INVALID_ARG, "null plan");
    if (p->batch)
        return 1;
    return (int)p->launches.size();
}

int fft3_plan_kernel_launches(fft3_plan p)
{
    if (!p)
        return fail(FFT3_ERR_INVALID_ARG, "null plan");
    if (p->batch)
        return batch_kernel_launches(p->batch);
    int n = 0;
    for (size_t k = 0; k < p->launches.size(); ++k) {
        if (pair_head(p, k)) {
            const int64_t K = p->launches[k].chunk, na = p->launches[k].args.g.A;
            n += 2 * (int)((na + K - 1) / K);
            ++k;
        } else {
            n += 1;
        }
    }
    return n;
}

int fft3_plan_describe(fft3_plan p, char *buf, size_t len)
{
    if (!p)
        return fail(FFT3_ERR_INVALID_ARG, "null plan");
    if (p->batch) {
        std::string bj;
        batch_describe(p->batch, &bj);
        if (buf && len > 0) {
            size_t c = std::min(len - 1, bj.size());
            memcpy(buf, bj.data(), c);
            buf[c] = 0;
        }
        return (int)bj.size();
    }
    std::string j = p->sched.json();
    // append the launch shapes
    std::string l = ",\"launches\":[";
    for (size_t i = 0; i < p->launches.size(); ++i) {
        const Launch &L = p->launches[i];
        l += (i ? "," : "") + std::string("{\"grid\":") + std::to_string(L.grid.x) +
             ",\"block\":" + std::to_string(L.block.x) + ",\"smem\":" + std::to_string(L.smem) +
             ",\"cluster\":" + std::to_string(L.cluster) + "}";
    }
    l += std::string("],\"host_direct\":") + (host_direct_ok(p) ? "true" : "false") + "}";
    j = j.substr(0, j.size() - 1) + l;
    if (buf && len > 0) {
        size_t c = std::min(len - 1, j.size());
        memcpy(buf, j.data(), c);
        buf[c] = 0;
    }
    return (int)j.size();
}

int fft3_twiddles(int n, int sign, const int64_t *d_m, int64_t count, double *d_out64, float *d_out32,
                  void *stream)
{
    if (n < 1 || count < 0 || !d_m || (sign != -1 && sign != 1))
        return fail(FFT3_ERR_INVALID_ARG, "bad argument to fft3_twiddles");
    if (count == 0)
        return FFT3_OK;
    int blocks = (int)std::min<int64_t>(4096, (count + 255) / 256);
    k_roots<<<blocks, 256, 0, (cudaStream_t)stream>>>(n, sign, d_m, count, d_out64, (float2 *)d_out32);
    CUDA_TRY(cudaGetLastError());
    return FFT3_OK;
}

int fft3_split_bf16(const float *d_x, int64_t count, uint16_t *d_hi, uint16_t *d_lo, void *stream)
{
    if (!d_x || !d_hi || !d_lo || count < 0)
        return fail(FFT3_ERR_INVALID_ARG, "bad argument to fft3_split_bf16");
    if (count == 0)
        return FFT3_OK;
    int blocks = (int)std::min<int64_t>(4096, (count + 255) / 256);
    k_split_bf16<<<blocks, 256, 0, (cudaStream_t)stream>>>(d_x, count, d_hi, d_lo);
    CUDA_TRY(cudaGetLastError());
    return FFT3_OK;
}

} // extern "C"

// ---------------------------------------------- allocation-free transform -- //
// fft3_execute_noalloc runs the rotated pencil-pencil-pencil schedule with its
// workspace and its twiddle tables in the fixed device arrays below instead of
// memory it allocates.  These arrays exist once per device for the life of the
// process (the loader reserves them with the module), every call shares them,
// and the data of the previous call stays in them; nothing in them needs to
// start at zero, because every call writes the twiddles and the whole
// workspace region it reads before reading it.
static __device__ __align__(256) float2 g_noalloc_ws[FFT3_NOALLOC_MAX_ELEMENTS];
static __device__ __align__(256) float2 g_noalloc_tw[FFT3_NOALLOC_MAX_TWIDDLES];
static __device__ __align__(256) unsigned g_noalloc_err[64];

namespace {

struct NoallocDevice {
    bool ready = false;
    float2 *ws = nullptr, *tw = nullptr;
    unsigned *err = nullptr;
};
std::mutex g_noalloc_mutex;
NoallocDevice g_noalloc[64];

// Host code cannot name a __device__ array's address directly: the symbol is a
// host-side stand-in.  Ask the runtime for the device address, once per device
// with that device current.
int noalloc_setup(int dev, NoallocDevice **out)
{
    if (dev < 0 || dev >= 64)
        return fail(FFT3_ERR_INVALID_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    NoallocDevice &d = g_noalloc[dev];
    if (!d.ready) {
        CUDA_TRY(cudaGetSymbolAddress((void **)&d.ws, g_noalloc_ws));
        CUDA_TRY(cudaGetSymbolAddress((void **)&d.tw, g_noalloc_tw));
        CUDA_TRY(cudaGetSymbolAddress((void **)&d.err, g_noalloc_err));
        d.ready = true;
    }
    *out = &d;
    return FFT3_OK;
}

} // namespace

namespace fft3 {
// Stage-major twiddles of one runtime line plan (fft_engine.cuh) computed on
// the device from the plan itself, so no exponent list has to be uploaded: the
// exponents and the FP64 roots come from the same helpers (roots.cuh) as the
// tables of regular plans, so both tables are identical.
__global__ void k_noalloc_line_roots(LineRt L, int total, float2 *out)
{
    if (L.nst == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0)
            out[0] = make_float2(1.f, 0.f);
        return;
    }
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const double2 w = root_fp64(stage_twiddle_exponent(L.n, L.rad, L.nst, e), L.n, FFT3_FORWARD);
        out[e] = make_float2((float)w.x, (float)w.y);
    }
}
} // namespace fft3

extern "C" int fft3_execute_noalloc(int n0, int n1, int n2, int batch, int direction, const void *in, void *out,
                                    void *stream)
{
    if (!in || !out)
        return fail(FFT3_ERR_INVALID_ARG, "null buffer");
    if (in == out)
        return fail(FFT3_ERR_INPLACE_UNSUPPORTED, "in-place execution is not supported (in == out)");
    if (n0 < 1 || n1 < 1 || n2 < 1 || batch < 1)
        return fail(FFT3_ERR_INVALID_ARG, "sizes and batch must be positive");
    const int64_t elems = (int64_t)n0 * n1 * n2 * batch;
    if (elems > FFT3_NOALLOC_MAX_ELEMENTS)
        return fail(FFT3_ERR_UNSUPPORTED_SIZE,
                    "fft3_execute_noalloc handles at most FFT3_NOALLOC_MAX_ELEMENTS (" +
                        std::to_string((long long)FFT3_NOALLOC_MAX_ELEMENTS) + ") complex values per call; got " +
                        std::to_string((long long)elems));
    fft3_options o{};
    o.variant = FFT3_PPP_ROTATE;
    fft3_plan_s P; // host-side description only; every device pointer below is static
    std::string err;
    int rc = build_schedule(n0, n1, n2, batch, FFT3_C64_FP32, FFT3_PENCIL3, direction, &o, &P.sched, &err);
    if (rc)
        return fail(rc, err);
    if (P.sched.tw_total > FFT3_NOALLOC_MAX_TWIDDLES)
        return fail(FFT3_ERR_UNSUPPORTED_SIZE, "twiddle tables exceed FFT3_NOALLOC_MAX_TWIDDLES");
    rc = check_device(&P.device);
    if (rc)
        return rc;
    NoallocDevice *nd = nullptr;
    rc = noalloc_setup(P.device, &nd);
    if (rc)
        return rc;
    P.elems = elems;
    P.d_tw = nd->tw;
    P.d_ws = nd->ws;
    P.ws_bytes = 0;
    P.d_err = nd->err;
    rc = build_launches(&P);
    if (rc)
        return rc;
    cudaStream_t st = (cudaStream_t)stream;
    for (const PassPlan &p : P.sched.passes) {
        const TwSeg &sg = P.sched.tw[p.tw_seg[0]];
        k_noalloc_line_roots<<<std::max(1, ((int)sg.m.size() + 255) / 256), 256, 0, st>>>(
            to_rt(p.line, 0), (int)sg.m.size(), nd->tw + sg.off);
        CUDA_TRY(cudaGetLastError());
    }
    return fft3_plan_execute(&P, in, out, stream);
}
