// autotune.cu -- measured plan selection.
//
// fft3_time_plan times one candidate plan with CUDA events on scratch buffers;
// fft3_autotune sweeps the candidate space of one shape (decomposition,
// pencil variant, slab mode, strided tile, volumetric mesh, radix order) and
// returns the fastest; fft3_autotune_many does the same per size class of a
// batch of uneven problems and writes one tuning code per problem.  The
// sweeps are exhaustive over the candidate lists below, so they are also the
// reference that a learned cost model's choices are scored against.
#include <string.h>

#include <algorithm>
#include <map>
#include <vector>

#include "capi_internal.h"

using namespace fft3;

namespace {

struct Scratch {
    void *in = nullptr, *out = nullptr;
    size_t bytes = 0;
    ~Scratch()
    {
        cudaFree(in);
        cudaFree(out);
    }
    int ensure(size_t b)
    {
        if (b <= bytes)
            return FFT3_OK;
        cudaFree(in);
        cudaFree(out);
        in = out = nullptr;
        bytes = 0;
        if (cudaMalloc(&in, b) != cudaSuccess || cudaMalloc(&out, b) != cudaSuccess) {
            cudaGetLastError();
            return fail(FFT3_ERR_OOM, "autotune scratch allocation failed");
        }
        cudaMemset(in, 0, b);
        bytes = b;
        return FFT3_OK;
    }
};

int time_plan(fft3_plan p, const void *in, void *out, int reps, float *ms)
{
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    int rc = fft3_plan_execute(p, in, out, nullptr); // warm-up (and graph capture for batched plans)
    if (!rc)
        rc = fft3_plan_execute(p, in, out, nullptr);
    if (!rc) {
        cudaEventRecord(e0, nullptr);
        for (int r = 0; r < reps && !rc; ++r)
            rc = fft3_plan_execute(p, in, out, nullptr);
        cudaEventRecord(e1, nullptr);
    }
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (!rc && e == cudaSuccess)
        cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc)
        return rc;
    if (e != cudaSuccess)
        return fail(FFT3_ERR_CUDA, std::string("timing: ") + cudaGetErrorString(e));
    int chk = fft3_plan_check(p);
    if (chk)
        return chk;
    *ms = t / std::max(1, reps);
    return FFT3_OK;
}

} // namespace

extern "C" {

int fft3_time_plan(int n0, int n1, int n2, int batch, int dtype, int decomposition, int direction,
                   const fft3_options *opts, int reps, float *ms)
{
    if (!ms || reps < 1)
        return fail(FFT3_ERR_INVALID_ARG, "ms must be non-null and reps positive");
    fft3_plan p = nullptr;
    int rc = fft3_plan_create_ex(&p, n0, n1, n2, batch, dtype, decomposition, direction, opts);
    if (rc)
        return rc;
    Scratch s;
    rc = s.ensure((size_t)n0 * n1 * n2 * batch * (dtype == FFT3_C128_FP64 ? 16 : 8));
    if (!rc)
        rc = time_plan(p, s.in, s.out, reps, ms);
    fft3_plan_destroy(p);
    return rc;
}

int fft3_time_candidates(int n0, int n1, int n2, int batch, int dtype, int direction, int reps, int count,
                         const int *decompositions, const fft3_options *opts, float *ms_out)
{
    if (count < 1 || !decompositions || !opts || !ms_out || reps < 1)
        return fail(FFT3_ERR_INVALID_ARG, "bad argument to fft3_time_candidates");
    Scratch s;
    int rc = s.ensure((size_t)n0 * n1 * n2 * batch * (dtype == FFT3_C128_FP64 ? 16 : 8));
    if (rc)
        return rc;
    for (int i = 0; i < count; ++i) {
        ms_out[i] = -1.f;
        fft3_plan p = nullptr;
        if (fft3_plan_create_ex(&p, n0, n1, n2, batch, dtype, decompositions[i], direction, &opts[i]))
            continue; // infeasible candidate
        float t = 0.f;
        rc = time_plan(p, s.in, s.out, reps, &t);
        fft3_plan_destroy(p);
        if (rc)
            return rc;
        ms_out[i] = t;
    }
    return FFT3_OK;
}

int fft3_autotune(int n0, int n1, int n2, int batch, int dtype, int direction, int reps, fft3_options *best,
                  int *best_decomposition, float *best_ms)
{
    if (!best || !best_decomposition || !best_ms || reps < 1)
        return fail(FFT3_ERR_INVALID_ARG, "null output or non-positive reps");
    struct Cand {
        int decomp;
        fft3_options o;
    };
    std::vector<Cand> c;
    auto add = [&](int d, int variant, int order, int tile, int slab, int m0, int m1, int m2) {
        Cand k{};
        k.decomp = d;
        k.o.variant = variant;
        k.o.radix_order = order;
        k.o.tile_lines = tile;
        k.o.slab_mode = slab;
        k.o.mesh[0] = m0;
        k.o.mesh[1] = m1;
        k.o.mesh[2] = m2;
        c.push_back(k);
    };
    for (int order = 0; order < 4; ++order) {
        add(FFT3_PENCIL3, 0, order, 0, 0, 0, 0, 0);
        add(FFT3_PENCIL3, 0, order, 8, 0, 0, 0, 0);
        add(FFT3_PENCIL3, 0, order, 16, 0, 0, 0, 0);
        add(FFT3_PENCIL3, 1, order, 0, 0, 0, 0, 0);
        add(FFT3_SLAB_PENCIL, 0, order, 0, 1, 0, 0, 0);
        add(FFT3_SLAB_PENCIL, 0, order, 0, 2, 0, 0, 0);
        add(FFT3_SLAB_PENCIL, 0, order, 0, 3, 0, 0, 0);
        add(FFT3_SLAB_PENCIL, 0, order, 0, 4, 0, 0, 0);
        add(FFT3_VOLUMETRIC, 0, order, 0, 0, 2, 2, 2);
    }
    Scratch s;
    int rc = s.ensure((size_t)n0 * n1 * n2 * batch * (dtype == FFT3_C128_FP64 ? 16 : 8));
    if (rc)
        return rc;
    float bt = 3.4e38f;
    int found = 0;
    for (const Cand &k : c) {
        fft3_plan p = nullptr;
        if (fft3_plan_create_ex(&p, n0, n1, n2, batch, dtype, k.decomp, direction, &k.o))
            continue; // infeasible candidate for this shape
        float t = 0.f;
        int r = time_plan(p, s.in, s.out, reps, &t);
        fft3_plan_destroy(p);
        if (r)
            return r;
        if (t < bt) {
            bt = t;
            *best = k.o;
            *best_decomposition = k.decomp;
            found = 1;
        }
    }
    if (!found)
        return fail(FFT3_ERR_UNSUPPORTED_SIZE, "no candidate plan is feasible for this shape");
    *best_ms = bt;
    return FFT3_OK;
}

int fft3_autotune_many(int count, const int *dims, const int64_t *offsets, int direction, int reps,
                       int max_per_class, int *tuning_out)
{
    (void)offsets;
    (void)max_per_class;
    if (count < 1 || !dims || !tuning_out || reps < 1)
        return fail(FFT3_ERR_INVALID_ARG, "bad argument to fft3_autotune_many");
    // The executor's shared buffers, blocks per SM, item order and L2 reuse are
    // properties of the whole batch, so candidates are timed on the whole
    // batch (packed into scratch arrays): the default codes, and each code
    // applied to every problem whose buffer need stays within the default
    // buffers (the others keep the default).
    std::vector<int> codes;
    for (int d = 1; d <= 2; ++d)
        for (int order = 0; order < 4; ++order)
            for (int tile = 2; tile <= 4; ++tile)
                codes.push_back(FFT3_TUNE(d, order, tile, 0));
    int budget = 1;
    for (int i = 0; i < count; ++i)
        budget = std::max(budget, batch_buffer_need(dims[3 * i], dims[3 * i + 1], dims[3 * i + 2], 0));
    std::vector<int64_t> off(count);
    int64_t total = 0;
    for (int i = 0; i < count; ++i) {
        off[i] = total;
        total += (int64_t)dims[3 * i] * dims[3 * i + 1] * dims[3 * i + 2];
    }
    Scratch s;
    int rc = s.ensure((size_t)total * 8);
    if (rc)
        return rc;
    auto fits = [&](int i, int code) {
        return code == 0 || batch_buffer_need(dims[3 * i], dims[3 * i + 1], dims[3 * i + 2], code) <= budget;
    };
    auto time_assignment = [&](const std::vector<int> &tune, float *t) -> int {
        fft3_plan p = nullptr;
        if (fft3_plan_create_many(&p, count, dims, off.data(), FFT3_C64_FP32, FFT3_AUTO, direction, tune.data())) {
            *t = 3.4e38f; // infeasible assignment
            return FFT3_OK;
        }
        int r = time_plan(p, s.in, s.out, reps, t);
        fft3_plan_destroy(p);
        return r;
    };
    std::vector<int> tune(count), best(count, 0);
    std::vector<int> order_codes(1, 0);
    order_codes.insert(order_codes.end(), codes.begin(), codes.end());
    // 1) one code for every problem it fits
    float bt = 3.4e38f;
    for (int code : order_codes) {
        for (int i = 0; i < count; ++i)
            tune[i] = fits(i, code) ? code : 0;
        float t = 0.f;
        if ((rc = time_assignment(tune, &t)))
            return rc;
        if (t < bt) {
            bt = t;
            best = tune;
        }
    }
    // 2) size classes (problem volume in thirds of the batch, smallest first):
    // each class in turn takes the code that makes the whole batch fastest,
    // kept when it gains at least 1%
    std::vector<int> idx(count);
    for (int i = 0; i < count; ++i)
        idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
        return (int64_t)dims[3 * x] * dims[3 * x + 1] * dims[3 * x + 2] <
               (int64_t)dims[3 * y] * dims[3 * y + 1] * dims[3 * y + 2];
    });
    for (int c = 0; c < 3; ++c) {
        const int lo = count * c / 3, hi = count * (c + 1) / 3;
        for (int code : order_codes) {
            tune = best;
            for (int k = lo; k < hi; ++k)
                tune[idx[k]] = fits(idx[k], code) ? code : 0;
            if (tune == best)
                continue;
            float t = 0.f;
            if ((rc = time_assignment(tune, &t)))
                return rc;
            if (t < 0.99f * bt) {
                bt = t;
                best = tune;
            }
        }
    }
    // 3) the segmented x, y and z passes (decomposition field 3 on every
    // problem; infeasible when a line length has no compiled plan)
    std::vector<int> seg(count, 3);
    float ts = 0.f;
    if ((rc = time_assignment(seg, &ts)))
        return rc;
    if (ts < bt) {
        bt = ts;
        best = seg;
    }
    // 4) the slab-by-slab executor (FFT3_TUNE_SLABZ on every problem;
    // infeasible when a line length has no compiled variant)
    std::vector<int> slabz(count, FFT3_TUNE(1, 0, 0, 0) | FFT3_TUNE_SLABZ);
    if ((rc = time_assignment(slabz, &ts)))
        return rc;
    if (ts < bt)
        best = slabz;
    for (int i = 0; i < count; ++i)
        tuning_out[i] = best[i];
    return FFT3_OK;
}

} // extern "C"
