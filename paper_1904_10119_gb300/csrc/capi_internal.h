// capi_internal.h -- shared internals of the C ABI translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/fft3.h"
#include "batched.h"
#include "geom.h"
#include "planner.h"
#include "plans.h"

namespace fft3 {

int fail(int code, const std::string &msg);

#define CUDA_TRY(x)                                                                                \
    do {                                                                                           \
        cudaError_t e_ = (x);                                                                      \
        if (e_ != cudaSuccess) {                                                                   \
            cudaGetLastError();                                                                    \
            return ::fft3::fail(e_ == cudaErrorMemoryAllocation ? FFT3_ERR_OOM : FFT3_ERR_CUDA,    \
                                std::string(#x) + ": " + cudaGetErrorString(e_));                  \
        }                                                                                          \
    } while (0)

struct Launch {
    const void *func = nullptr;
    dim3 grid, block;
    int smem = 0;
    int cluster = 1;
    int kind = 0;
    PassArgs args{};
    int src = BUF_IN, dst = BUF_OUT;
    bool reset_counters = false;
    bool slab_map = false; // k_slab_tma: 2D tensor map of the blocked workspace
    bool tma = false; // kernel takes two tensor maps after its PassArgs
    int stream_q = 0; // > 0: streamed strided pass, one 5D input map of Q decimated sub-lines
    int tc32 = 0;     // k_tc32: 1 = tiles by bulk copies (unused map), 2 = strided columns (4D input map)
    // two-stream pipelined pair: this pass (on the caller's stream) and the
    // next one (on the plan's side stream) run over chunks of `chunk` values
    // of a, the next pass's chunk c after this pass's chunk c
    int chunk = 0;
    bool pair_next = false;
    // identity probe of the same pass geometry
    PassGeom probe_g{};
    int probe_n = 1;
};

struct BatchState; // batched uneven plans (batched_host.cu)

int device_sms(int dev);
// Opts a kernel in to `smem` bytes of dynamic shared memory; max_shared also
// asks for the largest shared-memory carveout (the tensor-memory kernels,
// whose blocks fill an SM's shared memory; kernels that lean on L1 keep the
// driver's choice).
int prepare_func(const void *func, int smem, bool max_shared = false);
int occupancy_grid(const void *func, int threads, int smem, int64_t ntiles, int dev, dim3 *grid);
int check_device(int *dev);

// Batched plans
int batch_execute(fft3_plan p, const void *in, void *out, cudaStream_t st);
void batch_free(BatchState *b);
int batch_describe(const BatchState *b, std::string *json);
int batch_kernel_launches(const BatchState *b); // kernels in one execution of a batched plan
int batch_buffer_need(int n0, int n1, int n2, int code);

} // namespace fft3

struct fft3_plan_s {
    fft3::Schedule sched;
    int device = 0;
    int64_t elems = 0; // complex elements per array
    int esize = 8;     // bytes per complex element (16 for complex128)
    float2 *d_tw = nullptr; // twiddle table (double2 entries for complex128)
    float2 *d_ws = nullptr;
    size_t ws_bytes = 0;
    int *d_counters = nullptr;
    size_t counters_bytes = 0;
    unsigned *d_err = nullptr;
    std::vector<fft3::Launch> launches;
    float2 *d_stage_in = nullptr, *d_stage_out = nullptr;
    // pipelined host execution: a second set of staging buffers, the copy and
    // compute streams, and per-set events (input consumed, output produced, output drained)
    float2 *d_stage_in2 = nullptr, *d_stage_out2 = nullptr;
    cudaStream_t pipe_st[3] = {nullptr, nullptr, nullptr}; // H2D, compute, D2H
    cudaEvent_t pipe_ev[2][3] = {};                        // [set][input loaded, transform done, output drained]
    cudaStream_t last_stream = nullptr;
    cudaStream_t side = nullptr;                        // second stream of a pipelined pair
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;   // chunk hand-over and final join
    fft3::BatchState *batch = nullptr; // non-null for fft3_plan_create_many plans
};
