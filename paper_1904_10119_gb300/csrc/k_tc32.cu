// k_tc32.cu -- 1024-point line passes whose two 32-point DFT stages run as
// split-BF16 GEMMs on the fifth-generation tensor cores (tcgen05), with the
// lines on the MMA's M side.
//
// The line is split by Eq. ct (Section 2.1) with n0 = n1 = 32 in
// decimation-in-time order: for x[j], j = 32 j1 + j2,
//   (I)   for every j2: X1[j2][k1] = sum_j1 x[32 j1 + j2] w_32^{j1 k1},
//   (II)  twiddle: X1[j2][k1] *= w_1024^{j2 k1},
//   (III) transposition (j2, k1) -> (k1, j2),
//   (IV)  for every k1: X[k1 + 32 k2] = sum_j2 X1[j2][k1] w_32^{j2 k2}.
// A tile is 4 lines.  Stage (I) is one GEMM D = A B^T with M = 128 rows (4
// lines x 32 decimated sub-sequences j2), K = 64 (32 complex inputs, re and
// im interleaved) and N = 64 (32 complex outputs): B is the real-ified DFT_32,
//   B[2k+0][2j+0] = Re w,  B[2k+0][2j+1] = -Im w,
//   B[2k+1][2j+0] = Im w,  B[2k+1][2j+1] =  Re w,   w = w_32^{jk},
// so D[row][2k] and D[row][2k+1] are the real and imaginary parts of output
// k.  Stage (IV) is the same GEMM with rows (line, k1).  Both operands are
// split, v = v_hi + v_lo with v_hi = bf16(v), v_lo = bf16(v - v_hi), and
// three products are accumulated in FP32: A_lo B_hi + A_hi B_lo + A_hi B_hi
// (A_lo B_lo is dropped).  The twiddles (II) are applied in FP32.
//
// One persistent 512-thread block per SM (the occupancy of a kernel that
// allocates tensor memory is one block per SM) made of four independent
// groups of 128 threads; group g owns tensor-memory columns 128 g .. +127
// and a landing buffer, and transforms its own stream of tiles, so one
// group's MMAs and loads overlap the other groups' CUDA-core work.  In a
// group, thread t owns GEMM row t in both stages (tensor-memory lane t): it
// writes its row of A with tcgen05.st (high parts in columns 0-31, low parts
// in 32-63 of the group's region), one elected thread issues the twelve MMAs
// (4 K steps x 3 products, M = 128, N = 64, K = 16) into D (columns 64-127 of
// the region) and commits them to the group's mbarrier, and every thread
// reads its row of D back with tcgen05.ld.  B (DFT_32 high and low parts)
// sits in shared memory with the 128-byte swizzle, shared by the groups.
//
// Tiles arrive by TMA into the group's landing buffer (contiguous lines: one
// bulk copy of 32 KB; strided columns: four 4-column x 256-row boxes of a 4D
// tensor map).  The four groups of a block take the four adjacent 4-column
// tiles of a 16-column block, so between them they read and write whole
// 128-byte rows.  Once its inputs are in registers the landing buffer holds the
// tile's transposition (III) in a padded layout, and once stage (IV) has read
// that back it is refilled with the group's next tile, whose load overlaps the
// stage-(IV) MMAs and the output stores.
//
// Thread roles of the contiguous-line kernel (t = row within the group, tile
// lines l < 4): row t = 32 l + j2 (stage I), 32 l + k1 (IV), so every warp's
// shared-memory accesses cover 32 consecutive complex values or hit distinct
// banks through the padding.
#include <cuda_bf16.h>

#include "pass_kernels.cuh"
#include "plans.h"
#include "umma.cuh"

namespace fft3 {

namespace {

constexpr int kN = 1024;
constexpr int kLpt = kTc32Lpt;
constexpr uint32_t kTileBytes = (uint32_t)kLpt * kN * 8u; // 32 KB
constexpr int kPitchL = 34;                             // k1 pitch of the transposition (complex)
constexpr int kLineT = 32 * kPitchL;                    // line pitch of the transposition
constexpr int kLandBytes = kTc32LandBytes;              // 34816 >= 32768
static_assert(kLandBytes == kLpt * kLineT * 8, "the transposition fits the landing buffer");
constexpr int kBBytes = 64 * 128;                       // one 64 x 64 BF16 operand
constexpr int kTwOff = 2 * kBBytes;                     // w_1024^{j2 k1}, [k1][j2]
constexpr int kLandOff = kTwOff + kN * 8;
static_assert(kLandOff + kTc32Groups * kLandBytes + 1024 == kTc32SmemBytes,
              "dynamic shared memory (+ alignment slack)");
static_assert(kLandOff + kTcsQuarters * kTcsQuarterBytes + 1024 == kTcsSmemBytes && kTcsSmemBytes <= 227 * 1024,
              "dynamic shared memory of the strided kernel (+ alignment slack)");

// w = w_32^m for the DFT_32 operand (FP32 values of the FP64 generator) ->
// B_hi, B_lo in the 128-byte-swizzled K-major layout; the inverse transform
// uses the conjugate roots (the same factorisation with w_n^-1).
__device__ __forceinline__ void build_dft32_operand(uint8_t *bhi, uint8_t *blo, const float2 *w32, bool conj)
{
    for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
        const int n = e >> 6, kk = e & 63;
        const int kp = n >> 1, cp = n & 1, j = kk >> 1, c = kk & 1;
        const float2 w = conj ? cconj(w32[(kp * j) & 31]) : w32[(kp * j) & 31];
        const float v = (cp == c) ? w.x : (cp == 0 ? -w.y : w.y);
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(h));
        const int off = (n >> 3) * 1024 + (n & 7) * 128 + (((kk >> 3) ^ (n & 7)) << 4) + (kk & 7) * 2;
        *(uint16_t *)(bhi + off) = __bfloat16_as_ushort(h);
        *(uint16_t *)(blo + off) = __bfloat16_as_ushort(lo);
    }
}

// The twelve MMAs of one stage: D = A_lo B_hi + A_hi B_lo + A_hi B_hi.
__device__ __forceinline__ void issue_stage_mmas(uint32_t t_a, uint32_t t_d, uint32_t s_bhi, uint32_t s_blo)
{
    constexpr uint32_t idesc = idesc_bf16_f32(128, 64);
#pragma unroll
    for (int s = 0; s < 4; ++s)
        mma_bf16_ta(t_d, t_a + 32 + 8 * s, sdesc_sw128(s_bhi + 32 * s), idesc, s > 0);
#pragma unroll
    for (int s = 0; s < 4; ++s)
        mma_bf16_ta(t_d, t_a + 8 * s, sdesc_sw128(s_blo + 32 * s), idesc, true);
#pragma unroll
    for (int s = 0; s < 4; ++s)
        mma_bf16_ta(t_d, t_a + 8 * s, sdesc_sw128(s_bhi + 32 * s), idesc, true);
}

// Split 16 complex values into high and low parts and store them to this
// thread's row of A (columns col .. col+15 and 32+col .. 32+col+15).
__device__ __forceinline__ void store_a16(uint32_t t_row, int col, const float2 (&v)[16])
{
    uint32_t hi[16], lo[16];
#pragma unroll
    for (int i = 0; i < 16; ++i)
        split_c(v[i].x, v[i].y, hi[i], lo[i]);
    tmem_st16(t_row + col, hi);
    tmem_st16(t_row + 32 + col, lo);
}

// CTA-wide OR of a predicate.
__device__ __forceinline__ bool cta_any(bool p) { return __syncthreads_or(p ? 1 : 0) != 0; }

} // namespace

// Barrier of thread group g (named barrier 1 + g over its 128 threads), with
// an OR-reduction of a predicate.
template <int ID>
__device__ __forceinline__ bool bar_or(bool pred)
{
    uint32_t out;
    asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, %2, 128, p;\n\t"
                 "selp.u32 %0, 1, 0, q;\n\t}"
                 : "=r"(out)
                 : "r"(pred ? 1u : 0u), "n"(ID)
                 : "memory");
    return out != 0;
}
__device__ __forceinline__ bool group_or(int g, bool pred)
{
    switch (g) {
    case 0: return bar_or<1>(pred);
    case 1: return bar_or<2>(pred);
    case 2: return bar_or<3>(pred);
    default: return bar_or<4>(pred);
    }
}

// Contiguous lines: four independent groups, tiles of 4 lines loaded as one
// bulk copy each.
__global__ void __launch_bounds__(kTc32Threads, 1) k_tc32x(PassArgs a)
{
    extern __shared__ uint8_t dsm_raw[];
    __shared__ __align__(8) uint64_t full[kTc32Groups];
    __shared__ __align__(8) uint64_t mbar[kTc32Groups];
    __shared__ uint32_t s_tmem;
    uint8_t *dsm = (uint8_t *)(((uintptr_t)dsm_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *bhi = dsm, *blo = dsm + kBBytes;
    float2 *tw = (float2 *)(dsm + kTwOff);
    const int tid = threadIdx.x, g = tid >> 7, gt = tid & 127, warp = tid >> 5, lane = tid & 31;
    const int gw = warp & 3; // warp within the group = its tensor-memory lane quarter
    uint8_t *land = dsm + kLandOff + g * kLandBytes;
    const bool conj = a.conj != 0;

    build_dft32_operand(bhi, blo, a.tw + a.tw_split_off, conj);
    for (int i = tid; i < kN; i += blockDim.x)
        tw[i] = conj ? cconj(a.tw[i]) : a.tw[i];
    if (tid == 0) {
        for (int i = 0; i < kTc32Groups; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&mbar[i], 1);
        }
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(&s_tmem, 512);
        tmem_relinquish();
    }
    fence_proxy_async_smem(); // B, written by these threads, is read by the tensor cores
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // group g: A in columns 128 g .. +63, D in 128 g + 64 .. +127; row gt in lane gt
    const uint32_t t_a = s_tmem + ((uint32_t)(32 * gw) << 16) + 128 * g, t_d = t_a + 64;
    const uint32_t s_bhi = smem_u32(bhi), s_blo = smem_u32(blo);
    const uint64_t pol = l2_evict_first_policy();
    const int64_t stream = (int64_t)blockIdx.x * kTc32Groups + g, nstreams = (int64_t)gridDim.x * kTc32Groups;

    // Load of the group's k-th tile into its landing buffer (the group's thread 0).
    auto issue = [&](int64_t k) {
        const int64_t tile = stream + k * nstreams;
        if (tile >= a.ntiles)
            return;
        const TileId id = decode_tile(tile, a.tiles_c, a.g.A, kLpt);
        // lines beyond the array's last one are not loaded (their rows are never stored)
        const int nval = (int)min((int64_t)kLpt, a.g.C - id.c0);
        const float2 *src = a.in + id.c0 * a.g.ic + id.a * a.g.ia + id.b * a.g.ib;
        mbar_expect_tx(&full[g], (uint32_t)nval * kN * 8u);
        bulk_load(land, src, (uint32_t)nval * kN * 8u, &full[g], pol);
    };
    int64_t issued = -1; // (the group's thread 0) the last k whose load was issued
    if (gt == 0) {
        issue(0);
        issued = 0;
    }

    const float2 *lin = (const float2 *)land;
    float2 *tr = (float2 *)land;
    // stage (I) row gt = (line l1, sub-sequence j2); stage (IV) row gt = (line l2, output k1)
    const int l1 = gw, j2 = lane;
    const int l2 = l1, k1 = j2;
    uint32_t mph = 0;
    bool failed = false;
    int64_t k = 0;
    for (int64_t tile = stream; tile < a.ntiles; tile += nstreams, ++k) {
        const bool late = !mbar_wait(&full[g], (uint32_t)(k & 1), a.wait_budget);
        if (group_or(g, late)) {
            failed = true;
            break;
        }
        // ---- stage (I): row gt gathers its decimated sub-sequence x[32 j1 + j2]
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float2 v[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int j = 32 * (16 * h + i) + j2;
                v[i] = lin[l1 * kN + j];
            }
            store_a16(t_a, 16 * h, v);
        }
        tmem_wait_st();
        tc_fence_before();
        group_or(g, false);
        if (gt == 0) {
            tc_fence_after();
            issue_stage_mmas(t_a, t_d, s_bhi, s_blo);
            mma_commit(&mbar[g]);
        }
        const bool late1 = !mbar_wait(&mbar[g], mph, a.wait_budget);
        mph ^= 1;
        tc_fence_after();
        // ---- (II) twiddle and (III) transposition into the landing buffer
        {
            uint32_t d[64];
#pragma unroll
            for (int h = 0; h < 4; ++h)
                tmem_ld16(t_d + 16 * h, *(uint32_t(*)[16])(d + 16 * h));
            tmem_wait_ld();
#pragma unroll
            for (int kk1 = 0; kk1 < 32; ++kk1)
                tr[l1 * kLineT + kk1 * kPitchL + j2] =
                    cmul(make_float2(__uint_as_float(d[2 * kk1]), __uint_as_float(d[2 * kk1 + 1])), tw[kk1 * 32 + j2]);
        }
        tc_fence_before();
        if (group_or(g, late1)) {
            failed = true;
            break;
        }
        // ---- stage (IV): row gt = (line, k1) reads X1[j2][k1] for every j2
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float2 v[16];
            const float4 *src = (const float4 *)(tr + l2 * kLineT + k1 * kPitchL + 16 * h);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float4 q = src[i];
                v[2 * i] = make_float2(q.x, q.y);
                v[2 * i + 1] = make_float2(q.z, q.w);
            }
            store_a16(t_a, 16 * h, v);
        }
        tmem_wait_st();
        tc_fence_before();
        fence_proxy_async_smem(); // this thread's accesses to the landing buffer, before its refill
        group_or(g, false);
        if (gt == 0) {
            tc_fence_after();
            issue_stage_mmas(t_a, t_d, s_bhi, s_blo);
            mma_commit(&mbar[g]);
            issue(k + 1); // the landing buffer is read out: the group's next tile
            issued = k + 1;
        }
        const bool late2 = !mbar_wait(&mbar[g], mph, a.wait_budget);
        mph ^= 1;
        tc_fence_after();
        // ---- outputs X[k1 + 32 k2] of line l2
        const TileId id = decode_tile(tile, a.tiles_c, a.g.A, kLpt);
        const int64_t c = id.c0 + l2;
        const bool valid = !late2 && c < a.g.C;
        // element k = k1 + 32 k2 at k*ok, or blocked by 16 at (k/16)*oblk + (k%16)*ok
        float2 *op = a.out + c * a.g.oc + id.a * a.g.oa + id.b * a.g.ob +
                     (a.g.oblk ? (int64_t)(k1 >> 4) * a.g.oblk + (k1 & 15) * a.g.ok : (int64_t)k1 * a.g.ok);
        const int64_t ostep = a.g.oblk ? 2 * a.g.oblk : 32 * a.g.ok;
        {
            uint32_t d[64];
#pragma unroll
            for (int h = 0; h < 4; ++h)
                tmem_ld16(t_d + 16 * h, *(uint32_t(*)[16])(d + 16 * h));
            tmem_wait_ld();
            if (valid) {
#pragma unroll
                for (int k2 = 0; k2 < 32; ++k2)
                    op[k2 * ostep] = make_float2(__uint_as_float(d[2 * k2]), __uint_as_float(d[2 * k2 + 1]));
            }
        }
        tc_fence_before();
        if (group_or(g, late2)) {
            failed = true;
            break;
        }
    }
    if (failed && gt == 0) {
        // record the timeout and wait (bounded) for the copy still in flight
        // into this group's landing buffer before the block exits
        atomicOr(a.err, kErrWaitTimeout);
        for (int64_t v = k; v <= issued; ++v)
            if (stream + v * nstreams < a.ntiles && !mbar_wait(&full[g], (uint32_t)(v & 1), a.wait_budget))
                break;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        tmem_dealloc(s_tmem, 512);
}

// ---------------------------------------------------------------------------
// Strided columns (y and z lines): one block transforms one tile of 16
// adjacent columns at a time, loaded as four 32 KB quarters through a 5D
// tensor map {C, 32, 32, A, B} of the decimated sub-sequences x[32 j1 + j2]
// (box: 16 columns x 8 values of j2 x 32 values of j1, whole 128-byte rows).
//   stage (I):  group g transforms the sub-sequences j2 in [8g, 8g + 8) of the
//               16 columns (row t = (q, c), j2 = 8g + q, q = t / 16, c = t % 16)
//               and writes its twiddled outputs X1[c][j2][k1] back into its
//               own quarter, in place (slot of j1 := k1);
//   block barrier;
//   stage (IV): group g transforms the outputs k1 in [8g, 8g + 8) (row t =
//               (kk, c), k1 = 8g + kk), reading X1[c][j2][k1] for every j2
//               from the four quarters, and stores rows k1 + 32 k2: each warp
//               writes two whole 128-byte rows per instruction.
// Six quarter buffers rotate: quarter e of the block's i-th tile sits in
// buffer (4i + e) % 6, so the first two quarters of the next tile load while
// this tile is transformed, and the four buffers of a tile are refilled once
// every group has read them in stage (IV).
__global__ void __launch_bounds__(kTc32Threads, 1) k_tc32s(PassArgs a, const __grid_constant__ CUtensorMap tin)
{
    constexpr int NQ = kTcsQuarters;
    constexpr uint32_t QBYTES = kTcsQuarterBytes;
    extern __shared__ uint8_t dsm_raw[];
    __shared__ __align__(8) uint64_t full[NQ];
    __shared__ __align__(8) uint64_t mbar[kTc32Groups];
    __shared__ uint32_t s_tmem;
    uint8_t *dsm = (uint8_t *)(((uintptr_t)dsm_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *bhi = dsm, *blo = dsm + kBBytes;
    float2 *tw = (float2 *)(dsm + kTwOff);
    float2 *qbuf = (float2 *)(dsm + kLandOff); // NQ quarters of 4096 values
    const int tid = threadIdx.x, g = tid >> 7, gt = tid & 127, warp = tid >> 5;
    const int gw = warp & 3;
    const bool conj = a.conj != 0;

    build_dft32_operand(bhi, blo, a.tw + a.tw_split_off, conj);
    for (int i = tid; i < kN; i += blockDim.x)
        tw[i] = conj ? cconj(a.tw[i]) : a.tw[i];
    if (tid == 0) {
        for (int i = 0; i < NQ; ++i)
            mbar_init(&full[i], 1);
        for (int i = 0; i < kTc32Groups; ++i)
            mbar_init(&mbar[i], 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(&s_tmem, 512);
        tmem_relinquish();
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t t_a = s_tmem + ((uint32_t)(32 * gw) << 16) + 128 * g, t_d = t_a + 64;
    const uint32_t s_bhi = smem_u32(bhi), s_blo = smem_u32(blo);

    // Quarter L = 4 i + e of the block's tile sequence (thread 0 only).
    auto issue = [&](int64_t L) {
        const int64_t tile = blockIdx.x + (L >> 2) * (int64_t)gridDim.x;
        if (tile >= a.ntiles)
            return;
        const int b = (int)(L % NQ);
        const TileId id = decode_tile(tile, a.tiles_c, a.g.A, kTcsLpt);
        mbar_expect_tx(&full[b], QBYTES);
        tma_load_5d(qbuf + b * 4096, &tin, (int)id.c0, 8 * (int)(L & 3), 0, (int)id.a, (int)id.b, &full[b]);
    };
    int64_t issued = -1; // (thread 0) the last quarter issued
    if (tid == 0) {
        for (int64_t L = 0; L < NQ; ++L)
            issue(L);
        issued = NQ - 1;
    }
    const int q = gt >> 4, c = gt & 15;
    const int j2 = 8 * g + q, k1 = 8 * g + q; // stage (I) / stage (IV) index of this row
    uint32_t mph = 0;
    bool failed = false;
    int64_t i = 0;
    for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++i) {
        const int64_t L = 4 * i + g;
        const int b = (int)(L % NQ);
        float2 *mine = qbuf + b * 4096;
        const bool late = !mbar_wait(&full[b], (uint32_t)((L / NQ) & 1), a.wait_budget);
        // ---- stage (I): element (c, q, j1) of the quarter at (j1 * 8 + q) * 16 + c
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float2 v[16];
#pragma unroll
            for (int ii = 0; ii < 16; ++ii) {
                v[ii] = mine[((16 * h + ii) * 8 + q) * 16 + c];
            }
            store_a16(t_a, 16 * h, v);
        }
        tmem_wait_st();
        tc_fence_before();
        group_or(g, false);
        if (gt == 0) {
            tc_fence_after();
            issue_stage_mmas(t_a, t_d, s_bhi, s_blo);
            mma_commit(&mbar[g]);
        }
        const bool late1 = !mbar_wait(&mbar[g], mph, a.wait_budget);
        mph ^= 1;
        tc_fence_after();
        // ---- (II) twiddle w_1024^{j2 k1}, (III) in place: X1[c][j2][k1] at (k1 * 8 + q) * 16 + c
        {
            uint32_t d[64];
#pragma unroll
            for (int h = 0; h < 4; ++h)
                tmem_ld16(t_d + 16 * h, *(uint32_t(*)[16])(d + 16 * h));
            tmem_wait_ld();
#pragma unroll
            for (int kk1 = 0; kk1 < 32; ++kk1)
                mine[(kk1 * 8 + q) * 16 + c] =
                    cmul(make_float2(__uint_as_float(d[2 * kk1]), __uint_as_float(d[2 * kk1 + 1])), tw[kk1 * 32 + j2]);
        }
        tc_fence_before();
        if (cta_any(late || late1)) { // every quarter of the tile is transposed
            failed = true;
            break;
        }
        // ---- stage (IV): X1[c][j2][k1] for every j2, from quarter j2 / 8 of this tile
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float2 v[16];
#pragma unroll
            for (int ii = 0; ii < 16; ++ii) {
                const int jj = 16 * h + ii;
                const float2 *src = qbuf + (int)((4 * i + (jj >> 3)) % NQ) * 4096;
                v[ii] = src[(k1 * 8 + (jj & 7)) * 16 + c];
            }
            store_a16(t_a, 16 * h, v);
        }
        tmem_wait_st();
        tc_fence_before();
        fence_proxy_async_smem(); // this thread's accesses to the quarters, before their refill
        __syncthreads();          // every quarter of the tile is read out
        if (tid == 0) {
            for (int64_t Ln = 4 * i + NQ; Ln < 4 * i + NQ + 4; ++Ln)
                issue(Ln);
            issued = 4 * i + NQ + 3;
        }
        if (gt == 0) {
            tc_fence_after();
            issue_stage_mmas(t_a, t_d, s_bhi, s_blo);
            mma_commit(&mbar[g]);
        }
        const bool late2 = !mbar_wait(&mbar[g], mph, a.wait_budget);
        mph ^= 1;
        tc_fence_after();
        // ---- outputs X[k1 + 32 k2] of column c
        const TileId id = decode_tile(tile, a.tiles_c, a.g.A, kTcsLpt);
        const int64_t col = id.c0 + c;
        const bool valid = !late2 && col < a.g.C;
        float2 *op = a.out + col * a.g.oc + id.a * a.g.oa + id.b * a.g.ob + (int64_t)k1 * a.g.ok;
        const int64_t ostep = 32 * a.g.ok;
        {
            uint32_t d[64];
#pragma unroll
            for (int h = 0; h < 4; ++h)
                tmem_ld16(t_d + 16 * h, *(uint32_t(*)[16])(d + 16 * h));
            tmem_wait_ld();
            if (valid) {
#pragma unroll
                for (int k2 = 0; k2 < 32; ++k2)
                    op[k2 * ostep] = make_float2(__uint_as_float(d[2 * k2]), __uint_as_float(d[2 * k2 + 1]));
            }
        }
        tc_fence_before();
        if (cta_any(late2)) {
            failed = true;
            break;
        }
    }
    if (failed && tid == 0) {
        // record the timeout and wait (bounded) for the quarters still in flight
        atomicOr(a.err, kErrWaitTimeout);
        for (int64_t L = 4 * i; L <= issued; ++L)
            if (blockIdx.x + (L >> 2) * (int64_t)gridDim.x < a.ntiles &&
                !mbar_wait(&full[L % NQ], (uint32_t)((L / NQ) & 1), a.wait_budget))
                break;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        tmem_dealloc(s_tmem, 512);
}

const void *tc32_kernel(int mode) { return mode == 0 ? (const void *)&k_tc32x : (const void *)&k_tc32s; }

} // namespace fft3
