// geom.h -- plain (host and device) description of one pass of batched 1D
// DFTs; see pass_kernels.cuh for the meaning of every field.
#pragma once

#include <stdint.h>
#include <vector_types.h>

namespace fft3 {

struct PassGeom {
    int64_t C, A, B;
    int64_t ij, ic, ia, ib;
    int64_t ok, oc, oa, ob;
    // 0: output element k of a line at k*ok; > 0: at (k/16)*oblk + (k%16)*ok
    // (a line stored in blocks of 16, as the 16-column blocked layouts need)
    int64_t oblk;
    // Lines split into runs over blocks (the blocks an all-to-all exchanges):
    // ijb > 0: input element j at (j/ijb)*iblk + (j%ijb)*ij; okb > 0: output
    // element k at (k/okb)*oblk + (k%okb)*ok.  Only the runtime-radix kernels
    // (k_pass_g, k_pass_g64) and the layout probe take them.
    int64_t ijb, iblk, okb;
};

// Offset of element j of a line under the input (output) index of g.
__host__ __device__ __forceinline__ int64_t geom_in_elem(const PassGeom &g, int64_t j)
{
    return g.ijb > 0 ? (j / g.ijb) * g.iblk + (j % g.ijb) * g.ij : j * g.ij;
}
__host__ __device__ __forceinline__ int64_t geom_out_elem(const PassGeom &g, int64_t k)
{
    return g.okb > 0 ? (k / g.okb) * g.oblk + (k % g.okb) * g.ok
         : g.oblk   ? (k >> 4) * g.oblk + (k & 15) * g.ok
                    : k * g.ok;
}

// Error flag bits written by device code (read back by fft3_plan_check).
enum : unsigned {
    kErrWaitTimeout = 1u,
    kErrBadTile = 2u,
};

constexpr int kMaxStages = 12;

// A line transform with its radix list known only at run time.
struct LineRt {
    int n, T, nst, tw_off; // tw_off: offset of its stage-major table inside the pass table
    int rad[kMaxStages];
};

struct PassArgs {
    const float2 *in;
    float2 *out;
    PassGeom g;
    const float2 *tw; // the pass's twiddle tables (global memory), tw_len entries
    int tw_len;
    int conj;         // 1: inverse via conj(DFT(conj x))
    int64_t ntiles;
    int64_t tiles_c;
    int lpt;          // lines (or slabs) per tile
    LineRt L[2];      // runtime line plans: generic L[0]; slab x = L[0], y = L[1];
                      // volumetric rows (DFT_b) = L[0], columns (DFT_a) = L[1]
    int p, split_a, split_b, tw_split_off; // volumetric split n = a*b over p blocks
    int six_step;     // volumetric split with blocked ownership and three exchanges (k_vol)
    unsigned *err;    // device error flags (persistent kernels)
    int *counters;    // per-slab completion counters + ticket (persistent kernels)
    long long wait_budget; // clock cycles a bounded wait may spin before giving up
    int64_t nosignal_slab; // test hook: x tiles of this slab never signal (-1 = off)
};

} // namespace fft3
