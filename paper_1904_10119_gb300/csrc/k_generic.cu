// k_generic.cu -- pass kernels whose radix list is data: any 2*3*5-smooth line
// length up to 4096, the 2D slab pass of the slab-pencil decomposition for
// slabs that fit in one block's shared memory, the identity probe of a pass
// geometry, and the copy pass.
#include "pass_kernels.cuh"
#include "runtime_stages.cuh"

namespace fft3 {

// ------------------------------------------------------------ k_pass_g -- //
// One tile of `lpt` lines staged through shared memory (whichever mapping
// keeps the global accesses coalesced), the runtime radix stages, the tile
// stored back.  C = float2 (k_pass_g) or double2 (k_pass_g64: the complex128
// path, whose arrays and twiddle table hold double2).
template <class C>
__device__ __forceinline__ void pass_g_body(const PassArgs &a, const C *in, C *out, const C *twg)
{
    extern __shared__ __align__(16) unsigned char g_smem_raw[];
    C *smem = reinterpret_cast<C *>(g_smem_raw);
    const LineRt &L = a.L[0];
    const int n = L.n;
    const int P = line_pitch(n);
    C *tw = smem;
    C *b0 = smem + tw_slots(a.tw_len);
    C *b1 = b0 + a.lpt * P;
    for (int i = threadIdx.x; i < a.tw_len; i += blockDim.x)
        tw[i] = twg[i];
    const bool conj = a.conj != 0;
    const bool in_lines = a.g.ij == 1;  // lines contiguous in the input
    const bool out_lines = a.g.ok == 1; // lines contiguous in the output
    const int lpt = a.lpt;
    for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        __syncthreads();
        const TileId id = decode_tile(tile, a.tiles_c, a.g.A, lpt);
        const int64_t nval = min((int64_t)lpt, a.g.C - id.c0);
        const C *ib = in + id.c0 * a.g.ic + id.a * a.g.ia + id.b * a.g.ib;
        for (int e = threadIdx.x; e < lpt * n; e += blockDim.x) {
            int l, j;
            if (in_lines) { l = e / n; j = e - l * n; }
            else { l = e % lpt; j = e / lpt; }
            C v = Cx<C>::make(0, 0);
            if (l < nval)
                v = ib[l * a.g.ic + geom_in_elem(a.g, j)];
            b0[l * P + padpos(j)] = conj ? cconj(v) : v;
        }
        __syncthreads();
        const C *res = run_stages_lines(L, lpt, P, b0, b1, tw + L.tw_off);
        C *ob = out + id.c0 * a.g.oc + id.a * a.g.oa + id.b * a.g.ob;
        for (int e = threadIdx.x; e < lpt * n; e += blockDim.x) {
            int l, k;
            if (out_lines) { l = e / n; k = e - l * n; }
            else { l = e % lpt; k = e / lpt; }
            if (l < nval) {
                C v = res[l * P + padpos(k)];
                ob[l * a.g.oc + geom_out_elem(a.g, k)] = conj ? cconj(v) : v;
            }
        }
    }
}

__global__ void k_pass_g(PassArgs a) { pass_g_body<float2>(a, a.in, a.out, a.tw); }

__global__ void k_pass_g64(PassArgs a)
{
    pass_g_body<double2>(a, reinterpret_cast<const double2 *>(a.in), reinterpret_cast<double2 *>(a.out),
                         reinterpret_cast<const double2 *>(a.tw));
}

// -------------------------------------------------------------- k_slab -- //
// One n0 x n1 slab per tile, held in shared memory: x lines (rows, length n0)
// then y lines (columns, length n1), ping-ponging between two padded copies.
__global__ void k_slab(PassArgs a)
{
    extern __shared__ float2 smem[];
    const LineRt &X = a.L[0];
    const LineRt &Y = a.L[1];
    const int n0 = X.n, n1 = Y.n;
    const int P = line_pitch(n0);
    float2 *tw = smem;
    float2 *b0 = smem + tw_slots(a.tw_len);
    float2 *b1 = b0 + n1 * P;
    load_twiddles(tw, a.tw, a.tw_len);
    const bool conj = a.conj != 0;
    const int nel = n0 * n1;
    for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        __syncthreads();
        const int64_t sa = tile % a.g.A, sb = tile / a.g.A;
        const float2 *ib = a.in + sa * a.g.ia + sb * a.g.ib;
        float2 *ob = a.out + sa * a.g.oa + sb * a.g.ob;
        for (int e = threadIdx.x; e < nel; e += blockDim.x) {
            const int row = e / n0, col = e - row * n0;
            const float2 v = ib[e];
            b0[row * P + padpos(col)] = conj ? cconj(v) : v;
        }
        __syncthreads();
        float2 *r1 = run_stages_lines(X, n1, P, b0, b1, tw + X.tw_off);
        float2 *o1 = (r1 == b0) ? b1 : b0;
        float2 *r2 = run_stages_cols(Y, n0, P, r1, o1, tw + Y.tw_off);
        for (int e = threadIdx.x; e < nel; e += blockDim.x) {
            const int row = e / n0, col = e - row * n0;
            const float2 v = r2[row * P + padpos(col)];
            ob[e] = conj ? cconj(v) : v;
        }
    }
}

// ------------------------------------------------------- k_probe_pass -- //
// Identity line transform on the pass geometry: element j of every input
// line is written to element j of its output line.
__global__ void k_probe_pass(PassArgs a)
{
    const int64_t n = a.L[0].n;
    const int64_t total = n * a.g.C * a.g.A * a.g.B;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t j = e % n, r = e / n;
        const int64_t c = r % a.g.C;
        r /= a.g.C;
        const int64_t aa = r % a.g.A, b = r / a.g.A;
        a.out[geom_out_elem(a.g, j) + c * a.g.oc + aa * a.g.oa + b * a.g.ob] =
            a.in[geom_in_elem(a.g, j) + c * a.g.ic + aa * a.g.ia + b * a.g.ib];
    }
}

// --------------------------------------------------------------- k_copy -- //
__global__ void k_copy(const float2 *in, float2 *out, int64_t total)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i];
}

} // namespace fft3
