// k_vol.cu -- the volumetric decomposition's pass (Section 3.2, Fig. cuboid):
// one dimension's 1D DFTs, each line of length n = a*b split Cooley-Tukey
// style (Eq. ct, Eq. cteinstein) over a cluster of p thread blocks.
//
// The paper's 1D processor grid becomes the cluster.  Block r holds the rows
// i0 = r mod p of every line's matrix x~[i0, i1] = x[i0 + a*i1] (the
// elemental-cyclic distribution X~[(0)()]), i.e. the input elements j with
// j mod p = r.  It then
//   (I)   applies DFT_b to each of its rows,
//   (II)  scales by the twiddles w_n^{i0*k1}  -> T0[(0)()],
//   (III) takes part in the one exchange T1[()(0)] = T0[(0)()]: block r reads
//         the columns k1 = r mod p of every block's T0 straight out of the
//         peers' shared memory (distributed shared memory of the cluster),
//         which is the all-to-all followed by the local transposition T2,
//   (IV)  applies DFT_a to each of its columns and stores
//         y~[k1, k0] = y[k1 + b*k0], i.e. the outputs k with k mod p = r.
// Input and output are in the same elemental-cyclic distribution, and one
// exchange suffices because p | a and p | b (checked by the planner).
//
// With a.six_step the line is instead distributed in blocks (block r owns the
// elements [r n/p, (r+1) n/p) of input and output), the layout of the six-step
// algorithm of Section 2.2, which needs three exchanges: (0) every block
// gathers its cyclic rows from the owners of the blocked input (staged in its
// T1 region), then (I)-(IV) as above, and (V) every block gathers its blocked
// share of the output from the blocks that computed it (staged in its T0
// region) and stores it.  This is the comparison schedule for what the
// elemental-cyclic distribution saves.
#include <cooperative_groups.h>

#include "pass_kernels.cuh"
#include "runtime_stages.cuh"

namespace cg = cooperative_groups;

namespace fft3 {

__global__ void k_vol(PassArgs a)
{
    extern __shared__ float2 smem[];
    cg::cluster_group cluster = cg::this_cluster();
    const int p = a.p;
    const int r = (int)cluster.block_rank();
    const int A = a.split_a, B = a.split_b, n = A * B;
    const int ap = A / p, bp = B / p;
    const LineRt &LB = a.L[0]; // DFT_b on rows
    const LineRt &LA = a.L[1]; // DFT_a on columns
    const int Pb = line_pitch(B), Pa = line_pitch(A);
    const int lpt = a.lpt;
    float2 *tw = smem;
    float2 *T0 = smem + a.tw_len;                 // lpt*ap rows of length b
    float2 *T1 = T0 + lpt * ap * Pb;              // lpt*bp columns of length a
    float2 *X = T1 + lpt * bp * Pa;               // ping-pong partner
    load_twiddles(tw, a.tw, a.tw_len);
    const float2 *W = tw + a.tw_split_off;        // w_n^m, m < n
    const bool conj = a.conj != 0;
    const bool contig = a.g.ij == 1;
    const int64_t cid = blockIdx.x / p, ncl = gridDim.x / p;
    for (int64_t tile = cid; tile < a.ntiles; tile += ncl) {
        __syncthreads();
        const TileId id = decode_tile(tile, a.tiles_c, a.g.A, lpt);
        const int64_t nval = min((int64_t)lpt, a.g.C - id.c0);
        const float2 *ib = a.in + id.c0 * a.g.ic + id.a * a.g.ia + id.b * a.g.ib;
        const int cnt0 = lpt * ap * B;
        const int share = n / p; // elements of a line per block
        if (!a.six_step) {
            // load this block's cyclic share: rows i0 = r + p*u
            for (int e = threadIdx.x; e < cnt0; e += blockDim.x) {
                int l, u, i1;
                if (contig) { u = e % ap; int q = e / ap; i1 = q % B; l = q / B; }
                else { l = e % lpt; int q = e / lpt; i1 = q % B; u = q / B; }
                const int j = r + p * u + A * i1;
                float2 v = make_float2(0.f, 0.f);
                if (l < nval)
                    v = ib[l * a.g.ic + (int64_t)j * a.g.ij];
                T0[(l * ap + u) * Pb + padpos(i1)] = conj ? cconj(v) : v;
            }
        } else {
            // load this block's blocked share j = r*share + jj into T1 as [l][jj]
            for (int e = threadIdx.x; e < lpt * share; e += blockDim.x) {
                int l, jj;
                if (contig) { jj = e % share; l = e / share; }
                else { l = e % lpt; jj = e / lpt; }
                float2 v = make_float2(0.f, 0.f);
                if (l < nval)
                    v = ib[l * a.g.ic + (int64_t)(r * share + jj) * a.g.ij];
                T1[l * share + jj] = conj ? cconj(v) : v;
            }
            cluster.sync();
            // exchange (0): row i0 = r + p*u gathers x[i0 + A*i1] from block j / share
            for (int e = threadIdx.x; e < cnt0; e += blockDim.x) {
                const int i1 = e % B, q = e / B, u = q % ap, l = q / ap;
                const int j = r + p * u + A * i1;
                const float2 *src = cluster.map_shared_rank(T1, j / share);
                T0[(l * ap + u) * Pb + padpos(i1)] = src[l * share + j % share];
            }
            cluster.sync(); // every block's staged input is read before T1 is reused
        }
        __syncthreads();
        // (I) DFT_b on every local row
        float2 *R0 = run_stages_lines(LB, lpt * ap, Pb, T0, X, tw + LB.tw_off);
        // (II) twiddle w_n^{i0 k1}
        for (int e = threadIdx.x; e < lpt * ap * B; e += blockDim.x) {
            const int k1 = e % B, row = e / B, u = row % ap;
            const int i0 = r + p * u;
            float2 *q = R0 + row * Pb + padpos(k1);
            *q = cmul(*q, W[(i0 * k1) % n]);
        }
        cluster.sync();
        // (III) exchange: column k1 = r + p*v gathers T0[i0][k1] from block i0 mod p
        for (int e = threadIdx.x; e < lpt * bp * A; e += blockDim.x) {
            const int i0 = e % A, q = e / A, v = q % bp, l = q / bp;
            const int owner = i0 % p, u = i0 / p, k1 = r + p * v;
            const float2 *src = cluster.map_shared_rank(R0, owner);
            T1[(l * bp + v) * Pa + padpos(i0)] = src[(l * ap + u) * Pb + padpos(k1)];
        }
        cluster.sync();
        // (IV) DFT_a on every local column
        float2 *R1 = run_stages_lines(LA, lpt * bp, Pa, T1, X, tw + LA.tw_off);
        float2 *ob = a.out + id.c0 * a.g.oc + id.a * a.g.oa + id.b * a.g.ob;
        if (a.six_step) {
            cluster.sync(); // every block's columns are transformed
            // exchange (V): output k = r*share + kk, k = k1 + B*k0, computed by
            // block k1 mod p as its column v = k1 / p; staged in T0 as [l][kk]
            for (int e = threadIdx.x; e < lpt * share; e += blockDim.x) {
                const int kk = e % share, l = e / share;
                const int k = r * share + kk, k1 = k % B, k0 = k / B;
                const float2 *src = cluster.map_shared_rank(R1, k1 % p);
                T0[l * share + kk] = src[(l * bp + k1 / p) * Pa + padpos(k0)];
            }
            cluster.sync(); // the peers' results are read before the next tile reuses them
            for (int e = threadIdx.x; e < lpt * share; e += blockDim.x) {
                int l, kk;
                if (contig) { kk = e % share; l = e / share; }
                else { l = e % lpt; kk = e / lpt; }
                if (l < nval) {
                    const float2 val = T0[l * share + kk];
                    ob[l * a.g.oc + (int64_t)(r * share + kk) * a.g.ok] = conj ? cconj(val) : val;
                }
            }
            continue;
        }
        const int cnt1 = lpt * bp * A;
        for (int e = threadIdx.x; e < cnt1; e += blockDim.x) {
            int l, v, k0;
            if (contig) { v = e % bp; int q = e / bp; k0 = q % A; l = q / A; }
            else { l = e % lpt; int q = e / lpt; k0 = q % A; v = q / A; }
            if (l < nval) {
                const int k = r + p * v + B * k0;
                const float2 val = R1[(l * bp + v) * Pa + padpos(k0)];
                ob[l * a.g.oc + (int64_t)k * a.g.ok] = conj ? cconj(val) : val;
            }
        }
    }
}

} // namespace fft3
