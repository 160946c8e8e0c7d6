// planner.cpp -- lowers a decomposition of the 3D DFT to a schedule of passes.
//
// Decompositions (paper Sections 2.3, 2.4 and 3.2):
//   pencil-pencil-pencil  DFT_{n0}, then DFT_{n1}, then DFT_{n2}.  Three variants:
//     natural: the x pass writes `out`, the y and z passes run in place on
//              strided lines of `out` (tiles of adjacent columns);
//     rotate:  each pass reads contiguous lines and stores its result rotated,
//              xyz -> yzx -> zxy -> xyz (Section 2.4), so the next pass's lines
//              are contiguous again; the rotation is the store epilogue;
//     blocked: the y pass stores into a workspace laid out [x/16][z][y][x%16]
//              (a redistribution fused into its store, Section 3.1), so each of
//              its 16-column tiles is one contiguous block and the z pass reads
//              rows 16*n1 values apart instead of n0*n1; the z pass stores the
//              natural layout.  The default of FFT3_AUTO where it applies.
//   slab-pencil           2D DFT of every n0 x n1 slab (x lines then y lines
//                         on data kept on chip or in L2), then DFT_{n2}.
//   volumetric            every dimension's 1D DFT split n = a*b (Eq. ct) over
//                         a cluster of p blocks that hold the line in
//                         elemental-cyclic order; one exchange per dimension
//                         when p | a and p | b (Section 3.2).
// Parallelism limits of Section 2.5 become the tile counts of each pass; the
// divisibility condition of Section 3.2 is checked for every volumetric split.
#include "planner.h"

#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <sstream>

#include "plans.h"
#include "roots.cuh"

namespace fft3 {

// ------------------------------------------------------ fixed-plan table -- //
#define FFT3_META_ROW(ID, N, T, ...) {ID, N, T, 0, {__VA_ARGS__}},
static FixedPlanMeta g_meta[] = {FFT3_FIXED_PLANS(FFT3_META_ROW)};
#undef FFT3_META_ROW
static const int g_nmeta = (int)(sizeof(g_meta) / sizeof(g_meta[0]));

static void init_meta()
{
    static bool done = false;
    if (done)
        return;
    for (int i = 0; i < g_nmeta; ++i) {
        int c = 0;
        while (c < 8 && g_meta[i].rad[c] > 0)
            ++c;
        g_meta[i].nrad = c;
    }
    done = true;
}

#define FFT3_VOLC_META(N, A, B, P, LPT, TA, RA, TB, RB) {N, A, B, P, LPT, LPT *(A / P) * TB, TA, TB, {RA}, {RB}, nullptr},
static const VolcKernel g_volc_meta[] = {FFT3_VOLC_LIST(FFT3_VOLC_META)};
#undef FFT3_VOLC_META

const VolcKernel *volc_meta(int *count)
{
    *count = (int)(sizeof(g_volc_meta) / sizeof(g_volc_meta[0]));
    return g_volc_meta;
}

#define FFT3_CSTREAM_META(N, Q, R1, R2, G, S, LPT, P) {N, Q, R1, R2, G, S, LPT, P, G * LPT * R2, nullptr, {nullptr, nullptr}},
static const CStreamKernel g_cstream_meta[] = {FFT3_CSTREAM_LIST(FFT3_CSTREAM_META)};
#undef FFT3_CSTREAM_META

const CStreamKernel *cstream_meta(int *count)
{
    *count = (int)(sizeof(g_cstream_meta) / sizeof(g_cstream_meta[0]));
    return g_cstream_meta;
}

int fixed_plan_count() { return g_nmeta; }
const FixedPlanMeta &fixed_plan_meta(int id)
{
    init_meta();
    return g_meta[id];
}

static inline int tw_slots_h(int len) { return ((len > 0 ? len : 1) + 15) / 16 * 16; }
static inline int padpos_h(int p) { return p + (p >> 4); }
static inline int pitch_h(int n) { return (padpos_h(n - 1) + 1) | 1; }

// ----------------------------------------------------------- factorise --- //
static bool smooth235(int n, int *e2, int *e3, int *e5)
{
    *e2 = *e3 = *e5 = 0;
    if (n < 1)
        return false;
    while (n % 2 == 0) { n /= 2; ++*e2; }
    while (n % 3 == 0) { n /= 3; ++*e3; }
    while (n % 5 == 0) { n /= 5; ++*e5; }
    return n == 1;
}

int factorize(int n, int order, int *rad, int cap)
{
    int e2, e3, e5;
    if (!smooth235(n, &e2, &e3, &e5))
        return FFT3_ERR_UNSUPPORTED_SIZE;
    std::vector<int> r;
    int mode = order % 4;
    if (mode == 0 || mode == 1) { // radix 16 first, then 8/4/2, then 5s and 3s
        for (int i = 0; i < e2 / 4; ++i) r.push_back(16);
        if (e2 % 4) r.push_back(1 << (e2 % 4));
        for (int i = 0; i < e5; ++i) r.push_back(5);
        for (int i = 0; i < e3; ++i) r.push_back(3);
        if (mode == 1) std::reverse(r.begin(), r.end());
    } else if (mode == 2) { // radix 4 first
        for (int i = 0; i < e2 / 2; ++i) r.push_back(4);
        if (e2 % 2) r.push_back(2);
        for (int i = 0; i < e3; ++i) r.push_back(3);
        for (int i = 0; i < e5; ++i) r.push_back(5);
    } else { // radix 8 first
        for (int i = 0; i < e2 / 3; ++i) r.push_back(8);
        if (e2 % 3) r.push_back(1 << (e2 % 3));
        for (int i = 0; i < e3; ++i) r.push_back(3);
        for (int i = 0; i < e5; ++i) r.push_back(5);
    }
    if ((int)r.size() > cap)
        return FFT3_ERR_UNSUPPORTED_SIZE;
    for (size_t i = 0; i < r.size(); ++i)
        rad[i] = r[i];
    return (int)r.size();
}

// Candidates for a line: fixed plans of that length (in table order).
static std::vector<int> fixed_candidates(int n)
{
    init_meta();
    std::vector<int> c;
    for (int i = 0; i < g_nmeta; ++i)
        if (g_meta[i].n == n)
            c.push_back(i);
    return c;
}

static int choose_line(int n, int order, bool allow_fixed, LineChoice *lc, std::string *err)
{
    lc->n = n;
    std::vector<int> fc = allow_fixed ? fixed_candidates(n) : std::vector<int>();
    if (!fc.empty()) {
        const FixedPlanMeta &m = g_meta[fc[order % fc.size()]];
        lc->fixed = m.id;
        lc->T = m.T;
        lc->nst = m.nrad;
        for (int i = 0; i < m.nrad; ++i)
            lc->rad[i] = m.rad[i];
        return FFT3_OK;
    }
    if (n > kMaxLine) {
        *err = "line length " + std::to_string(n) + " exceeds " + std::to_string(kMaxLine);
        return FFT3_ERR_UNSUPPORTED_SIZE;
    }
    int k = factorize(n, order, lc->rad, kMaxStages);
    if (k < 0) {
        *err = "line length " + std::to_string(n) + " has a prime factor other than 2, 3, 5";
        return k;
    }
    lc->fixed = -1;
    lc->nst = k;
    int maxr = 1;
    for (int i = 0; i < k; ++i)
        maxr = std::max(maxr, lc->rad[i]);
    lc->T = std::max(1, n / maxr);
    return FFT3_OK;
}

// Stage-major twiddle exponents of a line choice (fft_engine.cuh header).
static void line_twiddles(const LineChoice &lc, std::vector<int64_t> *m)
{
    int64_t total = 0, NS = 1;
    for (int s = 0; s < lc.nst; ++s) {
        total += (lc.rad[s] - 1) * NS;
        NS *= lc.rad[s];
    }
    for (int64_t e = 0; e < total; ++e)
        m->push_back(stage_twiddle_exponent(lc.n, lc.rad, lc.nst, e));
}

static int add_seg(Schedule *s, int n, std::vector<int64_t> m)
{
    TwSeg seg;
    seg.n = n;
    seg.m = std::move(m);
    seg.off = s->tw_total;
    s->tw_total += ((int64_t)seg.m.size() + 15) / 16 * 16;
    s->tw.push_back(std::move(seg));
    return (int)s->tw.size() - 1;
}

static int line_seg(Schedule *s, const LineChoice &lc)
{
    std::vector<int64_t> m;
    line_twiddles(lc, &m);
    if (m.empty())
        m.push_back(0);
    return add_seg(s, lc.n, std::move(m));
}

void generic_launch_shape_elem(int n, int T, bool strided, int tw_len, int esize, int *lpt, int *threads,
                               int *smem)
{
    int P = pitch_h(n);
    // strided lines: tiles of 16 (complex64) or 8 (complex128) columns, 128-byte rows
    int l = strided ? 128 / esize : std::max(1, 256 / T);
    while (l > 1 && T * l > 1024)
        l /= 2;
    auto bytes = [&](int ll) { return tw_slots_h(tw_len) * esize + 2 * ll * P * esize; };
    while (l > 1 && bytes(l) > kSmemLimit)
        l /= 2;
    *lpt = l;
    *threads = std::max(32, std::min(1024, (T * l + 31) / 32 * 32));
    *smem = bytes(l);
}

void generic_launch_shape(int n, int T, bool strided, int tw_len, int *lpt, int *threads, int *smem)
{
    generic_launch_shape_elem(n, T, strided, tw_len, 8, lpt, threads, smem);
}

// --------------------------------------------------------- geometries ---- //
static PassGeom geom_natural(int d, int64_t n0, int64_t n1, int64_t n2, int64_t batch)
{
    PassGeom g{};
    int64_t N = n0 * n1 * n2;
    if (d == 0) { // x lines: c = y, a = z, b = batch
        g.C = n1; g.A = n2; g.B = batch;
        g.ij = 1; g.ic = n0; g.ia = n0 * n1; g.ib = N;
    } else if (d == 1) { // y lines: c = x, a = z, b = batch
        g.C = n0; g.A = n2; g.B = batch;
        g.ij = n0; g.ic = 1; g.ia = n0 * n1; g.ib = N;
    } else { // z lines: c = x + n0*y, a = batch
        g.C = n0 * n1; g.A = batch; g.B = 1;
        g.ij = n0 * n1; g.ic = 1; g.ia = N; g.ib = 0;
    }
    g.ok = g.ij; g.oc = g.ic; g.oa = g.ia; g.ob = g.ib;
    return g;
}

// Rotation xyz -> yzx -> zxy -> xyz (Section 2.4).  Pass d reads the layout in
// which dimension d is fastest and writes the layout in which d+1 is fastest.
static PassGeom geom_rotate(int d, int64_t n0, int64_t n1, int64_t n2, int64_t batch)
{
    int64_t n[3] = {n0, n1, n2};
    int64_t da = n[d], db = n[(d + 1) % 3], dc = n[(d + 2) % 3];
    PassGeom g{};
    int64_t N = n0 * n1 * n2;
    // input layout (da fastest, then db, then dc); lines along da:
    // c = index along db, a = index along dc, b = batch
    g.C = db; g.A = dc; g.B = batch;
    g.ij = 1; g.ic = da; g.ia = da * db; g.ib = N;
    // output layout (db fastest, then dc, then da)
    g.oc = 1; g.oa = db; g.ok = db * dc; g.ob = N;
    return g;
}

static void set_tiles(PassPlan *p)
{
    p->tiles_c = (p->g.C + p->lpt - 1) / p->lpt;
    p->ntiles = p->tiles_c * p->g.A * p->g.B;
}

// The TMA-pipelined strided kernel needs the same geometry on both sides,
// 16-byte multiples for every stride TMA walks, whole tiles and whole boxes.
static bool tma_ok(const PassGeom &g, int n, int lpt)
{
    if (lpt <= 0 || g.ic != 1 || g.oc != 1 || g.ij != g.ok || g.ia != g.oa || g.ib != g.ob)
        return false;
    if (g.C % lpt || (g.ij * 8) % 16 || (g.ia * 8) % 16 || (g.B > 1 && (g.ib * 8) % 16))
        return false;
    int br = n < 256 ? n : 256;
    if (n % br)
        return false;
    if (g.C > 0x7fffffff || g.A > 0x7fffffff || g.B > 0x7fffffff)
        return false;
    return 2 * n * lpt * 8 + 8192 * 8 <= kSmemLimit;
}

// Streamed strided pass for a line of length n: the compiled entry for n
// picked by `order` among the entries for n, if the input geometry suits its
// TMA map {C, Q, M, A, B} (16-byte multiples for every stride the map walks).
// `pair` = 1 keeps each line in one block (a pencil pass); `pair` = 2 takes
// the entries whose line is split over a cluster of two blocks (a volumetric
// split of the line, Section 3.2).
static int cstream_pick(int n, int order, const PassGeom &g, int pair)
{
    if (g.ic != 1 || g.oc != 1 || (g.ij * 8) % 16 || (g.ia * 8) % 16 || (g.B > 1 && (g.ib * 8) % 16))
        return -1;
    if (g.C > 0x7fffffff || g.A > 0x7fffffff || g.B > 0x7fffffff)
        return -1;
    int cnt = 0;
    const CStreamKernel *m = cstream_meta(&cnt);
    std::vector<int> ids;
    for (int i = 0; i < cnt; ++i)
        if (m[i].n == n && m[i].pair == pair &&
            cstream_smem_p(n, m[i].q, m[i].q / m[i].pair, m[i].lpt, m[i].groups * m[i].stages) <= kSmemLimit)
            ids.push_back(i);
    if (ids.empty())
        return -1;
    return ids[(size_t)std::max(0, order) % ids.size()];
}

// Kind, tile, line and launch shape of a streamed pass with compiled entry ci.
static void set_cstream(PassPlan *p, int ci)
{
    int cnt = 0;
    const CStreamKernel &m = cstream_meta(&cnt)[ci];
    p->kind = PK_CSTREAM;
    p->cstream = ci;
    p->lpt = m.lpt;
    p->p = m.pair;
    p->line = LineChoice{};
    p->line.n = m.n;
    p->line.fixed = -1;
    p->line.T = m.threads / m.lpt;
    p->line.nst = 3;
    p->line.rad[0] = m.r1;
    p->line.rad[1] = m.r2;
    p->line.rad[2] = m.q;
    p->threads = m.threads;
    p->smem_bytes = cstream_smem_p(m.n, m.q, m.q / m.pair, m.lpt, m.groups * m.stages);
}

// Kind, tile, line, twiddles and launch shape of a tcgen05 radix-32 pass of
// 1024-point lines (k_tc32.cu): twiddles w_1024^{j2 k1} stored [k1][j2], then
// w_32^m for the DFT_32 operand.
static void set_tc32(Schedule *s, PassPlan *p, int kind)
{
    p->kind = kind;
    p->lpt = kind == PK_TCX ? kTc32Lpt : kTcsLpt;
    p->threads = kTc32Threads;
    p->smem_bytes = kind == PK_TCX ? kTc32SmemBytes : kTcsSmemBytes;
    p->tc_mode = 0;
    p->line = LineChoice{};
    p->line.n = 1024;
    p->line.fixed = -1;
    p->line.T = 32;
    p->line.nst = 2;
    p->line.rad[0] = p->line.rad[1] = 32;
    std::vector<int64_t> tw(1024), w32(32);
    for (int i = 0; i < 1024; ++i)
        tw[i] = (int64_t)(i % 32) * (i / 32);
    for (int i = 0; i < 32; ++i)
        w32[i] = i;
    p->tw_seg[0] = add_seg(s, 1024, std::move(tw));
    p->tw_seg[2] = add_seg(s, 32, std::move(w32));
    set_tiles(p);
}

// A single 1D pass on dimension d with geometry g.
static int make_line_pass(Schedule *s, int d, int n, const PassGeom &g, bool rotate, int src, int dst,
                          PassPlan *out, std::string *err)
{
    PassPlan p;
    p.dim = d;
    p.g = g;
    p.src = src;
    p.dst = dst;
    int order = s->opts.radix_order;
    int rc = choose_line(n, order, true, &p.line, err);
    if (rc)
        return rc;
    const bool contig_in = g.ij == 1;
    const bool strided_in = g.ic == 1 && g.oc == 1;
    if (g.ijb > 0 || g.okb > 0) {
        // lines in runs over exchange blocks: the runtime-radix kernels
        rc = choose_line(n, order, false, &p.line, err);
        if (rc)
            return rc;
        const bool c128 = s->dtype == FFT3_C128_FP64;
        p.kind = c128 ? PK_G64 : PK_G;
        p.tw_seg[0] = line_seg(s, p.line);
        generic_launch_shape_elem(n, p.line.T, !contig_in, (int)s->tw[p.tw_seg[0]].m.size(), c128 ? 16 : 8,
                                  &p.lpt, &p.threads, &p.smem_bytes);
        if (p.smem_bytes > kSmemLimit) {
            *err = "pass needs more shared memory than a block has";
            return FFT3_ERR_UNSUPPORTED_SIZE;
        }
        set_tiles(&p);
        *out = p;
        return FFT3_OK;
    }
    // tc_stages 0: the tcgen05 radix-32 kernels for 1024-point lines, the first
    // shared-memory radix-16 stage (mma.sync) elsewhere; 1, 2: the mma.sync
    // radix-16 modes; 3: the first shared-memory radix-16 stage everywhere
    const int tc_opt = s->opts.tc_stages;
    const int tc_mode = tc_opt == 3 ? 0 : std::min(2, std::max(0, tc_opt));
    if (s->dtype == FFT3_C128_FP64) {
        // complex128, 16-byte elements: the compile-time FP64 passes (k_pass64.cu)
        // where the length has a fixed plan, else the runtime radix list (k_pass_g64)
        const bool contig = contig_in && g.ok == 1;
        if (p.line.fixed >= 0 && !rotate && (contig || (strided_in && p.line.T * kLpt64Strided <= 1024))) {
            p.kind = contig ? PK_J64 : PK_C64;
            p.tw_seg[0] = line_seg(s, p.line);
            const int twl = tw_slots_h((int)s->tw[p.tw_seg[0]].m.size());
            p.lpt = contig ? lpt_j(p.line.T) : kLpt64Strided;
            p.threads = p.line.T * p.lpt;
            p.smem_bytes = (twl + (contig ? p.lpt * pitch_h(n) : p.lpt * n)) * 16;
            if (p.smem_bytes <= kSmemLimit) {
                set_tiles(&p);
                *out = p;
                return FFT3_OK;
            }
        }
        rc = choose_line(n, order, false, &p.line, err);
        if (rc)
            return rc;
        p.kind = PK_G64;
        p.tw_seg[0] = line_seg(s, p.line);
        generic_launch_shape_elem(n, p.line.T, !contig_in, (int)s->tw[p.tw_seg[0]].m.size(), 16, &p.lpt,
                                  &p.threads, &p.smem_bytes);
        if (p.smem_bytes > kSmemLimit) {
            *err = "pass needs more shared memory than a block has";
            return FFT3_ERR_UNSUPPORTED_SIZE;
        }
        set_tiles(&p);
        *out = p;
        return FFT3_OK;
    }
    if (s->dtype == FFT3_C64_SPLITBF16_TC && !rotate && n == 1024 && tc_opt == 0 && s->opts.tile_lines == 0) {
        // both 32-point stages of the line as split-BF16 GEMMs on the tcgen05 tensor cores
        // (k_tc32.cu): contiguous lines whose 4-line tiles are one bulk copy, or strided
        // columns in 16-column tiles the 5D tensor map walks (16-byte multiples for
        // every stride)
        const bool al = (g.ia * 8) % 16 == 0 && (g.B <= 1 || (g.ib * 8) % 16 == 0);
        const bool lines = contig_in && g.ic == n && al;
        const bool cols = strided_in && (g.ij * 8) % 16 == 0 && al && g.C <= 0x7fffffff && g.A <= 0x7fffffff &&
                          g.B <= 0x7fffffff;
        if (lines || cols) {
            set_tc32(s, &p, lines ? PK_TCX : PK_TCS);
            *out = p;
            return FFT3_OK;
        }
    }
    if (s->dtype == FFT3_C64_SPLITBF16_TC && !rotate && strided_in && n > 1 && s->opts.tile_lines == 0) {
        // streamed strided pass whose 16 x 16 sub-line transforms run on the tensor cores
        int cnt = 0;
        const CStreamKernel *cm = cstream_meta(&cnt);
        const int ci = cstream_pick(n, order, g, 1);
        int tci = -1;
        for (int i = 0; i < cnt && tci < 0; ++i)
            if (cm[i].n == n && cm[i].pair == 1 && cm[i].r1 == 16 && cm[i].r2 == 16 && ci >= 0)
                tci = i;
        if (tci >= 0) {
            set_cstream(&p, tci);
            p.tc_mode = tc_mode;
            p.tw_seg[0] = line_seg(s, p.line);
            std::vector<int64_t> w16(16);
            for (int i = 0; i < 16; ++i)
                w16[i] = i;
            p.tw_seg[2] = add_seg(s, 16, std::move(w16)); // w_16^m for the DFT_16 matrix
            p.smem_bytes += 16 * 8;
            set_tiles(&p);
            *out = p;
            return FFT3_OK;
        }
    }
    if (s->dtype == FFT3_C64_SPLITBF16_TC && !rotate && n >= 128) {
        // prefer a candidate plan that has tensor-core kernels for this layout
        std::vector<int> fc = fixed_candidates(n);
        for (size_t k = 0; k < fc.size(); ++k) {
            const FixedPlanMeta &m = g_meta[fc[(k + order) % fc.size()]];
            const bool has16 = tc_mask_host(m.rad, m.nrad, tc_mode) != 0;
            const bool jok = contig_in && g.ok == 1 && tc_j_ok(n, m.T, has16);
            const bool cok = strided_in && tc_c_ok(n, m.T, has16);
            if (!jok && !cok)
                continue;
            p.line.n = n;
            p.line.fixed = m.id;
            p.line.T = m.T;
            p.line.nst = m.nrad;
            for (int i = 0; i < m.nrad; ++i)
                p.line.rad[i] = m.rad[i];
            p.kind = jok ? PK_JTC : PK_CTC;
            p.lpt = jok ? lpt_j(m.T) : lpt_c_tc();
            p.tc_mode = tc_mode;
            p.tw_seg[0] = line_seg(s, p.line);
            std::vector<int64_t> w16(16);
            for (int i = 0; i < 16; ++i)
                w16[i] = i;
            p.tw_seg[2] = add_seg(s, 16, std::move(w16));
            const int twl = tw_slots_h((int)s->tw[p.tw_seg[0]].m.size()) + 16;
            p.threads = m.T * p.lpt;
            p.smem_bytes = twl * 8 + 2 * p.lpt * (jok ? pitch_h(n) : n) * 8;
            set_tiles(&p);
            *out = p;
            return FFT3_OK;
        }
    }
    // strided tiles: 16 adjacent columns (128-byte rows) unless 8 are asked for;
    // lengths with a compiled streamed kernel use it unless tile_lines asks for
    // another (kTileTma: the TMA double-buffered kernel, 8/16: the plain one)
    int want_c = s->opts.tile_lines == 8 ? 8 : 16;
    if (p.line.fixed >= 0 && rotate && contig_in && g.oc == 1) {
        p.kind = PK_JROT;
        p.lpt = lpt_rot(p.line.T);
    } else if (p.line.fixed >= 0 && !rotate && contig_in && g.ok == 1 && n > 1) {
        p.kind = PK_J;
        p.lpt = lpt_j(p.line.T);
    } else if (!rotate && strided_in && n > 1 && (s->opts.tile_lines == 0 || s->opts.tile_lines == kTileStream) &&
               cstream_pick(n, order, g, 1) >= 0) {
        set_cstream(&p, cstream_pick(n, order, g, 1));
    } else if (p.line.fixed >= 0 && !rotate && strided_in && n > 1 && s->opts.tile_lines == kTileTma &&
               tma_ok(g, n, lpt_tma(n, p.line.T))) {
        p.kind = PK_CTMA;
        p.lpt = lpt_tma(n, p.line.T);
    } else if (p.line.fixed >= 0 && !rotate && strided_in && lpt_c(p.line.T, want_c) > 0 && n > 1) {
        p.kind = PK_C;
        p.lpt = lpt_c(p.line.T, want_c);
    } else {
        // runtime radix list (also used for n == 1 layout changes)
        if (p.line.fixed >= 0) {
            LineChoice lc;
            rc = choose_line(n, order, false, &lc, err);
            if (rc)
                return rc;
            p.line = lc;
        }
        p.kind = PK_G;
    }
    p.tw_seg[0] = line_seg(s, p.line);
    int tw_len = (int)s->tw[p.tw_seg[0]].m.size();
    if (p.kind == PK_G) {
        generic_launch_shape(n, p.line.T, !contig_in, tw_len, &p.lpt, &p.threads, &p.smem_bytes);
    } else if (p.kind == PK_J) {
        p.threads = p.line.T * p.lpt;
        p.smem_bytes = tw_slots_h(tw_len) * 8 + p.lpt * pitch_h(n) * 8;
    } else if (p.kind == PK_JROT) {
        p.threads = p.line.T * p.lpt;
        p.smem_bytes = tw_slots_h(tw_len) * 8 + p.lpt * pitch_h(n) * 8;
    } else if (p.kind == PK_CTMA) {
        p.threads = p.line.T * p.lpt;
        p.smem_bytes = tw_slots_h(tw_len) * 8 + 2 * p.lpt * n * 8;
    } else if (p.kind == PK_CSTREAM) {
        // launch shape set with the kind
    } else {
        p.threads = p.line.T * p.lpt;
        p.smem_bytes = tw_slots_h(tw_len) * 8 + p.lpt * n * 8;
    }
    if (p.smem_bytes > kSmemLimit) {
        *err = "pass needs more shared memory than a block has";
        return FFT3_ERR_UNSUPPORTED_SIZE;
    }
    set_tiles(&p);
    *out = p;
    return FFT3_OK;
}

// Volumetric split of a line of length n over p blocks: n = a*b with p | a
// and p | b (Section 3.2).  Prefers a close to sqrt(n).
static bool volumetric_split(int n, int p, int *a, int *b)
{
    int best = -1;
    for (int aa = p; aa <= n; aa += p) {
        if (n % aa)
            continue;
        int bb = n / aa;
        if (bb % p)
            continue;
        if (best < 0 || std::abs(aa - bb) < std::abs(best - n / best) ||
            (std::abs(aa - bb) == std::abs(best - n / best) && aa > best))
            best = aa;
    }
    if (best < 0)
        return false;
    *a = best;
    *b = n / best;
    return true;
}

static int vol_smem(int p, int a, int b, int lpt, int twlen)
{
    int sub_b = lpt * (a / p) * pitch_h(b); // T0: lpt*(a/p) rows of length b
    int sub_a = lpt * (b / p) * pitch_h(a); // T1: lpt*(b/p) columns of length a
    int big = std::max(sub_a, sub_b);
    return twlen * 8 + (sub_b + sub_a + big) * 8;
}

static LineChoice fixed_line(int n, int T, const int *rad)
{
    LineChoice lc;
    lc.n = n;
    lc.fixed = -1;
    lc.T = T;
    lc.nst = 0;
    while (lc.nst < 4 && rad[lc.nst] > 0) {
        lc.rad[lc.nst] = rad[lc.nst];
        ++lc.nst;
    }
    return lc;
}

// Compile-time split of a strided line when one is compiled for (n, p).
static bool make_volc_pass(Schedule *s, int d, int n, int p, const PassGeom &g, int src, int dst, PassPlan *out)
{
    if (g.ic != 1 || g.oc != 1)
        return false;
    int cnt = 0;
    const VolcKernel *vk = volc_meta(&cnt);
    for (int i = 0; i < cnt; ++i) {
        // tile_lines (16, 32 or 64) picks the tile width; 0 takes the first compiled one
        if (vk[i].n != n || vk[i].p != p || (s->opts.tile_lines > 1 && vk[i].lpt != s->opts.tile_lines))
            continue;
        PassPlan q;
        q.kind = PK_VOLC;
        q.volc = i;
        q.dim = d;
        q.g = g;
        q.src = src;
        q.dst = dst;
        q.p = p;
        q.split_a = vk[i].a;
        q.split_b = vk[i].b;
        q.line = fixed_line(vk[i].b, vk[i].tb, vk[i].rb);  // DFT_B on rows
        q.line2 = fixed_line(vk[i].a, vk[i].ta, vk[i].ra); // DFT_A on columns
        q.tw_seg[0] = line_seg(s, q.line);
        q.tw_seg[1] = line_seg(s, q.line2);
        std::vector<int64_t> m(n);
        for (int k = 0; k < n; ++k)
            m[k] = k;
        q.tw_seg[2] = add_seg(s, n, std::move(m));
        int twlen = 0;
        for (int k = 0; k < 3; ++k)
            twlen += tw_slots_h((int)s->tw[q.tw_seg[k]].m.size());
        q.lpt = vk[i].lpt;
        q.threads = vk[i].threads;
        q.smem_bytes = twlen * 8 + 2 * (n / p) * q.lpt * 8;
        set_tiles(&q);
        *out = q;
        return true;
    }
    return false;
}

static int make_vol_pass(Schedule *s, int d, int n, int p, const PassGeom &g, int src, int dst,
                         PassPlan *out, std::string *err)
{
    // a strided line split over a cluster pair whose halves of the decimated
    // sub-lines stream in by TMA (k_cstream.cu), unless tile_lines asks for
    // the compiled splits of k_volc.cu
    // the blocked six-step comparison schedule runs on the runtime-radix cluster kernel
    const bool six = s->opts.variant == FFT3_VOL_BLOCKED_SIX_STEP;
    const int ci = !six && p == 2 && s->opts.tile_lines <= kTileStream ? cstream_pick(n, s->opts.radix_order, g, 2)
                                                                       : -1;
    if (ci >= 0) {
        PassPlan q;
        q.dim = d;
        q.g = g;
        q.src = src;
        q.dst = dst;
        set_cstream(&q, ci);
        q.tw_seg[0] = line_seg(s, q.line);
        set_tiles(&q);
        *out = q;
        return FFT3_OK;
    }
    if (!six && make_volc_pass(s, d, n, p, g, src, dst, out))
        return FFT3_OK;
    PassPlan q;
    q.kind = PK_VOL;
    q.six_step = six;
    q.dim = d;
    q.g = g;
    q.src = src;
    q.dst = dst;
    q.p = p;
    if (!volumetric_split(n, p, &q.split_a, &q.split_b)) {
        *err = "volumetric split of " + std::to_string(n) + " over " + std::to_string(p) +
               " blocks needs n = a*b with p | a and p | b";
        return FFT3_ERR_UNSUPPORTED_SIZE;
    }
    int rc = choose_line(q.split_b, s->opts.radix_order, false, &q.line, err); // rows: DFT_b
    if (rc)
        return rc;
    rc = choose_line(q.split_a, s->opts.radix_order, false, &q.line2, err); // columns: DFT_a
    if (rc)
        return rc;
    q.tw_seg[0] = line_seg(s, q.line);
    q.tw_seg[1] = line_seg(s, q.line2);
    std::vector<int64_t> m(n);
    for (int i = 0; i < n; ++i)
        m[i] = i; // w_n^i, indexed by (i0*k1) mod n
    q.tw_seg[2] = add_seg(s, n, std::move(m));
    int twlen = 0;
    for (int k = 0; k < 3; ++k)
        twlen += tw_slots_h((int)s->tw[q.tw_seg[k]].m.size());
    const bool strided = g.ic == 1;
    int lpt = strided ? (s->opts.tile_lines == 8 ? 8 : 16) : std::max(1, 512 / std::max(1, n / p / 4));
    while (lpt > 1 && vol_smem(p, q.split_a, q.split_b, lpt, twlen) > kSmemLimit)
        lpt /= 2;
    q.lpt = lpt;
    q.smem_bytes = vol_smem(p, q.split_a, q.split_b, lpt, twlen);
    if (q.smem_bytes > kSmemLimit) {
        *err = "volumetric pass does not fit in shared memory";
        return FFT3_ERR_UNSUPPORTED_SIZE;
    }
    q.threads = std::max(256, (std::max(q.line.T, q.line2.T) + 31) / 32 * 32);
    set_tiles(&q);
    *out = q;
    return FFT3_OK;
}

// Slab 2D pass in one block's shared memory: fits when two copies of the
// padded slab fit.
static int slab_smem(int n0, int n1, int twlen) { return twlen * 8 + 2 * n1 * pitch_h(n0) * 8; }

static int make_slab_pass(Schedule *s, int n0, int n1, int64_t n2, int64_t batch, PassPlan *out,
                          std::string *err)
{
    PassPlan q;
    q.kind = PK_SLAB;
    q.dim = 3;
    q.src = BUF_IN;
    q.dst = BUF_OUT;
    int rc = choose_line(n0, s->opts.radix_order, false, &q.line, err);
    if (rc)
        return rc;
    rc = choose_line(n1, s->opts.radix_order, false, &q.line2, err);
    if (rc)
        return rc;
    q.tw_seg[0] = line_seg(s, q.line);
    q.tw_seg[1] = line_seg(s, q.line2);
    int twlen = tw_slots_h((int)s->tw[q.tw_seg[0]].m.size()) +
                tw_slots_h((int)s->tw[q.tw_seg[1]].m.size());
    q.smem_bytes = slab_smem(n0, n1, twlen);
    if (q.smem_bytes > kSmemLimit)
        return FFT3_ERR_UNSUPPORTED_SIZE;
    int64_t N = (int64_t)n0 * n1 * n2;
    // one slab per tile; slabs indexed by (a = z, b = batch)
    q.g = PassGeom{};
    q.g.C = 1; q.g.A = n2; q.g.B = batch;
    q.g.ij = 1; q.g.ic = 0; q.g.ia = (int64_t)n0 * n1; q.g.ib = N;
    q.g.ok = 1; q.g.oc = 0; q.g.oa = q.g.ia; q.g.ob = N;
    q.lpt = 1;
    int teams = std::max(1, std::max(n1, n0));
    int T = std::max(q.line.T, q.line2.T);
    // enough threads for one team of the longer line, up to 512 for the rest
    q.threads = std::min(512, std::max(64, (teams * T + 31) / 32 * 32));
    q.threads = std::max(q.threads, (T + 31) / 32 * 32);
    set_tiles(&q);
    *out = q;
    return FFT3_OK;
}

// Slab pass with x and y tiles in one persistent launch, the slab kept in L2
// between its x and y stages (compiled for square slabs with a fixed plan).
static bool slab_l2_supported(int n0, int n1) { return n0 == n1 && (n0 == 1024 || n0 == 512 || n0 == 256); }

static int make_slab_l2_pass(Schedule *s, int n0, int n1, int64_t n2, int64_t batch, PassPlan *out,
                             std::string *err)
{
    PassPlan q;
    q.kind = PK_SLABL2;
    q.dim = 3;
    q.src = BUF_IN;
    q.dst = BUF_OUT;
    int rc = choose_line(n0, s->opts.radix_order, true, &q.line, err);
    if (rc)
        return rc;
    q.line2 = q.line;
    if (q.line.fixed < 0)
        return FFT3_ERR_UNSUPPORTED_SIZE;
    q.tw_seg[0] = line_seg(s, q.line);
    int twlen = tw_slots_h((int)s->tw[q.tw_seg[0]].m.size());
    q.lpt = kSlabL2Lpt;
    q.threads = q.line.T * q.lpt;
    if (q.threads > 1024)
        return FFT3_ERR_UNSUPPORTED_SIZE;
    q.smem_bytes = twlen * 8 + q.lpt * pitch_h(n0) * 8;
    int64_t N = (int64_t)n0 * n1 * n2;
    q.g = PassGeom{};
    q.g.C = n1; q.g.A = n2; q.g.B = batch;
    q.g.ij = 1; q.g.ic = n0; q.g.ia = (int64_t)n0 * n1; q.g.ib = N;
    q.g.ok = 1; q.g.oc = n0; q.g.oa = q.g.ia; q.g.ob = N;
    q.tiles_c = n1 / q.lpt; // x tiles per slab (= y tiles per slab for square slabs)
    q.ntiles = 2 * q.tiles_c * n2 * batch;
    *out = q;
    return FFT3_OK;
}

// Slab stage fused with the slab-to-pencil redistribution: x and y tiles of
// every square slab in one persistent launch (k_slab_blk), from `in` into the
// workspace laid out as z pencils [x/16][z][y][x%16].
static int make_slab_blk_pass(Schedule *s, int n0, int n1, int64_t n2, PassPlan *out, std::string *err)
{
    PassPlan q;
    int rc = make_slab_l2_pass(s, n0, n1, n2, 1, &q, err);
    if (rc)
        return rc;
    q.kind = PK_SLABBLK;
    q.dst = BUF_WS;
    q.g.ok = 1; q.g.oc = 16; q.g.oa = (int64_t)n1 * 16; q.g.ob = (int64_t)n1 * 16 * n2;
    // rows per x tile = columns per y tile; transforming warps + one producer
    // warp; twiddles, the padded work buffer and the ring of landing buffers
    // (k_slab_tma)
    const int want = s->opts.slab_lines;
    if (want != 0 && want != 4 && want != 8) {
        *err = "slab_lines must be 0, 4 or 8";
        return FFT3_ERR_INVALID_ARG;
    }
    q.lpt = want == 8 ? 8 : 4;
    q.threads = q.line.T * q.lpt + 32;
    const int twlen = tw_slots_h((int)s->tw[q.tw_seg[0]].m.size());
    q.smem_bytes = (twlen + (q.lpt * pitch_h(n0) + 15) / 16 * 16 + kSlabTmaBufs * q.lpt * n0) * 8;
    if (q.smem_bytes > kSmemLimit || q.threads > 1024)
        return FFT3_ERR_UNSUPPORTED_SIZE;
    q.tiles_c = n1 / q.lpt;
    q.ntiles = 2 * q.tiles_c * n2;
    *out = q;
    return FFT3_OK;
}

int layout_position(int layout, int64_t n0, int64_t n1, int64_t n2, int64_t batch, int64_t idx, int64_t *pos)
{
    const int64_t N = n0 * n1 * n2;
    if (idx < 0 || idx >= N * batch)
        return FFT3_ERR_INVALID_ARG;
    const int64_t b = idx / N, r = idx % N;
    const int64_t k0 = r % n0, k1 = (r / n0) % n1, k2 = r / (n0 * n1);
    switch (layout) {
    case FFT3_LAYOUT_NATURAL: *pos = idx; return FFT3_OK;
    case FFT3_LAYOUT_ROTATED: *pos = k2 + n2 * (k0 + n0 * k1) + N * b; return FFT3_OK;
    case FFT3_LAYOUT_PENCILS:
        if (batch != 1 || n0 % 16)
            return FFT3_ERR_UNSUPPORTED_SIZE;
        *pos = (k0 / 16) * 16 * n1 * n2 + k2 * 16 * n1 + k1 * 16 + k0 % 16;
        return FFT3_OK;
    default: return FFT3_ERR_INVALID_ARG;
    }
}

// Rank-local stages of the slab-pencil decomposition over a 1D grid of P
// processes (Section 2.4): the slab stage (the rank's n2/P slabs, 2D DFT) and
// the pencil stage (the z lines of the rank's n0/P x columns), with the
// all-to-all between them left to the caller.  The packing for the exchange
// is the slab stage's y-pass store: x = d*Xl + xl goes to block d as
// [d][z_local][y][x_local], and the receiving rank's blocks [src][z_local][y][x_local]
// are its natural [z][y][x_local] pencils, so no stage has a separate pack
// or unpack.  The inverse runs the pencil stage first (its natural output is
// already split by z into the blocks for each rank) and the slab stage last,
// reading the packed blocks.
static int build_dist_stage(Schedule *s, std::string *err)
{
    const int P = s->opts.dist_ranks, stage = s->opts.dist_stage;
    const int64_t n0 = s->n0, n1 = s->n1, n2 = s->n2;
    if (s->dtype != FFT3_C64_FP32 && s->dtype != FFT3_C128_FP64) {
        *err = "the distributed slab-pencil stages run in complex64 or complex128";
        return FFT3_ERR_UNSUPPORTED_SIZE;
    }
    if (s->batch != 1 || s->opts.layout != FFT3_LAYOUT_NATURAL) {
        *err = "the distributed slab-pencil stages need batch 1 and the natural layout";
        return FFT3_ERR_UNSUPPORTED_SIZE;
    }
    s->decomp = FFT3_SLAB_PENCIL;
    const bool fwd = s->direction == FFT3_FORWARD;
    PassPlan p;
    int rc = FFT3_OK;
    auto push = [&](int d, int n, const PassGeom &g, int src, int dst) {
        if (!rc)
            rc = make_line_pass(s, d, n, g, false, src, dst, &p, err);
        if (!rc)
            s->passes.push_back(p);
    };
    if (stage == 2) {
        // z lines of the rank's (n0/P) x n1 x n2 pencils, natural on both sides
        if (n2 > 1)
            push(2, (int)n2, geom_natural(2, n0, n1, n2, 1), BUF_IN, BUF_OUT);
        return rc;
    }
    if (n0 % P) {
        *err = "the slab stage needs the rank count to divide n0";
        return FFT3_ERR_UNSUPPORTED_SIZE;
    }
    const int64_t Xl = n0 / P;
    if (stage == 3) {
        // the second exchange's local side: packed blocks [d][z_local][y][x_local] to
        // natural slabs (forward, after the exchange) or back (inverse, before it), as
        // a pass of one-point lines: c = x_local, a = z_local*n1 + y, b = d
        PassGeom g{};
        g.C = Xl; g.A = n2 * n1; g.B = P;
        g.ij = 1; g.ok = 1; g.ic = 1; g.oc = 1;
        const int64_t pa = Xl, pb = n2 * n1 * Xl, na = n0, nb = Xl;
        g.ia = fwd ? pa : na; g.ib = fwd ? pb : nb;
        g.oa = fwd ? na : pa; g.ob = fwd ? nb : pb;
        push(0, 1, g, BUF_IN, BUF_OUT);
        return rc;
    }
    // y lines, columns xl of block d (a = z_local, b = d): natural n0 x n1 x n2 slabs on
    // one side, the packed blocks [d][z_local][y][x_local] on the other
    PassGeom nat{}, pk{};
    nat.C = pk.C = Xl; nat.A = pk.A = n2; nat.B = pk.B = P;
    nat.ij = n0; nat.ic = 1; nat.ia = n0 * n1; nat.ib = Xl;
    pk.ij = Xl; pk.ic = 1; pk.ia = n1 * Xl; pk.ib = n2 * n1 * Xl;
    PassGeom gy{};
    gy.C = Xl; gy.A = n2; gy.B = P;
    if (fwd) {
        gy.ij = nat.ij; gy.ic = nat.ic; gy.ia = nat.ia; gy.ib = nat.ib;
        gy.ok = pk.ij; gy.oc = pk.ic; gy.oa = pk.ia; gy.ob = pk.ib;
        push(0, (int)n0, geom_natural(0, n0, n1, n2, 1), BUF_IN, BUF_WS);
        push(1, (int)n1, gy, BUF_WS, BUF_OUT);
    } else {
        gy.ij = pk.ij; gy.ic = pk.ic; gy.ia = pk.ia; gy.ib = pk.ib;
        gy.ok = nat.ij; gy.oc = nat.ic; gy.oa = nat.ia; gy.ob = nat.ib;
        push(1, (int)n1, gy, BUF_IN, BUF_WS);
        push(0, (int)n0, geom_natural(0, n0, n1, n2, 1), BUF_WS, BUF_OUT);
    }
    s->need_ws = true;
    return rc;
}

// Rank-local stages of the pencil-pencil-pencil decomposition on a Py x Pz
// grid (Section 2.4): each stage is one pass of one dimension's lines whose
// store packs the blocks of the next all-to-all (the x pass by its rotated
// store xyz -> yzx, the y pass by storing y slowest), while the line the next
// stage reads arrives in Py (or Pz) runs, one per sending rank: the
// two-level line index of the pass geometry (ijb, iblk) reads it in place.
// Sizes: Xl = n0/Py, Yl = n1/Py, Yl2 = n1/Pz, Zl = n2/Pz; the plan's own
// dims are the rank's local array (stage 1: n0 x Yl x Zl, stage 2:
// Xl x n1 x Zl, stage 3: Xl x Yl2 x n2).  The inverse stores what the
// forward stage reads and reads what it stores.
static int build_dist_ppp(Schedule *s, std::string *err)
{
    const int Py = s->opts.dist_ranks, Pz = std::max(1, s->opts.dist_ranks2), stage = s->opts.dist_stage;
    const int64_t n0 = s->n0, n1 = s->n1, n2 = s->n2;
    if (s->dtype != FFT3_C64_FP32 && s->dtype != FFT3_C128_FP64) {
        *err = "the distributed pencil-pencil-pencil stages run in complex64 or complex128";
        return FFT3_ERR_UNSUPPORTED_SIZE;
    }
    if (s->batch != 1 || s->opts.layout != FFT3_LAYOUT_NATURAL) {
        *err = "the distributed pencil-pencil-pencil stages need batch 1 and the natural layout";
        return FFT3_ERR_UNSUPPORTED_SIZE;
    }
    s->decomp = FFT3_PENCIL3;
    const bool fwd = s->direction == FFT3_FORWARD;
    PassPlan p;
    int rc = FFT3_OK;
    auto push = [&](int d, int n, const PassGeom &g, bool rot) {
        if (!rc)
            rc = make_line_pass(s, d, n, g, rot, BUF_IN, BUF_OUT, &p, err);
        if (!rc)
            s->passes.push_back(p);
    };
    PassGeom g{};
    if (stage == 1) { // local n0 x Yl x Zl
        if (n0 % Py) {
            *err = "the x stage needs Py to divide n0";
            return FFT3_ERR_UNSUPPORTED_SIZE;
        }
        const int64_t Yl = n1, Zl = n2;
        if (fwd) {
            push(0, (int)n0, geom_rotate(0, n0, Yl, Zl, 1), true); // [x][z][y]: x blocks contiguous
        } else {
            g.C = Yl; g.A = Zl; g.B = 1;
            g.ij = Zl * Yl; g.ic = 1; g.ia = Yl;
            g.ok = 1; g.oc = n0; g.oa = n0 * Yl;
            push(0, (int)n0, g, false);
        }
    } else if (stage == 2) { // local Xl x n1 x Zl
        if (n1 % Py || n1 % Pz) {
            *err = "the y stage needs Py and Pz to divide n1";
            return FFT3_ERR_UNSUPPORTED_SIZE;
        }
        const int64_t Xl = n0, Zl = n2, Yl = n1 / Py;
        g.C = Xl; g.A = Zl; g.B = 1;
        if (fwd) {
            // in: [src][x][z][y_local], y = src Yl + y_local; out: [y][z][x]
            g.ij = 1; g.ijb = Yl; g.iblk = Xl * Zl * Yl; g.ic = Zl * Yl; g.ia = Yl;
            g.ok = Zl * Xl; g.oc = 1; g.oa = Xl;
        } else {
            g.ij = Zl * Xl; g.ic = 1; g.ia = Xl;
            g.ok = 1; g.okb = Yl; g.oblk = Xl * Zl * Yl; g.oc = Zl * Yl; g.oa = Yl;
        }
        push(1, (int)n1, g, false);
    } else { // stage 3, local Xl x Yl2 x n2
        if (n2 % Pz) {
            *err = "the z stage needs Pz to divide n2";
            return FFT3_ERR_UNSUPPORTED_SIZE;
        }
        const int64_t Xl = n0, Yl2 = n1, Zl = n2 / Pz;
        g.C = Xl; g.A = Yl2; g.B = 1;
        if (fwd) {
            // in: [src][y][z_local][x], z = src Zl + z_local; out: natural [z][y][x]
            g.ij = Xl; g.ijb = Zl; g.iblk = Yl2 * Zl * Xl; g.ic = 1; g.ia = Zl * Xl;
            g.ok = Xl * Yl2; g.oc = 1; g.oa = Xl;
        } else {
            g.ij = Xl * Yl2; g.ic = 1; g.ia = Xl;
            g.ok = Xl; g.okb = Zl; g.oblk = Yl2 * Zl * Xl; g.oc = 1; g.oa = Zl * Xl;
        }
        push(2, (int)n2, g, false);
    }
    return rc;
}

int build_schedule(int n0, int n1, int n2, int batch, int dtype, int decomp, int direction,
                   const fft3_options *opts, Schedule *out, std::string *err)
{
    init_meta();
    if (n0 < 1 || n1 < 1 || n2 < 1 || batch < 1) {
        *err = "sizes and batch must be positive";
        return FFT3_ERR_INVALID_ARG;
    }
    if (direction != FFT3_FORWARD && direction != FFT3_INVERSE) {
        *err = "direction must be FFT3_FORWARD (-1) or FFT3_INVERSE (+1)";
        return FFT3_ERR_INVALID_ARG;
    }
    if (dtype != FFT3_C64_FP32 && dtype != FFT3_C64_SPLITBF16_TC && dtype != FFT3_C128_FP64) {
        *err = "unknown dtype";
        return FFT3_ERR_INVALID_ARG;
    }
    if (decomp < 0 || decomp > FFT3_AUTO) {
        *err = "unknown decomposition";
        return FFT3_ERR_INVALID_ARG;
    }
    int ns[3] = {n0, n1, n2};
    for (int d = 0; d < 3; ++d) {
        int e2, e3, e5;
        if (!smooth235(ns[d], &e2, &e3, &e5)) {
            *err = "dimension " + std::to_string(ns[d]) + " has a prime factor other than 2, 3, 5";
            return FFT3_ERR_UNSUPPORTED_SIZE;
        }
        if (ns[d] > kMaxLine) {
            *err = "dimension " + std::to_string(ns[d]) + " exceeds " + std::to_string(kMaxLine);
            return FFT3_ERR_UNSUPPORTED_SIZE;
        }
    }
    Schedule s;
    s.n0 = n0; s.n1 = n1; s.n2 = n2; s.batch = batch;
    s.dtype = dtype; s.direction = direction;
    if (opts)
        s.opts = *opts;
    {
        const int dr = s.opts.dist_ranks, dr2 = s.opts.dist_ranks2, st = s.opts.dist_stage;
        const bool ppp = decomp == FFT3_PENCIL3;
        const bool bad = dr < 0 || dr2 < 0 || st < 0 || st > 3 ||
                         (st == 0 ? (dr > 1 || dr2 > 1)
                                  : ppp ? (dr < 1 || (int64_t)dr * std::max(1, dr2) < 2) : (dr < 2 || dr2 > 1));
        if (bad) {
            *err = "dist_stage 1, 2 or 3 goes with dist_ranks > 1 (slab-pencil) or a grid dist_ranks x "
                   "dist_ranks2 of more than one rank (pencil-pencil-pencil); all 0 for a one-GPU plan";
            return FFT3_ERR_INVALID_ARG;
        }
    }
    if (s.opts.dist_stage != 0) {
        if (decomp != FFT3_SLAB_PENCIL && decomp != FFT3_AUTO && decomp != FFT3_PENCIL3) {
            *err = "rank-local stages exist for the slab-pencil and pencil-pencil-pencil decompositions";
            return FFT3_ERR_UNSUPPORTED_SIZE;
        }
        int rc = decomp == FFT3_PENCIL3 ? build_dist_ppp(&s, err) : build_dist_stage(&s, err);
        if (rc)
            return rc;
        if (s.passes.empty()) {
            PassPlan p;
            p.kind = PK_COPY;
            p.src = BUF_IN;
            p.dst = BUF_OUT;
            p.g = PassGeom{};
            p.g.C = (int64_t)n0 * n1 * n2;
            p.g.A = 1; p.g.B = 1;
            p.g.ij = 1; p.g.ok = 1;
            p.threads = 256;
            s.passes.push_back(p);
        }
        *out = std::move(s);
        return FFT3_OK;
    }
    if (dtype == FFT3_C128_FP64) {
        // complex128 runs every line transform as one pass of the runtime-radix
        // FP64 kernel: pencil-pencil-pencil in natural order (the slab-pencil
        // and automatic choices lower to the same three passes)
        if (decomp == FFT3_VOLUMETRIC || s.opts.variant != FFT3_PPP_NATURAL ||
            s.opts.layout != FFT3_LAYOUT_NATURAL) {
            *err = "complex128 runs the natural pencil-pencil-pencil schedule";
            return FFT3_ERR_UNSUPPORTED_SIZE;
        }
        decomp = FFT3_PENCIL3;
    }
    if (decomp == FFT3_AUTO && dtype == FFT3_C64_SPLITBF16_TC) {
        decomp = FFT3_PENCIL3;
        if (s.opts.variant == FFT3_PPP_NATURAL && (int64_t)n0 * n1 * 8 >= (4ll << 20))
            s.opts.variant = FFT3_PPP_BLOCKED;
    }
    if (decomp == FFT3_AUTO) {
        // Fixed default when no cost model is loaded: slab-pencil when a whole
        // slab fits one block's shared memory (one HBM sweep fewer), else
        // pencil-pencil-pencil, whose strided passes stream their sub-lines
        // (measured faster than the L2-resident slab kernel at 1024 x 1024).
        int twl = 2 * tw_slots_h(n0) + 2 * tw_slots_h(n1);
        decomp = slab_smem(n0, n1, twl) <= kSmemLimit ? FFT3_SLAB_PENCIL : FFT3_PENCIL3;
        // and with the blocked intermediate when it applies and the natural z lines
        // would be at least 4 MiB apart (1024^3: 8.68 against 9.41 ms; at 512^3, 2 MiB
        // apart, the natural layout measured 1.053 against 1.067 ms)
        if (decomp == FFT3_PENCIL3 && s.opts.variant == FFT3_PPP_NATURAL && (int64_t)n0 * n1 * 8 >= (4ll << 20))
            s.opts.variant = FFT3_PPP_BLOCKED;
    }
    if (dtype == FFT3_C64_SPLITBF16_TC) {
        if (decomp != FFT3_PENCIL3 || s.opts.variant == FFT3_PPP_ROTATE) {
            *err = "the split-BF16 tensor-core path runs the pencil-pencil-pencil decomposition (natural or blocked)";
            return FFT3_ERR_UNSUPPORTED_SIZE;
        }
    }
    s.decomp = decomp;
    int64_t N = (int64_t)n0 * n1 * n2;
    int rc = FFT3_OK;
    int cur = BUF_IN;
    auto add_nat = [&](int d) -> int {
        if (ns[d] == 1)
            return FFT3_OK;
        PassPlan p;
        int r = make_line_pass(&s, d, ns[d], geom_natural(d, n0, n1, n2, batch), false, cur, BUF_OUT,
                               &p, err);
        if (r)
            return r;
        s.passes.push_back(p);
        cur = BUF_OUT;
        return FFT3_OK;
    };
    // Blocked intermediate (FFT3_PPP_BLOCKED): x pass natural, y pass from `out`
    // into the workspace laid out as [x/16][z][y][x%16] (a 16-column tile of y
    // lines is one contiguous block), z pass from the workspace back to `out`.
    auto blocked_fits = [&]() {
        if (!(batch == 1 && n0 % 16 == 0 && n1 > 1 && n2 > 1 &&
              (s.opts.tile_lines == 0 || s.opts.tile_lines == kTileStream)))
            return false;
        int cnt = 0;
        const CStreamKernel *cm = cstream_meta(&cnt);
        bool y = false, z = false;
        for (int i = 0; i < cnt; ++i) {
            y = y || (cm[i].n == n1 && cm[i].pair == 1 && cm[i].lpt == 16);
            z = z || (cm[i].n == n2 && cm[i].pair == 1 && cm[i].lpt == 16);
        }
        return y && z;
    };
    auto emit_blocked_z = [&]() -> int {
        const int64_t X = n0, Y = n1, Z = n2;
        PassPlan p;
        PassGeom gz{}; // columns x%16, lines z, a = y, b = x/16
        gz.C = 16; gz.A = Y; gz.B = X / 16;
        gz.ij = Y * 16; gz.ic = 1; gz.ia = 16; gz.ib = Z * Y * 16;
        gz.ok = X * Y; gz.oc = 1; gz.oa = X; gz.ob = 16;
        rc = make_line_pass(&s, 2, n2, gz, false, BUF_WS, BUF_OUT, &p, err);
        if (rc)
            return rc;
        s.passes.push_back(p);
        s.need_ws = true;
        return FFT3_OK;
    };
    auto emit_blocked = [&]() -> int {
        const int64_t X = n0, Y = n1, Z = n2;
        PassPlan p;
        rc = make_line_pass(&s, 0, n0, geom_natural(0, n0, n1, n2, batch), false, BUF_IN, BUF_OUT, &p, err);
        if (rc)
            return rc;
        s.passes.push_back(p);
        PassGeom gy{}; // columns x%16, lines y, a = x/16, b = z
        gy.C = 16; gy.A = X / 16; gy.B = Z;
        gy.ij = X; gy.ic = 1; gy.ia = 16; gy.ib = X * Y;
        gy.ok = 16; gy.oc = 1; gy.oa = Z * Y * 16; gy.ob = Y * 16;
        rc = make_line_pass(&s, 1, n1, gy, false, BUF_OUT, BUF_WS, &p, err);
        if (rc)
            return rc;
        s.passes.push_back(p);
        return emit_blocked_z();
    };
    const int layout = s.opts.layout;
    if (layout < FFT3_LAYOUT_NATURAL || layout > FFT3_LAYOUT_PENCILS) {
        *err = "unknown layout";
        return FFT3_ERR_INVALID_ARG;
    }
    if (layout != FFT3_LAYOUT_NATURAL) {
        // Permuted spectrum (Section 2.4): the forward plan leaves out the last
        // redistribution, the inverse plan starts from the permuted layout.
        if (decomp == FFT3_VOLUMETRIC) {
            *err = "permuted layouts come from the slab-pencil and pencil-pencil-pencil schedules";
            return FFT3_ERR_UNSUPPORTED_SIZE;
        }
        if (n0 < 2 || n1 < 2 || n2 < 2) {
            *err = "permuted layouts need every dimension > 1";
            return FFT3_ERR_UNSUPPORTED_SIZE;
        }
        const bool fwd = direction == FFT3_FORWARD;
        auto push = [&](int d, int n, const PassGeom &g, bool rot, int src, int dst) -> int {
            PassPlan p;
            int r = make_line_pass(&s, d, n, g, rot, src, dst, &p, err);
            if (!r)
                s.passes.push_back(p);
            return r;
        };
        if (layout == FFT3_LAYOUT_ROTATED) {
            if (dtype == FFT3_C64_SPLITBF16_TC) {
                *err = "the rotated layout has no split-BF16 tensor-core schedule";
                return FFT3_ERR_UNSUPPORTED_SIZE;
            }
            if (fwd) {
                // x and y passes rotate (xyz -> yzx -> zxy); the z pass transforms the
                // contiguous z lines of zxy in place of the final rotation
                rc = push(0, n0, geom_rotate(0, n0, n1, n2, batch), true, BUF_IN, BUF_OUT);
                if (!rc)
                    rc = push(1, n1, geom_rotate(1, n0, n1, n2, batch), true, BUF_OUT, BUF_WS);
                if (!rc)
                    rc = push(2, n2, geom_natural(0, n2, n0, n1, batch), false, BUF_WS, BUF_OUT);
            } else {
                // z lines are contiguous in zxy: transform them and rotate zxy -> xyz,
                // then the natural x and y passes
                rc = push(2, n2, geom_rotate(2, n0, n1, n2, batch), true, BUF_IN, BUF_WS);
                if (!rc)
                    rc = push(0, n0, geom_natural(0, n0, n1, n2, batch), false, BUF_WS, BUF_OUT);
                if (!rc)
                    rc = push(1, n1, geom_natural(1, n0, n1, n2, batch), false, BUF_OUT, BUF_OUT);
            }
        } else {
            if (batch != 1 || n0 % 16) {
                *err = "the pencils layout needs batch 1 and n0 % 16 == 0";
                return FFT3_ERR_UNSUPPORTED_SIZE;
            }
            const int64_t X = n0, Y = n1, Z = n2;
            PassGeom gb{}; // z lines of the blocked layout on both sides: columns x%16, a = y, b = x/16
            gb.C = 16; gb.A = Y; gb.B = X / 16;
            gb.ij = Y * 16; gb.ic = 1; gb.ia = 16; gb.ib = Z * Y * 16;
            gb.ok = gb.ij; gb.oc = 1; gb.oa = 16; gb.ob = gb.ib;
            if (fwd) {
                if (decomp == FFT3_SLAB_PENCIL && s.opts.slab_mode == 5 && slab_l2_supported(n0, n1)) {
                    PassPlan p;
                    rc = make_slab_blk_pass(&s, n0, n1, n2, &p, err);
                    if (!rc)
                        s.passes.push_back(p);
                } else {
                    PassGeom gy{}; // as the blocked schedule: y lines from `out` into the workspace
                    gy.C = 16; gy.A = X / 16; gy.B = Z;
                    gy.ij = X; gy.ic = 1; gy.ia = 16; gy.ib = X * Y;
                    gy.ok = 16; gy.oc = 1; gy.oa = Z * Y * 16; gy.ob = Y * 16;
                    rc = push(0, n0, geom_natural(0, n0, n1, n2, 1), false, BUF_IN, BUF_OUT);
                    if (!rc)
                        rc = push(1, n1, gy, false, BUF_OUT, BUF_WS);
                }
                if (!rc)
                    rc = push(2, n2, gb, false, BUF_WS, BUF_OUT);
            } else {
                PassGeom gyi{}; // y lines of the blocked workspace into natural order
                gyi.C = 16; gyi.A = X / 16; gyi.B = Z;
                gyi.ij = 16; gyi.ic = 1; gyi.ia = Z * Y * 16; gyi.ib = Y * 16;
                gyi.ok = X; gyi.oc = 1; gyi.oa = 16; gyi.ob = X * Y;
                rc = push(2, n2, gb, false, BUF_IN, BUF_WS);
                if (!rc)
                    rc = push(1, n1, gyi, false, BUF_WS, BUF_OUT);
                if (!rc)
                    rc = push(0, n0, geom_natural(0, n0, n1, n2, 1), false, BUF_OUT, BUF_OUT);
            }
        }
        if (rc)
            return rc;
        s.need_ws = true;
    } else if (decomp == FFT3_PENCIL3 && s.opts.variant == FFT3_PPP_BLOCKED && blocked_fits()) {
        rc = emit_blocked();
        if (rc)
            return rc;
    } else if (decomp == FFT3_PENCIL3 && s.opts.variant == FFT3_PPP_ROTATE) {
        int bufs[3][2] = {{BUF_IN, BUF_OUT}, {BUF_OUT, BUF_WS}, {BUF_WS, BUF_OUT}};
        for (int d = 0; d < 3; ++d) {
            PassPlan p;
            rc = make_line_pass(&s, d, ns[d], geom_rotate(d, n0, n1, n2, batch), true, bufs[d][0],
                                bufs[d][1], &p, err);
            if (rc)
                return rc;
            s.passes.push_back(p);
        }
        s.need_ws = true;
    } else if (decomp == FFT3_PENCIL3) {
        for (int d = 0; d < 3 && !rc; ++d)
            rc = add_nat(d);
    } else if (decomp == FFT3_SLAB_PENCIL) {
        bool z_done = false;
        int mode = s.opts.slab_mode;
        int twl = 2 * tw_slots_h(n0) + 2 * tw_slots_h(n1);
        bool fits_smem = slab_smem(n0, n1, twl) <= kSmemLimit;
        if (mode == 0) // the L2-resident slab kernel measured slower than x and y passes (256^2 to 1024^2)
            mode = fits_smem ? 1 : 3;
        PassPlan p;
        if (mode == 1 && fits_smem) {
            rc = make_slab_pass(&s, n0, n1, n2, batch, &p, err);
            if (rc)
                return rc;
            s.passes.push_back(p);
            cur = BUF_OUT;
        } else if (mode == 2 && slab_l2_supported(n0, n1)) {
            rc = make_slab_l2_pass(&s, n0, n1, n2, batch, &p, err);
            if (rc)
                return rc;
            s.passes.push_back(p);
            cur = BUF_OUT;
        } else if (mode == 5 && slab_l2_supported(n0, n1) && batch == 1 && n2 > 1) {
            rc = make_slab_blk_pass(&s, n0, n1, n2, &p, err);
            if (rc)
                return rc;
            s.passes.push_back(p);
            rc = emit_blocked_z();
            if (rc)
                return rc;
            z_done = true;
        } else if (mode == 1 || mode == 2 || mode == 5) {
            *err = "requested slab mode is not available for this slab size";
            return FFT3_ERR_UNSUPPORTED_SIZE;
        } else if (mode == 4 && n0 > 1 && n1 > 1) {
            // x lines and y lines of chunks of slabs, pipelined on two streams:
            // the y lines of chunk c (read back from L2) run beside the x lines
            // of chunk c+1.  Chunks of about 32 MiB.
            rc = add_nat(0);
            if (!rc)
                rc = add_nat(1);
            if (!rc) {
                const int64_t slab_bytes = (int64_t)n0 * n1 * 8;
                const int64_t want = s.opts.slab_chunk > 0 ? s.opts.slab_chunk : (32ll << 20) / slab_bytes;
                const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(n2, want));
                PassPlan &px = s.passes[s.passes.size() - 2], &py = s.passes.back();
                px.chunk = chunk;
                py.chunk = chunk;
                px.pair_next = true;
            }
        } else if (blocked_fits() && (int64_t)n0 * n1 * 8 >= (4ll << 20)) {
            // slab stage as x and y passes; the y pass stores the slabs redistributed
            // into z pencils ([x/16][z][y][x%16]), the z pass reads them back (where
            // the natural z lines would be at least 4 MiB apart, as for FFT3_AUTO)
            rc = emit_blocked();
            if (rc)
                return rc;
            z_done = true;
        } else {
            // unfused slab stage: x lines then y lines as two passes
            rc = add_nat(0);
            if (!rc)
                rc = add_nat(1);
        }
        if (!rc && !z_done)
            rc = add_nat(2);
    } else { // volumetric
        for (int d = 0; d < 3 && !rc; ++d) {
            if (ns[d] == 1)
                continue;
            int p = s.opts.mesh[d];
            bool explicit_mesh = p > 0;
            if (!explicit_mesh) {
                // Automatic mesh: the contiguous dimension stays whole (a split
                // of it buys no coalescing on one GPU); a strided dimension is
                // split over 4 blocks where a compiled split exists, else over 2
                // (the paper's smallest mesh extent).
                // The streamed cluster-pair split (measured faster than the
                // compiled 4-block splits) comes first.
                int cnt = 0;
                const VolcKernel *vk = volc_meta(&cnt);
                p = 2;
                for (int i = 0; i < cnt; ++i)
                    if (vk[i].n == ns[d] && vk[i].p == 4)
                        p = 4;
                if (cstream_pick(ns[d], 0, geom_natural(d, n0, n1, n2, batch), 2) >= 0)
                    p = 2;
                int a, b;
                if (d == 0 || !volumetric_split(ns[d], p, &a, &b))
                    p = 1;
            }
            if (p != 1 && p != 2 && p != 4 && p != 8) {
                *err = "volumetric mesh extents must be 1, 2, 4 or 8";
                return FFT3_ERR_INVALID_ARG;
            }
            PassGeom g = geom_natural(d, n0, n1, n2, batch);
            PassPlan q;
            if (p == 1) {
                rc = make_line_pass(&s, d, ns[d], g, false, cur, BUF_OUT, &q, err);
            } else {
                rc = make_vol_pass(&s, d, ns[d], p, g, cur, BUF_OUT, &q, err);
            }
            if (rc)
                return rc;
            s.passes.push_back(q);
            cur = BUF_OUT;
        }
    }
    if (rc)
        return rc;
    if (s.passes.empty()) {
        PassPlan p;
        p.kind = PK_COPY;
        p.src = BUF_IN;
        p.dst = BUF_OUT;
        p.g = PassGeom{};
        p.g.C = N * batch;
        p.g.A = 1; p.g.B = 1;
        p.g.ij = 1; p.g.ok = 1;
        p.threads = 256;
        s.passes.push_back(p);
    }
    (void)N;
    *out = std::move(s);
    return FFT3_OK;
}

// ---------------------------------------------------------------- JSON --- //
static const char *kind_name(int k)
{
    static const char *names[] = {"line_contig", "line_contig_rotate", "line_strided", "line_runtime",
                                  "slab_smem", "slab_l2", "volumetric_split", "copy", "unused",
                                  "line_strided_tma", "line_contig_tc", "line_strided_tc",
                                  "volumetric_split_fixed", "line_strided_stream", "slab_l2_blocked",
                                  "line_runtime_fp64", "line_contig_fp64", "line_strided_fp64",
                                  "line_contig_r32_tc", "line_strided_r32_tc"};
    return (k >= 0 && k <= 19) ? names[k] : "?";
}
static const char *buf_name(int b)
{
    return b == BUF_IN ? "in" : (b == BUF_OUT ? "out" : "workspace");
}
static const char *decomp_name(int d)
{
    return d == FFT3_SLAB_PENCIL ? "slab_pencil"
           : d == FFT3_PENCIL3  ? "pencil_pencil_pencil"
           : d == FFT3_VOLUMETRIC ? "volumetric" : "auto";
}

static void line_json(std::ostringstream &o, const LineChoice &l)
{
    o << "{\"n\":" << l.n << ",\"fixed\":" << l.fixed << ",\"T\":" << l.T << ",\"radices\":[";
    for (int i = 0; i < l.nst; ++i)
        o << (i ? "," : "") << l.rad[i];
    o << "]}";
}

std::string Schedule::json() const
{
    std::ostringstream o;
    int64_t N = (int64_t)n0 * n1 * n2 * batch;
    o << "{\"dims\":[" << n0 << "," << n1 << "," << n2 << "],\"batch\":" << batch
      << ",\"dtype\":" << dtype << ",\"direction\":" << direction << ",\"decomposition\":\""
      << decomp_name(decomp) << "\",\"variant\":" << opts.variant << ",\"layout\":\""
      << (opts.layout == FFT3_LAYOUT_ROTATED ? "rotated" : opts.layout == FFT3_LAYOUT_PENCILS ? "pencils" : "natural")
      << "\""
      << ",\"dist_ranks\":" << opts.dist_ranks << ",\"dist_ranks2\":" << opts.dist_ranks2
      << ",\"dist_stage\":" << opts.dist_stage
      << ",\"workspace_bytes\":" << (need_ws ? N * 8 : 0) << ",\"hbm_sweeps\":" << passes.size()
      << ",\"twiddle_entries\":" << tw_total << ",\"passes\":[";
    for (size_t i = 0; i < passes.size(); ++i) {
        const PassPlan &p = passes[i];
        o << (i ? "," : "") << "{\"kind\":\""
          << (p.kind == PK_CSTREAM && p.tc_mode >= 0 ? "line_strided_stream_tc" : kind_name(p.kind))
          << "\",\"dim\":" << p.dim
          << ",\"src\":\"" << buf_name(p.src) << "\",\"dst\":\"" << buf_name(p.dst)
          << "\",\"line\":";
        line_json(o, p.line);
        if (p.kind == PK_SLAB || p.kind == PK_VOL || p.kind == PK_SLABL2 || p.kind == PK_VOLC ||
            p.kind == PK_SLABBLK) {
            o << ",\"line2\":";
            line_json(o, p.line2);
        }
        o << ",\"lpt\":" << p.lpt << ",\"threads\":" << p.threads << ",\"smem\":" << p.smem_bytes
          << ",\"tiles\":" << p.ntiles;
        if (p.kind == PK_VOL || p.kind == PK_VOLC)
            o << ",\"p\":" << p.p << ",\"a\":" << p.split_a << ",\"b\":" << p.split_b
              << ",\"exchanges\":" << (p.six_step ? 3 : 1);
        if (p.kind == PK_CSTREAM && p.p > 1)
            o << ",\"p\":" << p.p;
        if (p.kind == PK_JTC || p.kind == PK_CTC || (p.kind == PK_CSTREAM && p.tc_mode >= 0))
            o << ",\"tc_stages\":" << p.tc_mode << ",\"mma\":\"mma.sync.m16n8k16\"";
        if (p.kind == PK_TCX || p.kind == PK_TCS)
            o << ",\"mma\":\"tcgen05.mma m128n64k16\"";
        if (p.kind == PK_CSTREAM) {
            int cnt = 0;
            const CStreamKernel &m = cstream_meta(&cnt)[p.cstream];
            o << ",\"q\":" << m.q << ",\"m\":" << m.n / m.q << ",\"groups\":" << m.groups
              << ",\"staging\":" << m.groups * m.stages << ",\"cluster\":" << m.pair;
        }
        if (p.chunk > 0)
            o << ",\"chunk\":" << p.chunk << ",\"pipelined_with\":\"" << (p.pair_next ? "next" : "previous")
              << "\"";
        const PassGeom &g = p.g;
        o << ",\"geom\":{\"C\":" << g.C << ",\"A\":" << g.A << ",\"B\":" << g.B << ",\"ij\":" << g.ij
          << ",\"ic\":" << g.ic << ",\"ia\":" << g.ia << ",\"ib\":" << g.ib << ",\"ok\":" << g.ok
          << ",\"oc\":" << g.oc << ",\"oa\":" << g.oa << ",\"ob\":" << g.ob;
        if (g.oblk)
            o << ",\"oblk\":" << g.oblk;
        if (g.ijb)
            o << ",\"ijb\":" << g.ijb << ",\"iblk\":" << g.iblk;
        if (g.okb)
            o << ",\"okb\":" << g.okb;
        o << "}}";
    }
    o << "]}";
    return o.str();
}

} // namespace fft3

namespace fft3 {
int choose_runtime_line(int n, int order, LineChoice *lc, std::string *err)
{
    return choose_line(n, order, false, lc, err);
}
void line_twiddle_exponents(const LineChoice &lc, std::vector<int64_t> *m) { line_twiddles(lc, m); }
} // namespace fft3
