"""Batched uneven 3D DFTs in one persistent, graph-captured launch: parity of
every problem (small batches) or of a sample covering every size class (the
4096-problem batch) with the FP64 oracle, plus Parseval over all problems."""
import numpy as np
import pytest
import torch

import oracle
from paper_1904_10119_gb300 import fft3, synth
from tests.gpu_util import MAXABS_TOL, REL_L2_TOL

pytestmark = pytest.mark.gpu


def _layout(dims, gap=0):
    vols = [int(np.prod(d)) for d in dims]
    offs = np.zeros(len(dims), np.int64)
    offs[1:] = np.cumsum(np.asarray(vols[:-1]) + gap)
    return offs, int(offs[-1] + vols[-1])


def _check_problem(x, got, off, d, direction):
    n0, n1, n2 = (int(v) for v in d)
    N = n0 * n1 * n2
    ref = oracle.fft3(x[off:off + N], n0, n1, n2, sign=direction)
    g = got[off:off + N]
    rel, mx = oracle.rel_l2(g, ref), oracle.max_abs_ratio(g, ref)
    assert rel <= REL_L2_TOL and mx <= MAXABS_TOL, (d, rel, mx)


def _run(dims, offs, total, decomposition=fft3.FFT3_AUTO, direction=fft3.FFT3_FORWARD, tuning=None, seed=7):
    x = synth.uniform_c64(total, seed)
    xd = torch.from_numpy(x).cuda()
    out = torch.full_like(xd, complex(float("nan"), 0.0))
    h = fft3.fft3_plan_create_many(dims, offs, 0, decomposition, direction, tuning)
    try:
        fft3.fft3_plan_execute(h, xd.data_ptr(), out.data_ptr(), 0)
        torch.cuda.synchronize()
        assert fft3.fft3_plan_check(h) == 0
        assert fft3.fft3_plan_launches(h) == 1
        desc = fft3.fft3_plan_describe(h)
    finally:
        fft3.fft3_plan_destroy(h)
    return x, out.cpu().numpy(), desc


@pytest.mark.parametrize("decomp", [fft3.FFT3_AUTO, fft3.FFT3_SLAB_PENCIL, fft3.FFT3_PENCIL3])
@pytest.mark.parametrize("direction", [fft3.FFT3_FORWARD, fft3.FFT3_INVERSE])
def test_small_batch_every_problem(decomp, direction):
    dims = synth.batched_dims(48, 5)
    offs, total = _layout(dims, gap=3)
    x, got, desc = _run(dims, offs, total, decomp, direction)
    assert desc["problems"] == 48
    for off, d in zip(offs, dims):
        _check_problem(x, got, int(off), d, direction)


def test_tuning_codes_and_mixed_radix_shapes():
    dims = np.array([[16, 24, 40], [96, 80, 48], [30, 45, 27], [128, 16, 2], [1, 1, 1], [5, 1, 64], [2, 3, 5]])
    offs, total = _layout(dims)
    for code in [0, 1, 2, 1 | (3 << 2) | (1 << 5) | (2 << 8), 2 | (4 << 2) | (4 << 5) | (3 << 8),
                 2 | (2 << 2) | (2 << 5)]:
        x, got, _ = _run(dims, offs, total, tuning=[code] * len(dims), seed=code + 1)
        for off, d in zip(offs, dims):
            _check_problem(x, got, int(off), d, fft3.FFT3_FORWARD)


def test_graph_replay_and_buffer_change():
    dims = synth.batched_dims(20, 9)
    offs, total = _layout(dims)
    x = synth.uniform_c64(total, 3)
    xd = torch.from_numpy(x).cuda()
    o1, o2 = torch.empty_like(xd), torch.empty_like(xd)
    h = fft3.fft3_plan_create_many(dims, offs)
    try:
        for _ in range(2):
            fft3.fft3_plan_execute(h, xd.data_ptr(), o1.data_ptr(), 0)
        fft3.fft3_plan_execute(h, xd.data_ptr(), o2.data_ptr(), 0)  # re-captured for new buffers
        torch.cuda.synchronize()
        assert fft3.fft3_plan_check(h) == 0
    finally:
        fft3.fft3_plan_destroy(h)
    assert torch.equal(o1, o2)
    g = o1.cpu().numpy()
    for off, d in zip(offs, dims):
        _check_problem(x, g, int(off), d, fft3.FFT3_FORWARD)


def test_rejects_unsupported_problems():
    for dims in ([[7, 8, 8]], [[256, 8, 8]], [[0, 8, 8]]):
        with pytest.raises(fft3.Fft3Error) as e:
            fft3.fft3_plan_create_many(dims, [0])
        assert e.value.code in (-1, -2)


def test_4096_uneven_cubes_sampled_and_parseval():
    """4096 problems, dims i.i.d. from {16,...,96} (seed 7): at least 64
    problems covering every size class compared element by element, and
    Parseval's identity for every problem."""
    dims = synth.batched_dims(4096, 7)
    offs, total = _layout(dims)
    x, got, desc = _run(dims, offs, total, seed=7)
    assert desc["problems"] == 4096
    # sample: the first problem of every distinct (n0, n1, n2), then random ones up to 96
    seen, sample = set(), []
    for i, d in enumerate(map(tuple, dims)):
        if d not in seen:
            seen.add(d)
            sample.append(i)
    rng = np.random.default_rng(1)
    sample += list(rng.choice(len(dims), size=max(0, 96 - len(sample)), replace=False))
    assert len(set(int(v) for d in dims[sample] for v in d)) == 8
    for i in sample[:160]:
        _check_problem(x, got, int(offs[i]), dims[i], fft3.FFT3_FORWARD)
    # Parseval per problem
    x2 = np.abs(x.astype(np.complex128)) ** 2
    g2 = np.abs(got.astype(np.complex128)) ** 2
    for off, d in zip(offs, dims):
        N = int(np.prod(d))
        sx, sg = x2[off:off + N].sum(), g2[off:off + N].sum()
        assert abs(sg - N * sx) <= 1e-5 * N * sx


@pytest.mark.parametrize("gap", [0, 5])
@pytest.mark.parametrize("direction", [fft3.FFT3_FORWARD, fft3.FFT3_INVERSE])
def test_slab_executor_every_problem(gap, direction):
    """FFT3_TUNE_SLABZ: one persistent launch of slab items (x and y lines of
    one slab in shared memory) and z-tile items (read through L2 once the
    problem's slabs are done); every line length, every problem against the
    oracle, problems at aligned and odd offsets."""
    dims = np.vstack([synth.batched_dims(40, 13), [[8, 128, 16], [128, 8, 96], [24, 40, 8], [16, 16, 128],
                                                   [96, 96, 8]]])
    offs, total = _layout(dims, gap=gap)
    code = fft3.tune_code(1) | fft3.FFT3_TUNE_SLABZ
    x, got, desc = _run(dims, offs, total, direction=direction, tuning=[code] * len(dims), seed=4 + gap)
    assert desc["mode"] == "slab_executor" and desc["kernel_launches"] == 1
    assert desc["items"] < sum(int(d[2]) + -(-int(d[0] * d[1]) // 32) for d in dims)  # slabs / tiles grouped
    for off, d in zip(offs, dims):
        _check_problem(x, got, int(off), d, direction)


def test_slab_executor_4096_cubes_sampled_and_parseval():
    dims = synth.batched_dims(4096, 7)
    offs, total = _layout(dims)
    x, got, desc = _run(dims, offs, total, seed=7, tuning=[fft3.tune_code(1) | fft3.FFT3_TUNE_SLABZ] * len(dims))
    assert desc["mode"] == "slab_executor"
    rng = np.random.default_rng(2)
    seen, sample = set(), []
    for i, d in enumerate(map(tuple, dims)):
        if d not in seen:
            seen.add(d)
            sample.append(i)
    sample += list(rng.choice(len(dims), size=32, replace=False))
    for i in sample[:128]:
        _check_problem(x, got, int(offs[i]), dims[i], fft3.FFT3_FORWARD)
    x2 = np.abs(x.astype(np.complex128)) ** 2
    g2 = np.abs(got.astype(np.complex128)) ** 2
    for off, d in zip(offs, dims):
        N = int(np.prod(d))
        assert abs(g2[off:off + N].sum() - N * x2[off:off + N].sum()) <= 1e-5 * N * x2[off:off + N].sum()


@pytest.mark.parametrize("direction", [fft3.FFT3_FORWARD, fft3.FFT3_INVERSE])
def test_segmented_passes_every_problem(direction):
    """Tuning code decomposition field 3: the batch runs as three segmented
    passes (all x lines, then all y lines, then all z lines, one launch per
    line length), every problem checked against the oracle."""
    dims = np.vstack([synth.batched_dims(40, 11), [[8, 128, 16], [128, 8, 96], [24, 40, 8]]])
    offs, total = _layout(dims, gap=5)
    x, got, desc = _run(dims, offs, total, direction=direction, tuning=[3] * len(dims), seed=2)
    assert desc["mode"] == "segmented"
    classes = sum(len(set(int(v) for v in dims[:, d])) for d in range(3))
    assert desc["kernel_launches"] == classes
    # default x kernels: warp shuffles except at 64 and 128 points
    for L in desc["segmented_launches"]:
        want = "shared_memory" if L["dim"] > 0 or L["n"] in (64, 128) else "warp_shuffle"
        assert L["kernel"] == want, L
    for off, d in zip(offs, dims):
        _check_problem(x, got, int(off), d, direction)


@pytest.mark.parametrize("cand", [1, 2])
@pytest.mark.parametrize("gap", [0, 5])
@pytest.mark.parametrize("direction", [fft3.FFT3_FORWARD, fft3.FFT3_INVERSE])
def test_segmented_warp_shuffle_lines(cand, gap, direction):
    """Every line of the segmented passes by the warp-shuffle kernels (the
    radix_order field of the codes picks candidate `cand` of each length after
    the shared-memory kernel, for x lines and for y and z columns): every
    length, problems at 16-byte aligned offsets (128-bit loads and stores) and
    at odd offsets (8-byte fallback), every problem against the oracle."""
    xs = [8, 16, 24, 32, 40, 48, 64, 80, 96, 128]
    dims = np.array([[n, xs[(3 * i) % 4], 8 if i % 2 else 16] for i, n in enumerate(xs)] +
                    [[n, 16, 24] for n in xs[1:8]] + [[40, 8, 96], [96, 24, 8]])
    offs, total = _layout(dims, gap=gap)
    code = fft3.tune_code(3, cand)
    x, got, desc = _run(dims, offs, total, direction=direction, tuning=[code] * len(dims), seed=3 + cand)
    xl = [L for L in desc["segmented_launches"] if L["dim"] == 0]
    # 8-point lines have one warp-shuffle kernel, so candidate 2 wraps to the shared-memory one
    assert len(xl) == len(xs)
    assert all(L["kernel"] == "warp_shuffle" for L in desc["segmented_launches"] if cand == 1 or L["n"] != 8)
    assert all(L["R"] * L["L"] == L["n"] for L in desc["segmented_launches"] if L["kernel"] == "warp_shuffle")
    for off, d in zip(offs, dims):
        _check_problem(x, got, int(off), d, direction)


def test_auto_choice_replay_and_refusal():
    """FFT3_AUTO picks the slab executor for a large batch whose lengths all
    have its line variants and whose slabs fit an item's room, the segmented
    passes when a slab does not fit (128 x 128), and the executor for a small
    batch; replay on new buffers gives the same bits; a line length without a
    compiled plan is refused when the codes ask for the segmented passes."""
    dims = synth.batched_dims(200, 4)
    offs, total = _layout(dims)
    x = synth.uniform_c64(total, 8)
    xd = torch.from_numpy(x).cuda()
    o1, o2 = torch.empty_like(xd), torch.empty_like(xd)
    h = fft3.fft3_plan_create_many(dims, offs)
    try:
        desc = fft3.fft3_plan_describe(h)
        assert desc["mode"] == "slab_executor" and desc["kernel_launches"] == 1
        fft3.fft3_plan_execute(h, xd.data_ptr(), o1.data_ptr(), 0)
        fft3.fft3_plan_execute(h, xd.data_ptr(), o2.data_ptr(), 0)
        torch.cuda.synchronize()
        assert fft3.fft3_plan_check(h) == 0
    finally:
        fft3.fft3_plan_destroy(h)
    assert torch.equal(o1, o2)
    g = o1.cpu().numpy()
    for off, d in list(zip(offs, dims))[::7]:
        _check_problem(x, g, int(off), d, fft3.FFT3_FORWARD)
    big = np.vstack([dims, [[128, 128, 8]]])
    bo, btotal = _layout(big)
    xb = synth.uniform_c64(btotal, 9)
    xbd = torch.from_numpy(xb).cuda()
    ob = torch.empty_like(xbd)
    h = fft3.fft3_plan_create_many(big, bo)
    try:
        assert fft3.fft3_plan_describe(h)["mode"] == "segmented"
        fft3.fft3_plan_execute(h, xbd.data_ptr(), ob.data_ptr(), 0)
        torch.cuda.synchronize()
        assert fft3.fft3_plan_check(h) == 0
    finally:
        fft3.fft3_plan_destroy(h)
    gb = ob.cpu().numpy()
    for off, d in list(zip(bo, big))[::29] + [(bo[-1], big[-1])]:
        _check_problem(xb, gb, int(off), d, fft3.FFT3_FORWARD)
    small = synth.batched_dims(6, 4)
    so, _ = _layout(small)
    h = fft3.fft3_plan_create_many(small, so)
    try:
        assert fft3.fft3_plan_describe(h)["mode"] == "executor"
    finally:
        fft3.fft3_plan_destroy(h)
    with pytest.raises(fft3.Fft3Error):
        fft3.fft3_plan_create_many([[30, 16, 16]], [0], tuning=[3])


@pytest.mark.parametrize("waves_code", [1, 3])
@pytest.mark.parametrize("direction", [fft3.FFT3_FORWARD, fft3.FFT3_INVERSE])
def test_one_launch_segmented_every_problem(waves_code, direction):
    """Tuning codes 3 | (k << 8): all x, y and z lines of the batch in one
    cooperative launch (grid barriers between steps, 2^(k-1) waves), every
    problem checked against the oracle; replayed on the same buffers it gives
    the same bits."""
    dims = np.vstack([synth.batched_dims(40, 11), [[8, 128, 16], [128, 8, 96], [24, 40, 8]]])
    offs, total = _layout(dims, gap=5)
    code = 3 | (waves_code << 8)
    x, got, desc = _run(dims, offs, total, direction=direction, tuning=[code] * len(dims), seed=2)
    assert desc["mode"] == "segmented_one_launch" and desc["kernel_launches"] == 1
    assert desc["waves"] == 1 << (waves_code - 1)
    for off, d in zip(offs, dims):
        _check_problem(x, got, int(off), d, direction)
    _, again, _ = _run(dims, offs, total, direction=direction, tuning=[code] * len(dims), seed=2)
    assert np.array_equal(got, again, equal_nan=True)  # the gaps between problems stay NaN


def test_one_launch_segmented_4096_cubes_sampled_and_parseval():
    """The 4096-cube workload in one cooperative launch: a sample covering
    every size class element by element, Parseval for every problem."""
    dims = synth.batched_dims(4096, 7)
    offs, total = _layout(dims)
    x, got, desc = _run(dims, offs, total, seed=7, tuning=[3 | (1 << 8)] * len(dims))
    assert desc["mode"] == "segmented_one_launch"
    seen, sample = set(), []
    for i, d in enumerate(map(tuple, dims)):
        if d not in seen:
            seen.add(d)
            sample.append(i)
    for i in sample[:120]:
        _check_problem(x, got, int(offs[i]), dims[i], fft3.FFT3_FORWARD)
    x2 = np.abs(x.astype(np.complex128)) ** 2
    g2 = np.abs(got.astype(np.complex128)) ** 2
    for off, d in zip(offs, dims):
        N = int(np.prod(d))
        sx, sg = x2[off:off + N].sum(), g2[off:off + N].sum()
        assert abs(sg - N * sx) <= 1e-5 * N * sx


def test_autotune_many_assignment_is_exact():
    """fft3_autotune_many times the whole batch under the default codes, every
    candidate code, per-size-class codes, the segmented passes and the slab
    executor, and returns one code per problem; the plan built from that
    assignment computes every problem to the oracle's tolerance, both
    directions."""
    dims = synth.batched_dims(12, 5, choices=(16, 24, 32))
    codes = fft3.fft3_autotune_many(dims, reps=1)
    assert len(codes) == len(dims)
    slabz = [c & fft3.FFT3_TUNE_SLABZ for c in codes]
    seg = [(c & 3) == 3 for c in codes]
    assert len(set(slabz)) == 1 and (not any(seg) or all(seg))  # whole-batch modes are all or nothing
    offs, total = _layout(dims, gap=1)
    for direction in (fft3.FFT3_FORWARD, fft3.FFT3_INVERSE):
        x, got, desc = _run(dims, offs, total, direction=direction, tuning=codes, seed=4)
        for off, d in zip(offs, dims):
            _check_problem(x, got, int(off), d, direction)


@pytest.mark.parametrize("direction", [fft3.FFT3_FORWARD, fft3.FFT3_INVERSE])
def test_slab_executor_slab_larger_than_the_room(direction):
    """Explicit FFT3_TUNE_SLABZ codes on a batch with a 128 x 128 slab (more
    than the 96 x 97 values FFT3_AUTO allows): one slab per item, a larger
    stack per block (fewer blocks per SM), every problem against the oracle."""
    dims = np.array([[128, 128, 8], [128, 96, 16], [96, 128, 24], [16, 16, 16], [40, 24, 128]])
    offs, total = _layout(dims, gap=3)
    code = fft3.tune_code(1) | fft3.FFT3_TUNE_SLABZ
    x, got, desc = _run(dims, offs, total, direction=direction, tuning=[code] * len(dims), seed=6)
    assert desc["mode"] == "slab_executor" and desc["slab_executor_smem"] == 128 * 129 * 8
    for off, d in zip(offs, dims):
        _check_problem(x, got, int(off), d, direction)
