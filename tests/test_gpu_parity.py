"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by
element, at sizes that span several tiles and a ragged tail, for every
decomposition, both directions, several radix orders and the degenerate
shapes (unit dimensions, a single element)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1904_10119_gb300 import fft3, synth
from tests.gpu_util import MAXABS_TOL, REL_L2_TOL, assert_parity, run_plan

pytestmark = pytest.mark.gpu

S, P, V = fft3.FFT3_SLAB_PENCIL, fft3.FFT3_PENCIL3, fft3.FFT3_VOLUMETRIC
FWD, INV = fft3.FFT3_FORWARD, fft3.FFT3_INVERSE


def test_config_64cubed_ppp_forward_against_direct_sum():
    """64^3 forward, pencil-pencil-pencil, FP32, seed 1, direct-sum oracle."""
    x = synth.uniform_c64((1, 64, 64, 64), 1)
    x, got, plan = run_plan((64, 64, 64), 1, P, FWD, x=x)
    ref = oracle.fft3(x.ravel(), 64, 64, 64, method=oracle.METHOD_DIRECT)
    assert oracle.rel_l2(got, ref) <= 1e-5 and oracle.max_abs_ratio(got, ref) <= 1e-4
    assert plan.launches() == 3


SHAPES = [((64, 64, 64), 1), ((96, 80, 48), 2), ((30, 25, 18), 1), ((1024, 8, 6), 1), ((8, 1024, 6), 1),
          ((6, 8, 1024), 1), ((512, 24, 10), 1), ((20, 512, 12), 1), ((256, 12, 40), 2),
          ((16, 16, 16), 3), ((128, 36, 50), 1), ((45, 27, 75), 1)]


@pytest.mark.parametrize("shape,batch", SHAPES)
@pytest.mark.parametrize("decomp", [S, P, V])
def test_forward_parity(shape, batch, decomp):
    x, got, _ = run_plan(shape, batch, decomp, FWD, seed=sum(shape) + batch)
    assert_parity(x, got, shape, batch, FWD)


@pytest.mark.parametrize("shape,batch", [((64, 64, 64), 1), ((96, 80, 48), 2), ((1024, 8, 6), 1),
                                         ((6, 8, 1024), 1), ((30, 25, 18), 1)])
@pytest.mark.parametrize("decomp", [S, P, V])
def test_inverse_parity(shape, batch, decomp):
    x, got, _ = run_plan(shape, batch, decomp, INV, seed=7 + batch)
    assert_parity(x, got, shape, batch, INV)


@pytest.mark.parametrize("shape,batch", [((64, 64, 64), 1), ((96, 80, 48), 2), ((1024, 12, 10), 1),
                                         ((10, 20, 1024), 1), ((16, 16, 16), 4), ((1, 32, 5), 2)])
def test_pencil3_rotate_parity(shape, batch):
    x, got, plan = run_plan(shape, batch, P, FWD, seed=3, variant=fft3.FFT3_PPP_ROTATE)
    assert_parity(x, got, shape, batch, FWD)
    assert fft3.fft3_plan_workspace_bytes(plan.handle) == np.prod(shape) * batch * 8
    x, got, _ = run_plan(shape, batch, P, INV, seed=4, variant=fft3.FFT3_PPP_ROTATE)
    assert_parity(x, got, shape, batch, INV)


@pytest.mark.parametrize("order", [0, 1, 2, 3])
@pytest.mark.parametrize("shape", [(1024, 16, 8), (512, 40, 6), (256, 256, 4), (64, 48, 96), (640, 6, 10)])
def test_radix_orders(shape, order):
    x, got, _ = run_plan(shape, 1, P, FWD, seed=order, radix_order=order)
    assert_parity(x, got, shape)


@pytest.mark.parametrize("kw,shape,direction", [
    ({}, (1024, 12, 10), FWD),                                  # contiguous pass
    ({"tile_lines": 16}, (24, 1024, 6), INV),                   # plain strided pass
    ({"tile_lines": 8}, (8, 6, 1024), FWD),
    ({"slab_mode": 5, "slab_lines": 4}, (1024, 1024, 3), FWD),  # fused slab stage
    ({"slab_mode": 5, "slab_lines": 8}, (1024, 1024, 2), INV)])
def test_radix32_register_plan(kw, shape, direction):
    """The 1024-point plan with two radix-32 stages (one whole 32-point
    butterfly per thread in registers; radix_order 4 among the 1024-point
    candidates) in the kernels that run compile-time plans."""
    decomp = S if "slab_mode" in kw else P
    x, got, plan = run_plan(shape, 1, decomp, direction, seed=11, radix_order=4, **kw)
    assert_parity(x, got, shape, 1, direction)
    assert any(p["line"]["radices"] == [32, 32] for p in plan.describe()["passes"])


@pytest.mark.parametrize("mode,shape", [(1, (64, 64, 20)), (1, (96, 96, 8)), (2, (256, 256, 6)),
                                        (2, (512, 512, 3)), (3, (256, 256, 6)), (3, (100, 60, 12))])
def test_slab_modes(mode, shape):
    x, got, plan = run_plan(shape, 1, S, FWD, seed=mode, slab_mode=mode)
    assert_parity(x, got, shape)
    kinds = [p["kind"] for p in plan.describe()["passes"]]
    assert kinds[0] == {1: "slab_smem", 2: "slab_l2", 3: "line_contig"}[mode] or mode == 3


@pytest.mark.parametrize("shape,direction,lines", [((256, 256, 6), FWD, 0), ((256, 256, 5), INV, 8),
                                                   ((512, 512, 3), FWD, 4), ((512, 512, 4), INV, 8),
                                                   ((1024, 1024, 2), INV, 0), ((1024, 1024, 5), FWD, 8),
                                                   ((256, 256, 1), FWD, 0)])
def test_slab_fused_blocked(shape, direction, lines):
    """slab_mode 5: x and y tiles of every slab in one persistent launch (TMA
    loads by a producer warp), stored as blocked z pencils in the workspace,
    then the z pass back to natural order; 4 and 8 lines per tile, fewer slabs
    than the ticket lag (3), and a single slab (refused: no z pass)."""
    if shape[2] == 1:
        with pytest.raises(fft3.Fft3Error):
            fft3.Plan(*shape, 1, decomposition=S, slab_mode=5)
        return
    x, got, plan = run_plan(shape, 1, S, direction, seed=sum(shape), slab_mode=5, slab_lines=lines)
    assert_parity(x, got, shape, 1, direction)
    passes = plan.describe()["passes"]
    assert [p["kind"] for p in passes][0] == "slab_l2_blocked" and len(passes) == 2
    assert passes[0]["dst"] == "workspace" and passes[1]["src"] == "workspace"


@pytest.mark.parametrize("shape,batch,chunk,direction", [((64, 64, 64), 1, 0, FWD), ((96, 80, 10), 2, 3, FWD),
                                                         ((256, 256, 12), 1, 5, INV), ((100, 60, 9), 1, 1, FWD),
                                                         ((1024, 16, 9), 1, 4, INV), ((30, 25, 18), 3, 18, FWD)])
def test_slab_pipelined_chunks(shape, batch, chunk, direction):
    """slab_mode 4: x and y passes interleaved chunk by chunk on two streams,
    including a ragged last chunk and a batch."""
    x, got, plan = run_plan(shape, batch, S, direction, seed=chunk + batch, slab_mode=4, slab_chunk=chunk)
    assert_parity(x, got, shape, batch, direction)
    passes = plan.describe()["passes"]
    K = passes[0]["chunk"]
    assert passes[0]["pipelined_with"] == "next" and passes[1]["pipelined_with"] == "previous"
    assert K == (chunk if chunk else min(shape[2], max(1, (32 << 20) // (shape[0] * shape[1] * 8))))
    nchunks = -(-shape[2] // K)
    assert plan.kernel_launches() == 2 * nchunks + 1 and plan.launches() == 3
    # per-pass execution: the pair runs at its first index, the second index is empty
    xt = torch.from_numpy(x).cuda()
    out = torch.empty_like(xt)
    for k in range(plan.launches()):
        fft3.fft3_plan_execute_pass(plan.handle, k, xt.data_ptr(), out.data_ptr(), 0)
    torch.cuda.synchronize()
    assert_parity(x, out.cpu().numpy(), shape, batch, direction)


@pytest.mark.parametrize("shape,batch,order,direction", [
    ((40, 1024, 6), 1, 0, FWD), ((40, 1024, 6), 1, 1, INV), ((40, 1024, 6), 1, 2, FWD),
    ((40, 1024, 6), 1, 3, INV), ((40, 1024, 6), 1, 4, FWD), ((40, 1024, 6), 1, 5, FWD),
    ((24, 6, 1024), 2, 0, FWD), ((24, 6, 1024), 2, 1, INV), ((24, 6, 1024), 1, 4, FWD),
    ((18, 512, 4), 1, 0, INV), ((18, 512, 4), 1, 1, FWD), ((18, 512, 4), 1, 2, INV), ((18, 512, 4), 2, 3, FWD),
    ((20, 6, 512), 1, 1, FWD), ((20, 6, 512), 1, 3, INV), ((512, 512, 3), 1, 0, FWD), ((45, 512, 2), 1, 0, FWD)])
def test_streamed_strided_pass(shape, batch, order, direction):
    """Strided 512/1024-point lines with their decimated sub-lines streamed by
    TMA (tile_lines 2): every compiled variant (one block, or a cluster pair
    sharing 32-column tiles), ragged column tiles, a batch, both directions; a
    row stride that is not a 16-byte multiple falls back to the plain strided
    kernel."""
    x, got, plan = run_plan(shape, batch, P, direction, seed=order + 20, tile_lines=2, radix_order=order)
    assert_parity(x, got, shape, batch, direction)
    kinds = [p["kind"] for p in plan.describe()["passes"]]
    assert ("line_strided_stream" in kinds) == (shape[0] % 2 == 0)


@pytest.mark.parametrize("shape,direction", [((16, 512, 512), FWD), ((48, 1024, 512), INV), ((32, 512, 1024), FWD)])
def test_pencil3_blocked_intermediate(shape, direction):
    """FFT3_PPP_BLOCKED: the y pass stores [x/16][z][y][x%16] into the workspace
    and the z pass reads it back to natural order."""
    x, got, plan = run_plan(shape, 1, P, direction, seed=41, variant=fft3.FFT3_PPP_BLOCKED)
    assert_parity(x, got, shape, 1, direction)
    d = plan.describe()
    assert [(p["src"], p["dst"]) for p in d["passes"]] == [("in", "out"), ("out", "workspace"), ("workspace", "out")]
    assert fft3.fft3_plan_workspace_bytes(plan.handle) == np.prod(shape) * 8


@pytest.mark.parametrize("mesh,shape", [((2, 2, 2), (64, 64, 64)), ((4, 4, 4), (64, 64, 64)),
                                        ((8, 2, 4), (256, 32, 64)), ((2, 8, 4), (36, 256, 16)),
                                        ((4, 2, 8), (1024, 16, 64)), ((1, 4, 2), (30, 64, 36))])
def test_volumetric_meshes(mesh, shape):
    x, got, plan = run_plan(shape, 1, V, FWD, seed=11, mesh=mesh)
    assert_parity(x, got, shape)
    d = plan.describe()
    for p in d["passes"]:
        if p["kind"] == "volumetric_split":
            assert p["a"] % p["p"] == 0 and p["b"] % p["p"] == 0


@pytest.mark.parametrize("mesh,shape,batch,direction", [((2, 2, 2), (64, 64, 64), 1, FWD),
                                                        ((4, 4, 4), (64, 64, 64), 1, INV),
                                                        ((8, 2, 4), (256, 32, 64), 1, FWD),
                                                        ((1, 4, 2), (30, 64, 36), 2, FWD),
                                                        ((0, 0, 0), (1024, 1024, 4), 1, INV),
                                                        ((1, 2, 4), (100, 60, 48), 1, FWD)])
def test_volumetric_blocked_six_step(mesh, shape, batch, direction):
    """Blocked ownership of every split line (Section 2.2, Eq. ctparallel): three
    exchanges instead of one, same result."""
    x, got, plan = run_plan(shape, batch, V, direction, seed=13, mesh=mesh, variant=fft3.FFT3_VOL_BLOCKED_SIX_STEP)
    assert_parity(x, got, shape, batch, direction)
    splits = [p for p in plan.describe()["passes"] if p["kind"] == "volumetric_split"]
    assert splits and all(p["exchanges"] == 3 for p in splits)


@pytest.mark.parametrize("shape,batch", [((1, 64, 16), 1), ((64, 1, 1), 2), ((1, 1, 1), 3), ((1, 1, 96), 1),
                                         ((2, 3, 5), 1), ((5, 1, 3), 4)])
@pytest.mark.parametrize("decomp", [S, P, V])
def test_degenerate_shapes(shape, batch, decomp):
    x, got, _ = run_plan(shape, batch, decomp, FWD, seed=5)
    assert_parity(x, got, shape, batch)


def test_closed_forms_on_gpu():
    n0, n1, n2 = 64, 48, 40
    N = n0 * n1 * n2
    x = np.zeros((1, n2, n1, n0), np.complex64)
    x[0, 0, 0, 0] = 1
    _, got, _ = run_plan((n0, n1, n2), 1, S, FWD, x=x)
    assert np.max(np.abs(got - 1)) < 1e-6
    x = np.full((1, n2, n1, n0), 0.5 + 0.25j, np.complex64)
    _, got, _ = run_plan((n0, n1, n2), 1, P, FWD, x=x)
    expect = np.zeros(N, np.complex128)
    expect[0] = (0.5 + 0.25j) * N
    assert np.max(np.abs(got.ravel() - expect)) < 1e-5 * N


def test_round_trip_is_N_times_identity():
    shape = (96, 64, 40)
    N = int(np.prod(shape))
    x = synth.uniform_c64((1, 40, 64, 96), 9)
    _, y, _ = run_plan(shape, 1, S, FWD, x=x)
    _, z, _ = run_plan(shape, 1, P, INV, x=y)
    assert oracle.rel_l2(z / N, x) < 2e-6


def test_hdr_inputs():
    shape = (128, 64, 32)
    x = synth.hdr_c64((1, 32, 64, 128), 6)
    for d in (S, P, V):
        _, got, _ = run_plan(shape, 1, d, FWD, x=x)
        assert_parity(x, got, shape)


def test_execute_host_buffers():
    shape = (64, 40, 24)
    x = synth.uniform_c64((2, 24, 40, 64), 12)
    h = fft3.fft3_plan_create_ex(*shape, 2, 0, S, FWD, fft3.make_options())
    try:
        xin = torch.from_numpy(x).pin_memory()
        out = torch.empty_like(xin).pin_memory()
        fft3.fft3_plan_execute_host(h, xin.data_ptr(), out.data_ptr(), 0)
        assert_parity(x, out.numpy(), shape, 2)
    finally:
        fft3.fft3_plan_destroy(h)


@pytest.mark.parametrize("decomp,opts,dtype", [
    (S, {}, fft3.FFT3_C64_FP32), (P, {}, fft3.FFT3_C64_FP32), (P, {"variant": fft3.FFT3_PPP_ROTATE}, fft3.FFT3_C64_FP32),
    (V, {}, fft3.FFT3_C64_FP32), (P, {}, fft3.FFT3_C64_SPLITBF16_TC), (P, {}, fft3.FFT3_C128_FP64)])
@pytest.mark.parametrize("direction", [FWD, INV])
def test_execute_host_direct_and_staged(decomp, opts, dtype, direction):
    """Host buffers, both ways: pinned buffers (the first pass reads the host
    input directly where the schedule allows) and pageable numpy buffers
    (staged copies) give the oracle's transform; the input is left unchanged."""
    shape, batch = (1024, 24, 40), 1
    n0, n1, n2 = shape
    c128 = dtype == fft3.FFT3_C128_FP64
    if c128:
        rng = np.random.default_rng(4)
        x = (rng.uniform(-1, 1, (n2, n1, n0)) + 1j * rng.uniform(-1, 1, (n2, n1, n0))).astype(np.complex128)
    else:
        x = synth.uniform_c64((batch, n2, n1, n0), 21)
    h = fft3.fft3_plan_create_ex(*shape, batch, dtype, decomp, direction, fft3.make_options(**opts))
    try:
        ref = oracle.fft3(x.ravel(), n0, n1, n2, batch, sign=direction)
        pinned_in = torch.from_numpy(x.copy()).pin_memory()
        pinned_out = torch.full_like(pinned_in, complex(float("nan"), float("nan"))).pin_memory()
        page_in = np.ascontiguousarray(x.copy())
        page_out = np.full_like(page_in, np.nan)
        page_out2 = np.full_like(page_in, np.nan)
        pinned_out2 = torch.full_like(pinned_in, complex(float("nan"), float("nan"))).pin_memory()
        # pinned, pageable, and the two mixes (the direct input path depends on the input only)
        for src, dst, keep in ((pinned_in.data_ptr(), pinned_out, pinned_in.numpy()),
                               (page_in.ctypes.data, page_out, page_in),
                               (pinned_in.data_ptr(), page_out2, pinned_in.numpy()),
                               (page_in.ctypes.data, pinned_out2, page_in)):
            fft3.fft3_plan_execute_host(h, src, dst.data_ptr() if hasattr(dst, "data_ptr") else dst.ctypes.data, 0)
            got = dst.numpy() if hasattr(dst, "numpy") else dst
            assert np.array_equal(keep, x), "input modified"
            rel, mx = oracle.rel_l2(got, ref), oracle.max_abs_ratio(got, ref)
            tol = (1e-12, 1e-11) if c128 else (REL_L2_TOL, MAXABS_TOL)
            assert rel <= tol[0] and mx <= tol[1], (rel, mx)
        assert fft3.fft3_plan_check(h) == 0
    finally:
        fft3.fft3_plan_destroy(h)


@pytest.mark.parametrize("shape,opts,pinned", [((64, 40, 24), {}, True), ((64, 512, 512), {"variant": 2}, True),
                                               ((64, 40, 24), {}, False)])
def test_execute_host_pipelined(shape, opts, pinned):
    """Five transforms of different inputs from and to host memory with the
    copies of neighbouring transforms overlapping, pinned and pageable host
    buffers, the natural and the blocked schedule; every output is checked,
    and the pipelined and the single-transform forms alternate on one plan."""
    n0, n1, n2 = shape
    xs = [synth.uniform_c64((1, n2, n1, n0), 30 + i) for i in range(5)]
    h = fft3.fft3_plan_create_ex(*shape, 1, 0, P, FWD, fft3.make_options(**opts))
    try:
        assert fft3.fft3_plan_describe(h)["host_direct"] is True
        if pinned:
            hin = [torch.from_numpy(x).pin_memory() for x in xs]
            hout = [torch.full_like(t, complex(float("nan"), 0.0)).pin_memory() for t in hin]
            ptr = lambda t: t.data_ptr()
            arr = lambda t: t.numpy()
        else:
            hin = [np.ascontiguousarray(x) for x in xs]
            hout = [np.full_like(x, np.nan) for x in xs]
            ptr = lambda t: t.ctypes.data
            arr = lambda t: t
        for _ in range(2):
            fft3.fft3_plan_execute_host_pipelined(h, [ptr(t) for t in hin], [ptr(t) for t in hout], 0)
            assert fft3.fft3_plan_check(h) == 0
            for x, o in zip(xs, hout):
                assert_parity(x, arr(o), shape)
            # the other form on the same plan, then this one again
            one = np.full_like(xs[0], np.nan)
            fft3.fft3_plan_execute_host(h, xs[0].ctypes.data, one.ctypes.data, 0)
            assert_parity(xs[0], one, shape)
        fft3.fft3_plan_execute_host_pipelined(h, [], [], 0)  # count 0 is a no-op
    finally:
        fft3.fft3_plan_destroy(h)


def test_per_pass_execution_composes_to_the_transform():
    shape = (256, 64, 32)
    x = synth.uniform_c64((1, 32, 64, 256), 13)
    xt = torch.from_numpy(x).cuda()
    out = torch.empty_like(xt)
    plan = fft3.Plan(*shape, 1, decomposition=P, variant=fft3.FFT3_PPP_ROTATE)
    for k in range(plan.launches()):
        fft3.fft3_plan_execute_pass(plan.handle, k, xt.data_ptr(), out.data_ptr(), 0)
    torch.cuda.synchronize()
    assert_parity(x, out.cpu().numpy(), shape)


def test_error_paths():
    xt = torch.zeros(8 * 8 * 8, dtype=torch.complex64, device="cuda")
    h = fft3.fft3_plan_create(8, 8, 8, 1, 0, P, FWD)
    try:
        with pytest.raises(fft3.Fft3Error) as e:
            fft3.fft3_plan_execute(h, xt.data_ptr(), xt.data_ptr(), 0)
        assert e.value.code == -6
        with pytest.raises(fft3.Fft3Error) as e:
            fft3.fft3_plan_execute_pass(h, 99, xt.data_ptr(), xt.data_ptr() + 4096, 0)
        assert e.value.code in (-1, -6)
    finally:
        fft3.fft3_plan_destroy(h)
    for bad in [(7, 8, 8), (8, 8, 11 * 2), (8192, 2, 2)]:
        with pytest.raises(fft3.Fft3Error) as e:
            fft3.fft3_plan_create(*bad, 1, 0, P, FWD)
        assert e.value.code == -2
    # the context is still usable
    x, got, _ = run_plan((16, 16, 16), 1, P, FWD)
    assert_parity(x, got, (16, 16, 16))


@pytest.mark.parametrize("shape,batch", [((64, 64, 64), 1), ((1024, 16, 16), 1), ((16, 1024, 32), 1),
                                         ((32, 48, 1024), 2), ((128, 256, 80), 1), ((40, 40, 40), 1)])
@pytest.mark.parametrize("direction", [FWD, INV])
def test_tma_strided_pass(shape, batch, direction):
    x, got, plan = run_plan(shape, batch, P, direction, seed=21, tile_lines=1)
    assert_parity(x, got, shape, batch, direction)
    kinds = [p["kind"] for p in plan.describe()["passes"]]
    if shape != (40, 40, 40):
        assert "line_strided_tma" in kinds


@pytest.mark.parametrize("layout,shape,batch,decomp,extra", [
    (fft3.FFT3_LAYOUT_ROTATED, (64, 48, 96), 1, P, {}),
    (fft3.FFT3_LAYOUT_ROTATED, (30, 25, 18), 3, P, {}),
    (fft3.FFT3_LAYOUT_ROTATED, (1024, 16, 9), 1, fft3.FFT3_AUTO, {}),
    (fft3.FFT3_LAYOUT_PENCILS, (64, 48, 10), 1, P, {}),
    (fft3.FFT3_LAYOUT_PENCILS, (256, 256, 6), 1, S, {}),
    (fft3.FFT3_LAYOUT_PENCILS, (1024, 1024, 4), 1, fft3.FFT3_AUTO, {}),
    (fft3.FFT3_LAYOUT_PENCILS, (512, 512, 3), 1, S, {"slab_mode": 5})])
def test_permuted_layouts(layout, shape, batch, decomp, extra):
    """Permuted spectrum (Section 2.4): a forward plan's output read back through
    the oracle's positions is the DFT; an inverse plan fed the permuted layout
    returns the natural-order inverse DFT."""
    n0, n1, n2 = shape
    name = {fft3.FFT3_LAYOUT_ROTATED: "rotated", fft3.FFT3_LAYOUT_PENCILS: "pencils"}[layout]
    pos = oracle.layout_positions(name, n0, n1, n2, batch)
    x, got, plan = run_plan(shape, batch, decomp, FWD, seed=n2 + batch, layout=layout, **extra)
    assert plan.describe()["layout"] == name
    assert_parity(x, got.ravel()[pos].reshape(got.shape), shape, batch, FWD)
    xs = synth.uniform_c64((batch, n2, n1, n0), n2 + batch + 1)
    buf = np.empty(xs.size, dtype=np.complex64)
    buf[pos] = xs.ravel()
    _, got_i, _ = run_plan(shape, batch, decomp, INV, x=buf.reshape(xs.shape), layout=layout, **extra)
    assert_parity(xs, got_i, shape, batch, INV)
