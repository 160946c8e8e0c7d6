"""The split-BF16 tensor-core path (radix-16 sub-DFTs as m16n8k16 BF16 MMAs,
hi + lo parts, three products, FP32 accumulation) against the FP64 oracle.

Error budget: representing an FP32 value by hi + lo BF16 parts leaves a
relative error of at most 2^-17 (hi keeps 8 significant bits, lo the next 8),
the same for the DFT matrix, and the dropped lo x lo product is of the same
order, so one tensor-core stage adds an RMS relative error of a few 1e-6.  The
errors of successive stages add in quadrature.  The default mode (tc_stages 0)
puts, per line, the first radix-16 stage whose operands are both in shared
memory on the tensor cores (the middle stage of a contiguous 16 x 16 x 4 line,
the first 16-point stage of each decimated sub-line of a streamed strided
line); mode 1 every such stage, mode 2 every radix-16 stage.  Every mode is
held to the FP32 bar of the task (rel-L2 <= 1e-5, max-abs <= 1e-4 max|X|);
the measured errors are 3-6e-6.
"""
import numpy as np
import pytest

import oracle
from paper_1904_10119_gb300 import fft3, synth
from tests.gpu_util import MAXABS_TOL, REL_L2_TOL, run_plan

pytestmark = pytest.mark.gpu

TC = fft3.FFT3_C64_SPLITBF16_TC
P = fft3.FFT3_PENCIL3


def _err(x, got, shape, batch, direction):
    n0, n1, n2 = shape
    ref = oracle.fft3(x.ravel(), n0, n1, n2, batch, sign=direction)
    return oracle.rel_l2(got, ref), oracle.max_abs_ratio(got, ref)


@pytest.mark.parametrize("shape,batch", [((1024, 16, 8), 1), ((16, 1024, 8), 1), ((8, 16, 1024), 1),
                                         ((512, 64, 16), 1), ((256, 256, 16), 1), ((128, 128, 128), 1),
                                         ((1024, 24, 10), 2), ((40, 1024, 6), 1), ((18, 512, 4), 2),
                                         ((24, 6, 512), 1)])
@pytest.mark.parametrize("direction", [fft3.FFT3_FORWARD, fft3.FFT3_INVERSE])
@pytest.mark.parametrize("mode", [1, 2, 3])
def test_tc_radix16_stages(shape, batch, direction, mode):
    x, got, plan = run_plan(shape, batch, P, direction, seed=3, dtype=TC, tc_stages=mode)
    kinds = [p["kind"] for p in plan.describe()["passes"]]
    # modes 1 and 3 leave lines without a radix-16 stage in shared memory on the FP32 kernels
    assert any(k.endswith("_tc") for k in kinds) or mode in (1, 3)
    if 1024 in shape[1:] or 512 in shape[1:]:
        assert "line_strided_stream_tc" in kinds
    rel, mx = _err(x, got, shape, batch, direction)
    print(f"TC mode {mode} {shape} b{batch} dir{direction}: rel-L2 {rel:.3e} max-abs {mx:.3e}")
    assert rel <= REL_L2_TOL and mx <= MAXABS_TOL


@pytest.mark.parametrize("shape", [(1024, 16, 8), (8, 16, 1024), (256, 256, 16), (128, 128, 128)])
def test_tc_default_mode_meets_fp32_bar(shape):
    n0, n1, n2 = shape
    x = synth.uniform_c64((1, n2, n1, n0), 5)
    h = fft3.fft3_plan_create_ex(n0, n1, n2, 1, TC, P, -1, _opts_first())
    try:
        import torch
        xd = torch.from_numpy(x).cuda()
        out = torch.empty_like(xd)
        fft3.fft3_plan_execute(h, xd.data_ptr(), out.data_ptr(), 0)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
    finally:
        fft3.fft3_plan_destroy(h)
    rel, mx = _err(x, got, shape, 1, -1)
    print(f"TC default mode {shape}: rel-L2 {rel:.3e} max-abs {mx:.3e}")
    assert rel <= REL_L2_TOL and mx <= MAXABS_TOL


def _opts_first():
    return fft3.make_options(tc_stages=0)


@pytest.mark.parametrize("shape,batch,decomp", [
    ((1024, 8, 4), 1, P),        # contiguous 1024-point lines: whole 4-line tiles
    ((1024, 6, 5), 2, P),        # ragged last tile (6 lines = 4 + 2), batch 2
    ((16, 1024, 8), 1, P),       # strided 1024-point y columns
    ((20, 1024, 3), 1, P),       # 20 columns = 5 tiles of 4
    ((8, 16, 1024), 1, P),       # strided z columns (plane stride)
    ((24, 10, 1024), 1, P),
    ((1024, 1024, 2), 1, P),     # x and y passes both on tcgen05
    ((64, 1024, 1024), 1, fft3.FFT3_AUTO),  # blocked intermediate: y stores into it, z reads it
])
@pytest.mark.parametrize("direction", [fft3.FFT3_FORWARD, fft3.FFT3_INVERSE])
def test_tcgen05_radix32_lines(shape, batch, decomp, direction):
    """1024-point lines as two radix-32 split-BF16 GEMMs on the tcgen05 tensor
    cores (the default split-BF16 mode): element by element against the oracle."""
    x, got, plan = run_plan(shape, batch, decomp, direction, seed=9, dtype=TC)
    kinds = [p["kind"] for p in plan.describe()["passes"]]
    n_r32 = sum(1 for k in kinds if k.endswith("r32_tc"))
    assert n_r32 == sum(1 for d in shape if d == 1024), kinds
    rel, mx = _err(x, got, shape, batch, direction)
    print(f"tcgen05 r32 {shape} b{batch} dir{direction} {kinds}: rel-L2 {rel:.3e} max-abs {mx:.3e}")
    assert np.all(np.isfinite(got))
    assert rel <= REL_L2_TOL and mx <= MAXABS_TOL


@pytest.mark.parametrize("mode,label", [(0, "first shared-memory radix-16 stage"), (2, "every radix-16 stage")])
def test_tc_hdr_inputs(mode, label):
    """High-dynamic-range inputs (|z| log-uniform in [1e-3, 1e3], uniform phase)."""
    shape = (1024, 32, 16)
    x = synth.hdr_c64((1, 16, 32, 1024), 6)
    _, got, _ = run_plan(shape, 1, P, -1, x=x, dtype=TC, tc_stages=mode)
    rel, mx = _err(x, got, shape, 1, -1)
    print(f"TC mode {mode} ({label}) HDR {shape}: rel-L2 {rel:.3e} max-abs {mx:.3e}")
    assert rel <= REL_L2_TOL and mx <= MAXABS_TOL


def test_tc_error_exceeds_fp32_error():
    """The split-BF16 path is measurably less accurate than FP32 (so the test
    would notice a silent fall back to the FP32 kernels)."""
    shape = (1024, 16, 16)
    x = synth.uniform_c64((1, 16, 16, 1024), 8)
    _, g32, _ = run_plan(shape, 1, P, -1, x=x)
    _, gtc, _ = run_plan(shape, 1, P, -1, x=x, dtype=TC)
    r32, _ = _err(x, g32, shape, 1, -1)
    rtc, _ = _err(x, gtc, shape, 1, -1)
    print(f"FP32 rel-L2 {r32:.3e}, TC rel-L2 {rtc:.3e}")
    assert r32 < 1e-6 and rtc > 2 * r32
