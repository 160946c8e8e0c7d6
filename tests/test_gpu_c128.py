"""complex128 path (the paper's own precision, Section 4: complex double):
FP64 butterflies and FP64 twiddles against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
from paper_1904_10119_gb300 import fft3, synth

pytestmark = pytest.mark.gpu

REL_L2_TOL_FP64 = 1e-12
MAXABS_TOL_FP64 = 1e-11


def _run(shape, batch, direction, seed, decomposition=fft3.FFT3_PENCIL3, x=None):
    n0, n1, n2 = shape
    if x is None:
        x = synth.uniform_c128((batch, n2, n1, n0), seed)
    xt = torch.from_numpy(x).cuda()
    out = torch.full_like(xt, complex(float("nan"), float("nan")))
    plan = fft3.Plan(n0, n1, n2, batch, decomposition=decomposition, direction=direction,
                     dtype=fft3.FFT3_C128_FP64)
    plan.execute(xt, out)
    torch.cuda.synchronize()
    assert plan.check() == 0, fft3.last_error()
    assert torch.equal(xt.cpu(), torch.from_numpy(x)), "input was modified"
    kinds = {p["kind"] for p in plan.describe()["passes"]}
    assert kinds <= {"line_runtime_fp64", "line_contig_fp64", "line_strided_fp64"}, kinds
    return x, out.cpu().numpy(), plan


@pytest.mark.parametrize("shape,batch,direction", [
    ((64, 48, 96), 1, fft3.FFT3_FORWARD), ((30, 25, 18), 3, fft3.FFT3_FORWARD),
    ((100, 60, 9), 1, fft3.FFT3_INVERSE), ((1024, 16, 9), 1, fft3.FFT3_FORWARD),
    ((4096, 2, 3), 1, fft3.FFT3_INVERSE), ((3, 4096, 2), 1, fft3.FFT3_FORWARD),
    ((256, 256, 8), 1, fft3.FFT3_FORWARD), ((5, 1, 1), 2, fft3.FFT3_FORWARD), ((512, 64, 32), 1, fft3.FFT3_INVERSE),
    ((64, 1024, 3), 1, fft3.FFT3_FORWARD), ((24, 16, 1024), 1, fft3.FFT3_INVERSE)])
def test_c128_parity(shape, batch, direction):
    """FP64 passes: the compiled ones (contiguous and strided lines of a fixed
    plan's length) and the runtime-radix one, ragged tiles included."""
    x, got, _ = _run(shape, batch, direction, seed=sum(shape) + batch)
    ref = oracle.fft3(x.ravel(), *shape, batch, sign=direction)
    assert np.all(np.isfinite(got))
    assert oracle.rel_l2(got, ref) <= REL_L2_TOL_FP64
    assert oracle.max_abs_ratio(got, ref) <= MAXABS_TOL_FP64


def test_c128_round_trip_and_decompositions():
    """inverse(forward(x)) = N x to FP64 accuracy; slab-pencil and the automatic
    choice lower to the same passes."""
    shape = (96, 40, 18)
    N = int(np.prod(shape))
    x, X, _ = _run(shape, 1, fft3.FFT3_FORWARD, seed=5, decomposition=fft3.FFT3_AUTO)
    _, back, _ = _run(shape, 1, fft3.FFT3_INVERSE, seed=0, x=X)
    assert oracle.rel_l2(back / N, x) <= REL_L2_TOL_FP64
    _, X2, plan = _run(shape, 1, fft3.FFT3_FORWARD, seed=5, decomposition=fft3.FFT3_SLAB_PENCIL)
    assert np.array_equal(X, X2) and len(plan.describe()["passes"]) == 3


def test_c128_refuses_other_schedules():
    for decomp, opts in ((fft3.FFT3_VOLUMETRIC, {}), (fft3.FFT3_PENCIL3, {"variant": fft3.FFT3_PPP_ROTATE}),
                         (fft3.FFT3_PENCIL3, {"layout": fft3.FFT3_LAYOUT_PENCILS})):
        with pytest.raises(fft3.Fft3Error):
            fft3.Plan(64, 64, 64, 1, decomposition=decomp, dtype=fft3.FFT3_C128_FP64, **opts)
