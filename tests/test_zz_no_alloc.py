"""The allocation-free entry point, fft3_execute_noalloc.

It serves callers that must not allocate device memory (a plugin whose host
application owns every device allocation, or a latency-critical loop that
cannot pay for cudaMalloc/cudaFree), so it keeps its workspace and twiddles in
fixed arrays inside the library.  Here it is called through the C ABI twice in
a row and each result is compared with the regular plan path
(fft3_plan_create + fft3_plan_execute) at the parity tolerance of the other
GPU tests.  The file sorts last so a stop-at-first-failure run has already
run every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1904_10119_gb300 import fft3, synth
from tests.gpu_util import MAXABS_TOL, REL_L2_TOL

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a = a.astype(np.complex128).ravel()
    b = b.astype(np.complex128).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b), np.max(np.abs(a - b)) / np.max(np.abs(b))


def _regular(shape, batch, direction, xd):
    out = torch.empty_like(xd)
    plan = fft3.Plan(*shape, batch, decomposition=fft3.FFT3_PENCIL3, direction=direction,
                     variant=fft3.FFT3_PPP_ROTATE)
    plan.execute(xd, out)
    torch.cuda.synchronize()
    plan.close()
    return out.cpu().numpy()


@pytest.mark.parametrize("shape,batch,direction", [((64, 48, 40), 2, fft3.FFT3_FORWARD),
                                                   ((128, 128, 128), 1, fft3.FFT3_INVERSE),
                                                   ((1024, 32, 30), 1, fft3.FFT3_FORWARD)])
def test_noalloc_matches_plan_path_on_two_calls_in_a_row(shape, batch, direction):
    n0, n1, n2 = shape
    assert batch * n0 * n1 * n2 <= fft3.FFT3_NOALLOC_MAX_ELEMENTS
    L = fft3.load()
    for call, seed in enumerate((31, 32)):
        x = synth.uniform_c64((batch, n2, n1, n0), seed)
        xd = torch.from_numpy(x).cuda()
        out = torch.full_like(xd, complex(float("nan"), 0.0))
        rc = L.fft3_execute_noalloc(n0, n1, n2, batch, direction, ctypes.c_void_p(xd.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr()), None)
        assert rc == 0, fft3.last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref = _regular(shape, batch, direction, xd)
        rel, mx = _rel(got, ref)
        assert rel <= REL_L2_TOL and mx <= MAXABS_TOL, (call, rel, mx)
        assert torch.equal(xd.cpu(), torch.from_numpy(x))


def test_noalloc_rejects_sizes_beyond_its_arrays():
    x = torch.zeros(16, dtype=torch.complex64, device="cuda")
    with pytest.raises(fft3.Fft3Error) as e:
        fft3.fft3_execute_noalloc(256, 128, 128, 1, fft3.FFT3_FORWARD, x.data_ptr(), x.data_ptr() + 64)
    assert e.value.code == -2
    assert "FFT3_NOALLOC_MAX_ELEMENTS" in fft3.last_error()
    with pytest.raises(fft3.Fft3Error) as e:
        fft3.fft3_execute_noalloc(8, 8, 8, 1, fft3.FFT3_FORWARD, x.data_ptr(), x.data_ptr())
    assert e.value.code == -6
