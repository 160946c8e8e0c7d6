"""The allocation-free entry point, fft3_execute_noalloc.

It serves callers that must not allocate device memory: a plugin whose host
application owns every device allocation and only lends it buffers, or a
latency-critical loop that cannot pay for cudaMalloc/cudaFree (which may
synchronise the device and can fail once memory is fragmented).  So it keeps
its workspace and twiddles in fixed arrays inside the library.

Here it is called through the C ABI twice in a row; each result is compared
with the FP64 oracle at the parity tolerance of the other GPU tests, and with
the regular plan path (fft3_plan_create + fft3_plan_execute of the same
rotated pencil-pencil-pencil schedule), which runs the same kernels on
twiddle tables built by the same helpers, so the two must agree bit for bit.
Around the second call the device's free memory and torch's allocator
counters must not change.  The file sorts last so a stop-at-first-failure run
has already run every other test; it also passes on its own in a fresh
process.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1904_10119_gb300 import fft3, synth
from tests.gpu_util import MAXABS_TOL, REL_L2_TOL

pytestmark = pytest.mark.gpu


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
def test_noalloc_matches_oracle_and_plan_path_on_two_calls_in_a_row(shape, batch, direction):
    n0, n1, n2 = shape
    assert batch * n0 * n1 * n2 <= fft3.FFT3_NOALLOC_MAX_ELEMENTS
    L = fft3.load()
    for call, seed in enumerate((31, 32)):
        x = synth.uniform_c64((batch, n2, n1, n0), seed)
        xd = torch.from_numpy(x).cuda()
        out = torch.full_like(xd, complex(float("nan"), 0.0))
        torch.cuda.synchronize()
        free0, alloc0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated(), \
            torch.cuda.memory_reserved()
        rc = L.fft3_execute_noalloc(n0, n1, n2, batch, direction, ctypes.c_void_p(xd.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr()), None)
        assert rc == 0, fft3.last_error()
        torch.cuda.synchronize()
        if call == 1:  # the first call may load the library's module (and its fixed arrays) on this device
            assert torch.cuda.mem_get_info()[0] == free0, "device memory changed across the call"
            assert torch.cuda.memory_allocated() == alloc0 and torch.cuda.memory_reserved() == reserved0
        got = out.cpu().numpy()
        ref = oracle.fft3(x.ravel(), n0, n1, n2, batch, sign=direction)
        rel, mx = oracle.rel_l2(got, ref), oracle.max_abs_ratio(got, ref)
        print(f"noalloc {shape} b{batch} call {call}: rel-L2 {rel:.3e} max-abs {mx:.3e}")
        assert rel <= REL_L2_TOL and mx <= MAXABS_TOL, (call, rel, mx)
        assert np.array_equal(got, _regular(shape, batch, direction, xd)), "differs from the plan path"
        assert torch.equal(xd.cpu(), torch.from_numpy(x))


def test_noalloc_rejects_sizes_beyond_its_arrays():
    x = torch.zeros(16, dtype=torch.complex64, device="cuda")
    with pytest.raises(fft3.Fft3Error) as e:
        fft3.fft3_execute_noalloc(256, 128, 128, 1, fft3.FFT3_FORWARD, x.data_ptr(), x.data_ptr() + 64)
    assert e.value.code == -2
    assert "FFT3_NOALLOC_MAX_ELEMENTS" in fft3.last_error()
    # within the element limit, but a line longer than any plan supports
    with pytest.raises(fft3.Fft3Error) as e:
        fft3.fft3_execute_noalloc(8192, 2, 1, 1, fft3.FFT3_FORWARD, x.data_ptr(), x.data_ptr() + 64)
    assert e.value.code == -2
    with pytest.raises(fft3.Fft3Error) as e:
        fft3.fft3_execute_noalloc(8, 8, 8, 1, fft3.FFT3_FORWARD, x.data_ptr(), x.data_ptr())
    assert e.value.code == -6
