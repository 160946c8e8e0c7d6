"""Helpers shared by the GPU parity tests (inputs from synth, expected values
from the FP64 oracle, the transform through the C ABI of libfft3.so)."""
import numpy as np
import torch

import oracle
from paper_1904_10119_gb300 import fft3, synth

# FP32 bar from the benchmark spec: rel-L2 <= 1e-5 and max-abs <= 1e-4 * max|X|.
REL_L2_TOL = 1e-5
MAXABS_TOL = 1e-4


def run_plan(shape, batch=1, decomposition=fft3.FFT3_PENCIL3, direction=fft3.FFT3_FORWARD, x=None,
             seed=1, dtype=fft3.FFT3_C64_FP32, **opts):
    n0, n1, n2 = shape
    if x is None:
        x = synth.uniform_c64((batch, n2, n1, n0), seed)
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    out = torch.full_like(xt, complex(float("nan"), float("nan")))
    plan = fft3.Plan(n0, n1, n2, batch, decomposition=decomposition, direction=direction, dtype=dtype,
                     **opts)
    plan.execute(xt, out)
    torch.cuda.synchronize()
    assert plan.check() == 0, fft3.last_error()
    assert torch.equal(xt.cpu(), torch.from_numpy(np.ascontiguousarray(x))), "input was modified"
    return x, out.cpu().numpy(), plan


def errors(x, got, shape, batch, direction):
    n0, n1, n2 = shape
    ref = oracle.fft3(np.asarray(x).ravel(), n0, n1, n2, batch, sign=direction)
    return oracle.rel_l2(got, ref), oracle.max_abs_ratio(got, ref)


def assert_parity(x, got, shape, batch=1, direction=fft3.FFT3_FORWARD):
    rel, mx = errors(x, got, shape, batch, direction)
    assert np.all(np.isfinite(got))
    assert rel <= REL_L2_TOL, f"rel-L2 {rel:.3e} for {shape} batch {batch}"
    assert mx <= MAXABS_TOL, f"max-abs ratio {mx:.3e} for {shape} batch {batch}"
    return rel, mx
