"""Bit-exact checks of the integer parts of the CUDA path: the fused
redistributions (layout probe against the rotation maps of Section 2.4), the
FP64 twiddle generator against the oracle's long-double roots, the split-BF16
rounding, and the bounded waits of the persistent slab kernel."""
import numpy as np
import pytest
import torch

import oracle
from paper_1904_10119_gb300 import fft3, synth

pytestmark = pytest.mark.gpu


def _index_payload(n):
    i = np.arange(n, dtype=np.int64)
    return ((i % 4096).astype(np.float32) + 1j * (i // 4096).astype(np.float32)).astype(np.complex64)


def _decode(a):
    a = np.asarray(a).ravel()
    return a.real.astype(np.int64) + 4096 * a.imag.astype(np.int64)


def _probe(plan, x, npasses):
    xt = torch.from_numpy(x).cuda()
    out = torch.full_like(xt, complex(-1.0, -1.0))
    fft3.fft3_plan_probe_layout(plan.handle, xt.data_ptr(), out.data_ptr(), npasses, 0)
    torch.cuda.synchronize()
    return _decode(out.cpu().numpy())


@pytest.mark.parametrize("shape,batch", [((8, 12, 20), 1), ((64, 64, 64), 1), ((1024, 6, 10), 2),
                                         ((3, 512, 5), 1)])
def test_rotation_probe_bit_exact(shape, batch):
    n0, n1, n2 = shape
    N = n0 * n1 * n2
    plan = fft3.Plan(n0, n1, n2, batch, decomposition=fft3.FFT3_PENCIL3, variant=fft3.FFT3_PPP_ROTATE)
    x = _index_payload(N * batch)
    src = np.arange(N * batch)
    layouts = ["xyz", "yzx", "zxy"]
    expect_pos = np.arange(N)  # current position of each source element within one batch entry
    for k in range(1, 4):
        got = _probe(plan, x, k)             # got[dst] = src
        expect_pos = oracle.rotation_dst_index(n0, n1, n2, layouts[k - 1])[expect_pos]
        for b in range(batch):
            exp = np.empty(N, np.int64)
            exp[expect_pos] = src[b * N:(b + 1) * N]
            assert np.array_equal(got[b * N:(b + 1) * N], exp), (k, b)
    # three rotations bring the data back to natural order
    assert np.array_equal(expect_pos, np.arange(N))


@pytest.mark.parametrize("decomp", [fft3.FFT3_SLAB_PENCIL, fft3.FFT3_PENCIL3, fft3.FFT3_VOLUMETRIC])
def test_natural_layout_probe_is_identity(decomp):
    shape = (96, 40, 30)
    plan = fft3.Plan(*shape, 2, decomposition=decomp)
    x = _index_payload(int(np.prod(shape)) * 2)
    got = _probe(plan, x, -1)
    assert np.array_equal(got, np.arange(x.size))


@pytest.mark.parametrize("n", [2, 3, 5, 16, 96, 1000, 1024, 4096, 3 * 2 ** 20, 1 << 30])
def test_twiddle_generator_fp64(n):
    rng = np.random.default_rng(n)
    m = np.concatenate([np.arange(min(n, 4096)), rng.integers(-4 * n, 4 * n, 4096),
                        np.array([0, n // 4, n // 2, 3 * n // 4, n - 1])]).astype(np.int64)
    dm = torch.from_numpy(m).cuda()
    o64 = torch.empty(2 * m.size, dtype=torch.float64, device="cuda")
    o32 = torch.empty(2 * m.size, dtype=torch.float32, device="cuda")
    for sign in (-1, 1):
        fft3.fft3_twiddles(n, sign, dm.data_ptr(), m.size, o64.data_ptr(), o32.data_ptr(), 0)
        torch.cuda.synchronize()
        g64 = o64.cpu().numpy().view(np.complex128)
        g32 = o32.cpu().numpy().view(np.complex64)
        ref = oracle.roots(n, m, sign)
        err = np.abs(g64 - ref)
        assert err.max() <= 4.5e-16, (n, err.max())   # within about 2 ulp of values in [0.5, 1]
        # float32 values are the round-to-nearest of the generator's doubles
        # (bit-exact), so each lies within half a float32 ulp, plus the double
        # error, of the oracle
        assert np.array_equal(g32.view(np.uint32), g64.astype(np.complex64).view(np.uint32))
        for part in ("real", "imag"):
            r = getattr(ref, part)
            g = getattr(g32, part).astype(np.float64)
            half_ulp = 0.5 * np.spacing(np.abs(r).astype(np.float32)).astype(np.float64)
            assert np.all(np.abs(g - r) <= half_ulp + 4.5e-16)
        # away from the tiny values the oracle's long-double evaluation leaves
        # at exact zeros of sin/cos, the float32 tables equal the oracle rounded
        big = (np.abs(ref.real) > 1e-6) & (np.abs(ref.imag) > 1e-6)
        if big.any():
            assert np.mean(g32[big] != ref[big].astype(np.complex64)) < 1e-3


def test_split_bf16_bit_exact():
    x = np.concatenate([synth.uniform_c64(1 << 16, 3).view(np.float32),
                        synth.hdr_c64(1 << 12, 4).view(np.float32),
                        np.array([0.0, -0.0, 1.0, 3.0e38, 1e-40, 1.0 + 2 ** -8], np.float32)])
    xt = torch.from_numpy(x).cuda()
    hi = torch.empty(x.size, dtype=torch.int16, device="cuda")
    lo = torch.empty(x.size, dtype=torch.int16, device="cuda")
    fft3.fft3_split_bf16(xt.data_ptr(), x.size, hi.data_ptr(), lo.data_ptr(), 0)
    torch.cuda.synchronize()
    h_ref, l_ref = oracle.split_bf16(x)
    gh = hi.cpu().numpy().view(np.uint16).astype(np.uint32) << 16
    gl = lo.cpu().numpy().view(np.uint16).astype(np.uint32) << 16
    assert np.array_equal(gh, h_ref.view(np.uint32))
    assert np.array_equal(gl, l_ref.view(np.uint32))


@pytest.mark.parametrize("mode", [2, 5])
def test_bounded_wait_expires_and_reports_timeout(mode):
    """A slab whose x tiles never signal makes its y tiles' waits run out: the
    kernel records the timeout and returns, the host reads FFT3_ERR_TIMEOUT,
    and the context stays usable (slab_mode 2: L2-resident slab kernel;
    5: the fused kernel with TMA loads, whose producer waits)."""
    shape = (256, 256, 4)
    x = synth.uniform_c64((1, 4, 256, 256), 2)
    xt = torch.from_numpy(x).cuda()
    out = torch.empty_like(xt)
    opts = fft3.make_options(slab_mode=mode)
    opts.reserved[0] = 1 + 1      # slab 1 never signals
    opts.reserved[1] = 2000       # each wait gives up after 2e6 cycles (about a millisecond)
    h = fft3.fft3_plan_create_ex(*shape, 1, 0, fft3.FFT3_SLAB_PENCIL, -1, opts)
    try:
        fft3.fft3_plan_execute(h, xt.data_ptr(), out.data_ptr(), 0)
        assert fft3.fft3_plan_check(h) == -5
        assert "wait" in fft3.last_error()
        assert fft3.fft3_plan_check(h) == 0          # the flag was cleared
    finally:
        fft3.fft3_plan_destroy(h)
    from tests.gpu_util import assert_parity, run_plan
    x, got, _ = run_plan(shape, 1, fft3.FFT3_SLAB_PENCIL, -1, x=x, slab_mode=mode)
    assert_parity(x, got, shape)


def test_tcgen05_schedule_probe_is_identity_at_1024cubed():
    """The 1024^3 split-BF16 schedule (tcgen05 passes on the blocked
    intermediate [x/16][z][y][x%16], line transforms replaced by the identity):
    after all three passes every element is back at its natural position,
    bit-exact; after the y pass element (x, y, z) sits in the workspace at
    (x/16)*16*Y*Z + z*16*Y + 16*y + x%16 (the probe copies it to `out`)."""
    n = 1024
    plan = fft3.Plan(n, n, n, 1, decomposition=fft3.FFT3_AUTO, dtype=fft3.FFT3_C64_SPLITBF16_TC)
    assert [p["kind"] for p in plan.describe()["passes"]] == ["line_contig_r32_tc"] + ["line_strided_r32_tc"] * 2
    N = n ** 3
    i = torch.arange(N, device="cuda", dtype=torch.int64)
    x = torch.complex((i % 4096).float(), (i // 4096).float())
    out = torch.full_like(x, complex(-1.0, -1.0))
    for npasses in (2, -1):
        fft3.fft3_plan_probe_layout(plan.handle, x.data_ptr(), out.data_ptr(), npasses, 0)
        torch.cuda.synchronize()
        got = out.real.long() + 4096 * out.imag.long()  # got[position] = natural index
        if npasses == -1:
            assert torch.equal(got, i)
        else:
            xx, yy, zz = i % n, (i // n) % n, i // (n * n)
            pos = (xx // 16) * 16 * n * n + zz * 16 * n + 16 * yy + xx % 16
            assert torch.equal(got[pos], i)
        del got
    plan.close()
