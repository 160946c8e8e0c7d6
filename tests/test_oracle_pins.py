"""Pins for the FP64 oracle against what the paper and the mathematics fix.

Each test ties an oracle routine to something other than itself: hand-worked
textbook values (tests/golden/), closed forms, invariants, brute force on
tiny shapes, agreement between two independent routines, and numpy's FFT as
an independent library cross-check.  A dropped term, a wrong sign or index,
or a transposed operand in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1904_10119_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#")


def _rand(shape, seed):
    return synth.uniform_c64(shape, seed).astype(np.complex128)


# ---------------------------------------------------------------- golden --- #
def test_golden_dft4_textbook():
    g = _golden("dft4_textbook.txt")
    x = g[:, 0] + 1j * g[:, 1]
    y = g[:, 2] + 1j * g[:, 3]
    for f in (oracle.dft1_direct, oracle.fft1_rec):
        assert np.max(np.abs(f(x) - y)) < 1e-14


def test_golden_dft3_textbook():
    g = _golden("dft3_textbook.txt")
    x = g[:, 0] + 1j * g[:, 1]
    y = g[:, 2] + 1j * g[:, 3]
    for f in (oracle.dft1_direct, oracle.fft1_rec):
        assert np.max(np.abs(f(x) - y)) < 1e-14


def test_golden_3d_2x2x2_textbook():
    g = _golden("dft3d_2x2x2_textbook.txt")
    x = g[:, 1].astype(np.complex128)
    y = g[:, 2].astype(np.complex128)
    for method in (oracle.METHOD_DIRECT, oracle.METHOD_FFT):
        got = oracle.fft3(x, 2, 2, 2, method=method).ravel()
        assert np.max(np.abs(got - y)) < 1e-13
    assert np.max(np.abs(oracle.bruteforce3(x, 2, 2, 2).ravel() - y)) < 1e-13


def test_golden_ct16_index_maps():
    g = _golden("ct16_index_maps.txt").astype(np.int64)
    assert np.array_equal(oracle.ct_input_map(4, 4), g[:4])
    assert np.array_equal(oracle.ct_output_map(4, 4), g[4:])


def test_golden_rote256_distribution():
    g = _golden("rote256_p4_distribution.txt").astype(np.int64)
    x = _rand(256, 11)
    y, loc_in, loc_out = oracle.rote_parallel_dft1(x, 16, 16, 4)
    for r, count, first, stride in g:
        expect = np.arange(first, 256, stride)
        assert expect.size == count
        assert np.array_equal(loc_in[r], expect)
        assert np.array_equal(loc_out[r], expect)
    ref = oracle.dft1_direct(x)
    assert oracle.rel_l2(y, ref) < 1e-13


# ----------------------------------------------------------- closed forms --- #
SHAPES = [(8, 6, 5), (4, 4, 4), (16, 3, 10), (12, 20, 9)]


@pytest.mark.parametrize("shape", SHAPES)
def test_delta_to_ones(shape):
    n0, n1, n2 = shape
    x = np.zeros(n0 * n1 * n2, np.complex128)
    x[0] = 1
    y = oracle.fft3(x, n0, n1, n2)
    assert np.max(np.abs(y - 1.0)) < 1e-13


@pytest.mark.parametrize("shape", SHAPES)
def test_constant_to_scaled_delta(shape):
    n0, n1, n2 = shape
    c = 0.75 - 0.5j
    N = n0 * n1 * n2
    y = oracle.fft3(np.full(N, c), n0, n1, n2).ravel()
    expect = np.zeros(N, np.complex128)
    expect[0] = c * N
    assert np.max(np.abs(y - expect)) < 1e-12 * N


@pytest.mark.parametrize("shape,k", [((8, 6, 5), (3, 1, 4)), ((12, 20, 9), (5, 17, 2)),
                                     ((16, 16, 16), (15, 0, 7))])
def test_single_exponential_to_spike(shape, k):
    """x[j] = exp(+2 pi i (k0 j0/n0 + k1 j1/n1 + k2 j2/n2)) transforms (forward,
    w = exp(-2 pi i/n)) to N at (k0, k1, k2) and zero elsewhere."""
    n0, n1, n2 = shape
    j2, j1, j0 = np.meshgrid(np.arange(n2), np.arange(n1), np.arange(n0), indexing="ij")
    phase = (k[0] * j0 % n0) / n0 + (k[1] * j1 % n1) / n1 + (k[2] * j2 % n2) / n2
    x = np.exp(2j * np.pi * phase)
    y = oracle.fft3(x.ravel(), n0, n1, n2)
    N = n0 * n1 * n2
    expect = np.zeros((n2, n1, n0), np.complex128)
    expect[k[2], k[1], k[0]] = N
    assert np.max(np.abs(y - expect)) < 1e-11 * N


@pytest.mark.parametrize("shape,at", [((8, 6, 5), (1, 2, 3)), ((9, 10, 4), (8, 0, 3))])
def test_shifted_delta_is_phase_ramp(shape, at):
    n0, n1, n2 = shape
    x = np.zeros((n2, n1, n0), np.complex128)
    x[at[2], at[1], at[0]] = 1
    y = oracle.fft3(x.ravel(), n0, n1, n2)
    k2, k1, k0 = np.meshgrid(np.arange(n2), np.arange(n1), np.arange(n0), indexing="ij")
    expect = np.exp(-2j * np.pi * ((at[0] * k0 % n0) / n0 + (at[1] * k1 % n1) / n1 +
                                   (at[2] * k2 % n2) / n2))
    assert np.max(np.abs(y - expect)) < 1e-13


# ------------------------------------------------------------- invariants --- #
def test_linearity():
    n0, n1, n2 = 12, 10, 8
    a, b = 0.3 - 1.1j, -2.0 + 0.25j
    x1, x2 = _rand(n0 * n1 * n2, 1), _rand(n0 * n1 * n2, 2)
    lhs = oracle.fft3(a * x1 + b * x2, n0, n1, n2)
    rhs = a * oracle.fft3(x1, n0, n1, n2) + b * oracle.fft3(x2, n0, n1, n2)
    assert oracle.rel_l2(lhs, rhs) < 1e-14


@pytest.mark.parametrize("shape", [(16, 16, 16), (30, 18, 20)])
def test_parseval(shape):
    n0, n1, n2 = shape
    x = _rand(n0 * n1 * n2, 3)
    y = oracle.fft3(x, n0, n1, n2)
    N = n0 * n1 * n2
    assert abs(np.sum(np.abs(y) ** 2) - N * np.sum(np.abs(x) ** 2)) < 1e-12 * N * np.sum(np.abs(x) ** 2)


@pytest.mark.parametrize("shape,batch", [((16, 12, 10), 1), ((8, 8, 8), 3)])
def test_inverse_round_trip_is_N_times_identity(shape, batch):
    n0, n1, n2 = shape
    N = n0 * n1 * n2
    x = _rand(batch * N, 4)
    y = oracle.fft3(x, n0, n1, n2, batch, sign=oracle.FORWARD)
    z = oracle.fft3(y, n0, n1, n2, batch, sign=oracle.INVERSE)
    assert oracle.rel_l2(z.ravel() / N, x) < 1e-14


def test_conjugate_symmetry_of_real_input():
    n0, n1, n2 = 10, 12, 6
    x = _rand(n0 * n1 * n2, 5).real.astype(np.complex128)
    y = oracle.fft3(x, n0, n1, n2)
    ridx = lambda n: (-np.arange(n)) % n
    mirrored = y[np.ix_(ridx(n2), ridx(n1), ridx(n0))]
    assert np.max(np.abs(y - np.conj(mirrored))) < 1e-12 * np.max(np.abs(y))


def test_separability_any_axis_order():
    """The 1D passes commute: z then y then x equals x then y then z."""
    n0, n1, n2 = 12, 9, 10
    x = _rand(n0 * n1 * n2, 6)
    ref = oracle.fft3(x, n0, n1, n2)
    t = oracle.fft3_dims(x, n0, n1, n2, dims=(2,))
    t = oracle.fft3_dims(t, n0, n1, n2, dims=(1,))
    t = oracle.fft3_dims(t, n0, n1, n2, dims=(0,))
    assert oracle.rel_l2(t, ref) < 1e-14


def test_batch_elements_are_independent():
    n0, n1, n2, B = 8, 6, 4, 3
    x = _rand(B * n0 * n1 * n2, 7).reshape(B, -1)
    y = oracle.fft3(x.ravel(), n0, n1, n2, B)
    for b in range(B):
        assert oracle.rel_l2(y[b], oracle.fft3(x[b], n0, n1, n2)) < 1e-15


# ------------------------------------------------------------ brute force --- #
@pytest.mark.parametrize("shape", [(4, 4, 4), (6, 6, 6), (2, 3, 5), (5, 3, 2), (7, 2, 3), (1, 4, 3)])
@pytest.mark.parametrize("sign", [oracle.FORWARD, oracle.INVERSE])
def test_bruteforce_matches_separable(shape, sign):
    n0, n1, n2 = shape
    x = _rand(n0 * n1 * n2, 8)
    bf = oracle.bruteforce3(x, n0, n1, n2, sign)
    for method in (oracle.METHOD_DIRECT, oracle.METHOD_FFT):
        assert oracle.rel_l2(oracle.fft3(x, n0, n1, n2, sign=sign, method=method), bf) < 1e-14


# ------------------------------------------------ two routines agree --- #
def test_recursive_fft_equals_direct_sum_all_smooth_sizes():
    sizes = synth.smooth_sizes(1, 1024) + [7, 11, 13, 14, 49, 77, 91, 98]
    for n in sizes:
        x = _rand(n, 1000 + n)
        for sign in (oracle.FORWARD, oracle.INVERSE):
            d = oracle.dft1_direct(x, sign)
            r = oracle.fft1_rec(x, sign)
            assert oracle.rel_l2(r, d) < 1e-12, n


@pytest.mark.parametrize("shape,batch", [((32, 24, 20), 2), ((64, 64, 64), 1), ((5, 96, 40), 1)])
def test_numpy_fft_cross_check(shape, batch):
    """Independent library cross-check of the oracle only (numpy's pocketfft)."""
    n0, n1, n2 = shape
    x = _rand(batch * n0 * n1 * n2, 9).reshape(batch, n2, n1, n0)
    y = oracle.fft3(x.ravel(), n0, n1, n2, batch).reshape(batch, n2, n1, n0)
    ref = np.fft.fftn(x, axes=(1, 2, 3))
    assert oracle.rel_l2(y, ref) < 1e-12
    yi = oracle.fft3(x.ravel(), n0, n1, n2, batch, sign=oracle.INVERSE).reshape(x.shape)
    assert oracle.rel_l2(yi, np.fft.ifftn(x, axes=(1, 2, 3)) * (n0 * n1 * n2)) < 1e-12


def test_fft1_lines_inplace_matches_fft3_pass():
    n0, n1, n2 = 16, 12, 10
    x = _rand(n0 * n1 * n2, 10)
    buf = x.copy()
    # lines along n1: line (i0, i2) starts at i0 + n0*n1*i2, element stride n0
    for i2 in range(n2):
        sub = buf[i2 * n0 * n1:(i2 + 1) * n0 * n1].copy()
        oracle.fft1_lines_inplace(sub, n1, n0, 1, n0)
        buf[i2 * n0 * n1:(i2 + 1) * n0 * n1] = sub
    ref = oracle.fft3_dims(x, n0, n1, n2, dims=(1,))
    assert oracle.rel_l2(buf, ref) < 1e-15


@pytest.mark.parametrize("shape,batch,sign", [((8, 6, 10), 1, -1), ((16, 4, 5), 2, 1)])
def test_fft3_inplace_equals_fft3(shape, batch, sign):
    """The in-place whole-transform form the CPU baseline times computes the
    same 3D DFT as the out-of-place oracle (and so inherits its pins)."""
    n0, n1, n2 = shape
    x = synth.uniform_c128((batch, n2, n1, n0), 11)
    buf = np.ascontiguousarray(x.reshape(-1)).copy()
    oracle.fft3_inplace(buf, n0, n1, n2, batch, sign=sign)
    ref = oracle.fft3(x.ravel(), n0, n1, n2, batch, sign=sign).ravel()
    assert np.array_equal(buf, ref)


# ------------------------------------------ distributions / simulations --- #
@pytest.mark.parametrize("n0,n1,p", [(4, 4, 2), (16, 16, 4), (8, 12, 4), (12, 6, 3), (32, 32, 8)])
def test_rote_parallel_dft1(n0, n1, p):
    n = n0 * n1
    x = _rand(n, 12)
    y, loc_in, loc_out = oracle.rote_parallel_dft1(x, n0, n1, p)
    assert oracle.rel_l2(y, oracle.dft1_direct(x)) < 1e-13
    for r in range(p):
        cyc = np.arange(r, n, p)
        assert np.array_equal(loc_in[r], cyc) and np.array_equal(loc_out[r], cyc)
        assert loc_in[r].size == n // p


def test_rote_requires_divisibility():
    with pytest.raises(AssertionError):
        oracle.rote_parallel_dft1(np.zeros(24), 6, 4, 4)


@pytest.mark.parametrize("shape,mesh", [((8, 8, 8), (2, 2, 2)), ((16, 8, 12), (4, 2, 2)),
                                        ((4, 16, 8), (2, 4, 2))])
def test_volumetric_simulation_equals_3d_dft(shape, mesh):
    n0, n1, n2 = shape
    x = _rand(n0 * n1 * n2, 13)
    got = oracle.volumetric3_sim(x, n0, n1, n2, mesh)
    assert oracle.rel_l2(got, oracle.fft3(x, n0, n1, n2)) < 1e-13


@pytest.mark.parametrize("shape,p", [((4, 3, 2), 2), ((6, 2, 4), 2), ((4, 2, 4), 4)])
def test_slab_pencil_simulation_against_brute_force(shape, p):
    """Fig. 3dslabpencil on a 1D grid: the pencils rank r ends with are the x
    range of rank r of the N^3 direct sum; with the second exchange, the z range
    of rank r; the inverse brings either back to N times the slabs."""
    n0, n1, n2 = shape
    rng = np.random.default_rng(p + n0)
    x = rng.standard_normal((n2, n1, n0)) + 1j * rng.standard_normal((n2, n1, n0))
    slabs = [x[r * (n2 // p):(r + 1) * (n2 // p)] for r in range(p)]
    ref = oracle.bruteforce3(x, n0, n1, n2).reshape(n2, n1, n0)
    pen = oracle.slab_pencil_sim(slabs, n0, n1, n2, p)
    nat = oracle.slab_pencil_sim(slabs, n0, n1, n2, p, natural=True)
    for r in range(p):
        assert np.allclose(pen[r], ref[:, :, r * (n0 // p):(r + 1) * (n0 // p)], atol=1e-12)
        assert np.allclose(nat[r], ref[r * (n2 // p):(r + 1) * (n2 // p)], atol=1e-12)
    N = n0 * n1 * n2
    for got in (oracle.slab_pencil_sim(pen, n0, n1, n2, p, oracle.INVERSE),
                oracle.slab_pencil_sim(nat, n0, n1, n2, p, oracle.INVERSE, natural=True)):
        for r in range(p):
            assert np.allclose(got[r] / N, slabs[r], atol=1e-12)


@pytest.mark.parametrize("shape,grid", [((4, 6, 2), (2, 2)), ((6, 6, 2), (3, 1)), ((2, 4, 4), (1, 4)),
                                        ((4, 6, 6), (2, 3))])
def test_pencil3_simulation_against_brute_force(shape, grid):
    """Fig. 3dpencilpencil on a py x pz grid: the brick rank (p, q) ends with is
    its x range p and y range q of the N^3 direct sum; the inverse returns N
    times the pencils."""
    n0, n1, n2 = shape
    py, pz = grid
    rng = np.random.default_rng(py * 10 + pz)
    x = rng.standard_normal((n2, n1, n0)) + 1j * rng.standard_normal((n2, n1, n0))
    pencils = [x[(r // py) * (n2 // pz):(r // py + 1) * (n2 // pz), (r % py) * (n1 // py):(r % py + 1) * (n1 // py)]
               for r in range(py * pz)]
    ref = oracle.bruteforce3(x, n0, n1, n2).reshape(n2, n1, n0)
    bricks = oracle.pencil3_sim(pencils, n0, n1, n2, py, pz)
    for r in range(py * pz):
        p, q = r % py, r // py
        want = ref[:, q * (n1 // pz):(q + 1) * (n1 // pz), p * (n0 // py):(p + 1) * (n0 // py)]
        assert bricks[r].shape == want.shape and np.allclose(bricks[r], want, atol=1e-12)
    back = oracle.pencil3_sim(bricks, n0, n1, n2, py, pz, oracle.INVERSE)
    for r in range(py * pz):
        assert np.allclose(back[r] / (n0 * n1 * n2), pencils[r], atol=1e-12)


def test_slab_pencil_simulation_one_rank_is_the_3d_dft():
    x = synth.uniform_c64((1, 6, 5, 8), 3).reshape(6, 5, 8)
    got = oracle.slab_pencil_sim([x], 8, 5, 6, 1)[0]
    assert oracle.rel_l2(got, oracle.fft3(x, 8, 5, 6)) < 1e-14
    with pytest.raises(AssertionError):
        oracle.slab_pencil_sim([x], 8, 5, 6, 4)       # 4 does not divide n2 = 6


def test_cyclic_and_blocked_owners():
    own, loc = oracle.cyclic_owner(8, 2)
    assert own.tolist() == [0, 1, 0, 1, 0, 1, 0, 1] and loc.tolist() == [0, 0, 1, 1, 2, 2, 3, 3]
    own, loc = oracle.blocked_owner(8, 2)
    assert own.tolist() == [0, 0, 0, 0, 1, 1, 1, 1] and loc.tolist() == [0, 1, 2, 3, 0, 1, 2, 3]


def test_rotation_three_times_is_identity_and_explicit():
    n0, n1, n2 = 2, 3, 4
    N = n0 * n1 * n2
    r1 = oracle.rotation_dst_index(n0, n1, n2, "xyz")
    r2 = oracle.rotation_dst_index(n0, n1, n2, "yzx")
    r3 = oracle.rotation_dst_index(n0, n1, n2, "zxy")
    assert sorted(r1.tolist()) == list(range(N))
    comp = r3[r2[r1]]
    assert np.array_equal(comp, np.arange(N))
    # element (x=1, y=2, z=3) at 1 + 2*2 + 6*3 = 23 goes to y + n1*(z + n2*x) = 2 + 3*(3 + 4) = 23
    assert r1[1 + n0 * (2 + n1 * 3)] == 2 + n1 * (3 + n2 * 1)
    # element (x=1, y=0, z=0) -> 0 + 3*(0 + 4*1) = 12
    assert r1[1] == 12


def test_golden_layout_positions():
    """The permuted spectrum orders (Section 2.4) against hand-worked entries."""
    rows = open(os.path.join(GOLDEN, "layout_positions_small.txt")).read().split("\n")
    seen = set()
    for line in rows:
        if not line.strip() or line.startswith("#"):
            continue
        name, *v = line.split()
        n0, n1, n2, batch, k0, k1, k2, b, want = map(int, v)
        pos = oracle.layout_positions(name, n0, n1, n2, batch)
        N = n0 * n1 * n2
        assert pos[k0 + n0 * (k1 + n1 * k2) + N * b] == want
        seen.add(name)
    assert seen == {"rotated", "pencils"}


@pytest.mark.parametrize("layout,shape,batch", [("rotated", (2, 3, 4), 1), ("rotated", (5, 3, 6), 2),
                                                ("pencils", (32, 2, 3), 1), ("pencils", (48, 5, 7), 1)])
def test_layout_positions_are_permutations_with_contiguous_lines(layout, shape, batch):
    """Every layout is a bijection onto the buffer; in the rotated order the z
    lines are contiguous, in the pencils order a z line steps by 16*n1 and a
    16-column row of x is contiguous."""
    n0, n1, n2 = shape
    pos = oracle.layout_positions(layout, n0, n1, n2, batch)
    assert np.array_equal(np.sort(pos), np.arange(n0 * n1 * n2 * batch))
    p = pos.reshape(batch, n2, n1, n0)
    if layout == "rotated":
        assert np.all(np.diff(p, axis=1) == 1)
    else:
        assert np.all(np.diff(p, axis=1) == 16 * n1)
        assert np.all(np.diff(p.reshape(batch, n2, n1, n0 // 16, 16), axis=-1) == 1)


# --------------------------------------------------------------- roots --- #
def test_roots_closed_forms():
    n = 8
    w = oracle.roots(n, np.arange(n))
    assert np.max(np.abs(np.abs(w) - 1)) <= 2.3e-16
    h = math.sqrt(0.5)
    assert abs(w[1] - (h - 1j * h)) < 1e-16
    assert abs(w[2] - (-1j)) < 1e-16 and abs(w[4] + 1) < 1e-16
    wi = oracle.roots(n, np.arange(n), oracle.INVERSE)
    assert np.max(np.abs(wi - np.conj(w))) == 0
    # exponent reduction is exact: w^(m + k*n) == w^m bit for bit
    big = oracle.roots(1024, np.array([5, 5 + 1024 * 977, -1019]))
    assert big[0] == big[1] == big[2]
    # group law
    n = 1000
    a = oracle.roots(n, np.arange(n))
    m, k = 137, 411
    assert abs(a[m] * a[k] - a[(m + k) % n]) < 4e-16
    assert abs(oracle.roots(3, [1])[0] - (-0.5 - 1j * math.sqrt(3) / 2)) < 2e-16


# ---------------------------------------------------------------- bf16 --- #
def test_bf16_round_to_nearest_even():
    """IEEE-754 round-to-nearest-even on explicit bit patterns."""
    src = np.array([0x3F800000, 0x3F808000, 0x3F818000, 0x3F808001, 0xBF808000, 0x7F7FFFFF,
                    0x00010000, 0x0000FFFF, 0x3F80FFFF], np.uint32)
    exp = np.array([0x3F80, 0x3F80, 0x3F82, 0x3F81, 0xBF80, 0x7F80, 0x0001, 0x0001, 0x3F81],
                   np.uint32)
    got = oracle.bf16_round(src.view(np.float32)).view(np.uint32)
    assert np.array_equal(got >> 16, exp)
    assert np.all((got & 0xFFFF) == 0)


def test_split_bf16_hi_lo():
    x = synth.uniform_c64(4096, 21).view(np.float32)
    hi, lo = oracle.split_bf16(x)
    assert np.all((hi.view(np.uint32) & 0xFFFF) == 0) and np.all((lo.view(np.uint32) & 0xFFFF) == 0)
    err = np.abs(x.astype(np.float64) - hi.astype(np.float64) - lo.astype(np.float64))
    assert np.all(err <= 2.0 ** -16 * np.abs(x.astype(np.float64)) + 1e-45)


# ----------------------------------------------------------------- MLP --- #
def _mlp_params(F=16, H=64, seed=0):
    rng = np.random.default_rng(seed)
    return [rng.normal(0, 1 / math.sqrt(F), (H, F)), rng.normal(0, 0.1, H),
            rng.normal(0, 1 / math.sqrt(H), (H, H)), rng.normal(0, 0.1, H),
            rng.normal(0, 1 / math.sqrt(H), (1, H)), rng.normal(0, 0.1, 1)]


def test_gelu_closed_values():
    assert oracle.gelu(np.array([0.0]))[0] == 0.0
    assert abs(oracle.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-15
    assert abs(oracle.gelu(np.array([-1.0]))[0] + 0.15865525393145707) < 1e-15
    assert abs(oracle.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-16


def test_mlp_gradients_against_finite_differences():
    F, H, B = 7, 9, 11
    params = _mlp_params(F, H, 3)
    rng = np.random.default_rng(4)
    X = rng.normal(size=(B, F))
    t = rng.normal(size=B)
    pred, cache = oracle.mlp_forward(params, X)
    grads = oracle.mlp_backward(params, cache, pred, t)
    h = 1e-6
    for pi, p in enumerate(params):
        flat = p.reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 7)):
            old = flat[idx]
            flat[idx] = old + h
            lp = oracle.mse_loss(oracle.mlp_forward(params, X)[0], t)
            flat[idx] = old - h
            lm = oracle.mse_loss(oracle.mlp_forward(params, X)[0], t)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            g = grads[pi].reshape(-1)[idx]
            assert abs(fd - g) <= 1e-6 * max(1.0, abs(g)), (pi, idx, fd, g)


def test_adam_first_step_moves_by_lr_times_sign():
    p = [np.array([1.0, -2.0, 3.0])]
    g = [np.array([0.5, -4.0, 1e-3])]
    m = [np.zeros(3)]
    v = [np.zeros(3)]
    new_p, new_m, new_v = oracle.adam_step(p, g, m, v, t=1, lr=0.01)
    assert np.allclose(new_p[0], p[0] - 0.01 * np.sign(g[0]), rtol=0, atol=1e-7)
    assert np.allclose(new_m[0], 0.1 * g[0]) and np.allclose(new_v[0], 0.001 * g[0] ** 2)


def test_sampled_outputs_equal_full_transform():
    n0, n1, n2 = 24, 20, 18
    x = _rand(n0 * n1 * n2, 31).reshape(n2, n1, n0)
    full = oracle.fft3(x.ravel(), n0, n1, n2)
    k0s, k1s, k2s = [0, 5, 23], [1, 19], [0, 7, 17]
    got = oracle.dft3_sampled(x, n0, n1, n2, k0s, k1s, k2s, chunk_rows=37)
    ref = full[np.ix_(k2s, k1s, k0s)].transpose(2, 1, 0)
    assert oracle.rel_l2(got, ref) < 1e-14
    gi = oracle.dft3_sampled(x, n0, n1, n2, k0s, k1s, k2s, sign=oracle.INVERSE)
    fi = oracle.fft3(x.ravel(), n0, n1, n2, sign=oracle.INVERSE)
    assert oracle.rel_l2(gi, fi[np.ix_(k2s, k1s, k0s)].transpose(2, 1, 0)) < 1e-14


@pytest.mark.parametrize("shape,sign", [((8, 6, 10), -1), ((12, 5, 9), 1)])
def test_dft3_line_equals_fft3_lines(shape, sign):
    """A whole output line along each dimension, by the separable definition
    with the other two frequencies fixed, equals the corresponding line of
    the full oracle transform."""
    n0, n1, n2 = shape
    x = synth.uniform_c128((n2, n1, n0), 21)
    ref = oracle.fft3(x.ravel(), n0, n1, n2, sign=sign).reshape(n2, n1, n0)
    for dim, ka, kb in ((0, 2, 3), (1, 5, 7), (2, 1, 4)):
        line = oracle.dft3_line(x, n0, n1, n2, dim, ka, kb, sign=sign, chunk=3)
        want = ref[kb, ka, :] if dim == 0 else ref[kb, :, ka] if dim == 1 else ref[:, kb, ka]
        assert np.max(np.abs(line - want)) <= 1e-12 * np.max(np.abs(want))

