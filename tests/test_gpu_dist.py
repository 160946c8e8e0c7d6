"""The rank-local plans of the distributed decompositions (Section 2.4:
slab-pencil on a 1D grid, Fig. 3dslabpencil; pencil-pencil-pencil on a 2D
grid, Fig. 3dpencilpencil) on one GPU: the ranks run one after another on the
same device, their all-to-alls replaced by device copies of the equal blocks
(no kernel waits on another).  Every rank's output is compared element by
element with the oracle's simulation of the distributed algorithm, and at
1024^3 the reassembled spectrum with sampled outputs, Parseval and whole
lines of the 3D DFT."""
import numpy as np
import pytest
import torch

import oracle
from paper_1904_10119_gb300 import fft3, synth
from paper_1904_10119_gb300.distributed import SlabPencil
from tests.gpu_util import MAXABS_TOL, REL_L2_TOL

pytestmark = pytest.mark.gpu

S = fft3.FFT3_SLAB_PENCIL
FWD, INV = fft3.FFT3_FORWARD, fft3.FFT3_INVERSE


def _local_inputs(x, P, spectrum, natural):
    n2, n1, n0 = x.shape
    if spectrum and not natural:
        return [np.ascontiguousarray(x[:, :, r * (n0 // P):(r + 1) * (n0 // P)]) for r in range(P)]
    return [np.ascontiguousarray(x[r * (n2 // P):(r + 1) * (n2 // P)]) for r in range(P)]


def emulate(dims, P, direction, natural, local, dtype=fft3.FFT3_C64_FP32):
    """Runs the P ranks' stages on this GPU; `local` are the ranks' device arrays."""
    n0, n1, n2 = dims
    mk = lambda d, st: fft3.Plan(*d, 1, S, direction, dtype, dist_ranks=P, dist_stage=st)
    plans = {1: mk((n0, n1, n2 // P), 1), 2: mk((n0 // P, n1, n2), 2)}
    if natural:
        plans[3] = mk((n0, n1, n2 // P), 3)
    blk = n0 * n1 * n2 // P ** 2

    def run(stage, arrays):
        outs = []
        for a in arrays:
            o = torch.full_like(a.reshape(-1), complex(float("nan"), float("nan")))
            plans[stage].execute(a.reshape(-1), o)
            outs.append(o)
        return outs

    def exchange(sends):   # rank r receives block r of every rank, in rank order
        return [torch.cat([sends[s][r * blk:(r + 1) * blk] for s in range(P)]) for r in range(P)]

    if direction == FWD:
        data = run(2, exchange(run(1, local)))
        if natural:
            data = run(3, exchange(data))
    else:
        data = [a.reshape(-1) for a in local]
        if natural:
            data = exchange(run(3, data))
        data = run(1, exchange(run(2, data)))
    torch.cuda.synchronize()
    for p in plans.values():
        assert p.check() == 0, fft3.last_error()
    return data, plans


CASES = [((64, 48, 32), 2), ((128, 20, 64), 4), ((96, 80, 48), 2), ((1024, 8, 16), 2), ((16, 1024, 8), 2),
         ((32, 16, 1024), 4), ((30, 25, 18), 2), ((8, 1, 4), 4)]


@pytest.mark.parametrize("dims,P", CASES)
@pytest.mark.parametrize("direction,natural", [(FWD, False), (FWD, True), (INV, False), (INV, True)])
def test_ranks_match_the_simulation(dims, P, direction, natural):
    n0, n1, n2 = dims
    x = synth.uniform_c64((1, n2, n1, n0), sum(dims) + P).reshape(n2, n1, n0)
    local = _local_inputs(x, P, direction == INV, natural)
    got, plans = emulate(dims, P, direction, natural, [torch.from_numpy(a).cuda() for a in local])
    ref = oracle.slab_pencil_sim(local, n0, n1, n2, P, direction, natural)
    peak = max(float(np.abs(r).max()) for r in ref)
    for r in range(P):
        g = got[r].cpu().numpy()
        assert np.all(np.isfinite(g)), f"rank {r} left elements unwritten"
        assert oracle.rel_l2(g, ref[r].ravel()) <= REL_L2_TOL
        assert float(np.abs(g - ref[r].ravel()).max()) <= MAXABS_TOL * peak
    # the slab stage stores straight into the packed blocks: two passes, no separate pack
    assert plans[1].launches() == 2 and plans[2].launches() == 1


@pytest.mark.parametrize("dims,P", [((64, 48, 32), 2), ((30, 25, 18), 2)])
def test_complex128_ranks(dims, P):
    n0, n1, n2 = dims
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, (n2, n1, n0)) + 1j * rng.uniform(-1, 1, (n2, n1, n0))
    for direction in (FWD, INV):
        local = _local_inputs(x, P, direction == INV, False)
        got, _ = emulate(dims, P, direction, False, [torch.from_numpy(a).cuda() for a in local],
                         dtype=fft3.FFT3_C128_FP64)
        ref = oracle.slab_pencil_sim(local, n0, n1, n2, P, direction)
        for r in range(P):
            assert oracle.rel_l2(got[r].cpu().numpy(), ref[r].ravel()) <= 1e-13


def test_one_rank_driver_is_the_slab_pencil_plan():
    """Without a process group the driver runs the one-GPU slab-pencil plan."""
    x = synth.uniform_c64((1, 24, 20, 32), 2)
    sp = SlabPencil(32, 20, 24)
    assert sp.P == 1 and sp.local_shape(True) == (24, 20, 32)
    xd = torch.from_numpy(x).cuda().reshape(24, 20, 32)
    out = torch.empty_like(xd)
    sp.execute(xd, out)
    torch.cuda.synchronize()
    ref = oracle.fft3(x.ravel(), 32, 20, 24)
    assert oracle.rel_l2(out.cpu().numpy(), ref) <= REL_L2_TOL


@pytest.mark.parametrize("P", [2, 4])
def test_1024cubed_spectrum_reassembled(P):
    """1024^3 forward over P emulated ranks: the pencils joined along x are the
    3D DFT (sampled outputs, Parseval, one whole line per dimension)."""
    from tests.test_gpu_fullsize import _sampled_check
    n = 1024
    x = synth.uniform_c64((1, n, n, n), 4).reshape(n, n, n)
    local = [torch.from_numpy(a).cuda() for a in _local_inputs(x, P, False, False)]
    got, plans = emulate((n, n, n), P, FWD, False, local)
    del local
    host = torch.empty((n, n, n), dtype=torch.complex64).pin_memory()
    for r in range(P):
        host[:, :, r * (n // P):(r + 1) * (n // P)].copy_(got[r].reshape(n, n, n // P))
    del got
    torch.cuda.empty_cache()
    _sampled_check(x, host.numpy(), n, FWD, 71 + P)


# ------------------------------------------------------------------------- #
# pencil-pencil-pencil on a Py x Pz grid                                    #
# ------------------------------------------------------------------------- #
P3 = fft3.FFT3_PENCIL3


def _ppp_local(x, grid, spectrum):
    n2, n1, n0 = x.shape
    Py, Pz = grid
    out = []
    for r in range(Py * Pz):
        p, q = r % Py, r // Py
        if spectrum:
            out.append(np.ascontiguousarray(x[:, q * (n1 // Pz):(q + 1) * (n1 // Pz), p * (n0 // Py):(p + 1) * (n0 // Py)]))
        else:
            out.append(np.ascontiguousarray(x[q * (n2 // Pz):(q + 1) * (n2 // Pz), p * (n1 // Py):(p + 1) * (n1 // Py)]))
    return out


def emulate_ppp(n, grid, direction, local, dtype=fft3.FFT3_C64_FP32):
    """The Py x Pz ranks' three stages on this GPU, the row and column
    all-to-alls as device copies; `local` are the ranks' device arrays."""
    n0, n1, n2 = n
    Py, Pz = grid
    R = Py * Pz
    dims = {1: (n0, n1 // Py, n2 // Pz), 2: (n0 // Py, n1, n2 // Pz), 3: (n0 // Py, n1 // Pz, n2)}
    plans = {k: fft3.Plan(*d, 1, P3, direction, dtype, dist_ranks=Py, dist_ranks2=Pz, dist_stage=k)
             for k, d in dims.items()}

    def run(k, arrays):
        outs = []
        for a in arrays:
            o = torch.full_like(a.reshape(-1), complex(float("nan"), float("nan")))
            plans[k].execute(a.reshape(-1), o)
            outs.append(o)
        return outs

    def exchange(sends, row):
        outs = []
        for r in range(R):
            p, q = r % Py, r // Py
            members = [q * Py + i for i in range(Py)] if row else [j * Py + p for j in range(Pz)]
            me = members.index(r)
            blk = sends[r].numel() // len(members)
            outs.append(torch.cat([sends[m][me * blk:(me + 1) * blk] for m in members]))
        return outs

    if direction == FWD:
        data = run(3, exchange(run(2, exchange(run(1, local), True)), False))
    else:
        data = run(1, exchange(run(2, exchange(run(3, local), False)), True))
    torch.cuda.synchronize()
    for p in plans.values():
        assert p.check() == 0, fft3.last_error()
    return data, plans


PPP_CASES = [((64, 48, 32), (2, 2)), ((128, 24, 40), (4, 2)), ((96, 80, 48), (2, 4)), ((60, 30, 18), (3, 2)),
             ((1024, 16, 16), (2, 2)), ((16, 1024, 8), (2, 2)), ((32, 16, 1024), (2, 4)), ((8, 4, 4), (1, 4))]


@pytest.mark.parametrize("n,grid", PPP_CASES)
@pytest.mark.parametrize("direction", [FWD, INV])
def test_ppp_ranks_match_the_simulation(n, grid, direction):
    n0, n1, n2 = n
    x = synth.uniform_c64((1, n2, n1, n0), sum(n) + grid[0]).reshape(n2, n1, n0)
    local = _ppp_local(x, grid, direction == INV)
    got, plans = emulate_ppp(n, grid, direction, [torch.from_numpy(a).cuda() for a in local])
    ref = oracle.pencil3_sim(local, n0, n1, n2, grid[0], grid[1], direction)
    peak = max(float(np.abs(r).max()) for r in ref)
    for r in range(len(ref)):
        g = got[r].cpu().numpy()
        assert np.all(np.isfinite(g)), f"rank {r} left elements unwritten"
        assert oracle.rel_l2(g, ref[r].ravel()) <= REL_L2_TOL
        assert float(np.abs(g - ref[r].ravel()).max()) <= MAXABS_TOL * peak
    assert all(p.launches() == 1 for p in plans.values())


def test_ppp_complex128_ranks():
    n, grid = (48, 40, 30), (2, 2)
    rng = np.random.default_rng(9)
    x = rng.uniform(-1, 1, n[::-1]) + 1j * rng.uniform(-1, 1, n[::-1])
    for direction in (FWD, INV):
        local = _ppp_local(x, grid, direction == INV)
        got, _ = emulate_ppp(n, grid, direction, [torch.from_numpy(a).cuda() for a in local], fft3.FFT3_C128_FP64)
        ref = oracle.pencil3_sim(local, *n, *grid, direction)
        for r in range(4):
            assert oracle.rel_l2(got[r].cpu().numpy(), ref[r].ravel()) <= 1e-13


def test_ppp_1024cubed_bricks_reassembled():
    """1024^3 forward on a 2 x 2 grid: the four bricks joined are the 3D DFT
    (sampled outputs, Parseval, one whole line per dimension)."""
    from tests.test_gpu_fullsize import _sampled_check
    n, grid = 1024, (2, 2)
    x = synth.uniform_c64((1, n, n, n), 4).reshape(n, n, n)
    local = [torch.from_numpy(a).cuda() for a in _ppp_local(x, grid, False)]
    got, _ = emulate_ppp((n, n, n), grid, FWD, local)
    del local
    host = torch.empty((n, n, n), dtype=torch.complex64).pin_memory()
    h = n // 2
    for r in range(4):
        p, q = r % 2, r // 2
        host[:, q * h:(q + 1) * h, p * h:(p + 1) * h].copy_(got[r].reshape(n, h, h))
    del got
    torch.cuda.empty_cache()
    _sampled_check(x, host.numpy(), n, FWD, 83)
