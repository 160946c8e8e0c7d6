"""The distributed decompositions of Section 2.4 on the host: slab-pencil on
a 1D grid (Fig. 3dslabpencil) and pencil-pencil-pencil on a 2D grid (Fig.
3dpencilpencil).  The rank-local stage schedules the planner lowers
(fft3_options.dist_ranks / dist_ranks2 / dist_stage) are replayed numerically
with an FP64 line DFT through their pass geometries, and the drivers that join
them with torch.distributed all-to-alls run as gloo ranks (one process per
rank, rendezvous on 127.0.0.1), both against the oracle's simulations."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1904_10119_gb300 import fft3

S = fft3.FFT3_SLAB_PENCIL
P3 = fft3.FFT3_PENCIL3
FWD, INV = fft3.FFT3_FORWARD, fft3.FFT3_INVERSE


def dist_schedule(dims, stage, P, direction=FWD, dtype=fft3.FFT3_C64_FP32):
    return fft3.fft3_plan_schedule(*dims, 1, dtype, S, direction,
                                   fft3.make_options(dist_ranks=P, dist_stage=stage))


class ReplayStage:
    """Executes a schedule on the host: every pass gathers its lines through the
    input geometry, multiplies them by the FP64 DFT matrix of the oracle and
    scatters them through the output geometry."""

    def __init__(self, schedule, sign):
        self.s, self.sign = schedule, sign

    def execute(self, x, out):
        total = x.numel()
        bufs = {"in": x.numpy().ravel().astype(np.complex128), "out": np.full(total, np.nan, np.complex128),
                "workspace": np.full(total, np.nan, np.complex128)}
        for p in self.s["passes"]:
            g = p["geom"]
            if p["kind"] == "copy":
                bufs[p["dst"]][:] = bufs[p["src"]]
                continue
            n = p["line"]["n"]
            j = np.arange(n)[:, None, None, None]
            c = np.arange(g["C"])[None, :, None, None]
            a = np.arange(g["A"])[None, None, :, None]
            b = np.arange(g["B"])[None, None, None, :]
            # a line in runs over exchange blocks: element j at (j / jb) * blk + (j % jb) * stride
            jin = (j // g["ijb"]) * g["iblk"] + (j % g["ijb"]) * g["ij"] if g.get("ijb") else j * g["ij"]
            jout = (j // g["okb"]) * g["oblk"] + (j % g["okb"]) * g["ok"] if g.get("okb") else j * g["ok"]
            src = (jin + c * g["ic"] + a * g["ia"] + b * g["ib"]).reshape(n, -1)
            dst = (jout + c * g["oc"] + a * g["oa"] + b * g["ob"]).reshape(n, -1)
            lines = oracle.dft_matrix(n, self.sign) @ bufs[p["src"]][src]
            bufs[p["dst"]][dst] = lines
        out.copy_(torch.from_numpy(bufs["out"]).to(out.dtype).reshape(out.shape))


def test_stage_schedules():
    """Slab stage: x pass into the workspace, y pass storing the packed blocks;
    pencil stage: one z pass; stage 3: one pass of one-point lines.  The
    inverse slab stage reads the packed blocks first."""
    s1 = dist_schedule((64, 32, 8), 1, 4)
    assert s1["decomposition"] == "slab_pencil" and (s1["dist_ranks"], s1["dist_stage"]) == (4, 1)
    assert [(p["dim"], p["src"], p["dst"]) for p in s1["passes"]] == [(0, "in", "workspace"), (1, "workspace", "out")]
    gy = s1["passes"][1]["geom"]
    assert (gy["C"], gy["A"], gy["B"]) == (16, 8, 4)
    assert (gy["ij"], gy["ia"], gy["ib"]) == (64, 64 * 32, 16)
    assert (gy["ok"], gy["oa"], gy["ob"]) == (16, 32 * 16, 8 * 32 * 16)
    si = dist_schedule((64, 32, 8), 1, 4, INV)
    assert [(p["dim"], p["src"], p["dst"]) for p in si["passes"]] == [(1, "in", "workspace"), (0, "workspace", "out")]
    s2 = dist_schedule((16, 32, 32), 2, 4)
    assert [(p["dim"], p["src"], p["dst"]) for p in s2["passes"]] == [(2, "in", "out")]
    assert s2["workspace_bytes"] == 0
    s3 = dist_schedule((64, 32, 8), 3, 4)
    assert len(s3["passes"]) == 1 and s3["passes"][0]["line"]["n"] == 1
    s1c = dist_schedule((64, 32, 8), 1, 2, dtype=fft3.FFT3_C128_FP64)
    assert s1c["dtype"] == fft3.FFT3_C128_FP64 and len(s1c["passes"]) == 2


INVALID, UNSUPPORTED = -1, -2   # FFT3_ERR_INVALID_ARG, FFT3_ERR_UNSUPPORTED_SIZE


@pytest.mark.parametrize("opts,code", [
    ({"dist_ranks": 2}, INVALID), ({"dist_stage": 1}, INVALID), ({"dist_ranks": 2, "dist_stage": 4}, INVALID),
    ({"dist_ranks": -2, "dist_stage": 1}, INVALID),
    ({"dist_ranks": 3, "dist_stage": 1}, UNSUPPORTED),   # 3 does not divide n0 = 64
    ({"dist_ranks": 3, "dist_stage": 3}, UNSUPPORTED),
    ({"dist_ranks": 2, "dist_stage": 1, "layout": fft3.FFT3_LAYOUT_PENCILS}, UNSUPPORTED)])
def test_stage_options_rejected(opts, code):
    with pytest.raises(fft3.Fft3Error) as e:
        fft3.fft3_plan_schedule(64, 32, 8, 1, 0, S, FWD, fft3.make_options(**opts))
    assert e.value.code == code


@pytest.mark.parametrize("decomp,dtype,batch", [(fft3.FFT3_VOLUMETRIC, fft3.FFT3_C64_FP32, 1),
                                                (S, fft3.FFT3_C64_SPLITBF16_TC, 1), (S, fft3.FFT3_C64_FP32, 2),
                                                (P3, fft3.FFT3_C64_SPLITBF16_TC, 1), (P3, fft3.FFT3_C64_FP32, 2)])
def test_stage_needs_one_slab_pencil_problem(decomp, dtype, batch):
    with pytest.raises(fft3.Fft3Error) as e:
        fft3.fft3_plan_schedule(64, 32, 8, batch, dtype, decomp, FWD, fft3.make_options(dist_ranks=2, dist_stage=1))
    assert e.value.code == UNSUPPORTED


def _local_inputs(dims, P, spectrum, natural, seed):
    n0, n1, n2 = dims
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, (n2, n1, n0)) + 1j * rng.uniform(-1, 1, (n2, n1, n0))
    if spectrum and not natural:
        return x, [np.ascontiguousarray(x[:, :, r * (n0 // P):(r + 1) * (n0 // P)]) for r in range(P)]
    return x, [np.ascontiguousarray(x[r * (n2 // P):(r + 1) * (n2 // P)]) for r in range(P)]


@pytest.mark.parametrize("dims,P", [((16, 6, 8), 2), ((12, 5, 8), 4), ((20, 1, 6), 2)])
@pytest.mark.parametrize("direction,natural", [(FWD, False), (FWD, True), (INV, False), (INV, True)])
def test_replayed_stages_match_the_simulation(dims, P, direction, natural):
    """Each rank's stages, replayed on the host, with the all-to-alls done by
    slicing: every rank's output equals the oracle's simulation to FP64
    rounding, and the forward spectrum reassembled equals the whole 3D DFT."""
    n0, n1, n2 = dims
    x, local = _local_inputs(dims, P, direction == INV, natural, seed=sum(dims) + P)
    st = {1: ReplayStage(dist_schedule((n0, n1, n2 // P), 1, P, direction), direction),
          2: ReplayStage(dist_schedule((n0 // P, n1, n2), 2, P, direction), direction),
          3: ReplayStage(dist_schedule((n0, n1, n2 // P), 3, P, direction), direction)}
    blk = n0 * n1 * n2 // P ** 2

    def run(stage, arrays):
        outs = []
        for a in arrays:
            o = torch.empty(a.size, dtype=torch.complex128)
            st[stage].execute(torch.from_numpy(a.ravel().copy()), o)
            outs.append(o.numpy())
        return outs

    def exchange(sends):   # rank r receives block r of every rank, in rank order
        return [np.concatenate([sends[s][r * blk:(r + 1) * blk] for s in range(P)]) for r in range(P)]

    if direction == FWD:
        data = run(2, exchange(run(1, local)))
        if natural:
            data = run(3, exchange(data))
    else:
        data = run(3, local) if natural else [a.ravel() for a in local]
        if natural:
            data = exchange(data)
        data = run(1, exchange(run(2, data)))
    ref = oracle.slab_pencil_sim(local, n0, n1, n2, P, direction, natural)
    scale = max(np.abs(r).max() for r in ref)
    for got, want in zip(data, ref):
        assert np.abs(got - want.ravel()).max() <= 1e-12 * scale
    if direction == FWD:
        whole = oracle.fft3(x, n0, n1, n2)
        joined = (np.concatenate([d.reshape(n2 // P, n1, n0) for d in data], axis=0) if natural else
                  np.concatenate([d.reshape(n2, n1, n0 // P) for d in data], axis=2))
        assert np.abs(joined - whole).max() <= 1e-12 * np.abs(whole).max()


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, cases, q):
    from paper_1904_10119_gb300.distributed import SlabPencil
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        for dims, direction, natural in cases:
            n0, n1, n2 = dims
            P = world
            st = {1: ReplayStage(dist_schedule((n0, n1, n2 // P), 1, P, direction), direction),
                  2: ReplayStage(dist_schedule((n0 // P, n1, n2), 2, P, direction), direction),
                  3: ReplayStage(dist_schedule((n0, n1, n2 // P), 3, P, direction), direction)}
            sp = SlabPencil(n0, n1, n2, direction, natural_spectrum=natural, dtype=fft3.FFT3_C128_FP64, stages=st)
            x, local = _local_inputs(dims, P, direction == INV, natural, seed=sum(dims))
            out = torch.empty(sp.local_shape(spectrum=direction == FWD), dtype=torch.complex128)
            sp.execute(torch.from_numpy(local[rank]), out)
            q.put((rank, dims, direction, natural, out.numpy()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,cases", [
    (2, [((16, 6, 8), FWD, False), ((16, 6, 8), FWD, True), ((16, 6, 8), INV, False), ((10, 3, 4), INV, True)]),
    (4, [((8, 5, 12), FWD, False), ((8, 5, 12), INV, True)])])
def test_driver_over_gloo(world, cases):
    """The driver's all-to-alls over gloo: each rank's output equals the
    oracle's simulation of the distributed algorithm for that rank."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, cases, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in range(world * len(cases))]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, dims, direction, natural, out in got:
        n0, n1, n2 = dims
        _, local = _local_inputs(dims, world, direction == INV, natural, seed=sum(dims))
        want = oracle.slab_pencil_sim(local, n0, n1, n2, world, direction, natural)[rank]
        assert out.shape == want.shape
        assert np.abs(out - want).max() <= 1e-12 * np.abs(want).max()


# ------------------------------------------------------------------------- #
# pencil-pencil-pencil on a Py x Pz grid                                    #
# ------------------------------------------------------------------------- #
def ppp_schedule(dims, stage, grid, direction=FWD):
    return fft3.fft3_plan_schedule(*dims, 1, 0, P3, direction,
                                   fft3.make_options(dist_ranks=grid[0], dist_ranks2=grid[1], dist_stage=stage))


def ppp_stages(n, grid, direction):
    n0, n1, n2 = n
    Py, Pz = grid
    dims = {1: (n0, n1 // Py, n2 // Pz), 2: (n0 // Py, n1, n2 // Pz), 3: (n0 // Py, n1 // Pz, n2)}
    return {k: ReplayStage(ppp_schedule(d, k, grid, direction), direction) for k, d in dims.items()}


def test_ppp_stage_schedules():
    """One pass per stage: the x pass with the rotated store (x blocks
    contiguous), the y and z passes reading their lines in Py / Pz runs
    (two-level line index, the runtime-radix kernel); the inverse stores in
    runs what the forward reads in runs."""
    s1 = ppp_schedule((8, 3, 2), 1, (2, 2))
    assert [p["kind"] for p in s1["passes"]] == ["line_contig_rotate"] and s1["decomposition"] == "pencil_pencil_pencil"
    g1 = s1["passes"][0]["geom"]
    assert (g1["ok"], g1["oc"], g1["oa"]) == (6, 1, 3)                      # out [x][z][y]
    g2 = ppp_schedule((4, 6, 2), 2, (2, 2))["passes"][0]["geom"]
    assert (g2["ijb"], g2["iblk"], g2["ij"], g2["ok"]) == (3, 24, 1, 8)     # y runs of n1/Py, out [y][z][x]
    g3 = ppp_schedule((4, 3, 4), 3, (2, 2))["passes"][0]["geom"]
    assert (g3["ijb"], g3["iblk"], g3["ij"], g3["ok"]) == (2, 24, 4, 12)    # z runs of n2/Pz, out [z][y][x]
    g3i = ppp_schedule((4, 3, 4), 3, (2, 2), INV)["passes"][0]["geom"]
    assert (g3i["okb"], g3i["oblk"], g3i["ok"], g3i["ij"]) == (2, 24, 4, 12)
    assert all(ppp_schedule(d, k, (2, 2))["workspace_bytes"] == 0
               for k, d in ((1, (8, 3, 2)), (2, (4, 6, 2)), (3, (4, 3, 4))))


@pytest.mark.parametrize("opts,dims,code", [
    ({"dist_ranks": 1, "dist_stage": 1}, (8, 4, 4), INVALID),                      # a 1 x 1 grid
    ({"dist_ranks": 0, "dist_ranks2": 2, "dist_stage": 2}, (8, 4, 4), INVALID),
    ({"dist_ranks2": 2}, (8, 4, 4), INVALID),                                       # grid without a stage
    ({"dist_ranks": 3, "dist_ranks2": 1, "dist_stage": 1}, (8, 4, 4), UNSUPPORTED),  # 3 does not divide n0
    ({"dist_ranks": 2, "dist_ranks2": 3, "dist_stage": 2}, (4, 8, 4), UNSUPPORTED),  # 3 does not divide n1
    ({"dist_ranks": 2, "dist_ranks2": 3, "dist_stage": 3}, (4, 4, 8), UNSUPPORTED)])  # 3 does not divide n2
def test_ppp_stage_options_rejected(opts, dims, code):
    with pytest.raises(fft3.Fft3Error) as e:
        fft3.fft3_plan_schedule(*dims, 1, 0, P3, FWD, fft3.make_options(**opts))
    assert e.value.code == code
    with pytest.raises(fft3.Fft3Error) as e:   # the slab-pencil grid is one-dimensional
        fft3.fft3_plan_schedule(8, 4, 4, 1, 0, S, FWD, fft3.make_options(dist_ranks=2, dist_ranks2=2, dist_stage=1))
    assert e.value.code == INVALID


def _ppp_inputs(n, grid, spectrum, seed):
    n0, n1, n2 = n
    Py, Pz = grid
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, (n2, n1, n0)) + 1j * rng.uniform(-1, 1, (n2, n1, n0))
    out = []
    for r in range(Py * Pz):
        p, q = r % Py, r // Py
        if spectrum:
            out.append(np.ascontiguousarray(x[:, q * (n1 // Pz):(q + 1) * (n1 // Pz), p * (n0 // Py):(p + 1) * (n0 // Py)]))
        else:
            out.append(np.ascontiguousarray(x[q * (n2 // Pz):(q + 1) * (n2 // Pz), p * (n1 // Py):(p + 1) * (n1 // Py)]))
    return x, out


@pytest.mark.parametrize("n,grid", [((8, 6, 4), (2, 2)), ((6, 6, 6), (3, 2)), ((4, 8, 6), (1, 2)), ((6, 3, 5), (3, 1)),
                                    ((12, 12, 8), (2, 4))])
@pytest.mark.parametrize("direction", [FWD, INV])
def test_ppp_replayed_stages_match_the_simulation(n, grid, direction):
    """Each rank's three stages replayed on the host, the row and column
    all-to-alls done by slicing: every rank's output equals the oracle's
    simulation, and the forward bricks reassembled equal the whole 3D DFT."""
    n0, n1, n2 = n
    Py, Pz = grid
    x, local = _ppp_inputs(n, grid, direction == INV, seed=sum(n) + Py)
    st = ppp_stages(n, grid, direction)
    R = Py * Pz

    def run(k, arrays):
        outs = []
        for a in arrays:
            o = torch.empty(a.size, dtype=torch.complex128)
            st[k].execute(torch.from_numpy(a.ravel().copy()), o)
            outs.append(o.numpy())
        return outs

    def exchange(sends, row):   # within each row (same q) or column (same p), blocks in member order
        outs = [None] * R
        for r in range(R):
            p, q = r % Py, r // Py
            members = [q * Py + i for i in range(Py)] if row else [j * Py + p for j in range(Pz)]
            me = members.index(r)
            blk = sends[r].size // len(members)
            outs[r] = np.concatenate([sends[m][me * blk:(me + 1) * blk] for m in members])
        return outs

    if direction == FWD:
        data = run(3, exchange(run(2, exchange(run(1, local), True)), False))
    else:
        data = run(1, exchange(run(2, exchange(run(3, local), False)), True))
    ref = oracle.pencil3_sim(local, n0, n1, n2, Py, Pz, direction)
    scale = max(np.abs(r).max() for r in ref)
    for got, want in zip(data, ref):
        assert np.abs(got - want.ravel()).max() <= 1e-12 * scale
    if direction == FWD:
        whole = oracle.fft3(x, n0, n1, n2)
        for r, got in enumerate(data):
            p, q = r % Py, r // Py
            brick = whole[:, q * (n1 // Pz):(q + 1) * (n1 // Pz), p * (n0 // Py):(p + 1) * (n0 // Py)]
            assert np.abs(got.reshape(brick.shape) - brick).max() <= 1e-12 * np.abs(whole).max()


def _ppp_rank_main(rank, world, port, grid, cases, q):
    from paper_1904_10119_gb300.distributed import Pencil3
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        for n, direction in cases:
            pp = Pencil3(*n, grid, direction, dtype=fft3.FFT3_C128_FP64, stages=ppp_stages(n, grid, direction))
            _, local = _ppp_inputs(n, grid, direction == INV, seed=sum(n))
            out = torch.empty(pp.local_shape(spectrum=direction == FWD), dtype=torch.complex128)
            pp.execute(torch.from_numpy(local[rank]), out)
            q.put((rank, n, direction, out.numpy()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("grid,cases", [((2, 2), [((8, 6, 4), FWD), ((8, 6, 4), INV)]),
                                        ((2, 1), [((4, 6, 3), FWD)]), ((1, 2), [((3, 4, 6), INV)])])
def test_ppp_driver_over_gloo(grid, cases):
    """The pencil-pencil-pencil driver's row and column all-to-alls over gloo
    (subgroups of the 2 x 2, 2 x 1 and 1 x 2 grids): each rank's output equals
    the oracle's simulation for that rank."""
    world = grid[0] * grid[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_ppp_rank_main, args=(r, world, port, grid, cases, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in range(world * len(cases))]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, n, direction, out in got:
        _, local = _ppp_inputs(n, grid, direction == INV, seed=sum(n))
        want = oracle.pencil3_sim(local, *n, grid[0], grid[1], direction)[rank]
        assert out.shape == want.shape
        assert np.abs(out - want).max() <= 1e-12 * np.abs(want).max()
