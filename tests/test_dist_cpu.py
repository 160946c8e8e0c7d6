"""The distributed slab-pencil decomposition (Section 2.4, Fig. 3dslabpencil)
on the host: the rank-local stage schedules the planner lowers
(fft3_options.dist_ranks / dist_stage), replayed numerically with an FP64 line
DFT through their pass geometries, and the driver that joins them with
torch.distributed all-to-alls, run as 2 and 4 gloo ranks (one process per
rank, rendezvous on 127.0.0.1) against the oracle's slab-pencil simulation."""
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
            src = (j * g["ij"] + c * g["ic"] + a * g["ia"] + b * g["ib"]).reshape(n, -1)
            dst = (j * g["ok"] + c * g["oc"] + a * g["oa"] + b * g["ob"]).reshape(n, -1)
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


@pytest.mark.parametrize("decomp,dtype,batch", [(fft3.FFT3_PENCIL3, fft3.FFT3_C64_FP32, 1),
                                                (fft3.FFT3_VOLUMETRIC, fft3.FFT3_C64_FP32, 1),
                                                (S, fft3.FFT3_C64_SPLITBF16_TC, 1), (S, fft3.FFT3_C64_FP32, 2)])
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
