"""The N > 1 path of bench.py on CPU: two ranks over gloo (one process per
rank, rendezvous on 127.0.0.1), the job time is the slowest rank's and the
whole-job value divides it by the number of replicas."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, q):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        local = 3.0 + 2.5 * rank          # rank 1 is the slow one
        t = bench.max_over_ranks(local, "cpu")
        q.put((rank, t, bench.job_ms_per_transform(t, world)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_over_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [g[1] for g in got] == [5.5, 5.5]      # both ranks see the slowest rank's time
    assert [g[2] for g in got] == [2.75, 2.75]    # two transforms per step of 5.5 ms


def test_single_process_needs_no_group():
    import bench
    assert not dist.is_initialized()
    assert bench.max_over_ranks(4.0, "cpu") == 4.0
    assert bench.job_ms_per_transform(4.0, 1) == 4.0


def test_reference_arm_runs_on_rank_0_only():
    """`bench.py --impl reference` (the FP64 oracle on the host cores): one JSON
    line from rank 0 with the contract's keys; any other rank exits 0 silently."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--n", "16", "--steps", "2",
           "--warmup", "3"]
    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    out = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=300, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads([ln for ln in out.stdout.splitlines() if ln.startswith("{")][-1])
    assert line["impl"] == "reference" and line["unit"] == "ms" and line["higher_is_better"] is False
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    # every step is one whole transform of the workload, so the value is the measured step time
    assert "full forward 16^3 transform" in line["cpu_baseline"]["sample"]
    assert line["ms_per_step"] == line["value"] and line["steps"] == 2
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    out = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=300, cwd=root)
    assert out.returncode == 0 and not out.stdout.strip()


def test_traffic_table_is_keyed_to_the_measured_kernels_sources():
    """bench.py reads profiles/traffic.txt only while the translation units of
    the measured kernels and every header they include are unchanged: the hash
    follows those files (and ignores the others)."""
    import importlib
    import shutil
    import tempfile
    import bench
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with tempfile.TemporaryDirectory() as tmp:
        shutil.copytree(os.path.join(root, "paper_1904_10119_gb300", "csrc"),
                        os.path.join(tmp, "paper_1904_10119_gb300", "csrc"))
        old = bench.ROOT
        try:
            bench.ROOT = tmp
            h0 = bench._csrc_sha()
            with open(os.path.join(tmp, "paper_1904_10119_gb300", "csrc", "k_segmented.cu"), "a") as f:
                f.write("\n// unrelated edit\n")
            assert bench._csrc_sha() == h0          # not in the closure
            with open(os.path.join(tmp, "paper_1904_10119_gb300", "csrc", "fft_engine.cuh"), "a") as f:
                f.write("\n// edit of an included header\n")
            assert bench._csrc_sha() != h0          # included by the measured kernels
        finally:
            bench.ROOT = old
    importlib.reload(bench)
