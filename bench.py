"""Benchmark: forward 3D complex DFT of 1024^3 complex64 on one GB300 (or N
replicas under torchrun), through the libfft3 C ABI.

Prints ONE JSON line (rank 0).  A step is one complete forward transform of a
1024 x 1024 x 1024 complex64 array (8 GiB, out-of-place) with the inputs
already resident in HBM; `value` is ms per transform for the whole job.
`e2e` times the same transform through fft3_plan_execute_host with pinned
host buffers (host-to-device copy, transform, device-to-host copy per step).
`roofline` reports the dominant pass against the measured HBM copy
bandwidth; `cpu_baseline` the FP64 oracle timed on whole transforms of the
same workload on the host cores (in place on one complex128 array).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "1024^3 c64 3D-DFT ms & HBM roofline %; split-BF16 TC vs FP32 at rel-L2≤1e-5"
HBM_FALLBACK_GBS = 6800.0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


# Translation units of the kernels whose DRAM traffic profiles/traffic.txt records
# (the streamed strided pass and the contiguous pass).
_TRAFFIC_UNITS = ("k_cstream.cu", "k_fixed_a.cu", "k_fixed_b.cu")


def _csrc_sha() -> str:
    """Hash of the sources those kernels compile from: their translation units
    and every header they include, directly or not."""
    d = os.path.join(ROOT, "paper_1904_10119_gb300", "csrc")
    seen, stack = set(), list(_TRAFFIC_UNITS)
    while stack:
        name = stack.pop()
        path = os.path.join(d, name)
        if name in seen or not os.path.exists(path):
            continue
        seen.add(name)
        for line in open(path):
            m = re.match(r'\s*#include\s+"([^"]+)"', line)
            if m and not m.group(1).startswith(".."):
                stack.append(os.path.normpath(m.group(1)))
    h = hashlib.sha256()
    for name in sorted(seen):
        with open(os.path.join(d, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def max_over_ranks(x: float, device) -> float:
    """The largest of x over the ranks of the default process group (x itself
    without one): the job's step time is that of its slowest rank."""
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    if torch.distributed.is_available() and torch.distributed.is_initialized() and \
            torch.distributed.get_world_size() > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_ms_per_transform(step_ms: float, world: int) -> float:
    """Whole-job ms per transform: the path shards by independent transforms
    (replicas), every rank runs one per step, so `world` transforms finish in
    one step of the slowest rank."""
    return step_ms / world


def _profiled_traffic(kernel_kind: str):
    """DRAM bytes per launch of `kernel_kind` from the committed ncu summary,
    if it was taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    sha = _csrc_sha()
    for line in open(path):
        m = re.match(r"\s*(\w+)\s+traffic_per_launch_bytes=(\d+)\s+source_sha=(\w+)", line)
        if m and m.group(1) == kernel_kind and m.group(3) == sha:
            return int(m.group(2))
    return None


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sms.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        sms.sort()
        med = sms[len(sms) // 2] if sms else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sms)}


# ----------------------------------------------------------- CPU oracle ---- #
def _mem_available() -> int:
    """Bytes of host memory available to a new allocation (/proc/meminfo)."""
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


def oracle_cube(n: int, reserve: int = 0) -> int:
    """Edge of the largest cube, n or n/2^k, whose complex128 array (plus the
    complex64 input it is widened from and `reserve` bytes) fits host memory."""
    avail = _mem_available() - reserve
    m = n
    while m > 64 and 24 * m ** 3 * 1.1 > avail:
        m //= 2
    return m


class OracleTransforms:
    """Whole transforms of the FP64 oracle: the forward 3D DFT of an m^3
    complex128 array (the seeded complex64 input widened exactly), computed in
    place by oracle.fft3_inplace: x, y and z lines at their real strides, one
    array of 16 m^3 bytes.  Each call to step() times one full transform (the
    array keeps the previous output; the values only grow by m^1.5 per
    transform, far from overflow)."""

    def __init__(self, n: int, src=None, threads: int | None = None, reserve: int = 0):
        import numpy as np

        import oracle
        from paper_1904_10119_gb300 import synth
        if threads:
            oracle.set_num_threads(threads)
        self.oracle = oracle
        self.cores = oracle.num_threads()
        self.n = n
        self.m = m = oracle_cube(n, reserve)
        self.buf = np.empty((m, m, m), dtype=np.complex128)
        if src is not None and m == n:
            np.copyto(self.buf, src.reshape(m, m, m))
        else:
            np.copyto(self.buf, synth.uniform_c64((m, m, m), 4))

    def step(self) -> float:
        """ms of one full in-place m^3 transform."""
        t0 = time.perf_counter()
        self.oracle.fft3_inplace(self.buf.reshape(-1), self.m, self.m, self.m)
        return (time.perf_counter() - t0) * 1e3

    def to_workload_ms(self, ms: float) -> float:
        """ms per n^3 transform: the measured value itself when m == n, else
        scaled by the 5 N log2 N operation count (stated in the sample)."""
        if self.m == self.n:
            return ms
        big, small = self.n ** 3, self.m ** 3
        return ms * (big * math.log2(big)) / (small * math.log2(small))

    def sample(self, reps: int) -> str:
        s = (f"{reps} full forward {self.m}^3 transform(s) of the FP64 oracle, in place on one complex128 array "
             f"(x, y and z lines at their real strides), {self.cores} OpenMP threads")
        if self.m != self.n:
            s += (f"; host memory ({_mem_available() >> 30} GiB available) does not hold a {self.n}^3 "
                  f"complex128 array, so the {self.m}^3 time is scaled to {self.n}^3 by 5 N log2 N")
        return s


# --------------------------------------------------------------- main ---- #
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1024, help="cube edge (ignored with --shape)")
    ap.add_argument("--shape", type=int, nargs=3, default=None, metavar=("N0", "N1", "N2"))
    ap.add_argument("--decomp", default="auto",
                    choices=["auto", "slab_pencil", "slab_pencil_pipelined", "slab_pencil_fused", "ppp", "ppp_rotate",
                             "ppp_blocked", "volumetric"])
    ap.add_argument("--tile-lines", type=int, default=0)
    ap.add_argument("--slab-mode", type=int, default=0)
    ap.add_argument("--slab-chunk", type=int, default=0)
    ap.add_argument("--slab-lines", type=int, default=0)
    ap.add_argument("--radix-order", type=int, default=0)
    ap.add_argument("--dtype", default="f32", choices=["f32", "splitbf16"],
                    help="splitbf16: radix-16 stages on the tensor cores (hi+lo BF16, FP32 accumulation)")
    ap.add_argument("--tc-stages", type=int, default=0)
    ap.add_argument("--no-extras", action="store_true", help="skip the per-decomposition and batched tables")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer measurement")
    ap.add_argument("--cpu-reps", type=int, default=1,
                    help="whole oracle transforms timed for cpu_baseline (0 skips the CPU oracle baseline)")
    ap.add_argument("--batched", type=int, default=0, metavar="COUNT",
                    help="only time COUNT uneven cubes (seed 7): the default batched plan (the slab executor), the "
                         "segmented passes, the persistent executor and the one-launch segmented form")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    n0, n1, n2 = args.shape if args.shape else (args.n, args.n, args.n)
    N = n0 * n1 * n2
    flops = 5.0 * N * math.log2(N)
    workload = f"fft3d_c64_{n0}x{n1}x{n2}_forward_out_of_place"

    if args.impl == "reference":
        if rank != 0:
            return 0
        assert n0 == n1 == n2, "the CPU reference arm times cubic workloads"
        ref = OracleTransforms(n0)
        for _ in range(args.warmup):
            ref.step()
        vals = [ref.step() for _ in range(args.steps)]
        step_ms = sum(vals) / len(vals)
        v = ref.to_workload_ms(step_ms)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": workload, "dims": [n0, n1, n2], "batch": 1,
                           "oracle_cube": [ref.m] * 3},
                "cpu_baseline": {"value": v, "unit": "ms", "cores": ref.cores, "kind": "oracle",
                                 "sample": ref.sample(args.steps)},
                "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0

    import numpy as np
    import torch

    from paper_1904_10119_gb300 import fft3, synth

    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    if args.batched > 0:
        hbm, _ = _peaks()
        print(json.dumps({"batched": bench_batched(fft3, synth, torch, hbm, args.batched)}), flush=True)
        return 0

    decomp_map = {"auto": (fft3.FFT3_AUTO, {}), "slab_pencil": (fft3.FFT3_SLAB_PENCIL, {}),
                  "slab_pencil_pipelined": (fft3.FFT3_SLAB_PENCIL, {"slab_mode": 4}),
                  "slab_pencil_fused": (fft3.FFT3_SLAB_PENCIL, {"slab_mode": 5}),
                  "ppp": (fft3.FFT3_PENCIL3, {}), "ppp_rotate": (fft3.FFT3_PENCIL3, {"variant": 1}),
                  "ppp_blocked": (fft3.FFT3_PENCIL3, {"variant": 2}),
                  "volumetric": (fft3.FFT3_VOLUMETRIC, {})}

    # inputs: seeded uniform[-1,1) complex64, generated on the host into pinned memory
    h_in = torch.empty((n2, n1, n0), dtype=torch.complex64).pin_memory()
    synth.uniform_c64((n2, n1, n0), 4 + rank, out=h_in.numpy())
    x = h_in.to("cuda")
    out = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream

    def time_plan(decomp, opts, steps, warmup):
        plan = fft3.Plan(n0, n1, n2, 1, decomposition=decomp, **opts)
        npass = plan.launches()
        for _ in range(warmup):
            plan.execute(x, out)
        barrier()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(npass + 1)] for _ in range(steps)]
        for s in range(steps):
            evs[s][0].record(stream)
            for k in range(npass):
                fft3.fft3_plan_execute_pass(plan.handle, k, x.data_ptr(), out.data_ptr(), sp)
                evs[s][k + 1].record(stream)
        barrier()
        step_ms = [evs[s][0].elapsed_time(evs[s][npass]) for s in range(steps)]
        pass_ms = [sum(evs[s][k].elapsed_time(evs[s][k + 1]) for s in range(steps)) / steps
                   for k in range(npass)]
        assert plan.check() == 0, fft3.last_error()
        return plan, step_ms, pass_ms

    decomp, opts = decomp_map[args.decomp]
    opts = dict(opts)
    for k, v in (("tile_lines", args.tile_lines), ("slab_mode", args.slab_mode), ("slab_chunk", args.slab_chunk),
                 ("slab_lines", args.slab_lines), ("radix_order", args.radix_order)):
        if v:
            opts[k] = v
    if args.dtype == "splitbf16":
        opts["dtype"] = fft3.FFT3_C64_SPLITBF16_TC
        opts["tc_stages"] = args.tc_stages
    sampler = ClockSampler(dev)
    sampler.start()
    t_wall0 = time.perf_counter()
    plan, step_ms, pass_ms = time_plan(decomp, opts, args.steps, args.warmup)
    t_wall = time.perf_counter() - t_wall0
    clocks = sampler.stop()
    desc = plan.describe()
    mean_ms = sum(step_ms) / len(step_ms)
    t_step = max_over_ranks(mean_ms, "cuda")
    value = job_ms_per_transform(t_step, world)

    # roofline of the dominant pass
    hbm, peak_kind = _peaks()
    dom = max(range(len(pass_ms)), key=lambda k: pass_ms[k])
    alg_bytes = 2 * 8 * N  # each pass reads and writes the array once
    # a pipelined pair (x and y lines chunk by chunk on two streams) is timed as
    # one entry and needs to read and write the array once in all
    pair = desc["passes"][dom].get("pipelined_with") == "next"
    dom_bytes = alg_bytes
    achieved = dom_bytes / (pass_ms[dom] * 1e-3) / 1e9
    dom_kind = desc["passes"][dom]["kind"] + ("+" + desc["passes"][dom + 1]["kind"] if pair else "")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": _profiled_traffic(dom_kind), "kernel": dom_kind, "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": dom_bytes, "launch_ms": pass_ms[dom]}
    sweeps = len(pass_ms)
    whole = {"passes": sweeps, "bytes": sweeps * alg_bytes,
             "frac_of_plan_passes": sweeps * alg_bytes / (t_step * 1e-3) / 1e9 / hbm,
             "frac_of_3pass": 3 * alg_bytes / (t_step * 1e-3) / 1e9 / hbm,
             "frac_of_3pass_nominal_7900GBs": 3 * alg_bytes / (t_step * 1e-3) / 1e9 / 7900.0}

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        h_out = torch.empty_like(h_in).pin_memory()
        eplan = fft3.fft3_plan_create_ex(n0, n1, n2, 1, opts.get("dtype", 0), decomp, -1,
                                         fft3.make_options(**{k: v for k, v in opts.items() if k != "dtype"}))
        # every step copies its input from pinned host memory, transforms, and copies
        # the result back (fft3_plan_execute_host, synchronous per call)
        fft3.fft3_plan_execute_host(eplan, h_in.data_ptr(), h_out.data_ptr(), sp)
        e2e_steps = max(1, min(args.steps, 5))
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            fft3.fft3_plan_execute_host(eplan, h_in.data_ptr(), h_out.data_ptr(), sp)
        barrier()
        e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
        assert fft3.fft3_plan_check(eplan) == 0, fft3.last_error()
        # the pipelined form (copy in of i+1, transform of i, copy out of i-1 overlapped)
        fft3.fft3_plan_execute_host_pipelined(eplan, [h_in.data_ptr()] * 2, [h_out.data_ptr()] * 2, sp)
        t0 = time.perf_counter()
        fft3.fft3_plan_execute_host_pipelined(eplan, [h_in.data_ptr()] * 4, [h_out.data_ptr()] * 4, sp)
        barrier()
        pipelined_ms = (time.perf_counter() - t0) * 1e3 / 4
        direct = bool(fft3.fft3_plan_describe(eplan).get("host_direct"))
        fft3.fft3_plan_destroy(eplan)
        del h_out
        e2e = {"value": job_ms_per_transform(max_over_ranks(e2e_ms, "cuda"), world), "unit": "ms",
               "h2d_bytes_per_step": 8 * N,
               "d2h_bytes_per_step": 8 * N, "steps": e2e_steps, "api": "fft3_plan_execute_host",
               "path": ("direct input: the first pass reads the pinned host input over the host link; the "
                        "result is copied to the pinned host output" if direct else
                        "staged: copies between pinned host memory and device arrays around the transform"),
               "pipelined_ms_per_transform": pipelined_ms}

    extras = {}
    if not args.no_extras and rank == 0:
        variants = dict(decomp_map)
        variants["volumetric_mesh4_compiled"] = (fft3.FFT3_VOLUMETRIC, {"mesh": (1, 4, 4), "tile_lines": 16})
        variants["ppp_plain_strided_kernel"] = (fft3.FFT3_PENCIL3, {"tile_lines": 16})
        # the cyclic split and the blocked six-step split on the same runtime-radix cluster kernel
        variants["volumetric_cyclic_runtime_kernel"] = (fft3.FFT3_VOLUMETRIC, {"mesh": (1, 2, 2), "tile_lines": 8})
        variants["volumetric_blocked_six_step"] = (fft3.FFT3_VOLUMETRIC, {"variant": fft3.FFT3_VOL_BLOCKED_SIX_STEP,
                                                                          "mesh": (1, 2, 2), "tile_lines": 8})
        variants["permuted_output_pencils"] = (fft3.FFT3_AUTO, {"layout": fft3.FFT3_LAYOUT_PENCILS})
        variants["permuted_output_rotated"] = (fft3.FFT3_PENCIL3, {"layout": fft3.FFT3_LAYOUT_ROTATED})
        tc = fft3.FFT3_C64_SPLITBF16_TC
        variants["split_bf16_tc_radix32_tcgen05"] = (fft3.FFT3_AUTO, {"dtype": tc})
        variants["split_bf16_tc_one_stage_per_line_mma_sync"] = (fft3.FFT3_AUTO, {"dtype": tc, "tc_stages": 3})
        variants["split_bf16_tc_shared_memory_stages_mma_sync"] = (fft3.FFT3_AUTO, {"dtype": tc, "tc_stages": 1})
        variants["split_bf16_tc_every_stage_mma_sync"] = (fft3.FFT3_AUTO, {"dtype": tc, "tc_stages": 2})
        for name, (d, o) in variants.items():
            if name == "auto":
                continue
            try:
                p, sm, pm = time_plan(d, o, max(3, args.steps // 2), 3)
                extras[name] = {"ms": sum(sm) / len(sm), "pass_ms": pm,
                                "kinds": [q["kind"] for q in p.describe()["passes"]]}
                p.close()
            except Exception as e:  # report, do not hide
                extras[name] = {"error": str(e)}
        try:
            pf = fft3.Plan(n0, n1, n2, 1, decomposition=decomp, **opts)
            pi = fft3.Plan(n0, n1, n2, 1, decomposition=decomp, direction=fft3.FFT3_INVERSE, **opts)
            for _ in range(3):
                pf.execute(x, out)
                pi.execute(out, x)
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = max(3, args.steps // 2)
            e0.record(stream)
            for _ in range(reps):
                pf.execute(x, out)
                pi.execute(out, x)
            e1.record(stream)
            barrier()
            extras["forward_plus_inverse_ms"] = e0.elapsed_time(e1) / reps
            pf.close()
            pi.close()
        except Exception as e:
            extras["forward_plus_inverse_ms"] = {"error": str(e)}
        try:
            extras["batched_4096_uneven"] = bench_batched(fft3, synth, torch, hbm)
        except Exception as e:  # noqa: BLE001
            extras["batched_4096_uneven"] = {"error": str(e)}
        try:
            extras["complex128_fp64"] = c128_table(fft3, synth, torch)
        except Exception as e:  # noqa: BLE001
            extras["complex128_fp64"] = {"error": str(e)}
        if n0 == n1 == n2 == 1024:
            try:
                extras["slab_pencil_rank_local"] = dist_table(fft3, torch, n0, hbm)
            except Exception as e:  # noqa: BLE001
                extras["slab_pencil_rank_local"] = {"error": str(e)}
            try:
                extras["smaller_cubes"] = size_table(fft3, synth, torch, (256, 512), decomp_map)
            except Exception as e:
                extras["smaller_cubes"] = {"error": str(e)}

    cpu = None
    if rank == 0 and world == 1 and args.cpu_reps > 0 and n0 == n1 == n2:
        try:
            ref = OracleTransforms(n0, src=h_in.numpy())
            ms = sum(ref.step() for _ in range(args.cpu_reps)) / args.cpu_reps
            cpu = {"value": ref.to_workload_ms(ms), "unit": "ms", "cores": ref.cores, "kind": "oracle",
                   "sample": ref.sample(args.cpu_reps)}
            del ref
        except Exception as e:
            cpu = {"value": None, "unit": "ms", "cores": None, "kind": "oracle", "sample": f"failed: {e}"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.dtype == "f32" else "bf16x3_f32acc", "data": "synthetic",
            "config": {"workload": workload, "dims": [n0, n1, n2], "batch": 1,
                       "decomposition": desc["decomposition"], "passes": [p["kind"] for p in desc["passes"]],
                       "options": opts, "parallelism": f"replicas{world}" if world > 1 else "single",
                       "inputs": "uniform[-1,1) complex64, seed 4+rank",
                       "l2": "no flush: each pass streams the whole array in and out, larger than the 129 MB L2"},
            "e2e": e2e,
            "gpu_launches": plan.kernel_launches() * args.steps,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gflops": flops / (t_step * 1e-3) / 1e9,
            "pass_ms": pass_ms,
            "whole_transform_hbm": whole,
            "step_ms_min_max": [min(step_ms), max(step_ms)],
            "timed_wall_s": t_wall,
            "decompositions": extras,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def size_table(fft3, synth, torch, sizes, decomp_map):
    """Forward and inverse ms of n^3 (one transform, out of place) under each
    decomposition, CUDA events over 10 back-to-back executions."""
    table = {}
    st = torch.cuda.current_stream()
    for n in sizes:
        x = torch.empty((n, n, n), dtype=torch.complex64).pin_memory()
        synth.uniform_c64((n, n, n), 2, out=x.numpy())
        x = x.to("cuda")
        out = torch.empty_like(x)
        row = {}
        for name, (d, o) in decomp_map.items():
            if name == "auto":
                continue
            ent = {}
            for dname, direction in (("fwd_ms", fft3.FFT3_FORWARD), ("inv_ms", fft3.FFT3_INVERSE)):
                p = fft3.Plan(n, n, n, 1, decomposition=d, direction=direction, **o)
                for _ in range(3):
                    p.execute(x, out)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                for _ in range(10):
                    p.execute(x, out)
                e1.record(st)
                torch.cuda.synchronize()
                assert p.check() == 0, fft3.last_error()
                ent[dname] = e0.elapsed_time(e1) / 10
                ent["kinds"] = [q["kind"] for q in p.describe()["passes"]]
                p.close()
            row[name] = ent
        table[f"{n}^3"] = row
        del x, out
    return table


def dist_table(fft3, torch, n, hbm, ranks=(2, 4, 8), reps=10):
    """Local work of one rank of the distributed decompositions (n^3 forward),
    each stage timed with CUDA events over `reps` back-to-back executions on
    this GPU.  Slab-pencil on a 1D grid of P processes: the slab stage on n/P
    slabs (x pass, y pass storing the blocks packed for the all-to-all) and the
    pencil stage on the n/P-wide x range (z pass).  Pencil-pencil-pencil on a
    Py x Pz grid: its x, y and z stages.  The all-to-alls between stages run
    over the interconnect and are not part of these numbers."""
    table = {}
    st = torch.cuda.current_stream()
    for P in ranks:
        loc = n * n * n // P
        a = torch.empty(loc, dtype=torch.complex64, device="cuda")
        a.real.uniform_(-1, 1)
        a.imag.uniform_(-1, 1)
        b = torch.empty_like(a)
        row = {}
        for name, dims, stage in (("slab_stage_ms", (n, n, n // P), 1), ("pencil_stage_ms", (n // P, n, n), 2)):
            p = fft3.Plan(*dims, 1, fft3.FFT3_SLAB_PENCIL, fft3.FFT3_FORWARD, dist_ranks=P, dist_stage=stage)
            for _ in range(3):
                p.execute(a, b)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(reps):
                p.execute(a, b)
            e1.record(st)
            torch.cuda.synchronize()
            assert p.check() == 0, fft3.last_error()
            row[name] = e0.elapsed_time(e1) / reps
            row[name.replace("_ms", "_kinds")] = [q["kind"] for q in p.describe()["passes"]]
            p.close()
        ms = row["slab_stage_ms"] + row["pencil_stage_ms"]
        row["local_ms"] = ms
        # three sweeps of the rank's data, each read and written once
        row["local_hbm_frac_of_measured"] = 3 * 2 * 8 * loc / (ms * 1e-3) / 1e9 / hbm
        row["exchange_bytes_per_rank"] = 8 * loc * (P - 1) // P
        table[f"P{P}"] = row
        del a, b
    # pencil-pencil-pencil on a Py x Pz grid: the three stages of one rank
    for Py, Pz in ((2, 2), (4, 2)):
        loc = n * n * n // (Py * Pz)
        a = torch.empty(loc, dtype=torch.complex64, device="cuda")
        a.real.uniform_(-1, 1)
        a.imag.uniform_(-1, 1)
        b = torch.empty_like(a)
        row = {}
        dims = {1: (n, n // Py, n // Pz), 2: (n // Py, n, n // Pz), 3: (n // Py, n // Pz, n)}
        for stage, d in dims.items():
            p = fft3.Plan(*d, 1, fft3.FFT3_PENCIL3, fft3.FFT3_FORWARD, dist_ranks=Py, dist_ranks2=Pz,
                          dist_stage=stage)
            for _ in range(3):
                p.execute(a, b)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(reps):
                p.execute(a, b)
            e1.record(st)
            torch.cuda.synchronize()
            assert p.check() == 0, fft3.last_error()
            row[f"stage{stage}_ms"] = e0.elapsed_time(e1) / reps
            row[f"stage{stage}_kind"] = p.describe()["passes"][0]["kind"]
            p.close()
        ms = row["stage1_ms"] + row["stage2_ms"] + row["stage3_ms"]
        row["local_ms"] = ms
        row["local_hbm_frac_of_measured"] = 3 * 2 * 8 * loc / (ms * 1e-3) / 1e9 / hbm
        table[f"pencil3_{Py}x{Pz}"] = row
        del a, b
    return table


def c128_table(fft3, synth, torch, sizes=(256, 512, 1024), reps=5):
    """complex128 (FP64 butterflies and twiddles) forward ms of n^3, out of
    place, CUDA events over `reps` back-to-back executions; GFLOP/s in the
    5 N log2 N convention (the path is bound by FP64 arithmetic)."""
    import math
    table = {}
    st = torch.cuda.current_stream()
    for n in sizes:
        # timing only: uniform[-1,1) parts drawn on the device (16 GiB at 1024^3)
        x = torch.empty((n, n, n), dtype=torch.complex128, device="cuda")
        x.real.uniform_(-1, 1)
        x.imag.uniform_(-1, 1)
        out = torch.empty_like(x)
        p = fft3.Plan(n, n, n, 1, decomposition=fft3.FFT3_PENCIL3, dtype=fft3.FFT3_C128_FP64)
        p.execute(x, out)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            p.execute(x, out)
        e1.record(st)
        torch.cuda.synchronize()
        assert p.check() == 0, fft3.last_error()
        ms = e0.elapsed_time(e1) / reps
        N = n ** 3
        table[f"{n}^3"] = {"fwd_ms": ms, "gflops": 5 * N * math.log2(N) / ms / 1e6,
                           "hbm_gbs": 3 * 2 * 16 * N / ms / 1e6}
        p.close()
        del x, out
    return table


def bench_batched(fft3, synth, torch, hbm, count=4096):
    """`count` independent 3D DFTs with dims drawn from {16..96} (seed 7), one
    graph-captured execution of the default plan (FFT3_AUTO: the slab executor,
    one persistent launch of slab and z-tile items, for a batch this size): ms
    per batch, GB/s, roofline fractions; the segmented x, y and z passes (24
    launches, tuning codes 3), the persistent executor (tuning codes 0) and the
    segmented passes as one cooperative launch timed beside it."""
    import numpy as np
    dims = synth.batched_dims(count, 7)
    vols = dims.prod(axis=1)
    offs = np.zeros(len(dims), np.int64)
    offs[1:] = np.cumsum(vols[:-1])
    total = int(vols.sum())
    x = torch.empty(total, dtype=torch.complex64, device="cuda")
    x.real.uniform_(-1, 1)
    x.imag.uniform_(-1, 1)
    out = torch.empty_like(x)
    st = torch.cuda.current_stream()

    def run(tuning):
        h = fft3.fft3_plan_create_many(dims, offs, tuning=tuning)
        for _ in range(3):
            fft3.fft3_plan_execute(h, x.data_ptr(), out.data_ptr(), st.cuda_stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 10
        e0.record(st)
        for _ in range(reps):
            fft3.fft3_plan_execute(h, x.data_ptr(), out.data_ptr(), st.cuda_stream)
        e1.record(st)
        torch.cuda.synchronize()
        assert fft3.fft3_plan_check(h) == 0
        desc = fft3.fft3_plan_describe(h)
        fft3.fft3_plan_destroy(h)
        return e0.elapsed_time(e1) / reps, desc

    ms, desc = run(None)
    ms_seg, dseg = run([3] * count)
    ms_exec, _ = run([0] * count)
    # the segmented passes in one cooperative launch, 2^(k-1) waves of problems
    one_launch = {}
    for k in (1, 3, 5, 7):
        t, d = run([3 | (k << 8)] * count)
        one_launch[f"waves_{d['waves']}"] = t
    one_sweep = 2 * 8 * total
    return {"ms": ms, "mode": desc["mode"], "kernel_launches": desc["kernel_launches"],
            "one_launch_ms": one_launch,
            "segmented_ms": ms_seg, "segmented_launches": dseg["kernel_launches"],
            "executor_ms": ms_exec, "elements": total, "problems": count, "items": desc["items"],
            "GBps_one_sweep": one_sweep / (ms * 1e-3) / 1e9,
            "frac_of_1_sweep": one_sweep / (ms * 1e-3) / 1e9 / hbm,
            "frac_of_3_sweeps": 3 * one_sweep / (ms * 1e-3) / 1e9 / hbm,
            "gflops": sum(5.0 * v * math.log2(v) for v in vols) / (ms * 1e-3) / 1e9}


if __name__ == "__main__":
    sys.exit(main())
