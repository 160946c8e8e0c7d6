"""Learned plan selection: a small perceptron (the library's fft3_mlp_*
kernels) predicts the log run time of a candidate plan for a shape; the
candidate with the lowest prediction is proposed.  Exhaustive timing of all
candidates (fft3_time_candidates / fft3_autotune) stays the fallback and is
the yardstick of the model's regret, regret = t(chosen) / t(best) - 1.

The paper leaves the choice of decomposition to the user and shows that none
wins everywhere (Section 4.3); this module makes the choice from measurements.

Command line (runs on a GPU):
  python -m paper_1904_10119_gb300.plansel --train-shapes 120 --test-shapes 200 --out plansel.json
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import time

import numpy as np

from . import fft3

SIZES = (16, 24, 32, 40, 48, 64, 80, 96, 128, 160, 192, 256, 320, 384, 512, 640, 768, 1024)

KINDS = ("line_contig", "line_contig_rotate", "line_strided", "line_runtime", "slab_smem", "slab_l2",
         "volumetric_split", "volumetric_split_fixed", "line_strided_stream", "line_strided_tma")
N_FEATURES = 12 + len(KINDS) + 10


def candidates():
    """(decomposition, options kwargs) of every candidate plan; index 0 is the
    fixed default (pencil-pencil-pencil, natural layout, radix order 0,
    streamed strided kernels where compiled)."""
    out = []
    for order in range(4):
        out.append((fft3.FFT3_PENCIL3, dict(radix_order=order)))
        out.append((fft3.FFT3_PENCIL3, dict(radix_order=order, tile_lines=16)))
    for order in range(2):
        out.append((fft3.FFT3_PENCIL3, dict(radix_order=order, variant=1)))
        out.append((fft3.FFT3_SLAB_PENCIL, dict(radix_order=order, slab_mode=1)))
        out.append((fft3.FFT3_SLAB_PENCIL, dict(radix_order=order, slab_mode=2)))
        out.append((fft3.FFT3_SLAB_PENCIL, dict(radix_order=order, slab_mode=3, tile_lines=8)))
        out.append((fft3.FFT3_VOLUMETRIC, dict(radix_order=order)))
    out.append((fft3.FFT3_SLAB_PENCIL, dict(slab_mode=4)))
    out.append((fft3.FFT3_VOLUMETRIC, dict(mesh=(2, 2, 2))))
    out.append((fft3.FFT3_VOLUMETRIC, dict(mesh=(1, 4, 4), tile_lines=16)))
    return out


def features(shape, batch, decomp, opts, schedule=None) -> np.ndarray:
    """Features of a (shape, plan) pair: sizes, the plan's options, and what
    the host planner lowers it to (passes by kernel kind, line lengths, radix
    stages, lines per tile, launches)."""
    n0, n1, n2 = shape
    order = opts.get("radix_order", 0)
    if schedule is None:
        schedule = fft3.fft3_plan_schedule(*shape, batch, 0, decomp, -1, fft3.make_options(**opts))
    passes = schedule["passes"]
    f = np.zeros(N_FEATURES, np.float32)
    f[0:3] = [math.log2(n0), math.log2(n1), math.log2(n2)]
    f[3] = math.log2(batch)
    f[4] = math.log2(n0 * n1 * n2 * batch)
    f[5 + {fft3.FFT3_SLAB_PENCIL: 0, fft3.FFT3_PENCIL3: 1, fft3.FFT3_VOLUMETRIC: 2}[decomp]] = 1.0
    f[8] = float(opts.get("variant", 0))
    f[9] = opts.get("slab_mode", 0) / 4.0
    f[10] = opts.get("tile_lines", 0) / 16.0
    f[11] = order / 3.0
    for p in passes:
        if p["kind"] in KINDS:
            f[12 + KINDS.index(p["kind"])] += 1.0
    k = 12 + len(KINDS)
    f[k] = len(passes)
    f[k + 1] = sum(p.get("chunk", 0) > 0 for p in passes)
    stages = [len(p["line"]["radices"]) for p in passes]
    f[k + 2] = float(sum(stages))
    f[k + 3] = float(max(stages) if stages else 0)
    f[k + 4] = float(sum(16 in p["line"]["radices"] for p in passes))
    f[k + 5] = float(np.mean([math.log2(max(1, p["lpt"])) for p in passes]))
    f[k + 6] = float(np.mean([p["threads"] / 1024.0 for p in passes]))
    f[k + 7] = float(np.mean([p["smem"] / (227.0 * 1024) for p in passes]))
    f[k + 8] = float(np.log2(max(1, min(p["tiles"] for p in passes))))
    f[k + 9] = float(schedule["hbm_sweeps"] + (0.5 if schedule["decomposition"] == "volumetric" else 0.0))
    return f


def _opts_array(cands):
    arr = (fft3.fft3_options * len(cands))()
    for i, (_, o) in enumerate(cands):
        arr[i] = fft3.make_options(**o)
    dec = (ctypes.c_int * len(cands))(*[d for d, _ in cands])
    return dec, arr


def time_shape(shape, batch=1, reps=3, cands=None) -> np.ndarray:
    """Measured ms of every candidate for one shape (-1 = infeasible)."""
    cands = cands or candidates()
    dec, arr = _opts_array(cands)
    ms = (ctypes.c_float * len(cands))()
    rc = fft3.load().fft3_time_candidates(*shape, batch, 0, -1, reps, len(cands), dec, arr, ms)
    if rc < 0:
        raise fft3.Fft3Error(rc, fft3.last_error())
    return np.array(list(ms), np.float32)


def sample_shapes(count, seed, max_volume=1 << 24, exclude=()):
    rng = np.random.default_rng(seed)
    seen = set(tuple(s) for s in exclude)
    out = []
    while len(out) < count:
        s = tuple(int(v) for v in rng.choice(SIZES, 3))
        if int(np.prod(s)) > max_volume or s in seen:
            continue
        seen.add(s)
        out.append(s)
    return out


def collect(shapes, batch=1, reps=3):
    """Timing table: list of (shape, ms array over candidates)."""
    return [(s, time_shape(s, batch, reps)) for s in shapes]


def to_xy(table, batch=1):
    """Features and targets: the log run time of each feasible candidate
    relative to the mean log run time of the shape's candidates (only the
    ranking within a shape matters for the choice)."""
    cands = candidates()
    X, y = [], []
    for shape, ms in table:
        valid = [(i, t) for i, t in enumerate(ms) if t > 0]
        if not valid:
            continue
        mean_log = float(np.mean([math.log(t) for _, t in valid]))
        for i, t in valid:
            d, o = cands[i]
            X.append(features(shape, batch, d, o))
            y.append(math.log(t) - mean_log)
    return np.asarray(X, np.float32), np.asarray(y, np.float32)


class CostModel:
    """Feature standardisation + the library perceptron; `members` networks
    with different seeds are trained on the same data and their predictions
    averaged (an ensemble lowers the variance of the ranking)."""

    def __init__(self, hidden=64, seed=0, members=1):
        self.hidden = hidden
        self.seed = seed
        self.members = members
        self.mu = self.sd = None
        self.mlps = []

    @property
    def mlp(self):
        return self.mlps[0] if self.mlps else None

    def fit(self, X, y, epochs=200, batch=128, lr=1e-3):
        self.mu = X.mean(0)
        self.sd = X.std(0) + 1e-6
        curve = None
        for m in range(self.members):
            s = self.seed + 101 * m
            net = fft3.Mlp(X.shape[1], self.hidden, s)
            c = net.train((X - self.mu) / self.sd, y, epochs=epochs, batch=batch, lr=lr, seed=s + 1)
            curve = c if curve is None else curve
            self.mlps.append(net)
        return curve

    def predict(self, X):
        Z = (X - self.mu) / self.sd
        return np.mean([net.predict(Z) for net in self.mlps], axis=0)

    def close(self):
        for net in self.mlps:
            net.close()
        self.mlps = []

    def ranking(self, shape, batch=1):
        """Candidate indices the planner accepts for this shape, best
        predicted first."""
        cands = candidates()
        ok = []
        for i, (d, o) in enumerate(cands):
            try:
                fft3.fft3_plan_schedule(*shape, batch, 0, d, -1, fft3.make_options(**o))
                ok.append(i)
            except fft3.Fft3Error:
                pass
        X = np.stack([features(shape, batch, *cands[i]) for i in ok])
        return [ok[j] for j in np.argsort(self.predict(X), kind="stable")]

    def choose(self, shape, batch=1):
        return self.ranking(shape, batch)[0]


def analytic_ranking(shape, batch=1):
    """Baseline without the model: fewest HBM sweeps (passes of the plan,
    volumetric penalised by half a sweep for its exchange), ties broken by
    candidate order."""
    scored = []
    for i, (d, o) in enumerate(candidates()):
        try:
            s = fft3.fft3_plan_schedule(*shape, batch, 0, d, -1, fft3.make_options(**o))
        except fft3.Fft3Error:
            continue
        scored.append((s["hbm_sweeps"] + (0.5 if s["decomposition"] == "volumetric" else 0.0), i))
    return [i for _, i in sorted(scored)]


def hybrid_ranking(model):
    """The analytic preference first (fewest HBM sweeps, volumetric penalised by
    half a sweep), the model's predicted run time among plans that tie on it."""
    def rank(shape, batch=1):
        order = model.ranking(shape, batch)
        pos = {c: k for k, c in enumerate(order)}
        key = {}
        for i, (d, o) in enumerate(candidates()):
            if i not in pos:
                continue
            s = fft3.fft3_plan_schedule(*shape, batch, 0, d, -1, fft3.make_options(**o))
            key[i] = (s["hbm_sweeps"] + (0.5 if s["decomposition"] == "volumetric" else 0.0), pos[i])
        return sorted(key, key=lambda i: key[i])
    return rank


def regrets(table, ranker):
    """regret = t(chosen) / t(best) - 1 per shape, where the chosen plan is the
    first of the ranking that can be created on the GPU (a proposal whose
    creation fails falls through to the next one at no measured cost)."""
    out = []
    for shape, ms in table:
        valid = ms > 0
        best = ms[valid].min()
        t = np.inf
        for c in ranker(shape):
            if ms[c] > 0:
                t = ms[c]
                break
        out.append(float(t / best - 1.0))
    return np.asarray(out)


def summarize(r):
    return {"mean": float(np.mean(r)), "median": float(np.median(r)), "p90": float(np.percentile(r, 90)),
            "max": float(np.max(r)), "zero_regret_frac": float(np.mean(r <= 1e-9))}


def run(train_shapes=400, test_shapes=200, seed=8, max_volume=1 << 24, reps=3, epochs=400, members=5):
    t0 = time.perf_counter()
    train = sample_shapes(train_shapes, seed, max_volume)
    test = sample_shapes(test_shapes, seed + 1000, max_volume, exclude=train)
    tab_train = collect(train, reps=reps)
    tab_test = collect(test, reps=reps)
    t_collect = time.perf_counter() - t0
    X, y = to_xy(tab_train)
    model = CostModel(seed=seed, members=members)
    curve = model.fit(X, y, epochs=epochs)
    res = {
        "train_shapes": len(train), "test_shapes": len(test), "train_plans": int(X.shape[0]),
        "candidates": len(candidates()), "collect_seconds": t_collect, "members": members,
        "loss_first": float(curve[0]), "loss_last": float(curve[-1]),
        "regret_mlp": summarize(regrets(tab_test, lambda s: model.ranking(s))),
        "regret_hybrid": summarize(regrets(tab_test, hybrid_ranking(model))),
        "regret_fixed_default": summarize(regrets(tab_test, lambda s: [0])),
        "regret_analytic": summarize(regrets(tab_test, analytic_ranking)),
        "exhaustive_ms_per_shape": float(np.mean([ms[ms > 0].sum() for _, ms in tab_test])),
    }
    model.close()
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train-shapes", type=int, default=400)
    ap.add_argument("--test-shapes", type=int, default=200)
    ap.add_argument("--seed", type=int, default=8)
    ap.add_argument("--max-volume", type=int, default=1 << 24)
    ap.add_argument("--epochs", type=int, default=400)
    ap.add_argument("--members", type=int, default=5, help="networks averaged in the cost model")
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    res = run(a.train_shapes, a.test_shapes, a.seed, a.max_volume, epochs=a.epochs, members=a.members)
    s = json.dumps(res, indent=1)
    print(s)
    if a.out:
        with open(a.out, "w") as f:
            f.write(s)


if __name__ == "__main__":
    main()
