"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds no DFT arithmetic: it only draws inputs.  Every draw uses
numpy's PCG64 bit generator (``numpy.random.Generator(PCG64(seed))``) and its
``random(dtype=float32)``, which returns k * 2^-24 for a 24-bit integer k, so
``2u - 1`` is exact in FP32.  Real and imaginary parts are drawn i.i.d.

Workloads follow the paper's experiments (cubic 64^3, 256^3, 1024^3 complex
arrays, Section 4.3) and the batched / mixed-radix shapes used to exercise
the planner.  The paper does not state its input values.
"""
from __future__ import annotations

import numpy as np

BATCH_DIM_CHOICES = (16, 24, 32, 40, 48, 64, 80, 96)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def uniform_c64(shape, seed: int, out: np.ndarray | None = None, chunk: int = 1 << 26) -> np.ndarray:
    """complex64 array of the given shape with re, im i.i.d. uniform[-1, 1).

    ``out`` may be a preallocated (e.g. pinned) complex64 array of the same
    size; it is filled in chunks so that large arrays need no temporary of
    their full size."""
    size = int(np.prod(shape))
    if out is None:
        out = np.empty(size, dtype=np.complex64)
    flat = out.reshape(-1).view(np.float32)
    assert flat.size == 2 * size
    rng = _rng(seed)
    for s in range(0, 2 * size, chunk):
        e = min(2 * size, s + chunk)
        u = rng.random(e - s, dtype=np.float32)
        np.multiply(u, np.float32(2.0), out=u)
        np.subtract(u, np.float32(1.0), out=u)
        flat[s:e] = u
    return out.reshape(shape)


def uniform_c128(shape, seed: int) -> np.ndarray:
    """complex128 array of the given shape with re, im i.i.d. uniform[-1, 1)
    drawn in double precision (53-bit mantissas, for the complex128 path)."""
    size = int(np.prod(shape))
    r = _rng(seed).random(2 * size, dtype=np.float64) * 2.0 - 1.0
    return r.view(np.complex128).reshape(shape)


def hdr_c64(shape, seed: int) -> np.ndarray:
    """complex64 with |z| = 10^U(-3,3) (log-uniform in [1e-3, 1e3]) and a
    uniform phase 2*pi*U(0,1); computed in FP64 and rounded once to FP32."""
    size = int(np.prod(shape))
    rng = _rng(seed)
    mag = 10.0 ** rng.uniform(-3.0, 3.0, size)
    ph = 2.0 * np.pi * rng.random(size)
    z = (mag * np.cos(ph)).astype(np.float32) + 1j * (mag * np.sin(ph)).astype(np.float32)
    return z.astype(np.complex64).reshape(shape)


def batched_dims(count: int, seed: int, choices=BATCH_DIM_CHOICES) -> np.ndarray:
    """(count, 3) int array of (n0, n1, n2), each dim drawn i.i.d. from `choices`."""
    rng = _rng(seed)
    idx = rng.integers(0, len(choices), size=(count, 3))
    return np.asarray(choices, dtype=np.int64)[idx]


def smooth_sizes(lo: int = 2, hi: int = 1024, primes=(2, 3, 5)) -> list[int]:
    """All integers in [lo, hi] whose prime factors are in `primes`."""
    out = []
    for n in range(max(1, lo), hi + 1):
        m = n
        for p in primes:
            while m % p == 0:
                m //= p
        if m == 1:
            out.append(n)
    return out
