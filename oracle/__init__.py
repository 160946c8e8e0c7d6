"""FP64 CPU oracle for the 3D complex DFT -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never imports,
links or executes it, and the oracle shares no code with the CUDA path: the
arithmetic lives in ``oracle.c`` (plain C, FP64, OpenMP over lines) and in
the small numpy routines below, each written from the paper
(Popovici, Schatz, Franchetti, Low, "A Flexible Framework for Parallel
Multi-Dimensional DFTs"):

* Section 2.1 -- the DFT as a dense matrix-vector product and the
  Cooley-Tukey four-stage factorisation (Eq. ct): ``dft1_direct``,
  ``fft1_rec``.
* Section 2.3 -- the 3D DFT as batches of 1D DFTs along n0, n1, n2 with n0
  fastest in memory: ``fft3``, ``fft3_dims``; brute force N^3 sum:
  ``bruteforce3``.
* Section 3.1 -- elemental-cyclic and blocked distributions, and the
  redistribution B[(0)()] = A[()(0)]: ``cyclic_owner``, ``blocked_owner``.
* Section 3.2 (Eq. cteinstein and the T0/T1/T2 equations that follow it) --
  the parallel 1D DFT on p processes with one all-to-all, simulated with p
  explicit local buffers: ``rote_parallel_dft1``; applied along each
  dimension of a cube distributed cyclically on a 3D mesh (the volumetric
  decomposition of Fig. cuboid): ``volumetric3_sim``.
* Section 2.4 -- the slab-pencil algorithm on a 1D grid of p processes
  (Fig. 3dslabpencil): 2D DFTs of each rank's slabs, an all-to-all, the 1D
  DFTs of each rank's z pencils, and the optional second exchange back to
  slabs, simulated with p explicit local arrays: ``slab_pencil_sim``.
* Section 2.4 -- the pencil-pencil-pencil algorithm on a py x pz grid
  (Fig. 3dpencilpencil): x DFTs, an all-to-all within each row of the grid,
  y DFTs, an all-to-all within each column, z DFTs, the spectrum left in
  bricks (the last redistribution dropped): ``pencil3_sim``.
* Section 2.4 -- the data rotations xyz -> yzx -> zxy of the
  pencil-pencil-pencil algorithm: ``rotation_dst_index``; the shuffled
  spectrum left when the last redistribution is dropped, and the blocked
  z-pencil order: ``layout_positions``.

Parity is pinned for every function here by ``tests/test_oracle_*.py``
against closed forms, invariants, brute force and an independent library
FFT; the MLP reference (``mlp_*``) is pinned by central finite differences.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

FORWARD = -1
INVERSE = +1


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (plain gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-o", _LIB, _SRC, "-lm"]
        subprocess.check_call(cmd)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        i64 = ctypes.c_int64
        L.oracle_dft1_direct.argtypes = [dp, dp, i64, ctypes.c_int]
        L.oracle_fft1_rec.argtypes = [dp, dp, i64, ctypes.c_int]
        L.oracle_fft3.argtypes = [dp, dp, i64, i64, i64, i64, ctypes.c_int, ctypes.c_int]
        L.oracle_fft3_dims.argtypes = [dp, dp, i64, i64, i64, i64, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int]
        L.oracle_fft1_lines.argtypes = [dp, i64, i64, i64, i64, ctypes.c_int, ctypes.c_int]
        L.oracle_bruteforce3.argtypes = [dp, dp, i64, i64, i64, ctypes.c_int]
        L.oracle_roots.argtypes = [i64, ctypes.POINTER(ctypes.c_int64), i64, ctypes.c_int, dp]
        L.oracle_num_threads.restype = ctypes.c_int
        L.oracle_set_num_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _c128(x) -> np.ndarray:
    """Exact widening to complex128 (float32 inputs are representable in FP64)."""
    return np.ascontiguousarray(np.asarray(x), dtype=np.complex128)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def set_num_threads(t: int) -> None:
    lib().oracle_set_num_threads(int(t))


# --------------------------------------------------------------------------- #
# Roots of unity (Section 2.1)                                                 #
# --------------------------------------------------------------------------- #
def roots(n: int, m, sign: int = FORWARD) -> np.ndarray:
    """w_n^m = exp(sign*2*pi*i*m/n) for integer exponents m (reduced mod n
    exactly), evaluated in long double and rounded once to complex128."""
    m = np.ascontiguousarray(np.asarray(m, dtype=np.int64).ravel())
    out = np.empty(m.size, dtype=np.complex128)
    lib().oracle_roots(int(n), m.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), m.size, int(sign),
                       _ptr(out))
    return out


def dft_matrix(n: int, sign: int = FORWARD) -> np.ndarray:
    """DFT_n = [w_n^{lk}] (Section 2.1), exponents reduced mod n in integers."""
    l = np.arange(n, dtype=np.int64)
    return roots(n, np.outer(l, l) % n, sign).reshape(n, n)


# --------------------------------------------------------------------------- #
# 1D and 3D transforms                                                          #
# --------------------------------------------------------------------------- #
def dft1_direct(x, sign: int = FORWARD) -> np.ndarray:
    """y = DFT_n x as the O(n^2) direct sum (Section 2.1)."""
    x = _c128(x).ravel()
    y = np.empty_like(x)
    lib().oracle_dft1_direct(_ptr(x), _ptr(y), x.size, int(sign))
    return y


def fft1_rec(x, sign: int = FORWARD) -> np.ndarray:
    """Recursive Cooley-Tukey FFT following Eq. ct (smallest prime factor
    first, direct DFT at the prime leaves)."""
    x = _c128(x).ravel()
    y = np.empty_like(x)
    lib().oracle_fft1_rec(_ptr(x), _ptr(y), x.size, int(sign))
    return y


METHOD_DIRECT, METHOD_FFT, METHOD_AUTO = 0, 1, 2


def fft3_dims(x, n0: int, n1: int, n2: int, batch: int = 1, sign: int = FORWARD,
              dims: Sequence[int] = (0, 1, 2), method: int = METHOD_AUTO) -> np.ndarray:
    """Batched 1D DFTs along the listed dimensions (0 = n0, fastest) of a
    (batch, n2, n1, n0) complex array, in the order 0, 1, 2 (Section 2.3)."""
    x = _c128(x)
    assert x.size == batch * n0 * n1 * n2
    y = np.empty_like(x)
    mask = 0
    for d in dims:
        mask |= 1 << int(d)
    lib().oracle_fft3_dims(_ptr(x), _ptr(y), n0, n1, n2, batch, int(sign), int(method), mask)
    return y.reshape(batch, n2, n1, n0) if batch > 1 else y.reshape(n2, n1, n0)


def fft3(x, n0: int, n1: int, n2: int, batch: int = 1, sign: int = FORWARD,
         method: int = METHOD_AUTO) -> np.ndarray:
    """3D DFT of a (batch, n2, n1, n0) array by the pencil-pencil-pencil
    definition (Section 2.3).  Inverse (sign=+1) is unnormalised."""
    return fft3_dims(x, n0, n1, n2, batch, sign, (0, 1, 2), method)


def fft3_inplace(buf: np.ndarray, n0: int, n1: int, n2: int, batch: int = 1, sign: int = FORWARD,
                 method: int = METHOD_AUTO) -> None:
    """The 3D DFT of fft3 (Section 2.3, pencil-pencil-pencil definition)
    computed in place on a contiguous complex128 buffer: one array instead of
    two, which is what lets the CPU baseline time whole 1024^3 transforms."""
    assert buf.dtype == np.complex128 and buf.flags.c_contiguous and buf.size == batch * n0 * n1 * n2
    lib().oracle_fft3_dims(_ptr(buf), _ptr(buf), n0, n1, n2, batch, int(sign), int(method), 7)


def fft1_lines_inplace(buf: np.ndarray, n: int, lines: int, line_stride: int, elem_stride: int,
                       sign: int = FORWARD, method: int = METHOD_AUTO) -> None:
    """In-place 1D DFTs of `lines` lines of a complex128 buffer (CPU baseline)."""
    assert buf.dtype == np.complex128 and buf.flags.c_contiguous
    lib().oracle_fft1_lines(_ptr(buf), n, lines, line_stride, elem_stride, int(sign), int(method))


def bruteforce3(x, n0: int, n1: int, n2: int, sign: int = FORWARD) -> np.ndarray:
    """Full N-term sum per output with one combined integer phase exponent."""
    x = _c128(x)
    assert x.size == n0 * n1 * n2
    y = np.empty_like(x)
    lib().oracle_bruteforce3(_ptr(x), _ptr(y), n0, n1, n2, int(sign))
    return y.reshape(n2, n1, n0)


# --------------------------------------------------------------------------- #
# Error measures used by every parity test                                      #
# --------------------------------------------------------------------------- #
def rel_l2(got, ref) -> float:
    got = np.asarray(got, dtype=np.complex128).ravel()
    ref = np.asarray(ref, dtype=np.complex128).ravel()
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(got - ref) / (den if den > 0 else 1.0))


def max_abs_ratio(got, ref) -> float:
    """max|got - ref| / max|ref|."""
    got = np.asarray(got, dtype=np.complex128).ravel()
    ref = np.asarray(ref, dtype=np.complex128).ravel()
    m = np.max(np.abs(ref)) if ref.size else 0.0
    return float(np.max(np.abs(got - ref)) / (m if m > 0 else 1.0)) if ref.size else 0.0


# --------------------------------------------------------------------------- #
# Distributions and redistributions (Section 3.1)                              #
# --------------------------------------------------------------------------- #
def cyclic_owner(n: int, p: int):
    """Elemental-cyclic distribution of a mode of length n over p processes:
    element i lives on process i mod p at local slot i div p."""
    i = np.arange(n, dtype=np.int64)
    return i % p, i // p


def blocked_owner(n: int, p: int):
    """Blocked distribution (the mode split eta = eta0*eta1 with eta0 = n/p the
    block): element i lives on process i div (n/p) at local slot i mod (n/p)."""
    b = n // p
    i = np.arange(n, dtype=np.int64)
    return i // b, i % b


def ct_input_map(n0: int, n1: int) -> np.ndarray:
    """x~[i0, i1] = x[i0 + n0*i1]: returns the flat source index of x~ as an
    (n0, n1) integer matrix (Section 2.1, Eq. ct)."""
    i0 = np.arange(n0, dtype=np.int64)[:, None]
    i1 = np.arange(n1, dtype=np.int64)[None, :]
    return i0 + n0 * i1


def ct_output_map(n0: int, n1: int) -> np.ndarray:
    """y~[k1, k0] = y[k1 + n1*k0]: flat index of y for each entry of the
    (n1, n0) output matrix (Section 2.1, Eq. ct)."""
    k1 = np.arange(n1, dtype=np.int64)[:, None]
    k0 = np.arange(n0, dtype=np.int64)[None, :]
    return k1 + n1 * k0


def rote_parallel_dft1(x, n0: int, n1: int, p: int, sign: int = FORWARD):
    """Parallel 1D DFT of n = n0*n1 on a 1D grid of p processes, Section 3.2.

    The input matrix x~ (n0 x n1, x~[i0,i1] = x[i0+n0*i1]) is distributed
    [(0)()]: its rows are elemental-cyclic, process r owning rows i0 = r mod p.
    Each process (I) applies DFT_{n1} to its rows and (II) scales by the
    twiddles w_n^{i0 k1} (the twiddle matrix has the same distribution), giving
    T0[(0)()].  The all-to-all T1[()(0)] = T0[(0)()] sends to process r the
    columns k1 = r mod p of every other process's rows; each process then
    transposes locally (T2[(0)()], rows k1) and applies DFT_{n0}, producing
    rows k1 = r mod p of y~ (n1 x n0, y~[k1,k0] = y[k1 + n1*k0]).

    Requires p | n0 and p | n1 (then one exchange suffices).  Returns
    ``(y, local_in, local_out)``: the assembled output and, per process, the
    flat indices of x it held on input and of y it holds on output.
    """
    assert n0 % p == 0 and n1 % p == 0, "one-exchange form needs p | n0 and p | n1"
    n = n0 * n1
    x = _c128(x).ravel()
    assert x.size == n
    xt = x[ct_input_map(n0, n1)]                      # (n0, n1)
    F1 = dft_matrix(n1, sign)
    F0 = dft_matrix(n0, sign)
    # local buffers: process r owns rows i0 = r, r+p, ...
    local_rows = [np.arange(r, n0, p) for r in range(p)]
    T0 = []
    for r in range(p):
        rows = xt[local_rows[r], :]                    # (n0/p, n1)
        t = rows @ F1                                  # (I) DFT_{n1} on each row
        i0 = local_rows[r][:, None]
        k1 = np.arange(n1)[None, :]
        t = t * roots(n, (i0 * k1) % n, sign).reshape(t.shape)   # (II) twiddle
        T0.append(t)
    # all-to-all: process r receives, from every s, the block T0_s[:, k1 = r mod p]
    recv = [[T0[s][:, r::p] for s in range(p)] for r in range(p)]
    Y_local = []
    for r in range(p):
        # T1 on process r: columns k1 = r mod p, all rows i0 (reassembled by owner)
        cols = np.arange(r, n1, p)
        T1 = np.empty((n0, cols.size), dtype=np.complex128)
        for s in range(p):
            T1[local_rows[s], :] = recv[r][s]
        T2 = T1.T                                      # local transpose: (n1/p, n0), rows k1
        Y_local.append(T2 @ F0)                        # DFT_{n0} along i0 -> y~[k1, k0]
    y = np.empty(n, dtype=np.complex128)
    out_map = ct_output_map(n0, n1)                   # (n1, n0)
    local_in, local_out = [], []
    for r in range(p):
        cols = np.arange(r, n1, p)
        y[out_map[cols, :].ravel()] = Y_local[r].ravel()
        local_in.append(np.sort(ct_input_map(n0, n1)[local_rows[r], :].ravel()))
        local_out.append(np.sort(out_map[cols, :].ravel()))
    return y, local_in, local_out


def volumetric3_sim(x, n0: int, n1: int, n2: int, mesh=(2, 2, 2), splits=None,
                    sign: int = FORWARD) -> np.ndarray:
    """Volumetric 3D DFT (Fig. cuboid, Section 3.2): the cube is distributed
    elemental-cyclic in all three dimensions over a p0 x p1 x p2 mesh and each
    dimension's 1D DFTs run as the parallel one-exchange algorithm of
    ``rote_parallel_dft1`` over that dimension's p_d processes.  ``splits``
    gives n_d = a_d * b_d for each dimension (default: a_d = the smallest
    multiple of p_d dividing n_d with p_d | n_d / a_d)."""
    x = _c128(x).reshape(n2, n1, n0)
    ns = (n0, n1, n2)
    if splits is None:
        splits = []
        for n, p in zip(ns, mesh):
            a = next(a for a in range(p, n + 1, p) if n % a == 0 and (n // a) % p == 0)
            splits.append((a, n // a))
    out = x.copy()
    for d, (n, p, (a, b)) in enumerate(zip(ns, mesh, splits)):
        assert a * b == n
        axis = 2 - d                                  # numpy axis of dimension d
        moved = np.moveaxis(out, axis, -1)
        flat = moved.reshape(-1, n)
        res = np.empty_like(flat)
        for l in range(flat.shape[0]):
            res[l], _, _ = rote_parallel_dft1(flat[l], a, b, p, sign)
        out = np.moveaxis(res.reshape(moved.shape), -1, axis)
    return np.ascontiguousarray(out)


def slab_pencil_sim(local_in, n0: int, n1: int, n2: int, p: int, sign: int = FORWARD,
                    natural: bool = False):
    """Slab-pencil 3D DFT on a 1D grid of p processes (Section 2.4,
    Fig. 3dslabpencil), each rank's data an explicit array (n0 fastest):

    * slabs: rank r holds z in [r n2/p, (r+1) n2/p) as a (n2/p, n1, n0) array;
    * pencils: rank r holds x in [r n0/p, (r+1) n0/p) as a (n2, n1, n0/p) array.

    Forward (sign -1): ``local_in`` are the slabs; every rank applies the 2D
    DFT to its slabs, an all-to-all gives rank r the columns of its x range
    from every rank, every rank applies the 1D DFTs along z, and with
    ``natural`` a second all-to-all returns the spectrum to slabs (otherwise
    the spectrum stays in pencils, the last redistribution dropped).  Inverse
    (sign +1): the same steps in reverse order, from pencils (or slabs with
    ``natural``) to slabs.  Returns the list of the p output arrays."""
    assert n0 % p == 0 and n2 % p == 0
    xl, zl = n0 // p, n2 // p

    def to_pencils(slabs):       # all-to-all: x range r of every rank's slabs to rank r
        return [np.concatenate([slabs[s][:, :, r * xl:(r + 1) * xl] for s in range(p)], axis=0)
                for r in range(p)]

    def to_slabs(pencils):       # all-to-all: z range r of every rank's pencils to rank r
        return [np.concatenate([pencils[s][r * zl:(r + 1) * zl] for s in range(p)], axis=2)
                for r in range(p)]

    def slab_dft(slabs):
        return [fft3_dims(a, n0, n1, zl, 1, sign, (0, 1)).reshape(zl, n1, n0) for a in slabs]

    def pencil_dft(pencils):
        return [fft3_dims(a, xl, n1, n2, 1, sign, (2,)).reshape(n2, n1, xl) for a in pencils]

    if sign == FORWARD:
        data = [_c128(a).reshape(zl, n1, n0) for a in local_in]
        data = pencil_dft(to_pencils(slab_dft(data)))
        return to_slabs(data) if natural else data
    if natural:
        data = to_pencils([_c128(a).reshape(zl, n1, n0) for a in local_in])
    else:
        data = [_c128(a).reshape(n2, n1, xl) for a in local_in]
    return slab_dft(to_slabs(pencil_dft(data)))


def pencil3_sim(local_in, n0: int, n1: int, n2: int, py: int, pz: int, sign: int = FORWARD):
    """Pencil-pencil-pencil 3D DFT on a py x pz grid of processes (Section 2.4,
    Fig. 3dpencilpencil), rank r = q py + p holding an explicit array (n0
    fastest):

    * pencils: rank (p, q) holds y in [p n1/py, (p+1) n1/py) and z in
      [q n2/pz, (q+1) n2/pz), all x, as a (n2/pz, n1/py, n0) array;
    * bricks: rank (p, q) holds x in [p n0/py, (p+1) n0/py), y in
      [q n1/pz, (q+1) n1/pz), all z, as a (n2, n1/pz, n0/py) array.

    Forward (sign -1): pencils in; x DFTs; an all-to-all among the ranks of
    each row q gives rank (p, q) the x range p of its row's y ranges; y DFTs;
    an all-to-all among the ranks of each column p gives it the y range q of
    its column's z ranges; z DFTs; bricks out.  Inverse (sign +1): the same
    steps in reverse order, bricks in, pencils out.  Returns the list of
    outputs in rank order."""
    assert n0 % py == 0 and n1 % py == 0 and n1 % pz == 0 and n2 % pz == 0
    xl, yl, y2, zl = n0 // py, n1 // py, n1 // pz, n2 // pz
    ranks = [(r % py, r // py) for r in range(py * pz)]
    idx = {pq: r for r, pq in enumerate(ranks)}

    def dft(a, axis):               # 1D DFTs along numpy axis `axis` of a 3D array
        a = np.ascontiguousarray(a)
        d2, d1, d0 = a.shape
        return fft3_dims(a, d0, d1, d2, 1, sign, (2 - axis,)).reshape(a.shape)

    if sign == FORWARD:
        a = [dft(_c128(t).reshape(zl, yl, n0), 2) for t in local_in]
        b = [dft(np.concatenate([a[idx[(s, q)]][:, :, p * xl:(p + 1) * xl] for s in range(py)], axis=1), 1)
             for p, q in ranks]
        return [dft(np.concatenate([b[idx[(p, s)]][:, q * y2:(q + 1) * y2, :] for s in range(pz)], axis=0), 0)
                for p, q in ranks]
    c = [dft(_c128(t).reshape(n2, y2, xl), 0) for t in local_in]
    b = [dft(np.concatenate([c[idx[(p, s)]][q * zl:(q + 1) * zl] for s in range(pz)], axis=1), 1)
         for p, q in ranks]
    return [dft(np.concatenate([b[idx[(s, q)]][:, p * yl:(p + 1) * yl, :] for s in range(py)], axis=2), 2)
            for p, q in ranks]


# --------------------------------------------------------------------------- #
# Rotations of the pencil-pencil-pencil algorithm (Section 2.4)                 #
# --------------------------------------------------------------------------- #
def rotation_dst_index(n0: int, n1: int, n2: int, kind: str) -> np.ndarray:
    """For a cube with dims (da, db, dc) stored a-fastest, the rotation that
    makes the next dimension fastest (xyz -> yzx) sends element (ia, ib, ic)
    to ib + db*(ic + dc*ia).  ``kind`` names the layout being rotated:
    'xyz' (dims n0,n1,n2), 'yzx' (dims n1,n2,n0) or 'zxy' (dims n2,n0,n1).
    Returns the destination flat index of each source flat index."""
    dims = {"xyz": (n0, n1, n2), "yzx": (n1, n2, n0), "zxy": (n2, n0, n1)}[kind]
    da, db, dc = dims
    ic, ib, ia = np.meshgrid(np.arange(dc), np.arange(db), np.arange(da), indexing="ij")
    dst = ib + db * (ic + dc * ia)
    return dst.ravel().astype(np.int64)


def layout_positions(layout: str, n0: int, n1: int, n2: int, batch: int = 1) -> np.ndarray:
    """Position of every natural flat index (k0 + n0*(k1 + n1*k2) + N*b) in a
    permuted spectrum.  'rotated' (Section 2.4): the cube after the rotations
    xyz -> yzx -> zxy with the redistribution back to xyz dropped, i.e. the
    two rotations of ``rotation_dst_index`` applied in turn.  'pencils': z
    pencils grouped by 16 columns of x, element (k0, k1, k2) at block k0 // 16,
    then k2, then k1, then k0 % 16 (n0 a multiple of 16, batch 1)."""
    N = n0 * n1 * n2
    if layout == "rotated":
        first = rotation_dst_index(n0, n1, n2, "xyz")
        second = rotation_dst_index(n0, n1, n2, "yzx")
        one = second[first]
        return (one[None, :] + N * np.arange(batch)[:, None]).ravel().astype(np.int64)
    if layout == "pencils":
        if batch != 1 or n0 % 16:
            raise ValueError("pencils: batch 1 and n0 % 16 == 0")
        k2, k1, k0 = np.meshgrid(np.arange(n2), np.arange(n1), np.arange(n0), indexing="ij")
        pos = (k0 // 16) * (n2 * n1 * 16) + k2 * (n1 * 16) + k1 * 16 + k0 % 16
        return pos.ravel().astype(np.int64)
    raise ValueError(layout)


# --------------------------------------------------------------------------- #
# Split-BF16 representation: round-to-nearest-even to bfloat16                  #
# --------------------------------------------------------------------------- #
def bf16_round(x) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned
    as float32.  Written from the IEEE-754 definition on the bit pattern:
    keep the top 16 bits, adding 0x7FFF plus the lowest kept bit first."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32)
    nan = np.isnan(f)
    out = np.where(nan, f, out)
    return out


def split_bf16(x):
    """x = hi + lo with hi = bf16(x), lo = bf16(x - hi); x - hi is exact in FP32."""
    f = np.asarray(x, dtype=np.float32)
    hi = bf16_round(f)
    lo = bf16_round(f - hi)
    return hi, lo


# --------------------------------------------------------------------------- #
# FP64 reference for the plan-cost MLP: in -> H -> H -> 1, GELU, MSE, Adam      #
# --------------------------------------------------------------------------- #
def _erf(x):
    from scipy.special import erf
    return erf(x)


def gelu(x):
    """GELU in its exact form 0.5 x (1 + erf(x / sqrt 2))."""
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    """d/dx GELU = Phi(x) + x phi(x)."""
    Phi = 0.5 * (1.0 + _erf(x / math.sqrt(2.0)))
    phi = np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)
    return Phi + x * phi


def mlp_forward(params, X):
    """params: [W1 (H,F), b1 (H), W2 (H,H), b2 (H), W3 (1,H), b3 (1)].
    Returns predictions (B,) and the cache for the backward pass."""
    W1, b1, W2, b2, W3, b3 = [np.asarray(p, dtype=np.float64) for p in params]
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    h1 = gelu(z1)
    z2 = h1 @ W2.T + b2
    h2 = gelu(z2)
    out = h2 @ W3.T + b3
    return out[:, 0], (X, z1, h1, z2, h2)


def mse_loss(pred, target) -> float:
    d = np.asarray(pred, dtype=np.float64) - np.asarray(target, dtype=np.float64)
    return float(np.mean(d * d))


def mlp_backward(params, cache, pred, target):
    """Gradients of the MSE loss with respect to every parameter."""
    W1, b1, W2, b2, W3, b3 = [np.asarray(p, dtype=np.float64) for p in params]
    X, z1, h1, z2, h2 = cache
    B = X.shape[0]
    g_out = (2.0 / B) * (np.asarray(pred, np.float64) - np.asarray(target, np.float64))[:, None]
    gW3 = g_out.T @ h2
    gb3 = g_out.sum(axis=0)
    g_h2 = g_out @ W3
    g_z2 = g_h2 * gelu_grad(z2)
    gW2 = g_z2.T @ h1
    gb2 = g_z2.sum(axis=0)
    g_h1 = g_z2 @ W2
    g_z1 = g_h1 * gelu_grad(z1)
    gW1 = g_z1.T @ X
    gb1 = g_z1.sum(axis=0)
    return [gW1, gb1, gW2, gb2, gW3, gb3]


def adam_step(params, grads, m, v, t: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba): bias-corrected first and second moments."""
    new_p, new_m, new_v = [], [], []
    for p, g, mi, vi in zip(params, grads, m, v):
        p = np.asarray(p, np.float64)
        g = np.asarray(g, np.float64)
        mi = beta1 * np.asarray(mi, np.float64) + (1.0 - beta1) * g
        vi = beta2 * np.asarray(vi, np.float64) + (1.0 - beta2) * g * g
        mhat = mi / (1.0 - beta1 ** t)
        vhat = vi / (1.0 - beta2 ** t)
        new_p.append(p - lr * mhat / (np.sqrt(vhat) + eps))
        new_m.append(mi)
        new_v.append(vi)
    return new_p, new_m, new_v


def dft3_sampled(x, n0: int, n1: int, n2: int, k0s, k1s, k2s, sign: int = FORWARD,
                 chunk_rows: int = 1 << 16) -> np.ndarray:
    """Selected outputs X[k0, k1, k2] (for k0 in k0s, k1 in k1s, k2 in k2s) of
    the 3D DFT of one (n2, n1, n0) array, by the separable definition of
    Section 2.3 restricted to those frequencies: a product with the selected
    columns of DFT_{n0}, then of DFT_{n1}, then of DFT_{n2}.  Cost is one
    sweep over x, so it serves arrays far too large for ``fft3``.
    Returns an array of shape (len(k0s), len(k1s), len(k2s))."""
    k0s, k1s, k2s = (np.asarray(k, dtype=np.int64) for k in (k0s, k1s, k2s))
    F0 = roots(n0, np.outer(np.arange(n0), k0s) % n0, sign).reshape(n0, k0s.size)
    F1 = roots(n1, np.outer(np.arange(n1), k1s) % n1, sign).reshape(n1, k1s.size)
    F2 = roots(n2, np.outer(np.arange(n2), k2s) % n2, sign).reshape(n2, k2s.size)
    rows = np.asarray(x).reshape(n2 * n1, n0)
    A = np.empty((n2 * n1, k0s.size), dtype=np.complex128)
    for s in range(0, n2 * n1, chunk_rows):
        e = min(n2 * n1, s + chunk_rows)
        A[s:e] = rows[s:e].astype(np.complex128) @ F0
    A = A.reshape(n2, n1, k0s.size)
    B = np.einsum("zyk,yl->zkl", A, F1)
    return np.einsum("zkl,zm->klm", B, F2)


def dft3_line(x, n0: int, n1: int, n2: int, dim: int, ka: int, kb: int, sign: int = FORWARD,
              chunk: int = 16) -> np.ndarray:
    """One whole output line of the 3D DFT of a (n2, n1, n0) array (Section 2.3,
    separable definition): every frequency along dimension `dim`, the other two
    fixed (ka, kb in increasing dimension order).  The two fixed dimensions are
    summed out first with their roots w^{j k} (one sweep over x, FP64), then
    the remaining vector gets the direct O(n^2) DFT along `dim`."""
    n = (n0, n1, n2)
    other = [d for d in range(3) if d != dim]
    k = {other[0]: ka, other[1]: kb}
    w = {d: roots(n[d], np.arange(n[d]) * k[d] % n[d], sign) for d in other}
    v = np.asarray(x).reshape(n2, n1, n0)
    acc = np.zeros(n[dim], dtype=np.complex128)
    for z0 in range(0, n2, chunk):
        blk = v[z0:z0 + chunk].astype(np.complex128)           # (z, y, x)
        if dim == 0:
            acc += w[1] @ np.tensordot(w[2][z0:z0 + chunk], blk, axes=(0, 0))
        elif dim == 1:
            acc += np.tensordot(w[2][z0:z0 + chunk], blk, axes=(0, 0)) @ w[0]
        else:
            acc[z0:z0 + chunk] = np.tensordot(blk, w[0], axes=(2, 0)) @ w[1]
    return dft1_direct(acc, sign)

