"""Thin ctypes binding of libfft3.so (include/fft3.h), with the C names.

Argument marshalling only: every step of a transform runs in the library's
CUDA kernels.  There is no CPU fallback -- :func:`load` raises when the
library has not been built, and the library itself returns an error when no
GPU is visible.
"""
from __future__ import annotations

import ctypes
import json
import os
import re

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfft3.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "fft3.h")

FFT3_C64_FP32 = 0
FFT3_C64_SPLITBF16_TC = 1
FFT3_C128_FP64 = 2
FFT3_SLAB_PENCIL, FFT3_PENCIL3, FFT3_VOLUMETRIC, FFT3_AUTO = 0, 1, 2, 3
FFT3_FORWARD, FFT3_INVERSE = -1, 1
FFT3_PPP_NATURAL, FFT3_PPP_ROTATE, FFT3_PPP_BLOCKED = 0, 1, 2
FFT3_LAYOUT_NATURAL, FFT3_LAYOUT_ROTATED, FFT3_LAYOUT_PENCILS = 0, 1, 2
FFT3_VOL_CYCLIC, FFT3_VOL_BLOCKED_SIX_STEP = 0, 1

STATUS = {
    0: "FFT3_OK", -1: "FFT3_ERR_INVALID_ARG", -2: "FFT3_ERR_UNSUPPORTED_SIZE", -3: "FFT3_ERR_OOM",
    -4: "FFT3_ERR_CUDA", -5: "FFT3_ERR_TIMEOUT", -6: "FFT3_ERR_INPLACE_UNSUPPORTED",
    -7: "FFT3_ERR_NO_DEVICE",
}
DECOMP = {"slab_pencil": FFT3_SLAB_PENCIL, "pencil3": FFT3_PENCIL3, "ppp": FFT3_PENCIL3,
          "volumetric": FFT3_VOLUMETRIC, "auto": FFT3_AUTO}


class Fft3Error(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class fft3_options(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("radix_order", ctypes.c_int), ("tile_lines", ctypes.c_int),
                ("mesh", ctypes.c_int * 3), ("slab_mode", ctypes.c_int), ("tc_stages", ctypes.c_int),
                ("slab_chunk", ctypes.c_int), ("slab_lines", ctypes.c_int), ("layout", ctypes.c_int),
                ("dist_ranks", ctypes.c_int), ("dist_stage", ctypes.c_int), ("dist_ranks2", ctypes.c_int),
                ("reserved", ctypes.c_int * 8)]


_lib = None
_P = ctypes.c_void_p


def load() -> ctypes.CDLL:
    """Load the in-tree libfft3.so (built by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    i, i64, sz = ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
    pi = ctypes.POINTER(ctypes.c_int)
    sig = {
        "fft3_plan_create": (i, [ctypes.POINTER(_P), i, i, i, i, i, i, i]),
        "fft3_plan_create_ex": (i, [ctypes.POINTER(_P), i, i, i, i, i, i, i, ctypes.POINTER(fft3_options)]),
        "fft3_plan_create_many": (i, [ctypes.POINTER(_P), i, pi, ctypes.POINTER(ctypes.c_int64), i, i, i, pi]),
        "fft3_plan_execute": (i, [_P, _P, _P, _P]),
        "fft3_plan_execute_host": (i, [_P, _P, _P, _P]),
        "fft3_plan_check": (i, [_P]),
        "fft3_plan_destroy": (i, [_P]),
        "fft3_plan_workspace_bytes": (sz, [_P]),
        "fft3_plan_launches": (i, [_P]),
        "fft3_plan_kernel_launches": (i, [_P]),
        "fft3_plan_execute_host_pipelined": (i, [_P, _P, _P, ctypes.c_int, _P]),
        "fft3_plan_describe": (i, [_P, ctypes.c_char_p, sz]),
        "fft3_plan_schedule": (i, [i, i, i, i, i, i, i, ctypes.POINTER(fft3_options), ctypes.c_char_p, sz]),
        "fft3_plan_schedule_many": (i, [i, pi, ctypes.POINTER(ctypes.c_int64), i, i, i, pi, ctypes.c_char_p, sz]),
        "fft3_factorize": (i, [i, i, pi, i]),
        "fft3_layout_positions": (i, [i, i, i, i, i, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                      i64]),
        "fft3_twiddles": (i, [i, i, _P, i64, _P, _P, _P]),
        "fft3_plan_probe_layout": (i, [_P, _P, _P, i, _P]),
        "fft3_plan_execute_pass": (i, [_P, i, _P, _P, _P]),
        "fft3_split_bf16": (i, [_P, i64, _P, _P, _P]),
        "fft3_time_plan": (i, [i, i, i, i, i, i, i, ctypes.POINTER(fft3_options), i, ctypes.POINTER(ctypes.c_float)]),
        "fft3_time_candidates": (i, [i, i, i, i, i, i, i, i, pi, ctypes.POINTER(fft3_options),
                                     ctypes.POINTER(ctypes.c_float)]),
        "fft3_autotune": (i, [i, i, i, i, i, i, i, ctypes.POINTER(fft3_options), pi, ctypes.POINTER(ctypes.c_float)]),
        "fft3_autotune_many": (i, [i, pi, ctypes.POINTER(ctypes.c_int64), i, i, i, pi]),
        "fft3_mlp_create": (i, [ctypes.POINTER(_P), i, i, ctypes.c_ulonglong]),
        "fft3_mlp_destroy": (i, [_P]),
        "fft3_mlp_num_params": (i, [_P]),
        "fft3_mlp_set_params": (i, [_P, _P]),
        "fft3_mlp_get_params": (i, [_P, _P]),
        "fft3_mlp_forward": (i, [_P, _P, i, _P, _P]),
        "fft3_mlp_grad": (i, [_P, _P, _P, i, _P, _P, _P]),
        "fft3_mlp_adam_step": (i, [_P, _P, ctypes.c_float, _P]),
        "fft3_mlp_train": (i, [_P, _P, _P, i, i, i, ctypes.c_float, ctypes.c_ulonglong, _P]),
        "fft3_mlp_predict": (i, [_P, _P, i, _P]),
        "fft3_execute_noalloc": (i, [i, i, i, i, i, _P, _P, _P]),
        "fft3_last_error": (ctypes.c_char_p, []),
        "fft3_version": (i, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def header_symbols() -> list[str]:
    """Entry points declared in include/fft3.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(fft3_\w+)\s*\(", txt, re.M)))


def last_error() -> str:
    return load().fft3_last_error().decode(errors="replace")


def _check(rc: int) -> int:
    if rc < 0:
        raise Fft3Error(rc, last_error())
    return rc


def make_options(variant=0, radix_order=0, tile_lines=0, mesh=(0, 0, 0), slab_mode=0, tc_stages=0,
                 slab_chunk=0, slab_lines=0, layout=0, dist_ranks=0, dist_stage=0, dist_ranks2=0) -> fft3_options:
    o = fft3_options()
    o.variant = int(variant)
    o.radix_order = int(radix_order)
    o.tile_lines = int(tile_lines)
    for k in range(3):
        o.mesh[k] = int(mesh[k])
    o.slab_mode = int(slab_mode)
    o.tc_stages = int(tc_stages)
    o.slab_chunk = int(slab_chunk)
    o.slab_lines = int(slab_lines)
    o.layout = int(layout)
    o.dist_ranks = int(dist_ranks)
    o.dist_stage = int(dist_stage)
    o.dist_ranks2 = int(dist_ranks2)
    return o


# ------------------------------------------------------------ C-name calls -- #
def fft3_plan_create(n0, n1, n2, batch=1, dtype=FFT3_C64_FP32, decomposition=FFT3_PENCIL3,
                     direction=FFT3_FORWARD) -> int:
    h = _P()
    _check(load().fft3_plan_create(ctypes.byref(h), n0, n1, n2, batch, dtype, decomposition, direction))
    return h.value


def fft3_plan_create_ex(n0, n1, n2, batch=1, dtype=FFT3_C64_FP32, decomposition=FFT3_PENCIL3,
                        direction=FFT3_FORWARD, opts: fft3_options | None = None) -> int:
    h = _P()
    _check(load().fft3_plan_create_ex(ctypes.byref(h), n0, n1, n2, batch, dtype, decomposition,
                                      direction, ctypes.byref(opts) if opts is not None else None))
    return h.value


def fft3_plan_create_many(dims, offsets, dtype=FFT3_C64_FP32, decomposition=FFT3_AUTO,
                          direction=FFT3_FORWARD, tuning=None) -> int:
    count = len(offsets)
    d = (ctypes.c_int * (3 * count))(*[int(v) for v in list(_flat(dims))])
    o = (ctypes.c_int64 * count)(*[int(v) for v in offsets])
    t = (ctypes.c_int * count)(*[int(v) for v in tuning]) if tuning is not None else None
    h = _P()
    _check(load().fft3_plan_create_many(ctypes.byref(h), count, d, o, dtype, decomposition, direction, t))
    return h.value


def fft3_plan_schedule_many(dims, offsets, dtype=FFT3_C64_FP32, decomposition=FFT3_AUTO,
                            direction=FFT3_FORWARD, tuning=None) -> dict:
    """Host-only description of the batched plan fft3_plan_create_many would build."""
    count = len(offsets)
    d = (ctypes.c_int * (3 * count))(*[int(v) for v in list(_flat(dims))])
    o = (ctypes.c_int64 * count)(*[int(v) for v in offsets])
    t = (ctypes.c_int * count)(*[int(v) for v in tuning]) if tuning is not None else None
    L = load()
    n = _check(L.fft3_plan_schedule_many(count, d, o, dtype, decomposition, direction, t, None, 0))
    buf = ctypes.create_string_buffer(n + 1)
    _check(L.fft3_plan_schedule_many(count, d, o, dtype, decomposition, direction, t, buf, n + 1))
    return json.loads(buf.value.decode())


def _flat(dims):
    for row in dims:
        for v in row:
            yield v


def fft3_plan_execute(plan: int, in_ptr: int, out_ptr: int, stream: int = 0) -> None:
    _check(load().fft3_plan_execute(_P(plan), _P(in_ptr), _P(out_ptr), _P(stream)))


FFT3_NOALLOC_MAX_ELEMENTS = 1 << 21


def fft3_execute_noalloc(n0, n1, n2, batch, direction, in_ptr: int, out_ptr: int, stream: int = 0) -> None:
    """Transform without any device allocation (fixed library-owned scratch;
    see include/fft3.h for the limits and the sharing rules)."""
    _check(load().fft3_execute_noalloc(n0, n1, n2, batch, direction, _P(in_ptr), _P(out_ptr), _P(stream)))


def fft3_plan_execute_host(plan: int, h_in: int, h_out: int, stream: int = 0) -> None:
    _check(load().fft3_plan_execute_host(_P(plan), _P(h_in), _P(h_out), _P(stream)))


def fft3_plan_check(plan: int) -> int:
    return load().fft3_plan_check(_P(plan))


def fft3_plan_destroy(plan: int) -> None:
    _check(load().fft3_plan_destroy(_P(plan)))


def fft3_plan_workspace_bytes(plan: int) -> int:
    return int(load().fft3_plan_workspace_bytes(_P(plan)))


def fft3_plan_launches(plan: int) -> int:
    return _check(load().fft3_plan_launches(_P(plan)))


def fft3_plan_execute_host_pipelined(plan: int, h_in_ptrs, h_out_ptrs, stream: int = 0) -> None:
    count = len(h_in_ptrs)
    assert len(h_out_ptrs) == count
    arr_in = (_P * max(1, count))(*[int(v) for v in h_in_ptrs])
    arr_out = (_P * max(1, count))(*[int(v) for v in h_out_ptrs])
    _check(load().fft3_plan_execute_host_pipelined(_P(plan), arr_in, arr_out, count, _P(stream)))


def fft3_plan_kernel_launches(plan: int) -> int:
    return _check(load().fft3_plan_kernel_launches(_P(plan)))


def fft3_plan_describe(plan: int) -> dict:
    L = load()
    n = _check(L.fft3_plan_describe(_P(plan), None, 0))
    buf = ctypes.create_string_buffer(n + 1)
    _check(L.fft3_plan_describe(_P(plan), buf, n + 1))
    return json.loads(buf.value.decode())


def fft3_plan_schedule(n0, n1, n2, batch=1, dtype=FFT3_C64_FP32, decomposition=FFT3_PENCIL3,
                       direction=FFT3_FORWARD, opts: fft3_options | None = None) -> dict:
    L = load()
    po = ctypes.byref(opts) if opts is not None else None
    n = _check(L.fft3_plan_schedule(n0, n1, n2, batch, dtype, decomposition, direction, po, None, 0))
    buf = ctypes.create_string_buffer(n + 1)
    _check(L.fft3_plan_schedule(n0, n1, n2, batch, dtype, decomposition, direction, po, buf, n + 1))
    return json.loads(buf.value.decode())


def fft3_layout_positions(layout: int, n0: int, n1: int, n2: int, batch: int = 1, idx=None):
    """Positions (int64 numpy array) of natural flat indices `idx` (default:
    all of them, in order) in the buffer of a permuted layout."""
    import numpy as np
    if idx is None:
        idx = np.arange(n0 * n1 * n2 * batch, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    pos = np.empty_like(idx)
    p64 = ctypes.POINTER(ctypes.c_int64)
    _check(load().fft3_layout_positions(layout, n0, n1, n2, batch, idx.ctypes.data_as(p64),
                                        pos.ctypes.data_as(p64), idx.size))
    return pos


def fft3_factorize(n: int, order: int = 0) -> list[int]:
    rad = (ctypes.c_int * 16)()
    k = _check(load().fft3_factorize(n, order, rad, 16))
    return [rad[i] for i in range(k)]


def fft3_twiddles(n: int, sign: int, d_m: int, count: int, d_out64: int | None, d_out32: int | None,
                  stream: int = 0) -> None:
    _check(load().fft3_twiddles(n, sign, _P(d_m), count, _P(d_out64 or 0) if d_out64 else None,
                                _P(d_out32) if d_out32 else None, _P(stream)))


def fft3_plan_probe_layout(plan: int, in_ptr: int, out_ptr: int, npasses: int = -1, stream: int = 0) -> None:
    _check(load().fft3_plan_probe_layout(_P(plan), _P(in_ptr), _P(out_ptr), npasses, _P(stream)))


def fft3_plan_execute_pass(plan: int, k: int, in_ptr: int, out_ptr: int, stream: int = 0) -> None:
    _check(load().fft3_plan_execute_pass(_P(plan), k, _P(in_ptr), _P(out_ptr), _P(stream)))


def fft3_split_bf16(d_x: int, count: int, d_hi: int, d_lo: int, stream: int = 0) -> None:
    _check(load().fft3_split_bf16(_P(d_x), count, _P(d_hi), _P(d_lo), _P(stream)))


def fft3_time_plan(n0, n1, n2, batch=1, dtype=FFT3_C64_FP32, decomposition=FFT3_PENCIL3,
                   direction=FFT3_FORWARD, opts: fft3_options | None = None, reps: int = 5) -> float:
    ms = ctypes.c_float()
    _check(load().fft3_time_plan(n0, n1, n2, batch, dtype, decomposition, direction,
                                 ctypes.byref(opts) if opts is not None else None, reps, ctypes.byref(ms)))
    return float(ms.value)


def fft3_autotune(n0, n1, n2, batch=1, dtype=FFT3_C64_FP32, direction=FFT3_FORWARD, reps: int = 3):
    """Returns (options, decomposition, ms) of the fastest candidate plan."""
    o = fft3_options()
    d = ctypes.c_int()
    ms = ctypes.c_float()
    _check(load().fft3_autotune(n0, n1, n2, batch, dtype, direction, reps, ctypes.byref(o), ctypes.byref(d),
                                ctypes.byref(ms)))
    return o, int(d.value), float(ms.value)


def fft3_autotune_many(dims, direction=FFT3_FORWARD, reps: int = 3, max_per_class: int = 32) -> list[int]:
    count = len(dims)
    d = (ctypes.c_int * (3 * count))(*[int(v) for v in list(_flat(dims))])
    t = (ctypes.c_int * count)()
    _check(load().fft3_autotune_many(count, d, None, direction, reps, max_per_class, t))
    return [int(t[i]) for i in range(count)]


FFT3_TUNE_SLABZ = 1 << 12  # or'ed into every tuning code: the slab-by-slab executor


def tune_code(decomp: int, radix_order: int = 0, tile_code: int = 0, items_code: int = 0) -> int:
    """FFT3_TUNE of include/fft3.h."""
    return decomp | ((radix_order + 1) << 2) | (tile_code << 5) | (items_code << 8)


class Mlp:
    """The library's plan-cost perceptron (fft3_mlp_*); numpy float32 in and out."""

    def __init__(self, n_features: int, hidden: int = 64, seed: int = 0):
        h = _P()
        _check(load().fft3_mlp_create(ctypes.byref(h), n_features, hidden, seed))
        self.handle = h.value
        self.F, self.H = n_features, hidden

    @property
    def num_params(self) -> int:
        return _check(load().fft3_mlp_num_params(_P(self.handle)))

    def get_params(self):
        import numpy as np
        p = np.empty(self.num_params, np.float32)
        _check(load().fft3_mlp_get_params(_P(self.handle), _P(p.ctypes.data)))
        return p

    def set_params(self, p) -> None:
        import numpy as np
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.num_params
        _check(load().fft3_mlp_set_params(_P(self.handle), _P(p.ctypes.data)))

    def train(self, X, y, epochs=200, batch=128, lr=1e-3, seed=0):
        import numpy as np
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.float32)
        curve = np.zeros(epochs, np.float32)
        _check(load().fft3_mlp_train(_P(self.handle), _P(X.ctypes.data), _P(y.ctypes.data), X.shape[0], epochs,
                                     batch, lr, seed, _P(curve.ctypes.data)))
        return curve

    def predict(self, X):
        import numpy as np
        X = np.ascontiguousarray(X, dtype=np.float32)
        out = np.empty(X.shape[0], np.float32)
        _check(load().fft3_mlp_predict(_P(self.handle), _P(X.ctypes.data), X.shape[0], _P(out.ctypes.data)))
        return out

    def close(self):
        if self.handle:
            load().fft3_mlp_destroy(_P(self.handle))
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------ torch convenience -- #
class Plan:
    """Owns one fft3 plan; `execute(x, out)` takes contiguous CUDA tensors of
    complex64 (complex128 for an FFT3_C128_FP64 plan)."""

    def __init__(self, n0, n1, n2, batch=1, decomposition=FFT3_PENCIL3, direction=FFT3_FORWARD,
                 dtype=FFT3_C64_FP32, **opts):
        self.shape = (n0, n1, n2)
        self.batch = batch
        self.dtype = dtype
        self.handle = fft3_plan_create_ex(n0, n1, n2, batch, dtype, decomposition, direction,
                                          make_options(**opts))

    def execute(self, x, out, stream=None) -> None:
        import torch
        want = torch.complex128 if self.dtype == FFT3_C128_FP64 else torch.complex64
        assert x.is_cuda and out.is_cuda and x.dtype == want and out.dtype == want
        assert x.is_contiguous() and out.is_contiguous()
        s = stream if stream is not None else torch.cuda.current_stream()
        fft3_plan_execute(self.handle, x.data_ptr(), out.data_ptr(), s.cuda_stream)

    def describe(self) -> dict:
        return fft3_plan_describe(self.handle)

    def launches(self) -> int:
        return fft3_plan_launches(self.handle)

    def kernel_launches(self) -> int:
        return fft3_plan_kernel_launches(self.handle)

    def check(self) -> int:
        return fft3_plan_check(self.handle)

    def close(self) -> None:
        if self.handle:
            fft3_plan_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
