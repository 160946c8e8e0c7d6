"""GB300-native batched 3D complex DFT (slab-pencil, pencil-pencil-pencil and
volumetric decompositions) behind a small C ABI.

The compute path is ``libfft3.so`` (hand-written CUDA for sm_103a, built
in-tree from ``csrc/``); :mod:`paper_1904_10119_gb300.fft3` is a thin ctypes
binding with the C names.  There is no CPU fallback: every entry point fails
loudly when the library or a GPU is missing.
"""
__all__ = ["fft3", "synth"]
