"""Slab-pencil 3D DFT distributed over a 1D grid of P processes (Section 2.4,
Fig. 3dslabpencil): one process per GPU, each running the rank-local plans of
``libfft3`` (``fft3_options.dist_ranks`` / ``dist_stage``) on its own device,
with the exchanges between them done by ``torch.distributed.all_to_all_single``
(NCCL between GPUs, gloo on the host).

Data distribution (n0 fastest, every local array contiguous):

* slabs: rank r holds z in [r n2/P, (r+1) n2/P) as a (n2/P, n1, n0) array;
* pencils: rank r holds x in [r n0/P, (r+1) n0/P) as a (n2, n1, n0/P) array.

Forward: slabs in; the slab stage (x and y passes, the y pass storing the
slabs packed by destination rank), one all-to-all, the pencil stage (z pass)
leaves the spectrum in pencils.  With ``natural_spectrum`` a second
all-to-all and the stage-3 unpack return it to slabs (the exchange the paper
notes can be dropped when the caller accepts the shuffled spectrum).  Inverse:
the reverse, from pencils (or slabs) back to slabs, unnormalised.

Needs P | n0 and P | n2.  With P = 1 the transform is the one-GPU slab-pencil
plan.  ``stages`` replaces the rank-local GPU plans by objects with an
``execute(x, out)`` method, keyed by dist_stage (1, 2, 3; key 0 the one-GPU
plan when P = 1), as tests do with a host replay of the same schedules.
"""
from __future__ import annotations

from . import fft3


class SlabPencil:
    def __init__(self, n0: int, n1: int, n2: int, direction: int = fft3.FFT3_FORWARD, group=None,
                 natural_spectrum: bool = False, dtype: int = fft3.FFT3_C64_FP32, stages=None):
        import torch
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.P = dist.get_world_size(group) if dist.is_initialized() else 1
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        P = self.P
        if n0 % P or n2 % P:
            raise ValueError(f"the rank count {P} must divide n0 = {n0} and n2 = {n2}")
        self.shape = (n0, n1, n2)
        self.direction = direction
        self.natural = bool(natural_spectrum)
        self.dtype = dtype
        self.local_elems = n0 * n1 * n2 // P
        self.cdtype = torch.complex128 if dtype == fft3.FFT3_C128_FP64 else torch.complex64
        if P == 1:
            self.single = stages[0] if stages else fft3.Plan(n0, n1, n2, 1, fft3.FFT3_SLAB_PENCIL, direction,
                                                             dtype)
            return
        self.single = None
        if stages is None:
            mk = lambda dims, st: fft3.Plan(*dims, 1, fft3.FFT3_SLAB_PENCIL, direction, dtype, dist_ranks=P,
                                            dist_stage=st)
            stages = {1: mk((n0, n1, n2 // P), 1), 2: mk((n0 // P, n1, n2), 2)}
            if self.natural:
                stages[3] = mk((n0, n1, n2 // P), 3)
        self.stages = stages
        self._bufs = None

    def local_shape(self, spectrum: bool):
        """Shape of this rank's array: the spectrum's (pencils unless
        natural_spectrum) or the signal's (slabs)."""
        n0, n1, n2 = self.shape
        P = self.P
        if spectrum and not self.natural:
            return (n2, n1, n0 // P)
        return (n2 // P, n1, n0)

    def _exchange(self, send, recv):
        import torch
        # P equal blocks of n0 n1 n2 / P^2 values along the first dimension
        self.dist.all_to_all_single(torch.view_as_real(recv), torch.view_as_real(send), group=self.group)

    def execute(self, x, out) -> None:
        """x and out: this rank's contiguous arrays (complex64, or complex128
        for an FFT3_C128_FP64 plan) in the input and output distribution."""
        import torch
        assert x.is_contiguous() and out.is_contiguous() and x.dtype == self.cdtype == out.dtype
        assert x.numel() == out.numel() == self.local_elems
        if self.single is not None:
            self.single.execute(x, out)
            return
        if self._bufs is None or self._bufs[0].device != x.device:
            self._bufs = tuple(torch.empty(self.local_elems, dtype=self.cdtype, device=x.device) for _ in range(2))
        send, recv = self._bufs
        st = self.stages
        if self.direction == fft3.FFT3_FORWARD:
            st[1].execute(x, send)
            self._exchange(send, recv)
            if self.natural:
                st[2].execute(recv, send)
                self._exchange(send, recv)
                st[3].execute(recv, out)
            else:
                st[2].execute(recv, out)
        else:
            if self.natural:
                st[3].execute(x, send)
                self._exchange(send, recv)
                st[2].execute(recv, send)
            else:
                st[2].execute(x, send)
            self._exchange(send, recv)
            st[1].execute(recv, out)
