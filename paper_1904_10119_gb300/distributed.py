"""3D DFTs distributed over several processes (Section 2.4): one process per
GPU, each running the rank-local plans of ``libfft3``
(``fft3_options.dist_ranks`` / ``dist_ranks2`` / ``dist_stage``) on its own
device, with the exchanges between them done by
``torch.distributed.all_to_all_single`` (NCCL between GPUs, gloo on the host).

``SlabPencil``: the slab-pencil decomposition on a 1D grid of P processes
(Fig. 3dslabpencil).  ``Pencil3``: the pencil-pencil-pencil decomposition on
a Py x Pz grid (Fig. 3dpencilpencil), one exchange within each row of the
grid and one within each column.

SlabPencil:

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


class Pencil3:
    """Pencil-pencil-pencil 3D DFT on a Py x Pz grid: rank r = q Py + p.

    Data distribution (n0 fastest, every local array contiguous):

    * pencils (forward input, inverse output): rank (p, q) holds y in
      [p n1/Py, (p+1) n1/Py) and z in [q n2/Pz, (q+1) n2/Pz), all x, as a
      (n2/Pz, n1/Py, n0) array;
    * bricks (forward output, inverse input): rank (p, q) holds x in
      [p n0/Py, (p+1) n0/Py) and y in [q n1/Pz, (q+1) n1/Pz), all z, as a
      (n2, n1/Pz, n0/Py) array (the last redistribution left out).

    Forward: stage 1 (x lines, stored packed by destination), an all-to-all
    among the Py ranks of the row, stage 2 (y lines, read in place from the Py
    received blocks, stored packed), an all-to-all among the Pz ranks of the
    column, stage 3 (z lines, read in place, stored as the brick).  Inverse:
    stages 3, 2, 1 with the exchanges between them in reverse order.  Needs
    Py | n0, Py | n1, Pz | n1, Pz | n2.  ``stages`` replaces the GPU plans by
    objects with ``execute(x, out)``, keyed 1, 2, 3."""

    def __init__(self, n0: int, n1: int, n2: int, grid, direction: int = fft3.FFT3_FORWARD,
                 dtype: int = fft3.FFT3_C64_FP32, stages=None):
        import torch
        import torch.distributed as dist
        self.dist = dist
        Py, Pz = (int(v) for v in grid)
        world = dist.get_world_size() if dist.is_initialized() else 1
        if Py * Pz != world:
            raise ValueError(f"grid {Py} x {Pz} needs {Py * Pz} ranks, the job has {world}")
        if n0 % Py or n1 % Py or n1 % Pz or n2 % Pz:
            raise ValueError(f"grid {Py} x {Pz} must divide n0, n1 (by both) and n2 = {n0}, {n1}, {n2}")
        self.grid = (Py, Pz)
        self.rank = dist.get_rank() if dist.is_initialized() else 0
        self.p, self.q = self.rank % Py, self.rank // Py
        self.shape = (n0, n1, n2)
        self.direction = direction
        self.local_elems = n0 * n1 * n2 // (Py * Pz)
        self.cdtype = torch.complex128 if dtype == fft3.FFT3_C128_FP64 else torch.complex64
        # every rank creates every group, in the same order
        self.row_group = self.col_group = None
        if world > 1:
            for q in range(Pz):
                g = dist.new_group([q * Py + p for p in range(Py)])
                if q == self.q:
                    self.row_group = g
            for p in range(Py):
                g = dist.new_group([q * Py + p for q in range(Pz)])
                if p == self.p:
                    self.col_group = g
        if stages is None:
            mk = lambda dims, st: fft3.Plan(*dims, 1, fft3.FFT3_PENCIL3, direction, dtype, dist_ranks=Py,
                                            dist_ranks2=Pz, dist_stage=st)
            stages = {1: mk((n0, n1 // Py, n2 // Pz), 1), 2: mk((n0 // Py, n1, n2 // Pz), 2),
                      3: mk((n0 // Py, n1 // Pz, n2), 3)}
        self.stages = stages
        self._bufs = None

    def local_shape(self, spectrum: bool):
        n0, n1, n2 = self.shape
        Py, Pz = self.grid
        return (n2, n1 // Pz, n0 // Py) if spectrum else (n2 // Pz, n1 // Py, n0)

    def _exchange(self, send, recv, group, size):
        import torch
        if size == 1:
            recv.copy_(send)
            return
        self.dist.all_to_all_single(torch.view_as_real(recv), torch.view_as_real(send), group=group)

    def execute(self, x, out) -> None:
        import torch
        assert x.is_contiguous() and out.is_contiguous() and x.dtype == self.cdtype == out.dtype
        assert x.numel() == out.numel() == self.local_elems
        if self._bufs is None or self._bufs[0].device != x.device:
            self._bufs = tuple(torch.empty(self.local_elems, dtype=self.cdtype, device=x.device) for _ in range(2))
        send, recv = self._bufs
        st = self.stages
        Py, Pz = self.grid
        if self.direction == fft3.FFT3_FORWARD:
            st[1].execute(x, send)
            self._exchange(send, recv, self.row_group, Py)
            st[2].execute(recv, send)
            self._exchange(send, recv, self.col_group, Pz)
            st[3].execute(recv, out)
        else:
            st[3].execute(x, send)
            self._exchange(send, recv, self.col_group, Pz)
            st[2].execute(recv, send)
            self._exchange(send, recv, self.row_group, Py)
            st[1].execute(recv, out)
