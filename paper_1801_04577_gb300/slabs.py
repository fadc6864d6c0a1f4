"""Domain decomposition of one lattice into y-slabs (host logic).

One time step needs, at every node, only the post-collision populations of
its eight neighbours (streaming, Eq. 11 and Eq. 21) and, at a wall link, the
temperature of the next node along the link (Eq. 27-28).  So a lattice splits
into slabs of whole rows; each slab keeps a ghost row on each side, and after
every step (and after the initialisation) each slab's first and last own rows,
all planes, go to its neighbours' ghost rows.  The slab kernels then reproduce
the whole lattice bit for bit; the FP64 reductions (residual, Nusselt numbers,
conservation sums) are partial sums added across slabs.

Two ways to hold the slabs:

* ``SlabGroup``: several slabs in one process (one GPU, or peer-accessible
  GPUs), exchanged by the library's strided device copies
  (``clbm_slabs_step``);
* one slab per process (``torch.distributed``, NCCL on GPUs): ``exchange``
  sends the packed edge rows to the neighbouring ranks and receives their
  rows for the ghost rows; ``allreduce_sums`` adds the reduction sums.

Only the topology and the message pattern live here; the data movement on the
GPU is the library's (``clbm_halo_pack`` / ``clbm_halo_unpack`` /
``clbm_halo_copy``).
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import clbm


def partition(ny: int, parts: int) -> List[Tuple[int, int]]:
    """Rows [y0, y0 + rows) of each of `parts` slabs, bottom to top, as equal
    as possible (the first ny % parts slabs get one row more)."""
    if parts < 1 or ny < parts:
        raise ValueError(f"cannot split {ny} rows into {parts} slabs")
    base, extra = divmod(ny, parts)
    out, y0 = [], 0
    for k in range(parts):
        rows = base + (1 if k < extra else 0)
        out.append((y0, rows))
        y0 += rows
    return out


def neighbours(rank: int, world: int, periodic: bool) -> Tuple[Optional[int], Optional[int]]:
    """(rank below, rank above) of slab `rank`; None where a box wall bounds it."""
    below = rank - 1 if rank > 0 else (world - 1 if periodic else None)
    above = rank + 1 if rank < world - 1 else (0 if periodic else None)
    return below, above


# Message tags: a first own row travels down (it becomes the ghost row above
# the slab below), a last own row travels up (the ghost row below the slab above).
TAG_DOWN, TAG_UP = 11, 12


def exchange(send_lo, send_hi, recv_lo, recv_hi, rank: int, world: int, periodic: bool,
             group=None) -> None:
    """Halo exchange of one slab per rank through torch.distributed.

    send_lo / send_hi: this rank's packed first / last own row; recv_lo /
    recv_hi: buffers for the ghost row below / above (the last own row of the
    rank below, the first own row of the rank above).  Tensors on the backend's
    device (CUDA for NCCL, CPU for gloo).  Buffers on a box-wall side are left
    untouched (pass None).  The operations are issued in the same order on
    every rank -- send down, send up, receive from above, receive from below --
    so that ranks joined by two messages (two slabs of a periodic lattice)
    match them in order even where the backend ignores tags.
    """
    import torch.distributed as dist

    below, above = neighbours(rank, world, periodic)
    if world == 1:
        if periodic:  # the slab is its own neighbour on both sides
            recv_hi.copy_(send_lo)
            recv_lo.copy_(send_hi)
        return
    ops = []
    if below is not None:
        ops.append(dist.P2POp(dist.isend, send_lo, below, group=group, tag=TAG_DOWN))
    if above is not None:
        ops.append(dist.P2POp(dist.isend, send_hi, above, group=group, tag=TAG_UP))
    if above is not None:
        ops.append(dist.P2POp(dist.irecv, recv_hi, above, group=group, tag=TAG_DOWN))
    if below is not None:
        ops.append(dist.P2POp(dist.irecv, recv_lo, below, group=group, tag=TAG_UP))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()


def allreduce_sums(sums: np.ndarray, device=None, group=None) -> np.ndarray:
    """Element-wise sum of every rank's reduction sums (FP64)."""
    import torch
    import torch.distributed as dist

    t = torch.as_tensor(np.ascontiguousarray(sums, np.float64), device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy()


class DistSlab:
    """One slab per process: the GPU slab of this rank, packed halo buffers on
    its device, and the exchange through torch.distributed.  With NCCL the
    packed rows travel between the GPUs directly; with gloo (whose send and
    receive take host tensors) they are staged through pinned host memory, so
    ranks may even share one GPU -- no kernel of one rank ever waits on another
    rank: each rank's host finishes the exchange before it launches its next
    step."""

    def __init__(self, w, precision: str = "f32", rounding: int = 0, stream: Optional[int] = None,
                 group=None):
        import torch
        import torch.distributed as dist

        self.group = group
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        self.world = dist.get_world_size(group) if dist.is_initialized() else 1
        self.staged = dist.is_initialized() and dist.get_backend(group) == "gloo"
        self.periodic = bool(w.params.periodic_y)
        self.y0, self.rows = partition(w.params.ny, self.world)[self.rank]
        # the library's work, the staging copies and the communication share one stream
        if stream is None:
            self.tstream = torch.cuda.Stream()
            stream = self.tstream.cuda_stream
        else:
            self.tstream = torch.cuda.ExternalStream(stream)
        self.slab = clbm.Slab(w.params, self.y0, self.rows, w.geom, precision, stream, w.init, rounding)
        nbytes = clbm.clbm_halo_bytes(self.slab.ctx)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.bufs = [torch.empty(nbytes, dtype=torch.uint8, device=dev) for _ in range(4)]
        if self.staged:
            self.host = [torch.empty(nbytes, dtype=torch.uint8).pin_memory() for _ in range(4)]
        self.exchange()

    def exchange(self):
        import torch
        send_lo, send_hi, recv_lo, recv_hi = self.bufs
        below, above = neighbours(self.rank, self.world, self.periodic)
        clbm.clbm_halo_pack(self.slab.ctx, 0, send_lo)
        clbm.clbm_halo_pack(self.slab.ctx, 1, send_hi)
        with torch.cuda.stream(self.tstream):
            if self.staged:
                hs_lo, hs_hi, hr_lo, hr_hi = self.host
                hs_lo.copy_(send_lo, non_blocking=True)
                hs_hi.copy_(send_hi, non_blocking=True)
                self.tstream.synchronize()
                exchange(hs_lo, hs_hi, hr_lo, hr_hi, self.rank, self.world, self.periodic, self.group)
                recv_lo.copy_(hr_lo, non_blocking=True)
                recv_hi.copy_(hr_hi, non_blocking=True)
            else:
                exchange(send_lo, send_hi, recv_lo, recv_hi, self.rank, self.world, self.periodic,
                         self.group)
        if below is not None:
            clbm.clbm_halo_unpack(self.slab.ctx, 0, recv_lo)
        if above is not None:
            clbm.clbm_halo_unpack(self.slab.ctx, 1, recv_hi)

    def step(self, n: int = 1):
        for _ in range(n):
            self.slab.step(1)
            self.exchange()

    def _dev(self):
        return None if self.staged else self.bufs[0].device

    def residual(self) -> float:
        s = allreduce_sums(self.slab.sums(clbm.REDUCE_RESIDUAL), device=self._dev(), group=self.group)
        return float(clbm.clbm_finish_sums(self.slab.ctx, clbm.REDUCE_RESIDUAL, s)[0])

    def nusselt(self, which: int, length: float, dT: float) -> float:
        s = allreduce_sums(self.slab.sums(clbm.REDUCE_NUSSELT, which), device=self._dev(),
                           group=self.group)
        return float(clbm.clbm_finish_sums(self.slab.ctx, clbm.REDUCE_NUSSELT, s, length, dT)[0])

    def totals(self) -> np.ndarray:
        s = allreduce_sums(self.slab.sums(clbm.REDUCE_TOTALS), device=self._dev(), group=self.group)
        return clbm.clbm_finish_sums(self.slab.ctx, clbm.REDUCE_TOTALS, s)

    def close(self):
        self.slab.close()


class SlabGroup:
    """`parts` slabs of one lattice in this process (one shared stream),
    advanced together: every step is one step of each slab followed by the
    halo copies between them."""

    def __init__(self, w, parts: int, precision: str = "f32", rounding: int = 0,
                 stream: Optional[int] = None, bounds: Optional[Sequence[Tuple[int, int]]] = None):
        self.w = w
        self.periodic = bool(w.params.periodic_y)
        self.bounds = list(bounds) if bounds is not None else partition(w.params.ny, parts)
        self.slabs = [clbm.Slab(w.params, y0, rows, w.geom, precision, stream, w.init, rounding)
                      for (y0, rows) in self.bounds]
        self.exchange()

    @property
    def ctxs(self):
        return [s.ctx for s in self.slabs]

    def exchange(self):
        clbm.clbm_slabs_exchange(self.ctxs, self.periodic)

    def step(self, n: int = 1):
        clbm.clbm_slabs_step(self.ctxs, self.periodic, n)

    def moments(self):
        parts = [s.moments() for s in self.slabs]
        return tuple(np.concatenate([p[k] for p in parts], axis=0) for k in range(4))

    def _sum(self, what, which=0):
        return np.sum([s.sums(what, which) for s in self.slabs], axis=0)

    def residual(self) -> float:
        return float(clbm.clbm_finish_sums(self.slabs[0].ctx, clbm.REDUCE_RESIDUAL,
                                           self._sum(clbm.REDUCE_RESIDUAL))[0])

    def nusselt(self, which: int, length: float, dT: float) -> float:
        return float(clbm.clbm_finish_sums(self.slabs[0].ctx, clbm.REDUCE_NUSSELT,
                                           self._sum(clbm.REDUCE_NUSSELT, which), length, dT)[0])

    def totals(self) -> np.ndarray:
        return clbm.clbm_finish_sums(self.slabs[0].ctx, clbm.REDUCE_TOTALS, self._sum(clbm.REDUCE_TOTALS))

    def close(self):
        for s in self.slabs:
            s.close()
