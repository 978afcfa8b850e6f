"""One 2D lattice decomposed along y into slabs, one rank (one GPU) per slab.

The step of Eq. (2.2) reads f^n at most three nodes away, and its only global
quantity is the speed bound abar_j of Eq. (2.19), a maximum over every node
that sets dt, lambda and alpha_j (Eqs. 2.20, 2.21).  A slab therefore keeps
its own rows plus three halo rows on each side that borders another slab, and
each step is

    1. abar := maximum over the ranks of each slab's bound (one all-reduce of
       d numbers);
    2. one step of every slab (the CUDA library; only the slab's own rows are
       written);
    3. each slab's three outermost rows on a side go to the neighbour across
       it, which stores them as its halo (point-to-point, both directions).

This module is host-side orchestration only: the partition, the collectives
and the bookkeeping.  Every step of the method runs in the library through
``lbmh.Slab``; with ``device_buffers`` the halo rows move between device
buffers (NCCL), otherwise through host memory (gloo).  The backend that holds
a slab can be replaced (``backend=``), which is how the orchestration is
tested on CPU ranks.
"""
import numpy as np

from . import lbmh
from . import workloads as W

GHOST = 3  # rows of f^n one node update reads on each side


def partition_rows(ny, world):
    """Balanced contiguous row ranges [(begin, end), ...], one per rank, each
    at least GHOST rows so that a neighbour's halo comes from one slab."""
    if world < 1 or ny < GHOST * world:
        raise ValueError(f"{ny} rows cannot be cut into {world} slabs of at least {GHOST} rows")
    cuts = [ny * r // world for r in range(world + 1)]
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def neighbours(rank, world, periodic):
    """(rank below, rank above) of a slab, None where the lattice ends."""
    lo = rank - 1 if rank > 0 else (world - 1 if periodic and world > 1 else None)
    hi = rank + 1 if rank < world - 1 else (0 if periodic and world > 1 else None)
    return lo, hi


def local_rows(ny, begin, end, halo):
    """Global row index of every local row of a slab (wrapped for a y-periodic lattice)."""
    return np.arange(begin - halo[0], end + halo[1]) % ny


class SlabRun:
    """The slab of this rank and the exchanges of a decomposed lattice.

    pb: the whole lattice (workloads.Problem, 2D).  group: a torch.distributed
    process group (None: the default group).  backend(pb, begin, end,
    precision) returns the object holding the slab (default: lbmh.Slab)."""

    def __init__(self, pb, rank, world, precision=lbmh.FP32, group=None, backend=None, device_buffers=False):
        import torch
        import torch.distributed as dist
        if pb.dim != 2:
            raise ValueError("slabs decompose 2D lattices")
        self.pb, self.rank, self.world, self.group = pb, rank, world, group
        self.dist, self.torch = dist, torch
        self.rows = partition_rows(pb.ny, world)
        self.begin, self.end = self.rows[rank]
        make = backend if backend is not None else (lambda p, b, e, prec: lbmh.Slab(p, b, e, precision=prec))
        self.slab = make(pb, self.begin, self.end, precision)
        self.halo = tuple(self.slab.halo)
        periodic = pb.bc[2] == W.PERIODIC
        self.lo, self.hi = neighbours(rank, world, periodic)
        if (self.lo is None) != (self.halo[0] == 0) or (self.hi is None) != (self.halo[1] == 0):
            raise RuntimeError("slab halo rows do not match the partition")
        self.device_buffers = device_buffers
        nb = int(self.slab.halo_bytes)
        if device_buffers:
            dev = torch.device("cuda", torch.cuda.current_device())
            self._send = [torch.empty(nb, dtype=torch.uint8, device=dev) for _ in range(2)]
            self._recv = [torch.empty(nb, dtype=torch.uint8, device=dev) for _ in range(2)]
            self._coll_device = dev
        else:
            self._send = [torch.empty(nb, dtype=torch.uint8) for _ in range(2)]
            self._recv = [torch.empty(nb, dtype=torch.uint8) for _ in range(2)]
            self._coll_device = torch.device("cpu")
        self.steps = 0

    # -- collectives -------------------------------------------------------
    def _max_bound(self, local):
        t = self.torch.tensor([float(v) for v in local], dtype=self.torch.float64, device=self._coll_device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        return t.cpu().tolist()

    def _exchange(self):
        """Each side with a neighbour: own outermost rows out, the neighbour's in.
        Sends are issued high side first and receives low side first, so that
        two ranks that are each other's neighbour on both sides (a periodic
        lattice in two slabs) match messages in order even where tags are
        ignored; tags name the sending side."""
        dist = self.dist
        for side in (0, 1):
            if (self.lo, self.hi)[side] is not None:
                self._get(side, self._send[side])
        reqs = []
        if self.hi is not None:
            reqs.append(dist.isend(self._send[1], self.hi, group=self.group, tag=1))
        if self.lo is not None:
            reqs.append(dist.isend(self._send[0], self.lo, group=self.group, tag=0))
        if self.lo is not None:
            reqs.append(dist.irecv(self._recv[0], self.lo, group=self.group, tag=1))
        if self.hi is not None:
            reqs.append(dist.irecv(self._recv[1], self.hi, group=self.group, tag=0))
        for r in reqs:
            r.wait()
        for side in (0, 1):
            if (self.lo, self.hi)[side] is not None:
                self._set(side, self._recv[side])

    def _get(self, side, buf):
        if self.device_buffers:
            self.slab.halo_get(side, buf)
        else:
            self.slab.halo_get(side, buf.numpy())

    def _set(self, side, buf):
        if self.device_buffers:
            self.slab.halo_set(side, buf)
        else:
            self.slab.halo_set(side, buf.numpy())

    # -- the decomposed lattice ---------------------------------------------
    def local_state(self, U):
        """This slab's rows (halo included) of a whole-lattice state U[m][ny][nx]."""
        U = np.asarray(U, dtype=np.float64).reshape((self.pb.nfields, self.pb.ny, self.pb.nx))
        return np.ascontiguousarray(U[:, local_rows(self.pb.ny, self.begin, self.end, self.halo), :])

    def set_state(self, U):
        """f := f^eq(U0) on every slab with alpha^0, lambda^0 from the global
        speed bound of U0 (U: the whole lattice, on every rank)."""
        Ul = self.local_state(U)
        abar = self._max_bound(self.slab.state_speed_bound(Ul))
        self.slab.set_state_bound(Ul, abar)
        self.steps = 0
        return self

    def step(self, n=1):
        for _ in range(int(n)):
            self.slab.set_speed_bound(self._max_bound(self.slab.get_speed_bound()))
            self.slab.step(1)
            self._exchange()
            self.steps += 1
        return self

    def moments(self):
        """U of this slab's own rows, FP64 [m][end - begin][nx]."""
        U = self.slab.moments()
        return U[:, self.halo[0]:U.shape[1] - self.halo[1], :]

    def gather_moments(self):
        """U of the whole lattice on rank 0 (None on the other ranks)."""
        torch, dist = self.torch, self.dist
        mine = torch.from_numpy(np.ascontiguousarray(self.moments()))
        if self.rank != 0:
            dist.send(mine, 0, group=self.group)
            return None
        parts = [mine.numpy()]
        for r in range(1, self.world):
            b, e = self.rows[r]
            buf = torch.empty((self.pb.nfields, e - b, self.pb.nx), dtype=torch.float64)
            dist.recv(buf, r, group=self.group)
            parts.append(buf.numpy())
        return np.concatenate(parts, axis=1)

