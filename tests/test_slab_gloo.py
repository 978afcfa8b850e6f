"""Slab decomposition of one 2D lattice along y (paper_2609_18177_b300.slab),
checked on CPU ranks: gloo process groups of two and three ranks run the
orchestration of the decomposed step (global maximum of the speed bound of
Eq. 2.19, one step per slab, exchange of three halo rows) with every slab held
by the FP64 oracle, and the gathered rows must equal the oracle stepping the
whole lattice.

Systems without position-dependent terms (Euler, reactive Euler) must agree
bit for bit: every node sees the same f^n, the same speed bound and the same
arithmetic.  With the bed source the oracle's slab computes node positions
from its own local origin, which may round differently in the last bit, so
shallow water is held to 1e-13.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2609_18177_b300 import slab as S
from paper_2609_18177_b300 import workloads as W


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleSlab:
    """A slab held by the oracle, with the interface of lbmh.Slab."""

    def __init__(self, pb, begin, end, precision=None):
        import oracle
        self.oracle = oracle
        whole = begin == 0 and end == pb.ny
        periodic = pb.bc[2] == W.PERIODIC
        self.halo = (3 if not whole and (begin > 0 or periodic) else 0,
                     3 if not whole and (end < pb.ny or periodic) else 0)
        self.row0 = begin - self.halo[0]
        nyl = end - begin + self.halo[0] + self.halo[1]
        bc = list(pb.bc)
        if self.halo[0]:
            bc[2] = W.OUTFLOW  # the rows beyond a halo are never needed
        if self.halo[1]:
            bc[3] = W.OUTFLOW
        dy = pb.dx
        self.pb = pb.with_(ny=nyl, y0=pb.y0 + self.row0 * dy, y1=pb.y0 + (self.row0 + nyl) * dy, bc=tuple(bc))
        self.nyl = nyl
        self.halo_bytes = pb.nvel * pb.nfields * 3 * pb.nx * 8
        self.run = None
        self.abar = None

    def state_speed_bound(self, U):
        return list(self.oracle.alpha_bar(self.pb, U)[:2])

    def set_state_bound(self, U, abar):
        """f := f^eq(U) with alpha, lambda from abar, as the oracle's own
        initialisation forms them (Eqs. 2.20, 2.21)."""
        pb = self.pb
        U = np.asarray(U, dtype=np.float64).reshape((pb.nfields, self.nyl, pb.nx))
        self.run = self.oracle.Run(pb, U)
        dt = pb.cfl * pb.dx / (abar[0] + abar[1])
        lam = pb.dx / dt
        alpha = [abar[0] + pb.eps, abar[1] + pb.eps]
        f = self.run.f
        for j in range(self.nyl):
            for i in range(pb.nx):
                f[:, :, j, i] = self.oracle.equilibrium(pb, U[:, j, i], alpha, lam)

    def get_speed_bound(self):
        U = np.ascontiguousarray(self.moments()[:, self.halo[0]:self.nyl - self.halo[1], :])
        w = U.shape[1]
        return list(self.oracle.alpha_bar(self.pb.with_(ny=w, y1=self.pb.y0 + w * self.pb.dx), U)[:2])

    def set_speed_bound(self, abar):
        self.abar = list(abar)

    def step(self, n=1):
        self.run.step(n, abar=self.abar + [0.0])

    def _rows(self, out):
        return out.view(np.float64).reshape((self.pb.nvel * self.pb.nfields, 3, self.pb.nx))

    def halo_get(self, side, out):
        r = self.halo[0] if side == 0 else self.nyl - self.halo[1] - 3
        f = self.run.f.reshape((-1, self.nyl, self.pb.nx))
        self._rows(out)[...] = f[:, r:r + 3, :]

    def halo_set(self, side, rows):
        r = 0 if side == 0 else self.nyl - 3
        f = self.run.f.reshape((-1, self.nyl, self.pb.nx))
        f[:, r:r + 3, :] = self._rows(rows)

    def moments(self):
        return self.run.moments()


CASES = {
    "riemann_outflow": lambda: W.riemann_2d_seeded(40, seed=3, cfl=0.9),
    "euler_periodic": lambda: (lambda pb: (pb, W.random_state(pb, seed=5)))(
        W.Problem(system=W.EULER, dim=2, nx=24, ny=30, y1=30 / 24, cfl=0.8)),
    "reactive_reflect": lambda: (lambda pb: (pb, W.random_state(pb, seed=6)))(
        W.Problem(system=W.REACTIVE, dim=2, nx=20, ny=27, y1=27 / 20, cfl=0.7, gamma=1.2, q=5.0, K=40.0, Ti=2.0,
                  bc=(W.OUTFLOW, W.OUTFLOW, W.REFLECT, W.REFLECT))),
    "swe_bed_outflow": lambda: (lambda pb: (pb, W.random_state(pb, seed=7)))(
        W.Problem(system=W.SWE, dim=2, nx=22, ny=26, y1=26 / 22, cfl=0.6, bc=(W.OUTFLOW,) * 4,
                  bed_amp=0.3, bed_w2=0.05, bed_xc=0.4, bed_yc=0.6)),
}
STEPS = 8


def _rank(rank, world, port, case, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.join(root, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    from paper_2609_18177_b300 import slab as S2
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pb, U0 = CASES[case]()
    run = S2.SlabRun(pb, rank, world, backend=lambda p, b, e, prec: OracleSlab(p, b, e, prec))
    run.set_state(U0).step(STEPS)
    U = run.gather_moments()
    if rank == 0:
        out["U"] = U
    dist.barrier()
    dist.destroy_process_group()


def _decomposed(case, world):
    with mp.get_context("spawn").Manager() as mgr:  # no fork of this multi-threaded process
        out = mgr.dict()
        mp.spawn(_rank, args=(world, _free_port(), case, out), nprocs=world, join=True)
        return out["U"]


@pytest.mark.parametrize("case,world", [("riemann_outflow", 2), ("euler_periodic", 2), ("euler_periodic", 3),
                                        ("reactive_reflect", 3), ("swe_bed_outflow", 2)])
def test_slabs_equal_the_whole_lattice(case, world):
    import oracle
    pb, U0 = CASES[case]()
    whole = oracle.Run(pb, U0).step(STEPS).moments()
    got = _decomposed(case, world)
    assert got.shape == whole.shape
    if pb.system == W.SWE:
        scale = np.abs(whole).reshape(pb.nfields, -1).max(axis=1)
        err = np.abs(got - whole).reshape(pb.nfields, -1).max(axis=1) / scale
        assert np.all(err <= 1e-13), err
    else:
        assert np.array_equal(got, whole), np.abs(got - whole).max()


def test_partition_and_neighbours():
    assert S.partition_rows(10, 3) == [(0, 3), (3, 6), (6, 10)]
    with pytest.raises(ValueError):
        S.partition_rows(8, 3)  # a slab of fewer than three rows
    assert S.neighbours(0, 3, periodic=False) == (None, 1)
    assert S.neighbours(2, 3, periodic=False) == (1, None)
    assert S.neighbours(0, 3, periodic=True) == (2, 1)
    assert S.neighbours(0, 2, periodic=True) == (1, 1)
    assert S.neighbours(0, 1, periodic=True) == (None, None)
    assert list(S.local_rows(10, 0, 3, (3, 3))) == [7, 8, 9, 0, 1, 2, 3, 4, 5]


def test_oracle_slab_halo_geometry():
    pb, _ = CASES["euler_periodic"]()
    a = OracleSlab(pb, 0, 15)
    assert a.halo == (3, 3) and a.row0 == -3 and a.nyl == 21
    b = OracleSlab(pb.with_(bc=(W.OUTFLOW,) * 4), 0, 15)
    assert b.halo == (0, 3) and b.row0 == 0
