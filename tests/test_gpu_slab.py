"""Slabs of a 2D lattice decomposed along y, on the GPU (lbmh_create_slab and
the speed-bound and halo entry points).

(1) In one process: the slabs of a lattice are held side by side on cuda:0
and the host plays the ranks in turn (maximum of the speed bounds, one step of
each slab, each slab's outermost rows copied into the neighbour's halo through
device buffers).  No kernel waits on another.  The rows of the slabs must equal
the single lattice stepped by the same fused kernel bit for bit, in FP32 and
FP64, for every system and boundary kind, on lattices wider than one strip.
(2) Two processes on cuda:0, gloo between them, run the orchestration module
(paper_2609_18177_b300.slab) with host-staged halos: the same bits again.
"""
import os
import socket

import numpy as np
import pytest

from paper_2609_18177_b300 import lbmh
from paper_2609_18177_b300 import slab as S
from paper_2609_18177_b300 import workloads as W

pytestmark = pytest.mark.gpu
STEPS = 9


def _problem(name):
    if name == "riemann_outflow":
        return W.riemann_2d_seeded(130, seed=3, cfl=0.9)
    if name == "euler_periodic":
        pb = W.Problem(system=W.EULER, dim=2, nx=250, ny=61, y1=61 / 250, cfl=0.8)
        return pb, W.random_state(pb, seed=5)
    if name == "swe_bed_outflow":
        pb = W.Problem(system=W.SWE, dim=2, nx=131, ny=47, y1=47 / 131, cfl=0.6, bc=(W.OUTFLOW,) * 4,
                       bed_amp=0.3, bed_w2=0.05, bed_xc=0.4, bed_yc=0.2)
        return pb, W.random_state(pb, seed=7)
    if name == "reactive_reflect_inflow_sponge":
        pb = W.Problem(system=W.REACTIVE, dim=2, nx=140, ny=40, y1=40 / 140, cfl=0.7, gamma=1.2, q=5.0, K=40.0,
                       Ti=2.0, bc=(W.OUTFLOW, W.INFLOW, W.REFLECT, W.REFLECT), sponge_width=0.1,
                       u_in=(1.0, -0.5, 0.0, 8.0, 1.0))
        return pb, W.random_state(pb, seed=6)
    if name == "dam_break_bump":
        return W.dam_break_bump(96)
    raise KeyError(name)


NAMES = ["riemann_outflow", "euler_periodic", "swe_bed_outflow", "reactive_reflect_inflow_sponge", "dam_break_bump"]


def _whole(pb, U0, prec, steps):
    with lbmh.Solver(pb, precision=prec, kernel=lbmh.KERNEL_FUSED) as s:
        s.set_state(U0).step(steps)
        return s.moments(), s.info()


def _in_process(pb, U0, prec, world, steps):
    import torch
    rows = S.partition_rows(pb.ny, world)
    slabs = [lbmh.Slab(pb, b, e, precision=prec) for (b, e) in rows]
    periodic = pb.bc[2] == W.PERIODIC
    nbr = [S.neighbours(r, world, periodic) for r in range(world)]
    local = [np.ascontiguousarray(U0.reshape(pb.nfields, pb.ny, pb.nx)[:, S.local_rows(pb.ny, b, e, s.halo), :])
             for (b, e), s in zip(rows, slabs)]
    abar0 = np.max([s.state_speed_bound(u) for s, u in zip(slabs, local)], axis=0)
    for s, u in zip(slabs, local):
        s.set_state_bound(u, abar0)
    bufs = [[torch.empty(s.halo_bytes, dtype=torch.uint8, device="cuda") for _ in range(2)] for s in slabs]
    for _ in range(steps):
        ab = np.max([s.get_speed_bound() for s in slabs], axis=0)
        for s in slabs:
            s.set_speed_bound(ab).step(1)
        for r, s in enumerate(slabs):
            for side in (0, 1):
                if nbr[r][side] is not None:
                    s.halo_get(side, bufs[r][side])
        for r, s in enumerate(slabs):
            lo, hi = nbr[r]
            if lo is not None:
                s.halo_set(0, bufs[lo][1])
            if hi is not None:
                s.halo_set(1, bufs[hi][0])
    parts, infos = [], []
    for s in slabs:
        U = s.moments()
        parts.append(U[:, s.halo[0]:U.shape[1] - s.halo[1], :])
        infos.append(s.info())
        s.close()
    return np.concatenate(parts, axis=1), infos


@pytest.mark.parametrize("prec", [lbmh.FP32, lbmh.FP64], ids=["fp32", "fp64"])
@pytest.mark.parametrize("name", NAMES)
def test_slabs_hold_the_bits_of_the_whole_lattice(name, prec):
    pb, U0 = _problem(name)
    want, winfo = _whole(pb, U0, prec, STEPS)
    world = 3 if pb.ny >= 45 else 2
    got, infos = _in_process(pb, U0, prec, world, STEPS)
    assert got.shape == want.shape
    assert np.array_equal(got, want), np.abs(got - want).max()
    for inf in infos:  # every slab took the same steps with the same dt
        assert inf["steps"] == STEPS and inf["t"] == winfo["t"] and inf["last_dt"] == winfo["last_dt"]
    # the FP64 sums of the slabs' own rows add up to the whole lattice's
    tot = np.sum([inf["sum_U"] for inf in infos], axis=0)
    assert np.allclose(tot, winfo["sum_U"], rtol=1e-12, atol=1e-12 * np.abs(winfo["sum_U"]).max())


def test_slab_arguments():
    pb, U0 = _problem("riemann_outflow")
    with pytest.raises(lbmh.LbmhError):
        lbmh.Slab(pb, 10, 12)  # fewer than three rows
    with pytest.raises(lbmh.LbmhError):
        lbmh.Slab(pb, 0, pb.ny + 1)
    s = lbmh.Slab(pb, 0, 40)
    assert s.halo == (0, 3) and s.row0 == 0
    import torch
    buf = torch.empty(s.halo_bytes, dtype=torch.uint8, device="cuda")
    s.set_state_bound(np.ascontiguousarray(U0.reshape(pb.nfields, pb.ny, pb.nx)[:, :43]), [3.0, 3.0])
    with pytest.raises(lbmh.LbmhError):
        s.halo_get(0, buf)  # no neighbour below the first slab
    s.halo_get(1, buf)
    s.close()


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank(rank, world, port, name, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    from paper_2609_18177_b300 import slab as S2
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pb, U0 = _problem(name)
    run = S2.SlabRun(pb, rank, world, precision=lbmh.FP32)
    run.set_state(U0).step(STEPS)
    U = run.gather_moments()
    if rank == 0:
        out["U"] = U
    run.slab.close()
    dist.barrier()
    dist.destroy_process_group()


def test_two_processes_on_one_gpu_with_gloo():
    import torch.multiprocessing as mp
    name = "euler_periodic"
    pb, U0 = _problem(name)
    want, _ = _whole(pb, U0, lbmh.FP32, STEPS)
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(2, _free_port(), name, out), nprocs=2, join=True)
        got = out["U"]
    assert np.array_equal(got, want), np.abs(got - want).max()
