"""Batches (many lattices of uneven sizes, one persistent launch per step)
against the same lattices run alone, against the single-lattice path and
against the FP64 oracle.

Every node of a batched lattice goes through the same arithmetic whatever the
work split and whatever else shares the batch, so a lattice's result is
bitwise the same alone (a batch of one) and in any mix, including lattices
admitted or removed around it.  Against the single-lattice fused kernel (a
separately compiled kernel, whose FMA contractions may differ) the bar is the
precision's rounding level.
"""
import numpy as np
import pytest

import oracle
from paper_2609_18177_b300 import lbmh
from paper_2609_18177_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    lbmh.load()


def alone(pb, U0, nsteps, precision):
    """The lattice in a batch of its own."""
    b = lbmh.Batch(pb.system, precision=precision, capacity_bytes=2 * lbmh.Batch.footprint(pb, precision) + (1 << 20),
                   max_instances=1)
    slot = b.add(pb, U0)
    b.step(nsteps)
    U = b.moments(slot)
    b.close()
    return U


def single(pb, U0, nsteps, precision):
    """The lattice through the single-lattice handle (fused kernel)."""
    s = lbmh.Solver(pb, precision=precision, kernel=lbmh.KERNEL_FUSED).set_state(U0).step(nsteps)
    U = s.moments()
    s.close()
    return U


def rel_max(a, b):
    scale = np.abs(b).reshape(b.shape[0], -1).max(axis=1)
    return (np.abs(a - b).reshape(b.shape[0], -1).max(axis=1) / np.where(scale > 0, scale, 1.0)).max()


def rel_l1(a, b):
    scale = np.abs(b).reshape(b.shape[0], -1).sum(axis=1)
    return (np.abs(a - b).reshape(b.shape[0], -1).sum(axis=1) / np.where(scale > 0, scale, 1.0)).max()


def close_at_rounding_level(a, b, precision):
    """The FP32 bar of the oracle parity tests (relative L1 <= 2e-5 and relative
    max <= 5e-4 per field: near-dry cells switch between the wet and the dry
    branch on a last-bit difference of h); FP64: relative max <= 1e-12."""
    if precision == lbmh.FP32:
        return rel_l1(a, b) <= 2e-5 and rel_max(a, b) <= 5e-4
    return rel_max(a, b) <= 1e-12


def swe_mix():
    out = []
    for n in (64, 100, 130, 257, 75):
        out.append(W.dam_break_bump(n))
    return out


@pytest.mark.parametrize("precision", [lbmh.FP32, lbmh.FP64], ids=["fp32", "fp64"])
def test_batch_equals_alone_bitwise(precision):
    b = lbmh.Batch(W.SWE, precision=precision, capacity_bytes=1 << 28, max_instances=16)
    cases = swe_mix()
    slots = [b.add(pb, U0) for pb, U0 in cases]
    assert all(s is not None for s in slots)
    b.step(10)
    for (pb, U0), slot in zip(cases, slots):
        Ub = b.moments(slot)
        Ua = alone(pb, U0, 10, precision)
        assert np.array_equal(Ub, Ua), (pb.nx, np.abs(Ub - Ua).max())
        Us = single(pb, U0, 10, precision)
        assert close_at_rounding_level(Ub, Us, precision), (pb.nx, rel_l1(Ub, Us), rel_max(Ub, Us))
    b.close()


def test_batch_fp64_matches_oracle():
    b = lbmh.Batch(W.EULER, precision=lbmh.FP64, capacity_bytes=1 << 27, max_instances=8)
    cases = [W.riemann_2d_seeded(n, seed=s) for n, s in ((48, 1), (131, 2), (70, 3))]
    slots = [b.add(pb, U0) for pb, U0 in cases]
    b.step(8)
    for (pb, U0), slot in zip(cases, slots):
        r = oracle.Run(pb, U0).step(8)
        Uo = r.moments()
        Ub = b.moments(slot)
        scale = np.abs(Uo).reshape(pb.nfields, -1).max(axis=1)
        err = np.abs(Ub - Uo).reshape(pb.nfields, -1).max(axis=1) / scale
        assert np.all(err <= 1e-12), err
    b.close()


def test_fp32_batched_dam_break_to_T_meets_the_contract_against_the_oracle():
    """The batched workload's smallest sampled lattice (n = 274, seed 0 of the
    256-lattice recipe) in an FP32 batch beside two other dam breaks, to
    T = 0.1 (271 steps), against the FP64 oracle run as many steps: the
    accuracy contract's norm within the shallow-water tolerance."""
    from paper_2609_18177_b300 import accuracy as A
    cases = [W.dam_break_bump(n) for n in (274, 97, 160)]
    cap = sum(lbmh.Batch.footprint(pb, lbmh.FP32) for pb, _ in cases) + (8 << 20)
    b = lbmh.Batch(W.SWE, precision=lbmh.FP32, capacity_bytes=cap, max_instances=4)
    slots = [b.add(pb.with_(precision=lbmh.FP32), U0, T=0.1) for pb, U0 in cases]
    while True:
        b.step(30)
        done, t, steps, status = b.poll()
        if all(done[s] == 1 for s in slots):
            break
    pb, U0 = cases[0]
    nsteps = int(steps[slots[0]])
    assert 260 <= nsteps <= 280 and t[slots[0]] >= 0.1, (nsteps, t[slots[0]])
    r = oracle.Run(pb, U0).step(nsteps)  # the same number of steps (dt from each path's own speed bound)
    err = A.contract_l1(b.moments(slots[0]), r.moments(), pb.system, pb.dim)
    assert err["max"] <= A.tolerance(W.SWE), err
    b.close()


def test_step_targets_end_times_and_poll():
    b = lbmh.Batch(W.EULER, precision=lbmh.FP32, capacity_bytes=1 << 27, max_instances=8)
    pb, U0 = W.riemann_2d_seeded(80, seed=4)
    s5 = b.add(pb, U0, max_steps=5)
    s12 = b.add(pb, U0, max_steps=12)
    sT = b.add(pb, U0, T=0.01)
    b.step(20)
    done, t, steps, status = b.poll()
    assert steps[s5] == 5 and steps[s12] == 12 and done[s5] == 1 and done[s12] == 1
    assert done[sT] == 1 and t[sT] >= 0.01
    assert np.array_equal(b.moments(s5), alone(pb, U0, 5, lbmh.FP32))
    assert np.array_equal(b.moments(s12), alone(pb, U0, 12, lbmh.FP32))
    b.close()


def test_admission_by_footprint_and_reuse_of_freed_space():
    pb, U0 = W.riemann_2d_seeded(100, seed=5)
    fp = lbmh.Batch.footprint(pb, lbmh.FP32)
    assert fp > 0
    b = lbmh.Batch(W.EULER, precision=lbmh.FP32, capacity_bytes=int(2.5 * fp), max_instances=8)
    a1 = b.add(pb, U0)
    a2 = b.add(pb, U0)
    assert a1 is not None and a2 is not None
    assert b.add(pb, U0) is None  # the arena is full: admission refused
    assert b.info()["active"] == 2
    b.step(3)
    b.remove(a1)
    a3 = b.add(pb, U0)  # admitted into the freed space, mid-run of a2
    assert a3 is not None
    b.step(4)
    done, t, steps, status = b.poll()
    assert steps[a2] == 7 and steps[a3] == 4
    assert np.array_equal(b.moments(a3), alone(pb, U0, 4, lbmh.FP32))
    assert np.array_equal(b.moments(a2), alone(pb, U0, 7, lbmh.FP32))
    b.close()


def test_autotune_keeps_results_and_graph_replay():
    b = lbmh.Batch(W.REACTIVE, precision=lbmh.FP32, capacity_bytes=1 << 28, max_instances=8)
    cases = [W.reactive_circle(n) for n in (64, 150, 97)]
    slots = [b.add(pb, U0) for pb, U0 in cases]
    ms = b.autotune(steps_per_candidate=2)  # 8 candidates x (1 + 2) real steps
    assert ms > 0
    b.step(7)  # graph replay for 6 steps plus single launches
    done, t, steps, status = b.poll()
    for (pb, U0), slot in zip(cases, slots):
        assert steps[slot] == 31
        # the tuner may pick another ring depth (another kernel binary) than the
        # batch of one uses: compare at FP32 rounding level
        assert rel_max(b.moments(slot), alone(pb, U0, 31, lbmh.FP32)) <= 1e-4
    b.close()
