"""Failure detection on the GPU without a GPU fault.

Every device-side wait of the row pipeline is bounded.  A test hook
(LBMH_TEST_FIRST_WAIT_POLLS, read when a handle is created) sets the number of
polls of each CTA's first row-load wait; at 0 that wait gives up at once, as a
wait on a load that never lands would after its limit.  The CTA then stops
consuming, waits for the loads it has in flight with the full limit (so no
bulk copy is left pending when it exits) and sets the timeout bit, which the
host reads as LBMH_ERR_TIMEOUT.  Nothing hangs or faults, and the device stays
usable: a normal handle created next matches the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2609_18177_b300 import lbmh
from paper_2609_18177_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [lbmh.FP32, lbmh.FP64], ids=["fp32", "fp64"])
def test_a_row_wait_that_runs_out_reports_timeout_and_the_device_stays_usable(prec, monkeypatch):
    pb, U0 = W.riemann_2d_seeded(200, seed=4, cfl=0.9)
    monkeypatch.setenv("LBMH_TEST_FIRST_WAIT_POLLS", "0")
    s = lbmh.Solver(pb, precision=prec, kernel=lbmh.KERNEL_FUSED)
    monkeypatch.delenv("LBMH_TEST_FIRST_WAIT_POLLS")
    s.set_state(U0).step(3)
    with pytest.raises(lbmh.LbmhError) as ei:
        s.moments()
    assert ei.value.code == lbmh.ERR_TIMEOUT
    assert s.info()["status"] & 4  # the timeout bit is sticky
    s.close()
    # the same device, a handle created without the hook: the step is correct
    ref = oracle.Run(pb, U0).step(5).moments()
    with lbmh.Solver(pb, precision=lbmh.FP64, kernel=lbmh.KERNEL_FUSED) as s2:
        U = s2.set_state(U0).step(5).moments()
        assert s2.info()["status"] == 0
    scale = np.abs(ref).reshape(pb.nfields, -1).max(axis=1)
    err = np.abs(U - ref).reshape(pb.nfields, -1).max(axis=1) / scale
    assert np.all(err <= 1e-12), err


def test_batch_with_a_row_wait_that_runs_out_marks_its_lattices(monkeypatch):
    """The batch kernel shares the row pipeline: a lattice whose first row wait
    gives up is reported finished with the timeout bit, and the batch's other
    calls keep working."""
    pb, U0 = W.dam_break_bump(96)
    pb = pb.with_(precision=lbmh.FP32)
    cap = 2 * lbmh.Batch.footprint(pb, lbmh.FP32) + (8 << 20)
    monkeypatch.setenv("LBMH_TEST_FIRST_WAIT_POLLS", "0")
    b = lbmh.Batch(W.SWE, precision=lbmh.FP32, capacity_bytes=cap, max_instances=2)
    slot = b.add(pb, U0, max_steps=10)
    monkeypatch.delenv("LBMH_TEST_FIRST_WAIT_POLLS")
    b.step(4)
    done, t, steps, status = b.poll()
    b.close()
    assert status[slot] & 4, status[slot]
    assert done[slot] == 1
