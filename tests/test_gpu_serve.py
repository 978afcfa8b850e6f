"""The continuous-batching server: every request finishes with exactly its
step count, and each result is bitwise the same as the request run alone
(a batch of one), although it shared the device with other requests that
arrived, were admitted (some after waiting for arena space) and left around it.
"""
import numpy as np
import pytest

import oracle
from paper_2609_18177_b300 import accuracy as A
from paper_2609_18177_b300 import lbmh
from paper_2609_18177_b300 import serve as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    lbmh.load()


def test_served_results_equal_alone_and_queueing_happens():
    # every request arrives at t = 0, so the small arena must defer some of them
    trace = S.poisson_trace(12, rate=0.0, seed=3, n_range=(64, 160), steps_range=(20, 70))
    inputs = {r.rid: S.make_problem(r) for r in trace}
    biggest = max(lbmh.Batch.footprint(pb, lbmh.FP32) for pb, _ in inputs.values())
    srv = S.Server(capacity_bytes=int(2.2 * biggest), max_instances=8, chunk=8, keep_results=True)
    results, stats = srv.run(trace, inputs=inputs, max_seconds=120)
    srv.close()
    assert stats["completed"] == len(trace)
    assert stats["p50_latency_s"] <= stats["p99_latency_s"]
    by_id = {r.rid: r for r in results}
    for req in trace:
        res = by_id[req.rid]
        assert res.steps == req.steps
        pb, U0 = inputs[req.rid]
        assert np.array_equal(res.U, S.run_alone(req, pb, U0)), req
    assert stats["deferred_admissions"] > 0  # some requests queued for arena space


def test_served_fp32_results_of_each_system_meet_the_contract_against_the_oracle():
    """One small request of each system (sizes and step counts like the
    smallest ones of the served trace), served in FP32 together, against the
    FP64 oracle run the same number of steps: the accuracy contract's norm and
    the system's frozen tolerance."""
    trace = [S.Request(rid=0, kind="euler", n=151, steps=314, seed=5, arrival=0.0),
             S.Request(rid=1, kind="swe", n=192, steps=238, seed=6, arrival=0.0),
             S.Request(rid=2, kind="reactive", n=144, steps=210, seed=7, arrival=0.0)]
    inputs = {r.rid: S.make_problem(r) for r in trace}
    cap = 4 * max(lbmh.Batch.footprint(pb, lbmh.FP32) for pb, _ in inputs.values())
    srv = S.Server(capacity_bytes=cap, max_instances=4, chunk=32, keep_results=True)
    results, stats = srv.run(trace, inputs=inputs, max_seconds=300)
    srv.close()
    assert stats["completed"] == len(trace)
    for res in results:
        pb, U0 = inputs[res.rid]
        ref = oracle.Run(pb, U0).step(res.steps).moments()
        err = A.contract_l1(res.U, ref, pb.system, pb.dim)
        assert err["max"] <= A.tolerance(pb.system), (res.kind, err)
