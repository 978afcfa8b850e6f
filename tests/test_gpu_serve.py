"""The continuous-batching server: every request finishes with exactly its
step count, and each result is bitwise the same as the request run alone
(a batch of one), although it shared the device with other requests that
arrived, were admitted (some after waiting for arena space) and left around it.
"""
import numpy as np
import pytest

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
