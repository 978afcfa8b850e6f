"""Host-side helpers of bench.py that decide what its JSON line reports: the
clock record of the timed region (a throttled run must be recognisable), the
recorded DRAM traffic (valid only for the kernel sources, lattice, size and
precision it was captured on) and the roofline denominator."""
import json

import numpy as np
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class FakeProc:
    def __init__(self, out):
        self.out = out

    def terminate(self):
        pass

    def communicate(self, timeout=None):
        return self.out, ""


def sampler_with(lines):
    s = bench.ClockSampler(0)
    s.proc = FakeProc("\n".join(lines))
    return s.stop()


def test_clock_record_median_max_and_reasons():
    # index, sm MHz, max sm MHz, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    lines = ["0, 2032, 2032, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 1980, 2032, 1090.0, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 2032, 2032, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "garbage line"]
    c = sampler_with(lines)
    assert c["sm_mhz"] == 2032.0 and c["sm_max_mhz"] == 2032.0 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"]


def test_clock_record_flags_thermal_slowdown():
    lines = ["0, 1500, 2032, 1000.0, 0x60, Not Active, Active, Active, Not Active"] * 3
    c = sampler_with(lines)
    assert c["reasons"] == ["hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert c["sm_mhz"] == 1500.0


def test_clock_record_without_samples():
    assert sampler_with([])["reasons"] == ["no samples"]


@pytest.fixture
def fake_root(monkeypatch):
    d = os.path.join(ROOT, "_build", "bench_helpers")  # git-ignored build folder
    shutil.rmtree(d, ignore_errors=True)
    os.makedirs(os.path.join(d, "profiles"))
    monkeypatch.setattr(bench, "ROOT", d)
    yield d
    shutil.rmtree(d, ignore_errors=True)


def test_recorded_traffic_only_for_the_captured_sources_and_case(fake_root):
    assert bench.recorded_traffic("step_fused", "riemann2d", 8192, "fp32") is None  # no file
    entry = {"source_hash": bench.source_hash(), "lattice": "riemann2d", "n": 8192, "precision": "fp32",
             "bytes_per_launch": 1.25e10}
    with open(os.path.join(fake_root, "profiles", "traffic.json"), "w") as fh:
        json.dump({"step_fused": entry}, fh)
    assert bench.recorded_traffic("step_fused", "riemann2d", 8192, "fp32") == 1.25e10
    assert bench.recorded_traffic("step_fused", "riemann2d", 4096, "fp32") is None
    assert bench.recorded_traffic("step_fused", "riemann2d", 8192, "fp64") is None
    assert bench.recorded_traffic("step_fused", "reactive", 8192, "fp32") is None
    assert bench.recorded_traffic("other_kernel", "riemann2d", 8192, "fp32") is None
    entry["source_hash"] = "0" * 16  # the kernels changed since the capture
    with open(os.path.join(fake_root, "profiles", "traffic.json"), "w") as fh:
        json.dump({"step_fused": entry}, fh)
    assert bench.recorded_traffic("step_fused", "riemann2d", 8192, "fp32") is None


def test_measured_peak_or_fallback(fake_root):
    assert bench.measured_peaks() == (6400.0, "fallback")
    with open(os.path.join(fake_root, "MEASURED_PEAKS.json"), "w") as fh:
        json.dump({"hbm_gbs": 6484.6}, fh)
    assert bench.measured_peaks() == (6484.6, "measured")


def test_contract_norm_weighs_momentum_as_a_vector():
    """The accuracy contract's norm: scalar fields by sum|e|/sum|ref|, the
    momentum by sum ||e_m|| / sum ||m|| per node, so a near-zero component is
    measured against the whole momentum."""
    from paper_2609_18177_b300 import accuracy as A
    ref = np.zeros((3, 2, 2))
    ref[0] = 1.0                       # h
    ref[1] = [[3.0, 3.0], [3.0, 3.0]]  # hu
    ref[2] = [[4.0, 0.0], [0.0, 0.0]]  # hv: non-zero at one node only
    got = ref.copy()
    got[0, 0, 0] += 0.04
    got[2, 1, 1] += 1e-3              # 2.5e-4 of sum|hv| alone; 1e-3 / 14 of the momentum
    e = A.contract_l1(got, ref, A.SWE, 2)
    assert e["h"] == pytest.approx(0.04 / 4.0)
    # ||m|| per node: 5, 3, 3, 3 -> 14; the error vector (0, 1e-3) at one node
    assert e["momentum"] == pytest.approx(1e-3 / 14.0)
    assert e["max"] == pytest.approx(0.01)
    # Euler 2D: rho, momentum, E; reactive adds rho*Y
    assert [k for k, _ in A.quantities(A.EULER, 2)] == ["rho", "momentum", "E"]
    assert [k for k, _ in A.quantities(A.REACTIVE, 2)] == ["rho", "momentum", "E", "rhoY"]
    assert A.quantities(A.EULER, 1)[1] == ("momentum", [1])


def test_contract_norm_torch_matches_numpy():
    import torch
    from paper_2609_18177_b300 import accuracy as A
    rng = np.random.default_rng(3)
    ref = rng.uniform(0.5, 2.0, (4, 9, 7))
    got = ref * (1 + 1e-3 * rng.standard_normal(ref.shape))
    a = A.contract_l1(got, ref, A.EULER, 2)
    b = A.contract_l1_torch(torch.from_numpy(got), torch.from_numpy(ref), A.EULER, 2)
    for k in a:
        assert b[k] == pytest.approx(a[k], rel=1e-12)


def test_contract_norm_measures_unburnt_gas_against_the_density():
    """rho*Y of a burnt-out state is ~0: its error is taken relative to the
    density, not to its own vanishing sum."""
    from paper_2609_18177_b300 import accuracy as A
    ref = np.ones((5, 4, 4))
    ref[4] = 1e-300              # burnt: rho*Y decayed towards zero
    got = ref.copy()
    got[4] = 1e-38               # an FP32 run stops at its smallest normal numbers
    e = A.contract_l1(got, ref, A.REACTIVE, 2)
    assert e["rhoY"] == pytest.approx(1e-38)
    assert e["max"] == pytest.approx(1e-38)
