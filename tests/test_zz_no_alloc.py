"""The allocation-free step (lbmh_step_static).

lbmh_step_static serves callers that cannot allocate device memory (host
callbacks and graph nodes where cudaMalloc is illegal, frozen memory pools,
real-time loops): it runs the unfused FP64 step with all of its scratch in the
library's static device array.  Two calls in a row must reproduce two steps of
a handle that runs the same kernels with scratch from cudaMalloc, and two
steps of the FP64 oracle; the caller's arrays may sit anywhere inside a larger
allocation, and nothing outside them may be read or written.  This file is
collected last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

import oracle
from paper_2609_18177_b300 import lbmh
from paper_2609_18177_b300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12
GUARD = 4099  # doubles of sentinel before, between and after the caller's arrays


def rel_err(a, b):
    scale = np.abs(b).max()
    return np.abs(a - b).max() / (scale if scale > 0 else 1.0)


def field_rel_err(a, b, m):
    """max abs difference over max abs value, per conserved field (the parity norm)."""
    a = np.moveaxis(a, 1, 0).reshape(m, -1)
    b = np.moveaxis(b, 1, 0).reshape(m, -1)
    scale = np.abs(b).max(axis=1)
    return np.abs(a - b).max(axis=1) / np.where(scale > 0, scale, 1.0)


CASES = [(W.EULER, 2, W.OUTFLOW), (W.SWE, 2, W.PERIODIC), (W.REACTIVE, 1, W.OUTFLOW), (W.ADVECTION, 2, W.PERIODIC)]


def make_case(system, dim, bc):
    nx, ny = (67, 29) if dim == 2 else (301, 1)
    kw = dict(dim=dim, nx=nx, ny=ny, y1=ny / nx if dim == 2 else 1.0, bc=(bc,) * 4, cfl=0.8)
    extra = {W.SWE: dict(bed_amp=0.3, bed_w2=0.05, bed_xc=0.4, bed_yc=0.2),
             W.REACTIVE: dict(gamma=1.2, q=5.0, K=40.0, Ti=2.0),
             W.ADVECTION: dict(adv=(0.8, -0.45))}.get(system, {})
    pb = W.Problem(system=system, **kw, **extra)
    return pb, W.random_state(pb, seed=9)


@pytest.mark.parametrize("system,dim,bc", CASES)
def test_static_step_matches_handle_and_oracle_two_calls(system, dim, bc):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    pb, U0 = make_case(system, dim, bc)
    ref = lbmh.Solver(pb, precision=lbmh.FP64, kernel=lbmh.KERNEL_UNFUSED).set_state(U0)
    f0 = ref.get_f()
    orc = oracle.Run(pb, U0)
    orc.f[...] = f0.reshape(orc.f.shape)
    # the caller's two arrays inside one larger allocation, fenced by NaN sentinels
    n = f0.size
    arena = torch.full((3 * GUARD + 2 * n,), float("nan"), dtype=torch.float64, device="cuda")
    fa = arena[GUARD:GUARD + n].view(f0.shape)
    fb = arena[2 * GUARD + n:2 * GUARD + 2 * n].view(f0.shape)
    fa.copy_(torch.from_numpy(f0))
    for call in range(2):  # two calls in a row, ping-ponging the caller's arrays
        src, dst = (fa, fb) if call == 0 else (fb, fa)
        dt, status = lbmh.step_static(pb, src, dst, want_status=True)
        assert status & 1 == 0
        ref.step(1)
        orc.step(1)
        got = dst.cpu().numpy()
        assert rel_err(got, ref.get_f()) <= TOL, (call, rel_err(got, ref.get_f()))
        err = field_rel_err(got, orc.f.reshape(got.shape), pb.nfields)
        assert np.all(err <= TOL), (call, err)
        assert dt == pytest.approx(ref.info()["last_dt"], rel=1e-14)
        assert dt == pytest.approx(orc.info[2], rel=1e-13)
    guards = torch.cat([arena[:GUARD], arena[GUARD + n:2 * GUARD + n], arena[2 * GUARD + 2 * n:]])
    assert bool(torch.isnan(guards).all()), "the static step wrote outside the caller's arrays"
    ref.close()


def test_static_step_reports_status_bits():
    """A state that the step makes non-physical fails the call; the status bits
    are those of the handle path."""
    import torch
    pb, U0 = make_case(W.EULER, 2, W.OUTFLOW)
    ref = lbmh.Solver(pb, precision=lbmh.FP64, kernel=lbmh.KERNEL_UNFUSED).set_state(U0)
    f0 = torch.from_numpy(ref.get_f()).cuda()
    f0[0, 0, 5, 7] = -50.0  # negative density at one node
    out = torch.empty_like(f0)
    with pytest.raises(lbmh.LbmhError) as ei:
        lbmh.step_static(pb, f0, out, want_status=True)
    assert ei.value.code == lbmh.ERR_NONPHYSICAL
    ref.close()


def test_static_step_rejects_grids_beyond_the_static_scratch():
    import torch
    pb = W.Problem(system=W.EULER, dim=2, nx=1024, ny=1024)
    f = torch.zeros((5, 4, 1024, 1024), dtype=torch.float64, device="cuda")
    g = torch.empty_like(f)
    with pytest.raises(lbmh.LbmhError) as ei:
        lbmh.step_static(pb, f, g)
    assert ei.value.code == lbmh.ERR_INVALID_ARG
    assert "static scratch" in str(ei.value)
