"""The allocation-free step (lbmh_step_static) against the regular handle path.

lbmh_step_static serves callers that cannot allocate device memory: it runs
the unfused step with all of its scratch in the library's static device
array.  Two calls in a row must reproduce two steps of a handle that runs the
same (unfused, FP64) kernels with scratch from cudaMalloc.  This file is
collected last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

from paper_2609_18177_b300 import lbmh
from paper_2609_18177_b300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12


def rel_err(a, b):
    scale = np.abs(b).max()
    return np.abs(a - b).max() / (scale if scale > 0 else 1.0)


@pytest.mark.parametrize("system,dim,bc", [
    (W.EULER, 2, W.OUTFLOW), (W.SWE, 2, W.PERIODIC), (W.REACTIVE, 1, W.OUTFLOW), (W.ADVECTION, 2, W.PERIODIC),
])
def test_static_step_matches_handle_two_calls(system, dim, bc):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    nx, ny = (67, 29) if dim == 2 else (301, 1)
    kw = dict(dim=dim, nx=nx, ny=ny, y1=ny / nx if dim == 2 else 1.0, bc=(bc,) * 4, cfl=0.8)
    extra = {W.SWE: dict(bed_amp=0.3, bed_w2=0.05, bed_xc=0.4, bed_yc=0.2),
             W.REACTIVE: dict(gamma=1.2, q=5.0, K=40.0, Ti=2.0),
             W.ADVECTION: dict(adv=(0.8, -0.45))}.get(system, {})
    pb = W.Problem(system=system, **kw, **extra)
    U0 = W.random_state(pb, seed=9)
    ref = lbmh.Solver(pb, precision=lbmh.FP64, kernel=lbmh.KERNEL_UNFUSED).set_state(U0)
    f0 = ref.get_f()
    fa = torch.from_numpy(f0).cuda()
    fb = torch.empty_like(fa)
    for call in range(2):  # two calls in a row, ping-ponging the caller's arrays
        src, dst = (fa, fb) if call == 0 else (fb, fa)
        dt = lbmh.step_static(pb, src, dst)
        ref.step(1)
        expect = ref.get_f()
        assert rel_err(dst.cpu().numpy(), expect) <= TOL, (call, rel_err(dst.cpu().numpy(), expect))
        assert dt == pytest.approx(ref.info()["last_dt"], rel=1e-14)
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
