"""FP64 parity of the CUDA path with the oracle where the workloads are large
or long (the accuracy contract of the batched and roofline runs).

(1) The shallow-water dam break over a bump (the batched workload, n = 274):
within the horizon over which one ulp of input stays at rounding level in the
oracle itself (5 steps, tests/test_oracle_sensitivity.py) the FP64 GPU path
matches the oracle to 1e-12; after 20 steps it is no further from the oracle
than the oracle is from itself under a one-ulp input change (times 10).

(2) Windows of a large lattice of the seeded 2D Riemann workload: the GPU's
distributions before and after one step are cut into 64 x 64 windows plus the
three-node halo the update reads; the oracle steps each window with the GPU's
global speed bound (Eq. 2.19: the only quantity of a step that is not local),
and the window's interior must match the GPU's result -- at the first step and
after hundreds of steps, when shocks and contacts cross the lattice.  FP64 at
4096 x 4096 to 1e-12; FP32 at 8192 x 8192, the roofline run's size and kernel
instance, to one FP32 step's rounding.
"""
import numpy as np
import pytest

import oracle
from paper_2609_18177_b300 import lbmh
from paper_2609_18177_b300 import workloads as W
from test_oracle_sensitivity import HORIZON, STEPS, parity_spread, spread_history

pytestmark = pytest.mark.gpu


def test_fp64_dam_break_stays_within_the_schemes_own_rounding_spread():
    pb, U0 = W.dam_break_bump(274)
    orc = oracle.Run(pb, U0)
    with lbmh.Solver(pb, precision=lbmh.FP64, kernel=lbmh.KERNEL_FUSED) as s:
        s.set_state(U0)
        for k in range(1, STEPS + 1):
            s.step(1)
            orc.step(1)
            if k == HORIZON:
                h, m = parity_spread(orc.moments(), s.moments())
                assert h <= 1e-12 and m <= 1e-12, (h, m)
        h, m = parity_spread(orc.moments(), s.moments())
    own = spread_history()[0][-1]
    assert h <= 10 * own[0] and m <= 10 * own[1], ((h, m), own)


def window_problem(pb, i0, i1, j0, j1):
    """The lattice's columns [i0, i1) x rows [j0, j1) as a problem of its own
    (same mesh; sides inside the lattice become outflow: the nodes they affect
    lie in the halo, whose results are discarded)."""
    dx = pb.dx
    bc = (pb.bc[0] if i0 == 0 else W.OUTFLOW, pb.bc[1] if i1 == pb.nx else W.OUTFLOW,
          pb.bc[2] if j0 == 0 else W.OUTFLOW, pb.bc[3] if j1 == pb.ny else W.OUTFLOW)
    return pb.with_(nx=i1 - i0, ny=j1 - j0, x0=pb.x0 + i0 * dx, x1=pb.x0 + i1 * dx,
                    y0=pb.y0 + j0 * dx, y1=pb.y0 + j1 * dx, bc=bc)


def window_err(pb, fb, fa, abar, a0, b0, size=64):
    """Step the window [a0, a0+size) x [b0, b0+size) with the oracle from the
    GPU's distributions before the step (fb: the window plus its halo, cut at
    the lattice's edges) and compare its interior with the GPU's after the step
    (fa): per field, max |difference| / max |oracle| over velocities and nodes."""
    i0, i1 = max(0, a0 - 3), min(pb.nx, a0 + size + 3)
    j0, j1 = max(0, b0 - 3), min(pb.ny, b0 + size + 3)
    wp = window_problem(pb, i0, i1, j0, j1)
    r = oracle.Run(wp, np.ones((pb.nfields, j1 - j0, i1 - i0)))
    r.f[...] = fb
    r.step(1, abar=list(abar) + [0.0])
    o = r.f[:, :, b0 - j0:b0 - j0 + size, a0 - i0:a0 - i0 + size]
    o2 = np.moveaxis(o, 1, 0).reshape(pb.nfields, -1)
    g2 = np.moveaxis(fa, 1, 0).reshape(pb.nfields, -1)
    return np.abs(g2 - o2).max(axis=1) / np.abs(o2).max(axis=1)


# (n, precision, steps before the second check, bound): FP64 at half the
# roofline size; FP32 at the roofline run's own size and kernel instance (the
# oracle steps the window from the GPU's FP32 distributions, so the bound is
# one FP32 step's rounding: MUFU reciprocals and square roots, <= 2 ulp each)
WINDOW_CASES = [(4096, lbmh.FP64, 300, 1e-12), (8192, lbmh.FP32, 100, 2e-5)]


@pytest.mark.parametrize("n,prec,later,bound", WINDOW_CASES, ids=["4096-fp64", "8192-fp32"])
def test_windows_of_a_large_lattice_match_the_oracle(n, prec, later, bound):
    import torch
    size = 64
    pb, U0 = W.riemann_2d_seeded(n, seed=0, cfl=0.9)
    rng = np.random.default_rng(11)
    wins = [(0, 0), (n - size, n - size), (n // 2 - 32, n // 2 - 32), (n // 2 - 32, n // 4), (n // 4, n // 2 - 32),
            tuple(int(v) for v in rng.integers(3, n - size - 3, 2))]
    f_before = torch.empty((5, 4, n, n), dtype=torch.float64, device="cuda")
    f_after = torch.empty_like(f_before)
    with lbmh.Solver(pb, precision=prec, kernel=lbmh.KERNEL_FUSED) as s:
        s.set_state(U0)
        for when in (0, later):
            if when:
                s.step(when - 1)
            abar = s.info()["abar"]
            s.get_f(out=f_before)
            s.step(1)
            s.get_f(out=f_after)
            for (a0, b0) in wins:
                fb = f_before[:, :, max(0, b0 - 3):b0 + size + 3, max(0, a0 - 3):a0 + size + 3].cpu().numpy()
                fa = f_after[:, :, b0:b0 + size, a0:a0 + size].cpu().numpy()
                err = window_err(pb, fb, fa, abar, a0, b0, size)
                assert np.all(err <= bound), (when, a0, b0, err)
