"""Pin the oracle to the numbers the paper prints (Tables 5.1, 5.2, 5.3, 5.5).

Time control: every step recomputes abar from U^n (Eq. 2.19) and
dt = CFL dx / sum abar (Eq. 2.21); the run stops at the first t_n >= T and the
exact solution is evaluated at that t_n.  (Clipping the last step so that
t = T changes lambda for one step and moves the Table 5.1/5.2 errors 2-30x away
from the printed values, so the paper did not do that.)
"""
import math

import numpy as np
import pytest

import oracle
from conftest import load_golden
from paper_2609_18177_b300.exact import total_variation
from paper_2609_18177_b300 import workloads as W


def run_until(pb, U0, T):
    r = oracle.Run(pb, U0)
    while r.t < T:
        r.step(1)
    return r


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def table(name):
    return {int(r[0]): float(r[2]) for r in load_golden(name)}


def advection_error(N):
    pb, U0 = W.advection_1d(N, "sine", cfl=0.9)
    r = run_until(pb, U0, 1.0)
    X, _ = W.cell_centres(pb)
    return rel_l2(r.moments()[0], np.sin(2 * np.pi * (X - r.t)))


def test_table_5_1_smooth_advection():
    """Table 5.1: errors within 8% of the paper at N = 400, 800, 1600 and order ~2."""
    paper = table("table_5_1_smooth_advection.txt")
    errs = {N: advection_error(N) for N in (400, 800, 1600)}
    for N, e in errs.items():
        assert 0.90 < e / paper[N] < 1.08, (N, e, paper[N])
    assert math.log2(errs[400] / errs[800]) > 1.9
    assert math.log2(errs[800] / errs[1600]) > 1.9


def entropy_1d_error(N):
    pb, U0 = W.entropy_wave_1d(N)
    r = run_until(pb, U0, 1.0)
    X, _ = W.cell_centres(pb)
    return rel_l2(r.moments()[0], 1.0 + 0.2 * np.sin(2 * np.pi * (X - r.t)))


def test_table_5_2_entropy_wave_1d():
    """Table 5.2: density errors within 6% of the paper at N = 400, 800; order >= 1.9."""
    paper = table("table_5_2_entropy_wave_1d.txt")
    e400, e800 = entropy_1d_error(400), entropy_1d_error(800)
    assert 0.95 < e400 / paper[400] < 1.06
    assert 0.95 < e800 / paper[800] < 1.06
    assert math.log2(e400 / e800) > 1.9


def entropy_2d_error(N):
    pb, U0 = W.entropy_wave_2d(N)
    r = run_until(pb, U0, 0.3)
    X, Y = W.cell_centres(pb)
    return rel_l2(r.moments()[0], 1.0 + 0.2 * np.sin(2 * np.pi * (X + Y - 2 * r.t)))


def test_table_5_3_entropy_wave_2d_orders():
    """Table 5.3: the pre-asymptotic convergence orders (1.51, 1.71) are reproduced
    within 0.08.  The absolute errors sit a constant factor 1.43-1.50 above the
    printed ones at every N; the test bounds that factor.

    Error measures tried against the printed values (ratio ours / paper at
    N = 40, 80, 160): relative L2 of the density at the final t_n (kept):
    1.43, 1.48, 1.50; exact solution at T = 0.3 instead of t_n: 1.43, 1.49,
    1.51; absolute discrete L2 sqrt(sum e^2 / N): 1.44, 1.49, 1.51; the
    state of the last step before T: 1.42, 1.48, 1.50; a clipped last step
    landing on T: 1.41, 1.47, 1.50; relative L2 over all four conserved
    fields: 0.74, 0.76, 0.77; relative L1 of the density: 1.27, 1.24, 1.17;
    max norm: 2.16, 2.47, 2.85; L2 relative to the wave's amplitude
    (rho - 1): 10.2, 10.6, 10.7.  None matches within a few percent at every N,
    so the difference is not in how the error is measured, and the band
    stays."""
    paper = table("table_5_3_entropy_wave_2d.txt")
    errs = {N: entropy_2d_error(N) for N in (40, 80, 160)}
    for (a, b) in ((40, 80), (80, 160)):
        ours = math.log2(errs[a] / errs[b])
        theirs = math.log2(paper[a] / paper[b])
        assert abs(ours - theirs) < 0.08, (a, b, ours, theirs)
    for N, e in errs.items():
        assert 1.3 < e / paper[N] < 1.6, (N, e / paper[N])


def test_table_5_5_sod_total_variation():
    """Table 5.5: TV(rho, u, p) on [0.15, 0.35] within 0.005 of the paper (N = 600)."""
    (row,) = load_golden("table_5_5_sod_tv.txt")
    paper = [float(v) for v in row[1:4]]
    pb, U0 = W.sod(600)
    r = run_until(pb, U0, 0.2)
    U = r.moments()[:, 0, :]
    X, _ = W.cell_centres(pb)
    X = X[0]
    rho = U[0]
    u = U[1] / rho
    p = (pb.gamma - 1.0) * (U[2] - 0.5 * rho * u * u)
    sel = (X >= 0.15) & (X <= 0.35)
    ours = [total_variation(rho[sel]), total_variation(u[sel]), total_variation(p[sel])]
    for a, b in zip(ours, paper):
        assert abs(a - b) < 0.005, (ours, paper)
