"""Oracle (pull form, C) against the brute-force push form of Eq. (2.2) (Python)
on tiny grids: every system, both dimensions, periodic and outflow boundaries."""
import numpy as np
import pytest

import brute_force_lbm as BF
import oracle
from paper_2609_18177_b300 import workloads as W


def cases():
    out = []
    for dim in (1, 2):
        nx, ny = (9, 1) if dim == 1 else (7, 6)
        y1 = ny / nx if dim == 2 else 1.0
        for bc in (W.PERIODIC, W.OUTFLOW):
            base = dict(dim=dim, nx=nx, ny=ny, y1=y1, bc=(bc,) * 4, cfl=0.8)
            out.append((f"adv{dim}d-{bc}", W.Problem(system=W.ADVECTION, adv=(0.8, -0.5), **base)))
            out.append((f"euler{dim}d-{bc}", W.Problem(system=W.EULER, **base)))
            out.append((f"swe{dim}d-{bc}", W.Problem(system=W.SWE, bed_amp=0.4, bed_w2=0.05,
                                                      bed_xc=0.4, bed_yc=0.3, **base)))
            out.append((f"react{dim}d-{bc}", W.Problem(system=W.REACTIVE, gamma=1.2, q=5.0,
                                                        K=40.0, Ti=2.0, **base)))
    return out


@pytest.mark.parametrize("name,pb", cases(), ids=[c[0] for c in cases()])
def test_push_form_matches_oracle(name, pb):
    U0 = W.random_state(pb, seed=11)
    r = oracle.Run(pb, U0)
    f = r.f.copy()
    for _ in range(3):
        f, dt = BF.step(pb, f)
        r.step(1)
        assert r.info[2] == pytest.approx(dt, rel=1e-14)
        scale = np.abs(r.f).max(axis=(0, 2, 3), keepdims=True)
        assert np.all(np.abs(f - r.f) <= 1e-13 * scale), np.abs(f - r.f).max()


def test_push_form_wet_dry():
    pb = W.Problem(system=W.SWE, dim=1, nx=10, x0=-1, x1=1, cfl=0.9, bc=(W.OUTFLOW,) * 4)
    X, _ = W.cell_centres(pb)
    U0 = W.swe_conservative(pb, np.where(X <= 0.0, 2.0, 0.0), 0.0)
    r = oracle.Run(pb, U0)
    f = r.f.copy()
    for _ in range(4):
        f, dt = BF.step(pb, f)
        r.step(1)
        assert np.all(np.abs(f - r.f) <= 1e-13 * np.abs(r.f).max())


@pytest.mark.parametrize("dim", [1, 2])
def test_push_form_bed_with_dry_cells(dim):
    """The bed-slope source next to dry nodes: a dam break towards the
    Gaussian bump, whose top sticks out of a shallow pool (h = 0 there), and
    one node with 0 < h < h_dry (dry, at rest).  The pure-Python push-form
    stepper applies Section 5's bed source and the dry-node rule on its own;
    the oracle must agree with it to rounding."""
    if dim == 1:
        pb = W.Problem(system=W.SWE, dim=1, nx=12, x0=-1.0, x1=1.0, cfl=0.9, bc=(W.OUTFLOW,) * 4,
                       bed_amp=0.5, bed_w2=0.1, bed_xc=0.2)
    else:
        pb = W.Problem(system=W.SWE, dim=2, nx=8, ny=7, x0=-1.0, x1=1.0, y0=-0.875, y1=0.875, cfl=0.9,
                       bc=(W.OUTFLOW,) * 4, bed_amp=0.5, bed_w2=0.1, bed_xc=0.2, bed_yc=0.0)
    X, Y = W.cell_centres(pb)
    b = pb.bed_amp * np.exp(-((X - pb.bed_xc) ** 2 + (Y - pb.bed_yc) ** 2 if dim == 2 else (X - pb.bed_xc) ** 2)
                            / pb.bed_w2)
    h = np.where(X <= -0.4, 1.5, np.maximum(0.0, 0.3 - b))
    assert np.any(h == 0.0) and np.any(h > 0.0)
    # one node in the pool beyond the bump with 0 < h < h_dry and momentum h u
    # (u = 1 if it were wet): the rule takes it as dry, at rest
    i = np.argmax(X.ravel() > 0.6)
    h.flat[i] = 0.5 * pb.h_dry
    u = np.zeros_like(h)
    u.flat[i] = 1.0
    U0 = W.swe_conservative(pb, h, u)
    r = oracle.Run(pb, U0)
    f = r.f.copy()
    for _ in range(4):
        f, dt = BF.step(pb, f)
        r.step(1)
        assert r.info[2] == pytest.approx(dt, rel=1e-14)
        scale = np.abs(r.f).max(axis=(0, 2, 3), keepdims=True)
        assert np.all(np.abs(f - r.f) <= 1e-13 * scale), np.abs(f - r.f).max()


def boundary_cases():
    """Reflecting walls, fixed inflow and the sponge layer (Example 5.13's
    boundaries) on every system, including corners where two kinds meet."""
    out = []
    combos = {
        1: [((W.REFLECT, W.INFLOW, 0, 0), 0.35), ((W.INFLOW, W.REFLECT, 0, 0), 0.0),
            ((W.OUTFLOW, W.REFLECT, 0, 0), 0.5)],
        2: [((W.OUTFLOW, W.INFLOW, W.REFLECT, W.REFLECT), 0.3),
            ((W.REFLECT, W.REFLECT, W.PERIODIC, W.PERIODIC), 0.0),
            ((W.INFLOW, W.OUTFLOW, W.INFLOW, W.REFLECT), 0.45)],
    }
    for dim in (1, 2):
        nx, ny = (9, 1) if dim == 1 else (7, 6)
        y1 = ny / nx if dim == 2 else 1.0
        for bc, sponge in combos[dim]:
            base = dict(dim=dim, nx=nx, ny=ny, y1=y1, bc=bc, cfl=0.8, sponge_width=sponge)
            tag = f"{dim}d-" + "".join("POR I"[b] for b in bc[:2 * dim]) + (f"-s{sponge}" if sponge else "")
            for name, pb in (("adv", W.Problem(system=W.ADVECTION, adv=(0.8, -0.5), **base)),
                             ("euler", W.Problem(system=W.EULER, **base)),
                             ("swe", W.Problem(system=W.SWE, bed_amp=0.4, bed_w2=0.05, bed_xc=0.4, bed_yc=0.3,
                                               **base)),
                             ("react", W.Problem(system=W.REACTIVE, gamma=1.2, q=5.0, K=40.0, Ti=2.0, **base))):
                u_in = tuple(W.random_state(pb, seed=5).reshape(pb.nfields, -1)[:, 0])
                out.append((f"{name}{tag}", pb.with_(u_in=u_in)))
    return out


@pytest.mark.parametrize("name,pb", boundary_cases(), ids=[c[0] for c in boundary_cases()])
def test_push_form_matches_oracle_reflect_inflow_sponge(name, pb):
    U0 = W.random_state(pb, seed=13)
    r = oracle.Run(pb, U0)
    f = r.f.copy()
    for _ in range(3):
        f, dt = BF.step(pb, f)
        r.step(1)
        assert r.info[2] == pytest.approx(dt, rel=1e-14)
        scale = np.abs(r.f).max(axis=(0, 2, 3), keepdims=True)
        assert np.all(np.abs(f - r.f) <= 1e-13 * scale), np.abs(f - r.f).max()
