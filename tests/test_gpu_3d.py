"""The 3D (D3Q7) path against the FP64 oracle: advection, Euler and reactive
Euler, periodic and outflow sides, ragged grids, FP64 (relative max error <=
1e-12 per field) and FP32 (relative L1 <= 2e-5, relative max <= 5e-4);
checkpoints, time targets and the unsupported combinations."""
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


def rel_max(g, o):
    m = o.shape[0]
    g2, o2 = g.reshape(m, -1), o.reshape(m, -1)
    s = np.abs(o2).max(axis=1)
    return np.abs(g2 - o2).max(axis=1) / np.where(s > 0, s, 1.0)


def rel_l1(g, o):
    m = o.shape[0]
    g2, o2 = g.reshape(m, -1), o.reshape(m, -1)
    s = np.abs(o2).sum(axis=1)
    return np.abs(g2 - o2).sum(axis=1) / np.where(s > 0, s, 1.0)


def case(system, bc, nx=23, ny=19, nz=17, seed=2):
    h = 1.0 / nx
    kw = dict(system=system, dim=3, nx=nx, ny=ny, nz=nz, y1=ny * h, z1=nz * h, cfl=0.8, bc=(bc,) * 4,
              bc_z=(bc, bc), adv=(0.7, -0.45, 0.35))
    if system == W.REACTIVE:
        kw.update(gamma=1.2, q=5.0, K=40.0, Ti=2.0)
    pb = W.Problem(**kw)
    return pb, W.random_state(pb, seed=seed)


CASES = [(s, bc) for s in (W.ADVECTION, W.EULER, W.REACTIVE) for bc in (W.PERIODIC, W.OUTFLOW)]
IDS = [f"{W.SYSTEM_NAMES[s]}-{'per' if bc == 0 else 'out'}" for s, bc in CASES]


KERNELS = [(lbmh.KERNEL_FUSED, "fused"), (lbmh.KERNEL_UNFUSED, "four-kernel")]


@pytest.mark.parametrize("kernel", [k for k, _ in KERNELS], ids=[n for _, n in KERNELS])
@pytest.mark.parametrize("precision", [lbmh.FP64, lbmh.FP32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("system,bc", CASES, ids=IDS)
def test_3d_matches_oracle(system, bc, precision, kernel):
    pb, U0 = case(system, bc)
    pb = pb.with_(precision=precision)
    r = oracle.Run(pb, U0)
    s = lbmh.Solver(pb, precision=precision, kernel=kernel).set_state(U0)
    assert s.info()["kernel"] == (lbmh.KERNEL_FUSED if kernel == lbmh.KERNEL_FUSED else lbmh.KERNEL_UNFUSED)
    for n in range(4):
        r.step(5)
        s.step(5)
        Ug, Uo = s.moments(), r.moments()
        assert s.nsteps == r.nsteps
        if precision == lbmh.FP64:
            assert np.all(rel_max(Ug, Uo) <= 1e-12), (5 * (n + 1), rel_max(Ug, Uo))
            assert abs(s.t - r.t) <= 1e-13 * r.t
        else:
            assert np.all(rel_l1(Ug, Uo) <= 2e-5), (5 * (n + 1), rel_l1(Ug, Uo))
            assert np.all(rel_max(Ug, Uo) <= 5e-4), (5 * (n + 1), rel_max(Ug, Uo))
    s.close()


def test_3d_checkpoint_resume_is_bitwise_and_time_target():
    pb, U0 = case(W.EULER, W.PERIODIC, nx=16, ny=16, nz=16)
    for prec in (lbmh.FP64, lbmh.FP32):
        a = lbmh.Solver(pb, precision=prec).set_state(U0).step(6)
        f = a.get_f()
        t, n = a.t, a.nsteps
        a.step(4)
        b = lbmh.Solver(pb, precision=prec).set_f(f, t, n).step(4)
        assert np.array_equal(a.get_f(), b.get_f())
        a.close()
        b.close()
    r = oracle.Run(pb, U0)
    s = lbmh.Solver(pb, precision=lbmh.FP64).set_state(U0)
    s.advance_to(0.02)
    while r.t < 0.02:
        r.step(1)
    assert s.info()["steps"] == r.nsteps
    assert np.all(rel_max(s.moments(), r.moments()) <= 1e-12)
    s.close()


def test_3d_unsupported_combinations():
    pb, _U0 = case(W.EULER, W.PERIODIC, nx=8, ny=8, nz=8)
    with pytest.raises(lbmh.LbmhError) as ei:
        lbmh.Solver(pb.with_(system=W.SWE), precision=lbmh.FP64)
    assert ei.value.code == lbmh.ERR_UNSUPPORTED
    s = lbmh.Solver(pb, precision=lbmh.FP64).set_state(W.random_state(pb, seed=1))
    with pytest.raises(lbmh.LbmhError):
        s.omega()
    s.close()


@pytest.mark.parametrize("kernel", [k for k, _ in KERNELS], ids=[n for _, n in KERNELS])
@pytest.mark.parametrize("precision", [lbmh.FP64, lbmh.FP32], ids=["fp64", "fp32"])
def test_3d_graph_replay_and_set_f_keep_moments_consistent(precision, kernel):
    """A step normally reuses the moments U^{n+1} that the previous collision
    wrote and refills only the ghost layers; the distributions set from
    outside (set_f) and the first step of every graph replay take the full
    moments pass.  Graph replays, single steps and the oracle must agree."""
    pb, U0 = case(W.REACTIVE, W.OUTFLOW)
    pb = pb.with_(precision=precision)
    a = lbmh.Solver(pb, precision=precision, kernel=kernel).set_state(U0).step(60)  # 0 single, 2 graph replays, 12 single
    b = lbmh.Solver(pb, precision=precision, kernel=kernel).set_state(U0)
    for _ in range(60):
        b.step(1)
    assert np.array_equal(a.get_f(), b.get_f())
    if precision == lbmh.FP64:
        r = oracle.Run(pb, U0).step(60)
        assert np.all(rel_max(a.moments(), r.moments()) <= 1e-12)
    # new distributions under an existing graph: the replay starts with the full pass
    f_other = lbmh.Solver(pb, precision=precision).set_state(W.random_state(pb, seed=7)).step(3).get_f()
    a.set_f(f_other, 0.0, 0)
    a.step(50)
    c = lbmh.Solver(pb, precision=precision, kernel=kernel).set_f(f_other, 0.0, 0)
    for _ in range(50):
        c.step(1)
    assert np.array_equal(a.get_f(), c.get_f())
    for s in (a, b, c):
        s.close()


def test_3d_int_and_64bit_offsets_give_the_same_bits(monkeypatch):
    """The four-kernel path's collision kernel indexes with int offsets where
    every offset of the lattice fits (up to ~390^3) and with 64-bit offsets
    beyond; the two instances do the same arithmetic.  LBMH_3D_INDEX64=1
    forces the 64-bit one on a small lattice."""
    pb, U0 = case(W.REACTIVE, W.OUTFLOW)
    for prec in (lbmh.FP64, lbmh.FP32):
        monkeypatch.delenv("LBMH_3D_INDEX64", raising=False)
        a = lbmh.Solver(pb, precision=prec, kernel=lbmh.KERNEL_UNFUSED).set_state(U0).step(12)
        monkeypatch.setenv("LBMH_3D_INDEX64", "1")
        b = lbmh.Solver(pb, precision=prec, kernel=lbmh.KERNEL_UNFUSED).set_state(U0).step(12)
        assert np.array_equal(a.get_f(), b.get_f())
        a.close()
        b.close()


@pytest.mark.parametrize("precision", [lbmh.FP64, lbmh.FP32], ids=["fp64", "fp32"])
def test_3d_speed_bounds_reported(precision):
    """lbmh_get_info reports the speed bound of the current state along x, y
    and z (Eq. 2.19): max over nodes of |u_j| + c, recomputed here from the
    state's moments."""
    pb, U0 = case(W.EULER, W.OUTFLOW)
    pb = pb.with_(precision=precision)
    s = lbmh.Solver(pb, precision=precision).set_state(U0).step(7)
    U = s.moments().reshape(5, -1)
    rho, m, E = U[0], U[1:4], U[4]
    p = (pb.gamma - 1.0) * (E - 0.5 * (m * m).sum(axis=0) / rho)
    c = np.sqrt(pb.gamma * p / rho)
    want = [float((np.abs(m[j] / rho) + c).max()) for j in range(3)]
    inf = s.info()
    got = [inf["abar"][0], inf["abar"][1], inf["abar_z"]]
    tol = 1e-12 if precision == lbmh.FP64 else 1e-5
    assert np.allclose(got, want, rtol=tol, atol=0.0), (got, want)
    s.close()


@pytest.mark.parametrize("precision", [lbmh.FP64, lbmh.FP32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("bc", [W.PERIODIC, W.OUTFLOW], ids=["per", "out"])
def test_3d_fused_over_several_tiles_and_chunks(bc, precision, monkeypatch):
    """A lattice of several 32 x 8 tiles with ragged edges in x and y, and z
    chunks of 8 planes with a ragged last chunk (the fused kernel marches each
    chunk with a fill of its own), against the oracle."""
    monkeypatch.setenv("LBMH_3D_ZCHUNK", "8")
    pb, U0 = case(W.EULER, bc, nx=70, ny=19, nz=29, seed=5)
    pb = pb.with_(precision=precision)
    s = lbmh.Solver(pb, precision=precision, kernel=lbmh.KERNEL_FUSED).set_state(U0)
    monkeypatch.delenv("LBMH_3D_ZCHUNK")
    r = oracle.Run(pb, U0).step(6)
    s.step(6)
    Ug, Uo = s.moments(), r.moments()
    if precision == lbmh.FP64:
        assert np.all(rel_max(Ug, Uo) <= 1e-12), rel_max(Ug, Uo)
    else:
        assert np.all(rel_l1(Ug, Uo) <= 2e-5), rel_l1(Ug, Uo)
        assert np.all(rel_max(Ug, Uo) <= 5e-4), rel_max(Ug, Uo)
    info = s.info()
    # the FP64 sums over the warps' partial slots: conservation under periodic sides
    if bc == W.PERIODIC:
        tot0 = U0.reshape(pb.nfields, -1).sum(axis=1)
        assert np.allclose(info["sum_U"], tot0, rtol=1e-10 if precision == lbmh.FP64 else 1e-5)
    s.close()


@pytest.mark.parametrize("kernel", [k for k, _ in KERNELS], ids=[n for _, n in KERNELS])
@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 3, 4), (5, 1, 7), (33, 9, 2), (3, 17, 1)],
                         ids=["1x1x1", "2x3x4", "5x1x7", "33x9x2", "3x17x1"])
def test_3d_tiny_and_degenerate_grids(shape, kernel):
    """Lattices of one node, one row or one plane along an axis, and tiles
    that are almost all ghost lanes, FP64 against the oracle (<= 1e-12) and
    FP32 at the FP32 bar, both sides kinds."""
    nx, ny, nz = shape
    for bc in (W.PERIODIC, W.OUTFLOW):
        for precision in (lbmh.FP64, lbmh.FP32):
            pb, U0 = case(W.EULER, bc, nx=nx, ny=ny, nz=nz, seed=4)
            pb = pb.with_(precision=precision)
            r = oracle.Run(pb, U0).step(6)
            with lbmh.Solver(pb, precision=precision, kernel=kernel).set_state(U0) as s:
                s.step(6)
                Ug, Uo = s.moments(), r.moments()
            if precision == lbmh.FP64:
                assert np.all(rel_max(Ug, Uo) <= 1e-12), (shape, bc, rel_max(Ug, Uo))
            else:
                assert np.all(rel_max(Ug, Uo) <= 5e-4), (shape, bc, rel_max(Ug, Uo))
