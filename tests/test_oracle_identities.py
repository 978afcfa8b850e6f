"""Pin the oracle to identities, theorems and exact solutions (CPU only).

Each test checks the oracle against something fixed independently of it:
  - (2.4): moments of the equilibrium;
  - the textbook wave speeds, through a finite-difference Jacobian of the flux;
  - omega = 1 turns the scheme into the global Lax-Friedrichs finite-volume
    scheme (independent numpy implementation below);
  - a spatially uniform state turns (2.2) with the midpoint source into the
    trapezoidal rule for the ODE U' = S(U);
  - conservation of sum_x U under periodic BCs when S = 0;
  - Theorem 4.2/4.3: the weighted norm ||f||_P never grows for linear systems;
  - omega in (1, 2] and omega -> 2 under refinement on smooth data (Section 2.2);
  - exact Riemann and dry-bed dam-break solutions (Examples 5.5, 5.6, 5.9).
"""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
from paper_2609_18177_b300.exact import riemann_profile, ritter
from paper_2609_18177_b300 import workloads as W

GAMMA = 1.4


def systems_1d_2d():
    out = []
    for dim in (1, 2, 3):
        n = 8
        out.append(W.Problem(system=W.EULER, dim=dim, nx=n, ny=n, nz=n))
        if dim < 3:
            out.append(W.Problem(system=W.SWE, dim=dim, nx=n, ny=n))
        out.append(W.Problem(system=W.REACTIVE, dim=dim, nx=n, ny=n, nz=n, gamma=1.2, q=50.0,
                             K=2566.4, Ti=50.0))
        out.append(W.Problem(system=W.ADVECTION, dim=dim, nx=n, ny=n, nz=n, adv=(0.7, -0.4, 0.3)))
    return out


def random_U(pb, rng):
    d = pb.dim
    if pb.system == W.ADVECTION:
        return rng.uniform(-1, 1, 1)
    if pb.system == W.SWE:
        h = rng.uniform(0.5, 2.0)
        vel = rng.uniform(-1, 1, d)
        return np.concatenate([[h], h * vel])
    rho = rng.uniform(0.5, 2.0)
    vel = rng.uniform(-1, 1, 3)[:d]
    p = rng.uniform(0.5, 2.0)
    Y = rng.uniform(0.1, 0.9)
    kin = 0.5 * rho * np.sum(vel ** 2)
    if pb.system == W.REACTIVE:
        E = p / (pb.gamma - 1) + kin + rho * pb.q * Y
        return np.concatenate([[rho], rho * vel, [E, rho * Y]])
    return np.concatenate([[rho], rho * vel, [p / (pb.gamma - 1) + kin]])


def fd_jacobian(pb, direction, U, h=1e-6):
    m = U.size
    J = np.zeros((m, m))
    for c in range(m):
        e = np.zeros(m)
        e[c] = h * max(1.0, abs(U[c]))
        J[:, c] = (oracle.flux(pb, direction, U + e) - oracle.flux(pb, direction, U - e)) / (2 * e[c])
    return J


def physical_speeds(pb, direction, U):
    """Textbook characteristic speeds from primitive variables."""
    d = pb.dim
    if pb.system == W.ADVECTION:
        return np.array([pb.adv[direction]])
    if pb.system == W.SWE:
        h = U[0]
        vn = U[1 + direction] / h
        c = math.sqrt(pb.g * h)
        return np.array([vn - c] + [vn] * (d - 1) + [vn + c])
    rho = U[0]
    vel = U[1:1 + d] / rho
    kin = 0.5 * rho * np.sum(vel ** 2)
    chem = pb.q * U[d + 2] if pb.system == W.REACTIVE else 0.0
    p = (pb.gamma - 1) * (U[d + 1] - kin - chem)
    c = math.sqrt(pb.gamma * p / rho)
    vn = vel[direction]
    m = U.size
    return np.array([vn - c] + [vn] * (m - 2) + [vn + c])


@pytest.mark.parametrize("pb", systems_1d_2d(), ids=lambda p: f"{W.SYSTEM_NAMES[p.system]}{p.dim}d")
def test_flux_jacobian_has_textbook_speeds_and_eigenvectors(pb):
    rng = np.random.default_rng(1)
    for _ in range(5):
        U = random_U(pb, rng)
        for direction in range(pb.dim):
            J = fd_jacobian(pb, direction, U)
            lam_fd = np.sort(np.linalg.eigvals(J).real)
            lam_tb = np.sort(physical_speeds(pb, direction, U))
            assert np.allclose(lam_fd, lam_tb, atol=1e-6), (lam_fd, lam_tb)
            lam = oracle.eigvals(pb, direction, U)
            assert np.allclose(np.sort(lam), lam_tb, atol=1e-12)
            R = oracle.right_eigvecs(pb, direction, U)
            L = oracle.left_eigvecs(pb, direction, U)
            # A R = R Lambda, L = R^{-1}
            assert np.allclose(J @ R, R * lam[None, :], atol=1e-5 * max(1, np.abs(J).max()))
            assert np.allclose(L @ R, np.eye(U.size), atol=1e-12)
            assert oracle.max_speed(pb, direction, U) == pytest.approx(np.abs(lam_tb).max(), rel=1e-14)


@pytest.mark.parametrize("pb", systems_1d_2d(), ids=lambda p: f"{W.SYSTEM_NAMES[p.system]}{p.dim}d")
def test_equilibrium_moments(pb):
    """(2.4): sum_k f^eq_k = U and sum_k v_kj f^eq_k = F_j with v_k = lambda e_k."""
    rng = np.random.default_rng(2)
    d = pb.dim
    for _ in range(5):
        U = random_U(pb, rng)
        alpha = rng.uniform(1.0, 3.0, d)
        lam = alpha.sum() / 0.7
        feq = oracle.equilibrium(pb, U, alpha, lam)
        assert np.allclose(feq.sum(axis=0), U, rtol=1e-14, atol=1e-14)
        for j in range(d):
            e = np.zeros(2 * d + 1)
            e[1 + j], e[1 + j + d] = 1.0, -1.0
            mom = (lam * e[:, None] * feq).sum(axis=0)
            assert np.allclose(mom, oracle.flux(pb, j, U), rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------------------------
# omega = 1  <=>  global Lax-Friedrichs finite volumes
# ---------------------------------------------------------------------------

def fv_flux(pb, U):
    """Independent numpy fluxes F_j(U) on whole grids, U shape (m, ny, nx)."""
    d = pb.dim
    out = []
    if pb.system == W.ADVECTION:
        return [pb.adv[j] * U for j in range(d)]
    if pb.system == W.SWE:
        h = U[0]
        vel = [U[1 + j] / h for j in range(d)]
        for j in range(d):
            F = [h * vel[j]] + [U[1 + i] * vel[j] + (0.5 * pb.g * h * h if i == j else 0.0) for i in range(d)]
            out.append(np.stack(F))
        return out
    rho = U[0]
    vel = [U[1 + j] / rho for j in range(d)]
    E = U[d + 1]
    chem = pb.q * U[d + 2] if pb.system == W.REACTIVE else 0.0  # heat of the unburnt gas
    p = (pb.gamma - 1) * (E - 0.5 * rho * sum(v * v for v in vel) - chem)
    for j in range(d):
        F = [rho * vel[j]] + [U[1 + i] * vel[j] + (p if i == j else 0.0) for i in range(d)]
        F.append(vel[j] * (E + p))
        if pb.system == W.REACTIVE:
            F.append(U[d + 2] * vel[j])
        out.append(np.stack(F))
    return out


def fv_speed(pb, U):
    d = pb.dim
    if pb.system == W.ADVECTION:
        return [abs(pb.adv[j]) for j in range(d)]
    if pb.system == W.SWE:
        c = np.sqrt(pb.g * U[0])
        return [float(np.max(np.abs(U[1 + j] / U[0]) + c)) for j in range(d)]
    rho = U[0]
    vel = [U[1 + j] / rho for j in range(d)]
    chem = pb.q * U[d + 2] if pb.system == W.REACTIVE else 0.0
    p = (pb.gamma - 1) * (U[d + 1] - 0.5 * rho * sum(v * v for v in vel) - chem)
    c = np.sqrt(pb.gamma * p / rho)
    return [float(np.max(np.abs(vel[j]) + c)) for j in range(d)]


def shift(pb, A, j, s):
    """A evaluated at index i + s along axis j (j=0: x), ghost values per BC."""
    axis = A.ndim - 1 - j
    n = A.shape[axis]
    idx = np.arange(n) + s
    periodic = (pb.bc[0] if j == 0 else pb.bc[2] if j == 1 else pb.bc_z[0]) == W.PERIODIC
    idx = idx % n if periodic else np.clip(idx, 0, n - 1)
    return np.take(A, idx, axis=axis)


def lf_step(pb, U):
    speeds = fv_speed(pb, U)
    dt = pb.cfl * pb.dx / sum(speeds)
    alpha = [s + pb.eps for s in speeds]
    F = fv_flux(pb, U)
    Un = U.copy()
    for j in range(pb.dim):
        Up, Um = shift(pb, U, j, +1), shift(pb, U, j, -1)
        Fp, Fm = shift(pb, F[j], j, +1), shift(pb, F[j], j, -1)
        Un = Un - dt / (2 * pb.dx) * (Fp - Fm) + alpha[j] * dt / (2 * pb.dx) * (Up - 2 * U + Um)
    return Un


LF_CASES = [
    ("sod_outflow", lambda: W.sod(64)),
    ("euler2d_periodic", lambda: (W.Problem(system=W.EULER, dim=2, nx=20, ny=20),)),
    ("swe2d_outflow", lambda: (W.Problem(system=W.SWE, dim=2, nx=18, ny=18, bc=(W.OUTFLOW,) * 4),)),
    ("advection1d", lambda: W.advection_1d(50, "pulse")),
    ("euler3d_periodic", lambda: (W.cube(W.EULER, 10),)),
    ("advection3d_outflow", lambda: (W.cube(W.ADVECTION, 9, adv=(0.6, -0.4, 0.5), bc=(W.OUTFLOW,) * 4,
                                              bc_z=(W.OUTFLOW, W.OUTFLOW)),)),
]


@pytest.mark.parametrize("name,make", LF_CASES, ids=[c[0] for c in LF_CASES])
def test_omega_one_is_global_lax_friedrichs(name, make):
    made = make()
    pb = made[0]
    U0 = made[1] if len(made) > 1 else W.random_state(pb, seed=3)
    pb = pb.with_(omega_mode=1, omega_fixed=1.0, cfl=0.8)
    r = oracle.Run(pb, U0)
    U = U0.reshape((pb.nfields,) + pb.shape()).copy()
    for _ in range(6):
        r.step(1)
        U = lf_step(pb, U)
        assert np.allclose(r.moments(), U, rtol=1e-12, atol=1e-12 * np.abs(U).max())


# ---------------------------------------------------------------------------
# inflow sides (Example 5.13) and the sponge, pinned without the push-form
# stepper: omega = 1 with an inflow side is the global Lax-Friedrichs scheme
# whose ghost node holds the inflow state (its flux enters the face between
# the ghost and the first node with the step's alpha), and a uniform inflow
# state is a steady solution
# ---------------------------------------------------------------------------

def shift_inflow(pb, A, j, s, ghost):
    """A at index i + s along axis j; an index beyond an INFLOW side reads
    `ghost` (one node's values, broadcast), others per the side's BC."""
    axis = A.ndim - 1 - j
    n = A.shape[axis]
    lo, hi = (pb.bc[0], pb.bc[1]) if j == 0 else (pb.bc[2], pb.bc[3])
    idx = np.arange(n) + s
    out = np.take(A, np.clip(idx, 0, n - 1) if lo != W.PERIODIC else idx % n, axis=axis)
    shape = [1] * A.ndim
    shape[0] = A.shape[0]
    g = np.asarray(ghost, dtype=np.float64).reshape(shape)
    for side, bad in ((lo, idx < 0), (hi, idx >= n)):
        if side == W.INFLOW and bad.any():
            sel = [slice(None)] * A.ndim
            sel[axis] = np.nonzero(bad)[0]
            out[tuple(sel)] = np.broadcast_to(g, out[tuple(sel)].shape)
    return out


def lf_step_inflow(pb, U):
    speeds = fv_speed(pb, U)
    dt = pb.cfl * pb.dx / sum(speeds)
    alpha = [s + pb.eps for s in speeds]
    m = U.shape[0]
    u_in = np.array(pb.u_in[:m])
    F = fv_flux(pb, U)
    Fin = [f.reshape(m) for f in fv_flux(pb, u_in.reshape((m,) + (1,) * (U.ndim - 1)))]
    Un = U.copy()
    for j in range(pb.dim):
        Up, Um = shift_inflow(pb, U, j, +1, u_in), shift_inflow(pb, U, j, -1, u_in)
        Fp, Fm = shift_inflow(pb, F[j], j, +1, Fin[j]), shift_inflow(pb, F[j], j, -1, Fin[j])
        Un = Un - dt / (2 * pb.dx) * (Fp - Fm) + alpha[j] * dt / (2 * pb.dx) * (Up - 2 * U + Um)
    return Un


INFLOW_CASES = [
    ("euler1d_inflow_hi", W.Problem(system=W.EULER, dim=1, nx=48, bc=(W.OUTFLOW, W.INFLOW, 0, 0),
                                    u_in=(1.3, -0.9, 4.0))),
    ("euler1d_inflow_lo_sponge", W.Problem(system=W.EULER, dim=1, nx=40, bc=(W.INFLOW, W.OUTFLOW, 0, 0),
                                           u_in=(0.8, 0.6, 2.5), sponge_width=0.3)),
    ("swe2d_inflow_lo", W.Problem(system=W.SWE, dim=2, nx=16, ny=12, y1=0.75,
                                  bc=(W.INFLOW, W.OUTFLOW, W.OUTFLOW, W.OUTFLOW), u_in=(1.4, 0.7, -0.2))),
    ("reactive2d_inflow_hi_sponge", W.Problem(system=W.REACTIVE, dim=2, nx=14, ny=10, y1=10 / 14, gamma=1.2,
                                              q=2.0, K=5.0, Ti=3.0, bc=(W.OUTFLOW, W.INFLOW, W.PERIODIC, W.PERIODIC),
                                              u_in=(1.0, -1.2, 0.1, 6.0, 1.0), sponge_width=0.2)),
]


@pytest.mark.parametrize("name,pb", INFLOW_CASES, ids=[c[0] for c in INFLOW_CASES])
def test_omega_one_with_inflow_sides_is_lax_friedrichs_with_the_inflow_ghost(name, pb):
    """omega = 1 (fixed; with a sponge, omega' = 1 + (1 - 1)(1 - sigma) = 1 too):
    the step is the global Lax-Friedrichs update whose neighbour beyond an
    inflow side is u_in.  A wrong alpha or lambda in the ghost's f^eq(u_in), or
    a ghost state other than u_in, changes the face flux and fails this."""
    if pb.system == W.REACTIVE:
        pb = pb.with_(K=0.0)  # no source: the identity is the homogeneous LF scheme
    U0 = W.random_state(pb, seed=8)
    pb = pb.with_(omega_mode=1, omega_fixed=1.0, cfl=0.8)
    r = oracle.Run(pb, U0)
    U = U0.reshape((pb.nfields,) + pb.shape()).copy()
    for _ in range(5):
        r.step(1)
        U = lf_step_inflow(pb, U)
        assert np.allclose(r.moments(), U, rtol=1e-12, atol=1e-12 * np.abs(U).max())


@pytest.mark.parametrize("name,pb", INFLOW_CASES, ids=[c[0] for c in INFLOW_CASES])
def test_uniform_inflow_state_is_steady(name, pb):
    """A lattice filled with the inflow state keeps that state with its inflow
    sides (and a sponge): f = f^eq everywhere, the ghosts hold f^eq(u_in) with
    the same alpha and lambda, streaming moves equal values.  Only rounding
    (sum_k f^eq_k(U) is U up to an ulp) moves it, and it does not grow.
    Without a source only (the Arrhenius source would burn the gas)."""
    pb = pb.with_(K=0.0)
    m = pb.nfields
    U0 = np.broadcast_to(np.array(pb.u_in[:m]).reshape((m,) + (1,) * len(pb.shape())),
                         (m,) + pb.shape()).copy()
    r = oracle.Run(pb, U0)
    for _ in range(4):
        r.step(10)
        U = r.moments()
        assert np.all(np.abs(U - U0) <= 4e-15 * np.abs(U0).max()), np.abs(U - U0).max()


# ---------------------------------------------------------------------------
# uniform state + source  <=>  trapezoidal rule for U' = S(U)
# ---------------------------------------------------------------------------

def test_uniform_reactive_state_is_trapezoidal_rule():
    pb = W.Problem(system=W.REACTIVE, dim=2, nx=4, ny=4, gamma=1.2, q=50.0, Ti=20.0, K=30.0,
                   cfl=0.9)
    rho, p, Y = 1.0, 12.0, 0.9
    U0 = W.euler_conservative(pb, np.full((4, 4), rho), 0.0, p, v=0.0, Y=Y)
    r = oracle.Run(pb, U0)
    z = rho * Y
    E = U0[3, 0, 0]

    def rate(zz):
        T = (pb.gamma - 1) * (E - pb.q * zz) / rho / rho
        return pb.K * zz * math.exp(-pb.Ti / T)

    for _ in range(20):
        r.step(1)
        dt = r.info[2]
        rhs = z - 0.5 * dt * rate(z)
        z = brentq(lambda zz: zz + 0.5 * dt * rate(zz) - rhs, 0.0, z, xtol=1e-16, rtol=1e-15)
        U = r.moments()
        assert np.allclose(U[4], z, rtol=1e-13, atol=0)
        assert np.allclose(U[3], E, rtol=1e-14)
        assert np.allclose(U[1:3], 0.0, atol=1e-14)
    assert z < 0.85 * rho * Y  # the reaction really ran


# ---------------------------------------------------------------------------
# conservation and stability
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("system", [W.EULER, W.SWE, W.ADVECTION, W.REACTIVE])
def test_periodic_conservation(system):
    kw = dict(gamma=1.2, q=5.0, K=0.0) if system == W.REACTIVE else {}
    pb = W.Problem(system=system, dim=2, nx=24, ny=20, y1=20 / 24, adv=(0.6, -0.3), cfl=0.9, **kw)
    U0 = W.random_state(pb, seed=5)
    r = oracle.Run(pb, U0)
    tot0 = U0.reshape(pb.nfields, -1).sum(axis=1)
    r.step(40)
    assert r.flags == 0
    tot = r.moments().reshape(pb.nfields, -1).sum(axis=1)
    scale = np.abs(U0).reshape(pb.nfields, -1).sum(axis=1)
    assert np.all(np.abs(tot - tot0) <= 1e-13 * scale), (tot - tot0) / scale


def test_bed_source_conserves_mass():
    pb, U0 = W.bump_lake(24)
    r = oracle.Run(pb, U0)
    r.step(30)
    assert abs(r.moments()[0].sum() - U0[0].sum()) <= 1e-13 * U0[0].sum()


def weighted_norm_sq(pb, f, alpha, lam):
    """||f||_P^2 = sum_x sum_k f_k^T A0 (a_k I + sum_j b_kj A_j)^{-1} f_k with A0 = I
    (Section 4); a_k, b_kj of the LF-type equilibrium (2.20)."""
    d, m = pb.dim, pb.m_linear
    A = np.asarray(pb.A)
    total = 0.0
    for k in range(2 * d + 1):
        if k == 0:
            Ek = (1.0 - sum(alpha) / lam) * np.eye(m)
        else:
            j = (k - 1) % d
            sgn = 1.0 if k <= d else -1.0
            Ek = alpha[j] / (2 * lam) * np.eye(m) + sgn / (2 * lam) * A[j]
        Winv = np.linalg.inv(Ek)
        fk = f[k].reshape(m, -1)
        total += float(np.einsum("in,ij,jn->", fk, Winv, fk))
    return total


@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("cfl", [0.3, 0.9])
def test_theorem_4_2_weighted_norm_non_increasing(dim, cfl):
    # Theorem 4.3 admits 0 < eps < (1/d)(1/CFL - 1) sum_j abar_j; take half of that
    # bound so that the weights (a_k I + sum_j b_kj A_j)^{-1} stay well conditioned
    # (eps = 1e-10 makes one of them ~1e10 and the norm pure rounding noise).
    n = 64 if dim == 1 else 24
    pb, U0 = W.acoustics_random(n, dim=dim, cfl=cfl, seed=7)
    A = np.asarray(pb.A)
    abar = [np.abs(np.linalg.eigvalsh(A[j])).max() for j in range(dim)]
    pb = pb.with_(eps=0.5 * (1.0 / dim) * (1.0 / cfl - 1.0) * sum(abar))
    r = oracle.Run(pb, U0)
    alpha = [a + pb.eps for a in abar]
    lam = sum(abar) / cfl
    prev = weighted_norm_sq(pb, r.f, alpha, r.info[3])
    assert r.info[3] == pytest.approx(lam, rel=1e-14)
    for _ in range(60):
        r.step(1)
        now = weighted_norm_sq(pb, r.f, alpha, r.info[3])
        assert now <= prev * (1 + 1e-13)
        prev = now


def test_omega_range_and_smooth_limit():
    """omega in (1, 2]; on smooth data max(2 - omega) shrinks ~ linearly with dx."""
    gaps = []
    for N in (100, 200, 400):
        pb, U0 = W.entropy_wave_1d(N)
        r = oracle.Run(pb, U0).step(1, want_omega=True)
        om = r.omega
        assert np.all(om > 1.0) and np.all(om <= 2.0)
        gaps.append(float(np.max(2.0 - om)))
    assert gaps[0] / gaps[1] > 1.7 and gaps[1] / gaps[2] > 1.7
    pb, U0 = W.advection_1d(200, "pulse")
    r = oracle.Run(pb, U0).step(1, want_omega=True)
    assert r.omega.min() < 1.25 and np.median(r.omega) > 1.99


def run_until(pb, U0, T):
    r = oracle.Run(pb, U0)
    while r.t < T:
        r.step(1)
    return r


@pytest.mark.parametrize("which", ["sod", "lax"])
def test_shock_tube_converges_to_exact_riemann_solution(which):
    make, T, left, right, bound = {
        "sod": (W.sod, 0.2, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0.008),
        "lax": (W.lax, 0.14, (0.445, 0.698, 3.528), (0.5, 0.0, 0.571), 0.02),
    }[which]
    errs = []
    for N in (150, 300, 600):
        pb, U0 = make(N)
        r = run_until(pb, U0, T)
        assert r.flags == 0
        X, _ = W.cell_centres(pb)
        rho_ex, u_ex, p_ex = riemann_profile(left, right, X[0], r.t)
        U = r.moments()[:, 0, :]
        errs.append(np.mean(np.abs(U[0] - rho_ex)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < bound


def test_dry_bed_dam_break_converges_to_ritter():
    errs = []
    for N in (150, 300, 600):
        pb, U0 = W.dry_dam_break_1d(N)
        r = run_until(pb, U0, 0.15)
        X, _ = W.cell_centres(pb)
        h_ex, _u = ritter(X[0], r.t)
        h = r.moments()[0, 0]
        assert h.min() > -1e-12
        errs.append(np.mean(np.abs(h - h_ex)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.01


def test_dry_threshold_keeps_front_speeds_physical():
    """Wet-dry dam break over the bump (reading A10): with the dry threshold
    1e-5 the speed bound stays at the physical front speed, and a perturbation
    at FP32 rounding level (1e-7) barely moves the depth."""
    pb, U0 = W.dam_break_bump(96)
    rng = np.random.default_rng(0)
    U1 = U0 * (1 + 1e-7 * rng.standard_normal(U0.shape))
    a, b = oracle.Run(pb, U0), oracle.Run(pb, U1)
    amax = 0.0
    while a.t < 0.1:
        a.step(1)
        amax = max(amax, a.info[0], a.info[1])
    while b.t < 0.1:
        b.step(1)
    assert amax < 6.0  # 2 sqrt(g h0) = 6.26 bounds the dry-bed front speed
    Ua, Ub = a.moments(), b.moments()
    l1_h = np.abs(Ua[0] - Ub[0]).sum() / np.abs(Ua[0]).sum()
    assert l1_h < 1e-5


def test_reflective_wall_equals_mirrored_full_domain():
    """A reflecting wall at y = 0 gives the upper half of the solution on the
    doubled domain whose initial data are the mirror image (v -> -v) below y = 0."""
    n = 12
    half = W.Problem(system=W.EULER, dim=2, nx=n, ny=n // 2, x0=0.0, x1=1.0, y0=0.0, y1=0.5, cfl=0.8,
                     bc=(W.PERIODIC, W.PERIODIC, W.REFLECT, W.OUTFLOW))
    full = half.with_(ny=n, y0=-0.5, bc=(W.PERIODIC, W.PERIODIC, W.OUTFLOW, W.OUTFLOW))
    Uh = W.random_state(half, seed=21)
    lower = Uh[:, ::-1, :].copy()
    lower[2] = -lower[2]
    Uf = np.concatenate([lower, Uh], axis=1)
    rh, rf = oracle.Run(half, Uh), oracle.Run(full, Uf)
    for _ in range(6):
        rh.step(1)
        rf.step(1)
        assert rh.info[2] == pytest.approx(rf.info[2], rel=1e-14)
    a, b = rh.moments(), rf.moments()[:, n // 2:, :]
    scale = np.abs(b).reshape(4, -1).max(axis=1)
    assert np.all(np.abs(a - b).reshape(4, -1).max(axis=1) <= 1e-12 * scale)


def test_sponge_blends_omega_toward_one():
    """omega' = 1 + (omega - 1)(1 - sigma(x)) with sigma = (1 + cos(pi x / L))/2
    on the sponge [x0, x0 + L]; unchanged beyond it."""
    pb = W.Problem(system=W.EULER, dim=1, nx=64, x0=0.0, x1=1.0, cfl=0.8, bc=(W.OUTFLOW,) * 4)
    U0 = W.random_state(pb, seed=4)
    f1 = oracle.Run(pb, U0).step(2).f  # a state off equilibrium; both runs step from it
    a = oracle.Run(pb, U0)
    a.f[...] = f1
    b = oracle.Run(pb.with_(sponge_width=0.25), U0)
    b.f[...] = f1
    a.step(1, want_omega=True)
    b.step(1, want_omega=True)
    x = (np.arange(64) + 0.5) / 64
    sigma = np.where(x < 0.25, 0.5 * (1 + np.cos(np.pi * x / 0.25)), 0.0)
    assert np.allclose(b.omega.ravel(), 1 + (a.omega.ravel() - 1) * (1 - sigma), rtol=0, atol=1e-14)
    assert np.array_equal(b.omega.ravel()[x >= 0.25], a.omega.ravel()[x >= 0.25])


def test_znd_profile_of_example_5_13():
    """The ZND generator of Example 5.13's initial data: (a) at the printed
    D_CJ the flow leaves the reaction zone sonic (Mach 1 at Y = 0 in the shock
    frame), (b) the states satisfy the three flux conservations, (c) the
    Rankine-Hugoniot von Neumann state is the strong shock of the upstream
    state, and (d) with the printed K the half-reaction length of the f = 1.1
    overdriven detonation is 1 (the normalisation K was chosen for)."""
    c = W.DETONATION_5_13
    g, q = c["gamma"], c["q"]
    Dcj = W.d_cj(g, q)
    rho, u, p, disc = W.znd_state(0.0, Dcj, g, q)
    assert abs(u) / np.sqrt(g * p / rho) == pytest.approx(1.0, abs=1e-6)
    D = np.sqrt(1.1) * Dcj
    Y = np.linspace(0.0, 1.0, 11)
    rho, u, p, disc = W.znd_state(Y, D, g, q)
    assert np.allclose(rho * u, -D, rtol=1e-13)
    assert np.allclose(p + rho * u * u, 1.0 + D * D, rtol=1e-13)
    assert np.allclose(g / (g - 1) * p / rho + 0.5 * u * u + q * Y, g / (g - 1) + 0.5 * D * D + q, rtol=1e-13)
    # normal-shock relations at Y = 1 (no reaction yet): rho2/rho1 = (g+1)M^2 / ((g-1)M^2 + 2)
    M2 = D * D / g
    assert rho[-1] == pytest.approx((g + 1) * M2 / ((g - 1) * M2 + 2), rel=1e-12)
    assert np.all(disc > 0)
    xi = np.linspace(0.0, 3.0, 3001)
    Yx = W.znd_profile(xi, D, g, q, c["Ti"], c["K"])
    half = np.interp(0.5, Yx[::-1], xi[::-1])
    assert half == pytest.approx(1.0, abs=2e-3)


def test_cellular_detonation_initial_data():
    pb, U0 = W.cellular_detonation(nx=120, ny=90)
    assert pb.bc == (W.OUTFLOW, W.INFLOW, W.REFLECT, W.REFLECT) and pb.sponge_width == 6.0
    assert pb.dx == pytest.approx(1.0 / 3.0) and pb.u_in[0] == 1.0 and pb.u_in[4] == 1.0
    X, Yc = W.cell_centres(pb)
    ahead = X > 30.0
    assert np.allclose(U0[0][ahead], 1.0) and np.allclose(U0[4][ahead], 1.0)
    Yf = U0[4] / U0[0]
    assert np.all(Yf[~ahead] < 1.0) and np.all(Yf >= 0.0)
    strip = (X >= 29.0) & (X <= 30.0)
    assert np.abs(U0[2][strip]).max() > 0 and np.all(U0[2][~strip] == 0.0)



# ---------------------------------------------------------------------------
# 3D (D3Q7)
# ---------------------------------------------------------------------------

def test_uniform_reactive_state_is_trapezoidal_rule_3d():
    pb = W.cube(W.REACTIVE, 4, gamma=1.2, q=50.0, Ti=20.0, K=30.0, cfl=0.9)
    rho, p, Y = 1.0, 12.0, 0.9
    U0 = W.euler_conservative(pb, np.full((4, 4, 4), rho), 0.0, p, v=0.0, w=0.0, Y=Y)
    r = oracle.Run(pb, U0)
    z, E = rho * Y, U0[4, 0, 0, 0]

    def rate(zz):
        T = (pb.gamma - 1) * (E - pb.q * zz) / rho / rho
        return pb.K * zz * math.exp(-pb.Ti / T)

    for _ in range(10):
        r.step(1)
        dt = r.info[2]
        rhs = z - 0.5 * dt * rate(z)
        z = brentq(lambda zz: zz + 0.5 * dt * rate(zz) - rhs, 0.0, z, xtol=1e-16, rtol=1e-15)
        U = r.moments()
        assert np.allclose(U[5], z, rtol=1e-13, atol=0)
        assert np.allclose(U[1:4], 0.0, atol=1e-14)
    assert z < 0.9 * rho * Y


@pytest.mark.parametrize("system", [W.EULER, W.ADVECTION, W.REACTIVE])
def test_periodic_conservation_3d(system):
    kw = dict(gamma=1.2, q=5.0, K=0.0) if system == W.REACTIVE else {}
    pb = W.cube(system, 10, adv=(0.6, -0.3, 0.45), cfl=0.9, **kw)
    U0 = W.random_state(pb, seed=5)
    r = oracle.Run(pb, U0)
    tot0 = U0.reshape(pb.nfields, -1).sum(axis=1)
    r.step(15)
    assert r.flags == 0
    tot = r.moments().reshape(pb.nfields, -1).sum(axis=1)
    scale = np.abs(U0).reshape(pb.nfields, -1).sum(axis=1)
    assert np.all(np.abs(tot - tot0) <= 1e-13 * scale), (tot - tot0) / scale


@pytest.mark.parametrize("system", [W.EULER, W.REACTIVE])
def test_axes_are_interchangeable_3d(system):
    """Cycling the axes (x, y, z) -> (y, z, x) of the data and of the velocity
    components cycles the solution: every direction is treated alike (a wrong
    stride, index or eigenvector along one axis would break this)."""
    kw = dict(gamma=1.2, q=5.0, K=40.0, Ti=2.0) if system == W.REACTIVE else {}
    pb = W.Problem(system=system, dim=3, nx=9, ny=9, nz=9, bc=(W.OUTFLOW,) * 4, bc_z=(W.OUTFLOW, W.OUTFLOW),
                   cfl=0.8, **kw)
    U0 = W.random_state(pb, seed=17)

    def cycle(U):
        # new (x, y, z) = old (y, z, x): array axes (z, y, x) -> (x, z, y); momenta follow
        V = np.transpose(U, (0, 3, 1, 2)).copy()
        V[[1, 2, 3]] = V[[2, 3, 1]]
        return V

    a = oracle.Run(pb, U0).step(8)
    b = oracle.Run(pb, cycle(U0)).step(8)
    Ua, Ub = cycle(a.moments()), b.moments()
    scale = np.abs(Ub).reshape(pb.nfields, -1).max(axis=1)
    assert np.all(np.abs(Ua - Ub).reshape(pb.nfields, -1).max(axis=1) <= 1e-12 * scale)
