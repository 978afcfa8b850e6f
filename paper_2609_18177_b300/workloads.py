"""Problem descriptions and seeded synthetic initial data.

This module holds no arithmetic of the lattice Boltzmann method: it states the
balance law to solve (system, domain, boundary conditions, CFL, physical
constants) and builds the initial conservative state U0[m][ny][nx] in FP64 for
the paper's test problems (Section 5) and for the seeded workloads derived from
them.  Both the CUDA path and the CPU oracle consume what it returns.

Nodes sit at cell centres x_i = x0 + (i + 1/2) dx of a uniform mesh.
"""
from dataclasses import dataclass, field, replace
from typing import Optional, Tuple

import numpy as np

ADVECTION, EULER, SWE, REACTIVE, LINEAR = 0, 1, 2, 3, 4
PERIODIC, OUTFLOW, REFLECT, INFLOW = 0, 1, 2, 3
SYSTEM_NAMES = {ADVECTION: "advection", EULER: "euler", SWE: "shallow_water",
                REACTIVE: "reactive_euler", LINEAR: "linear"}


@dataclass
class Problem:
    """Balance law (2.1) on a DdQ(2d+1) lattice; names follow the C ABI struct."""
    system: int
    dim: int
    nx: int
    ny: int = 1
    x0: float = 0.0
    x1: float = 1.0
    y0: float = 0.0
    y1: float = 1.0
    bc: Tuple[int, int, int, int] = (PERIODIC, PERIODIC, PERIODIC, PERIODIC)
    cfl: float = 0.5
    eps: float = 1e-10            # Section 5: epsilon = 1e-10 in all examples
    adv: Tuple[float, float] = (1.0, 0.0)
    gamma: float = 1.4
    g: float = 9.81
    bed_amp: float = 0.0
    bed_w2: float = 1.0
    bed_xc: float = 0.0
    bed_yc: float = 0.0
    K: float = 0.0
    Ti: float = 0.0
    q: float = 0.0
    m_linear: int = 0
    A: Optional[np.ndarray] = None
    omega_mode: int = 0           # 0: adaptive (2.12)/(2.16); 1: fixed omega_fixed
    omega_fixed: float = 1.0
    h_dry: float = 1e-5           # depth below which a node is dry (u = v = 0)
    nz: int = 1                   # 3D (D3Q7): nodes, extent and boundaries in z
    z0: float = 0.0
    z1: float = 1.0
    bc_z: Tuple[int, int] = (PERIODIC, PERIODIC)
    sponge_width: float = 0.0     # > 0: sponge layer of this width at x-lo (omega blended toward 1)
    u_in: Tuple[float, ...] = ()  # conservative state held by inflow ghost nodes
    precision: int = 0            # 0: FP64, 1: FP32 distributions (CUDA path only)

    @property
    def nfields(self) -> int:
        if self.system == ADVECTION:
            return 1
        if self.system == EULER:
            return self.dim + 2
        if self.system == SWE:
            return self.dim + 1
        if self.system == REACTIVE:
            return self.dim + 3
        return self.m_linear

    @property
    def nvel(self) -> int:
        return 2 * self.dim + 1

    @property
    def dx(self) -> float:
        return (self.x1 - self.x0) / self.nx

    @property
    def nodes(self) -> int:
        return self.nx * (self.ny if self.dim >= 2 else 1) * (self.nz if self.dim == 3 else 1)

    def shape(self):
        if self.dim == 3:
            return (self.nz, self.ny, self.nx)
        return (self.ny, self.nx) if self.dim == 2 else (1, self.nx)

    def with_(self, **kw) -> "Problem":
        return replace(self, **kw)


def cell_centres_3d(pb: Problem):
    """X, Y, Z node coordinates of a 3D lattice, shape (nz, ny, nx)."""
    h = pb.dx
    x = pb.x0 + (np.arange(pb.nx) + 0.5) * h
    y = pb.y0 + (np.arange(pb.ny) + 0.5) * h
    z = pb.z0 + (np.arange(pb.nz) + 0.5) * h
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def cell_centres(pb: Problem):
    x = pb.x0 + (np.arange(pb.nx) + 0.5) * pb.dx
    if pb.dim == 1:
        return x[None, :], np.zeros((1, pb.nx))
    dy = (pb.y1 - pb.y0) / pb.ny
    y = pb.y0 + (np.arange(pb.ny) + 0.5) * dy
    X, Y = np.meshgrid(x, y)
    return X, Y


# --------------------------------------------------------------------------
# primitive -> conservative (the definitions of U in Section 5)
# --------------------------------------------------------------------------

def euler_conservative(pb, rho, u, p, v=None, Y=None, w=None):
    rho = np.asarray(rho, dtype=np.float64)
    shp = rho.shape
    u = np.broadcast_to(np.asarray(u, dtype=np.float64), shp)
    p = np.broadcast_to(np.asarray(p, dtype=np.float64), shp)
    v = np.zeros(shp) if v is None else np.broadcast_to(np.asarray(v, dtype=np.float64), shp)
    w = np.zeros(shp) if w is None else np.broadcast_to(np.asarray(w, dtype=np.float64), shp)
    comps = [rho, rho * u]
    if pb.dim >= 2:
        comps.append(rho * v)
    if pb.dim == 3:
        comps.append(rho * w)
    E = p / (pb.gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    if pb.system == REACTIVE:
        Yv = np.broadcast_to(np.asarray(Y, dtype=np.float64), shp)
        E = E + rho * pb.q * Yv
        comps.append(E)
        comps.append(rho * Yv)
    else:
        comps.append(E)
    return np.stack(comps).astype(np.float64)


def swe_conservative(pb, h, u, v=None):
    h = np.asarray(h, dtype=np.float64)
    shp = h.shape
    u = np.broadcast_to(np.asarray(u, dtype=np.float64), shp)
    comps = [h, h * u]
    if pb.dim == 2:
        v = np.zeros(shp) if v is None else np.broadcast_to(np.asarray(v, dtype=np.float64), shp)
        comps.append(h * v)
    return np.stack(comps).astype(np.float64)


# --------------------------------------------------------------------------
# Section 5.1: linear advection
# --------------------------------------------------------------------------

def advection_1d(nx, profile="sine", cfl=0.5, pulse=(0.3, 0.5)):
    """u_t + u_x = 0 on [0,1], periodic.  profile 'sine': sin(2 pi x) (Example 5.1);
    'pulse': 1 on the closed interval `pulse`, else 0 (Example 5.2's square wave)."""
    pb = Problem(system=ADVECTION, dim=1, nx=nx, x0=0.0, x1=1.0, cfl=cfl, adv=(1.0, 0.0))
    X, _ = cell_centres(pb)
    if profile == "sine":
        u = np.sin(2 * np.pi * X)
    else:
        u = ((X >= pulse[0]) & (X <= pulse[1])).astype(np.float64)
    return pb, u[None, :, :]


def advection_2d(n, cfl=0.5, adv=(1.0, 0.5), seed=0):
    """2D advection of a smooth bump plus a square, periodic on [0,1]^2."""
    pb = Problem(system=ADVECTION, dim=2, nx=n, ny=n, cfl=cfl, adv=adv)
    X, Y = cell_centres(pb)
    rng = np.random.default_rng(seed)
    cx, cy = rng.uniform(0.3, 0.7, 2)
    u = np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / 0.01)
    u = u + ((np.abs(X - 0.25) < 0.1) & (np.abs(Y - 0.7) < 0.1))
    return pb, u[None]


# --------------------------------------------------------------------------
# Section 5.2: Euler
# --------------------------------------------------------------------------

def entropy_wave_1d(nx, cfl=0.6):
    """Example 5.3: rho = 1 + 0.2 sin(2 pi x), u = 1, p = 1, periodic on [0,1]."""
    pb = Problem(system=EULER, dim=1, nx=nx, cfl=cfl, gamma=1.4)
    X, _ = cell_centres(pb)
    return pb, euler_conservative(pb, 1.0 + 0.2 * np.sin(2 * np.pi * X), 1.0, 1.0)


def entropy_wave_2d(n, cfl=0.3):
    """Example 5.4: rho = 1 + 0.2 sin(2 pi (x+y)), u = v = p = 1, periodic on [0,1]^2."""
    pb = Problem(system=EULER, dim=2, nx=n, ny=n, cfl=cfl, gamma=1.4)
    X, Y = cell_centres(pb)
    return pb, euler_conservative(pb, 1.0 + 0.2 * np.sin(2 * np.pi * (X + Y)), 1.0, 1.0, v=1.0)


def shock_tube(nx, left, right, x0=0.0, x1=1.0, xs=0.5, cfl=0.3, gamma=1.4):
    """1D Riemann problem with primitive states (rho, u, p), transmissive BCs."""
    pb = Problem(system=EULER, dim=1, nx=nx, x0=x0, x1=x1, cfl=cfl, gamma=gamma,
                 bc=(OUTFLOW, OUTFLOW, OUTFLOW, OUTFLOW))
    X, _ = cell_centres(pb)
    L = X <= xs
    rho = np.where(L, left[0], right[0])
    u = np.where(L, left[1], right[1])
    p = np.where(L, left[2], right[2])
    return pb, euler_conservative(pb, rho, u, p)


def sod(nx, cfl=0.3):
    """Example 5.6 (Table 5.4 states), T = 0.2."""
    return shock_tube(nx, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), cfl=cfl)


def lax(nx, cfl=0.3):
    """Example 5.5 (Table 5.4 states), T = 0.14."""
    return shock_tube(nx, (0.445, 0.698, 3.528), (0.5, 0.0, 0.571), cfl=cfl)


def shu_osher(nx, cfl=0.3, xs=-4.0):
    """Example 5.7 on [-5,5], T = 1.8; interface at x = -4 (the paper gives only the states)."""
    pb = Problem(system=EULER, dim=1, nx=nx, x0=-5.0, x1=5.0, cfl=cfl, gamma=1.4,
                 bc=(OUTFLOW, OUTFLOW, OUTFLOW, OUTFLOW))
    X, _ = cell_centres(pb)
    L = X < xs
    rho = np.where(L, 3.857143, 1.0 + 0.2 * np.sin(5.0 * X))
    u = np.where(L, 2.629369, 0.0)
    p = np.where(L, 10.33333, 1.0)
    return pb, euler_conservative(pb, rho, u, p)


def riemann_2d(n, states, cfl=0.9, split=(0.5, 0.5)):
    """Four-quadrant 2D Riemann problem on [0,1]^2 with zero-gradient BCs.
    states: dict with keys 'ne','nw','sw','se' -> (rho, u, v, p)."""
    pb = Problem(system=EULER, dim=2, nx=n, ny=n, cfl=cfl, gamma=1.4,
                 bc=(OUTFLOW, OUTFLOW, OUTFLOW, OUTFLOW))
    X, Y = cell_centres(pb)
    E = X > split[0]
    N = Y > split[1]
    quads = {"ne": E & N, "nw": ~E & N, "sw": ~E & ~N, "se": E & ~N}
    rho = np.zeros(X.shape); u = np.zeros(X.shape); v = np.zeros(X.shape); p = np.zeros(X.shape)
    for key, mask in quads.items():
        r, uu, vv, pp = states[key]
        rho[mask], u[mask], v[mask], p[mask] = r, uu, vv, pp
    return pb, euler_conservative(pb, rho, u, p, v=v)


LAX_LIU_CONFIG4 = {  # Example 5.8
    "ne": (1.1, 0.0, 0.0, 1.1),
    "nw": (0.5065, 0.8939, 0.0, 0.35),
    "sw": (1.1, 0.8939, 0.8939, 1.1),
    "se": (0.5065, 0.0, 0.8939, 0.35),
}


def seeded_quadrant_states(seed):
    """Quadrant states drawn from a seed: rho in [0.1,1.5], |u|,|v| <= 1.2, p in [0.03,1.5]."""
    rng = np.random.default_rng(seed)
    out = {}
    for key in ("ne", "nw", "sw", "se"):
        rho = rng.uniform(0.1, 1.5)
        u, v = rng.uniform(-1.2, 1.2, 2)
        p = rng.uniform(0.03, 1.5)
        out[key] = (float(rho), float(u), float(v), float(p))
    return out


def riemann_2d_seeded(n, seed=0, cfl=0.9):
    return riemann_2d(n, seeded_quadrant_states(seed), cfl=cfl)


# --------------------------------------------------------------------------
# Section 5.3: shallow water (g = 9.81)
# --------------------------------------------------------------------------

def dry_dam_break_1d(nx, cfl=0.9):
    """Example 5.9: (h,u) = (2,0) for x <= 0, (0,0) otherwise on [-1,1], T = 0.15."""
    pb = Problem(system=SWE, dim=1, nx=nx, x0=-1.0, x1=1.0, cfl=cfl, g=9.81,
                 bc=(OUTFLOW, OUTFLOW, OUTFLOW, OUTFLOW))
    X, _ = cell_centres(pb)
    return pb, swe_conservative(pb, np.where(X <= 0.0, 2.0, 0.0), 0.0)


def circular_dam_break(n, cfl=0.4):
    """Example 5.10: h = 2 for r <= 0.5 else 1 on [-1,1]^2, T = 0.07."""
    pb = Problem(system=SWE, dim=2, nx=n, ny=n, x0=-1, x1=1, y0=-1, y1=1, cfl=cfl, g=9.81,
                 bc=(OUTFLOW,) * 4)
    X, Y = cell_centres(pb)
    h = np.where(X * X + Y * Y <= 0.25, 2.0, 1.0)
    return pb, swe_conservative(pb, h, 0.0, 0.0)


def dam_break_bump(n, cfl=0.4, dam_x=-0.5):
    """Wet-dry dam break over a Gaussian bump b = 0.8 exp(-r^2/0.02) on [-1,1]^2:
    h = 1 upstream of x = dam_x, dry (h = 0) downstream, at rest; outflow BCs."""
    pb = Problem(system=SWE, dim=2, nx=n, ny=n, x0=-1, x1=1, y0=-1, y1=1, cfl=cfl, g=9.81,
                 bc=(OUTFLOW,) * 4, bed_amp=0.8, bed_w2=0.02, bed_xc=0.0, bed_yc=0.0)
    X, Y = cell_centres(pb)
    h = np.where(X < dam_x, 1.0, 0.0)
    return pb, swe_conservative(pb, h, 0.0, 0.0)


def bump_lake(n, cfl=0.4, seed=0):
    """Small smooth depth perturbation over the bump (wet everywhere), periodic."""
    pb = Problem(system=SWE, dim=2, nx=n, ny=n, x0=-1, x1=1, y0=-1, y1=1, cfl=cfl, g=9.81,
                 bed_amp=0.3, bed_w2=0.05)
    X, Y = cell_centres(pb)
    rng = np.random.default_rng(seed)
    cx, cy = rng.uniform(-0.3, 0.3, 2)
    h = 1.0 + 0.1 * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / 0.02)
    return pb, swe_conservative(pb, h, 0.1, -0.05)


# --------------------------------------------------------------------------
# Section 5.4: reactive Euler, one-step Arrhenius kinetics
# --------------------------------------------------------------------------

def reactive_circle(n, gamma=1.2, K=2566.4, Ti=50.0, q=50.0, cfl=0.9):
    """Example 5.12: (rho,u,v,p,Y) = (1,0,0,80,0.2) inside r^2 <= 0.36, (1,0,0,10,0.8)
    outside, on [-1,1]^2, transmissive BCs, T = 0.04."""
    pb = Problem(system=REACTIVE, dim=2, nx=n, ny=n, x0=-1, x1=1, y0=-1, y1=1, cfl=cfl,
                 gamma=gamma, K=K, Ti=Ti, q=q, bc=(OUTFLOW,) * 4)
    X, Y = cell_centres(pb)
    inside = X * X + Y * Y <= 0.36
    p = np.where(inside, 80.0, 10.0)
    Yf = np.where(inside, 0.2, 0.8)
    return pb, euler_conservative(pb, np.ones(X.shape), 0.0, p, v=0.0, Y=Yf)


def detonation_1d(nx=None, dx=1.0 / 150, L=100.0, cfl=0.9):
    """Example 5.11 initial data on [0, L] (K = 145.68913, Ti = 50, q = 50, gamma = 1.4)."""
    if nx is None:
        nx = int(round(L / dx))
    pb = Problem(system=REACTIVE, dim=1, nx=nx, x0=0.0, x1=L, cfl=cfl, gamma=1.4,
                 K=145.68913, Ti=50.0, q=50.0, bc=(OUTFLOW,) * 4)
    X, _ = cell_centres(pb)
    left = X < 2.0
    rho = np.where(left, 2.5706, 1.0)
    u = np.where(left, 6.86089, 0.0)
    p = np.where(left, 80.02055, 1.0)
    Yf = np.where(left, 0.0, 1.0)
    return pb, euler_conservative(pb, rho, u, p, Y=Yf)


def d_cj(gamma, q):
    """Chapman-Jouguet detonation speed of Example 5.13 (upstream rho = p = 1)."""
    a = (gamma * gamma - 1.0) * q
    return float(np.sqrt(gamma + a + np.sqrt(a * (2.0 * gamma + a))))


def znd_state(Y, D, gamma, q):
    """Steady 1D ZND state at reaction progress Y behind a shock moving at D
    into (rho, u, p, Y) = (1, 0, 1, 1), in the shock-attached frame where the
    upstream gas arrives with u = -D: mass, momentum and energy fluxes equal
    the upstream ones, and of the two specific volumes they allow the shocked
    (smaller) one is taken.  Returns rho, u, p and the discriminant of the
    quadratic for the specific volume (zero at a sonic point)."""
    m = -D
    P = 1.0 + D * D
    H = gamma / (gamma - 1.0) + 0.5 * D * D + q
    a = m * m * (gamma + 1.0) / (2.0 * (gamma - 1.0))
    b = gamma * P / (gamma - 1.0)
    c = H - q * np.asarray(Y, dtype=np.float64)
    disc = b * b - 4.0 * a * c
    V = (b - np.sqrt(np.maximum(disc, 0.0))) / (2.0 * a)
    return 1.0 / V, m * V, P - m * m * V, disc


def znd_profile(xi, D, gamma, q, Ti, K):
    """Reaction progress Y at distances xi >= 0 behind the shock: the steady
    rate equation u dY/dx = -K Y exp(-Ti/T), T = p/rho, integrated from Y = 1
    at the shock (scipy LSODA, rtol 1e-10)."""
    from scipy.integrate import solve_ivp

    def rhs(_x, y):
        rho, u, p, _d = znd_state(y[0], D, gamma, q)
        return [K * y[0] * np.exp(-Ti * rho / p) / u]

    xi = np.asarray(xi, dtype=np.float64)
    top = float(xi.max()) if xi.size else 0.0
    if top <= 0.0:
        return np.ones_like(xi)
    sol = solve_ivp(rhs, [0.0, top], [1.0], method="LSODA", rtol=1e-10, atol=1e-14, dense_output=True)
    return np.clip(sol.sol(np.clip(xi, 0.0, top))[0], 0.0, 1.0)


DETONATION_5_13 = dict(gamma=1.2, q=2.0, Ti=20.0, K=1.13436364e6)


def cellular_detonation(nx=1200, ny=900, overdrive=1.1, k=6, x_front=30.0, cfl=0.3, sponge=6.0):
    """Example 5.13: [0,40] x [-15,15] (1200 x 900 nodes, dx = 1/30 at full
    size), gamma = 1.2, q = 2, Ti = 20, K = 1.13436364e6, shock-attached frame
    moving at D = sqrt(overdrive) D_CJ.  Unreacted (1, -D, 0, 1, 1) ahead of
    the front at x_front, the ZND profile behind it, v = 0.1 sin(2 pi k y / 30)
    in x_front - 1 <= x <= x_front.  Reflecting walls at y = +-15, fixed
    inflow of the unreacted state at x = 40, zero-gradient outflow at x = 0
    with a sponge over 0 <= x <= sponge."""
    c = DETONATION_5_13
    D = float(np.sqrt(overdrive)) * d_cj(c["gamma"], c["q"])
    pb = Problem(system=REACTIVE, dim=2, nx=nx, ny=ny, x0=0.0, x1=40.0, y0=-15.0, y1=15.0, cfl=cfl,
                 gamma=c["gamma"], K=c["K"], Ti=c["Ti"], q=c["q"], bc=(OUTFLOW, INFLOW, REFLECT, REFLECT),
                 sponge_width=sponge)
    unreacted = euler_conservative(pb, np.ones(1), -D, np.ones(1), v=0.0, Y=np.ones(1))[:, 0]
    pb = pb.with_(u_in=tuple(float(v) for v in unreacted))
    X, Yc = cell_centres(pb)
    xs = X[0]
    behind = xs <= x_front
    Yz = np.ones_like(xs)
    Yz[behind] = znd_profile(x_front - xs[behind], D, c["gamma"], c["q"], c["Ti"], c["K"])
    rho1, u1, p1, _d = znd_state(Yz, D, c["gamma"], c["q"])
    ones = np.ones_like(X)
    rho = np.where(behind, rho1, 1.0)[None, :] * ones
    u = np.where(behind, u1, -D)[None, :] * ones
    p = np.where(behind, p1, 1.0)[None, :] * ones
    Yf = np.where(behind, Yz, 1.0)[None, :] * ones
    v = np.where((X >= x_front - 1.0) & (X <= x_front), 0.1 * np.sin(2.0 * np.pi * k * Yc / 30.0), 0.0)
    return pb, euler_conservative(pb, rho, u, p, v=v, Y=Yf)


# --------------------------------------------------------------------------
# Section 4: linear symmetric systems (acoustics), oracle-side stability tests
# --------------------------------------------------------------------------

def acoustics_random(n, dim=1, a=1.0, cfl=0.9, seed=0, eps=1e-10):
    """u_t + A u_x = 0 with A = [[0,a],[a,0]] (symmetric, A0 = I); random discontinuous data."""
    A = np.zeros((dim, 2, 2))
    for j in range(dim):
        A[j] = [[0.0, a], [a, 0.0]] if j == 0 else [[0.0, 0.5 * a], [0.5 * a, 0.3 * a]]
    pb = Problem(system=LINEAR, dim=dim, nx=n, ny=n if dim == 2 else 1, cfl=cfl, m_linear=2,
                 A=A, eps=eps)
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((2,) + pb.shape())
    U[:, ..., : n // 3] += 2.0
    return pb, U


# --------------------------------------------------------------------------
# generic seeded states for parity tests
# --------------------------------------------------------------------------

def random_state(pb: Problem, seed=0, smooth=False):
    """Seeded physical state of any system: a smooth field plus (unless smooth)
    a few jumps, with positive density/pressure/depth."""
    if pb.dim == 3:
        return random_state_3d(pb, seed, smooth)
    rng = np.random.default_rng(seed)
    X, Y = cell_centres(pb)
    Lx = pb.x1 - pb.x0
    Ly = (pb.y1 - pb.y0) if pb.dim == 2 else 1.0
    xs = (X - pb.x0) / Lx
    ys = (Y - pb.y0) / Ly if pb.dim == 2 else np.zeros_like(X)

    def field_(lo, hi):
        k1, k2 = rng.integers(1, 4, 2)
        ph1, ph2 = rng.uniform(0, 2 * np.pi, 2)
        base = 0.5 + 0.25 * np.sin(2 * np.pi * k1 * xs + ph1) + 0.25 * np.cos(2 * np.pi * k2 * ys + ph2)
        if not smooth:
            cut = rng.uniform(0.3, 0.7)
            base = np.where(xs + 0.3 * ys > cut, base, 0.6 * base + 0.4 * rng.uniform())
        return lo + (hi - lo) * base

    if pb.system == ADVECTION:
        return field_(-1.0, 1.0)[None]
    if pb.system == LINEAR:
        return np.stack([field_(-1.0, 1.0) for _ in range(pb.m_linear)])
    if pb.system == SWE:
        return swe_conservative(pb, field_(0.5, 2.0), field_(-0.5, 0.5), field_(-0.5, 0.5))
    rho = field_(0.5, 2.0)
    u = field_(-0.8, 0.8)
    v = field_(-0.8, 0.8)
    p = field_(0.5, 2.0)
    Yf = field_(0.0, 1.0) if pb.system == REACTIVE else None
    return euler_conservative(pb, rho, u, p, v=v, Y=Yf)


def random_state_3d(pb: Problem, seed=0, smooth=False):
    """random_state on a 3D lattice (advection, Euler, reactive Euler)."""
    rng = np.random.default_rng(seed)
    X, Yc, Z = cell_centres_3d(pb)
    xs = (X - pb.x0) / (pb.x1 - pb.x0)
    ys = (Yc - pb.y0) / (pb.y1 - pb.y0)
    zs = (Z - pb.z0) / (pb.z1 - pb.z0)

    def field_(lo, hi):
        k = rng.integers(1, 4, 3)
        ph = rng.uniform(0, 2 * np.pi, 3)
        base = 0.5 + (np.sin(2 * np.pi * k[0] * xs + ph[0]) + np.cos(2 * np.pi * k[1] * ys + ph[1])
                      + np.sin(2 * np.pi * k[2] * zs + ph[2])) / 6.0
        if not smooth:
            cut = rng.uniform(0.3, 0.7)
            base = np.where(xs + 0.3 * ys + 0.2 * zs > cut, base, 0.6 * base + 0.4 * rng.uniform())
        return lo + (hi - lo) * base

    if pb.system == ADVECTION:
        return field_(-1.0, 1.0)[None]
    rho = field_(0.5, 2.0)
    u, v, w = field_(-0.8, 0.8), field_(-0.8, 0.8), field_(-0.8, 0.8)
    p = field_(0.5, 2.0)
    Yf = field_(0.0, 1.0) if pb.system == REACTIVE else None
    return euler_conservative(pb, rho, u, p, v=v, Y=Yf, w=w)


def cube(system, n, **kw):
    """A 3D (D3Q7) problem on [0,1]^3 with n^3 nodes."""
    return Problem(system=system, dim=3, nx=n, ny=n, nz=n, **kw)
