"""FP64 CPU oracle of the adaptive-relaxation Lax-Friedrichs-type LBM.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package smoke check and
by the CPU-baseline leg of the benchmark.  The product path (the CUDA library
and its Python binding) never imports this package, and this package imports
nothing from the product.

The arithmetic lives in ``lbm_oracle.c`` (plain C loops, FP64, no FP
contraction); this module only marshals numpy arrays through ctypes.  The
problem description is any object with the attributes listed in ``_FIELDS``
(the same names as the C ABI's problem struct).
"""
import ctypes
import os

import numpy as np

from . import build as _build

ADVECTION, EULER, SWE, REACTIVE, LINEAR = 0, 1, 2, 3, 4
PERIODIC, OUTFLOW, REFLECT, INFLOW = 0, 1, 2, 3
FLAG_NONPHYSICAL, FLAG_NOROOT = 1, 2


class _Problem(ctypes.Structure):
    _fields_ = [
        ("system", ctypes.c_int), ("dim", ctypes.c_int),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double),
        ("y0", ctypes.c_double), ("y1", ctypes.c_double),
        ("bc", ctypes.c_int * 4),
        ("nz", ctypes.c_int),
        ("z0", ctypes.c_double), ("z1", ctypes.c_double),
        ("bc_z", ctypes.c_int * 2),
        ("cfl", ctypes.c_double), ("eps", ctypes.c_double),
        ("adv", ctypes.c_double * 3),
        ("gamma", ctypes.c_double), ("g", ctypes.c_double),
        ("bed_amp", ctypes.c_double), ("bed_w2", ctypes.c_double),
        ("bed_xc", ctypes.c_double), ("bed_yc", ctypes.c_double),
        ("K", ctypes.c_double), ("Ti", ctypes.c_double), ("q", ctypes.c_double),
        ("m_linear", ctypes.c_int),
        ("A", ctypes.POINTER(ctypes.c_double)),
        ("omega_mode", ctypes.c_int), ("omega_fixed", ctypes.c_double),
        ("h_dry", ctypes.c_double),
        ("sponge_width", ctypes.c_double),
        ("u_in", ctypes.c_double * 8),
    ]


_lib = None


def use_native_build():
    """Load the copy of the oracle tuned for this machine's CPU (-march=native,
    built here on first use) instead of the portable one: for timing the
    oracle as a CPU baseline.  Must be called before any other oracle call."""
    global _lib
    if _lib is not None:
        raise RuntimeError("the oracle library is already loaded")
    _load(_build.build(native=True))


def set_threads(n):
    """OpenMP threads of the oracle's loops; returns the number in effect."""
    return lib().orc_set_threads(int(n))


def lib():
    if _lib is None:
        _load(_build.build())
    return _lib


def _load(path):
    global _lib
    L = ctypes.CDLL(path)
    P = ctypes.POINTER(_Problem)
    dp = ctypes.POINTER(ctypes.c_double)
    L.orc_nfields.argtypes = [P]
    L.orc_flux.argtypes = [P, ctypes.c_int, dp, dp]
    L.orc_flux.restype = None
    L.orc_eigvals.argtypes = [P, ctypes.c_int, dp, dp]
    L.orc_eigvals.restype = None
    L.orc_max_speed.argtypes = [P, ctypes.c_int, dp]
    L.orc_max_speed.restype = ctypes.c_double
    L.orc_right_eigvecs.argtypes = [P, ctypes.c_int, dp, dp]
    L.orc_right_eigvecs.restype = None
    L.orc_left_eigvecs.argtypes = [P, ctypes.c_int, dp, dp]
    L.orc_source.argtypes = [P, dp, ctypes.c_double, ctypes.c_double, dp]
    L.orc_source.restype = None
    L.orc_equilibrium.argtypes = [P, dp, dp, ctypes.c_double, dp]
    L.orc_equilibrium.restype = None
    L.orc_moments.argtypes = [P, dp, dp]
    L.orc_alpha_bar_U.argtypes = [P, dp, dp]
    L.orc_init.argtypes = [P, dp, dp, dp]
    L.orc_step.argtypes = [P, dp, dp, ctypes.c_double, dp, dp, dp]
    L.orc_advance.argtypes = [P, dp, dp, ctypes.c_double, ctypes.c_long,
                              ctypes.POINTER(ctypes.c_long)]
    L.orc_set_threads.argtypes = [ctypes.c_int]
    _lib = L


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c_problem(pb):
    """Build the C struct from a problem object (attribute names as in the C ABI)."""
    s = _Problem()
    s.system = int(pb.system)
    s.dim = int(pb.dim)
    s.nx = int(pb.nx)
    s.ny = int(pb.ny) if pb.dim >= 2 else 1
    s.nz = int(getattr(pb, "nz", 1)) if pb.dim == 3 else 1
    s.z0, s.z1 = float(getattr(pb, "z0", 0.0)), float(getattr(pb, "z1", 1.0))
    bz = tuple(getattr(pb, "bc_z", (PERIODIC, PERIODIC)))
    s.bc_z[0], s.bc_z[1] = int(bz[0]), int(bz[1])
    s.x0, s.x1, s.y0, s.y1 = float(pb.x0), float(pb.x1), float(pb.y0), float(pb.y1)
    for i in range(4):
        s.bc[i] = int(pb.bc[i])
    s.cfl, s.eps = float(pb.cfl), float(pb.eps)
    for i, v in enumerate(tuple(pb.adv)[:3]):
        s.adv[i] = float(v)
    s.gamma, s.g = float(pb.gamma), float(pb.g)
    s.bed_amp, s.bed_w2 = float(pb.bed_amp), float(pb.bed_w2)
    s.bed_xc, s.bed_yc = float(pb.bed_xc), float(pb.bed_yc)
    s.K, s.Ti, s.q = float(pb.K), float(pb.Ti), float(pb.q)
    s.m_linear = int(getattr(pb, "m_linear", 0))
    A = getattr(pb, "A", None)
    keep = None
    if A is not None:
        keep = np.ascontiguousarray(A, dtype=np.float64)
        s.A = _dp(keep)
    s.omega_mode = int(pb.omega_mode)
    s.omega_fixed = float(pb.omega_fixed)
    s.h_dry = float(pb.h_dry)
    s.sponge_width = float(getattr(pb, "sponge_width", 0.0))
    for i, v in enumerate(tuple(getattr(pb, "u_in", ()))[:8]):
        s.u_in[i] = float(v)
    return s, keep


def nfields(pb):
    s, _k = _c_problem(pb)
    return lib().orc_nfields(ctypes.byref(s))


def nq(pb):
    return 2 * pb.dim + 1


def grid_shape(pb):
    if pb.dim == 3:
        return (pb.nz, pb.ny, pb.nx)
    return (pb.ny, pb.nx) if pb.dim == 2 else (1, pb.nx)


def flux(pb, direction, U):
    s, _k = _c_problem(pb)
    U = np.ascontiguousarray(U, dtype=np.float64)
    F = np.zeros_like(U)
    lib().orc_flux(ctypes.byref(s), direction, _dp(U), _dp(F))
    return F


def eigvals(pb, direction, U):
    s, _k = _c_problem(pb)
    U = np.ascontiguousarray(U, dtype=np.float64)
    lam = np.zeros_like(U)
    lib().orc_eigvals(ctypes.byref(s), direction, _dp(U), _dp(lam))
    return lam


def max_speed(pb, direction, U):
    s, _k = _c_problem(pb)
    U = np.ascontiguousarray(U, dtype=np.float64)
    return lib().orc_max_speed(ctypes.byref(s), direction, _dp(U))


def right_eigvecs(pb, direction, U):
    s, _k = _c_problem(pb)
    U = np.ascontiguousarray(U, dtype=np.float64)
    m = U.size
    R = np.zeros((m, m))
    lib().orc_right_eigvecs(ctypes.byref(s), direction, _dp(U), _dp(R))
    return R


def left_eigvecs(pb, direction, U):
    s, _k = _c_problem(pb)
    U = np.ascontiguousarray(U, dtype=np.float64)
    m = U.size
    L = np.zeros((m, m))
    rc = lib().orc_left_eigvecs(ctypes.byref(s), direction, _dp(U), _dp(L))
    if rc != 0:
        raise ArithmeticError("singular eigenvector matrix")
    return L


def source(pb, U, x=0.0, y=0.0):
    s, _k = _c_problem(pb)
    U = np.ascontiguousarray(U, dtype=np.float64)
    S = np.zeros_like(U)
    lib().orc_source(ctypes.byref(s), _dp(U), float(x), float(y), _dp(S))
    return S


def equilibrium(pb, U, alpha, lam):
    """f^eq_k(U) for k = 0..2d, shape (Q, m)."""
    s, _k = _c_problem(pb)
    U = np.ascontiguousarray(U, dtype=np.float64)
    a = np.zeros(3)
    a[: len(alpha)] = alpha
    feq = np.zeros((nq(pb), U.size))
    lib().orc_equilibrium(ctypes.byref(s), _dp(U), _dp(a), float(lam), _dp(feq))
    return feq


def moments(pb, f):
    s, _k = _c_problem(pb)
    f = np.ascontiguousarray(f, dtype=np.float64)
    U = np.zeros((f.shape[1],) + f.shape[2:])
    _check(lib().orc_moments(ctypes.byref(s), _dp(f), _dp(U)))
    return U


def alpha_bar(pb, U):
    s, _k = _c_problem(pb)
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = np.zeros(3)
    _check(lib().orc_alpha_bar_U(ctypes.byref(s), _dp(U), _dp(out)))
    return out[: max(pb.dim, 2)]


def _check(rc):
    if rc < 0:
        raise ValueError(f"oracle error {rc}")
    return rc


class Run:
    """A solve held by the oracle: distributions f[k][c][(z)][y][x] and time t."""

    def __init__(self, pb, U0):
        self.pb = pb
        self._s, self._keep = _c_problem(pb)
        self.m = lib().orc_nfields(ctypes.byref(self._s))
        shp = grid_shape(pb)
        U0 = np.ascontiguousarray(np.asarray(U0, dtype=np.float64).reshape((self.m,) + shp))
        self.f = np.zeros((nq(pb), self.m) + shp)
        self.info = np.zeros(5)  # abar_x, abar_y, dt, lambda, abar_z
        _check(lib().orc_init(ctypes.byref(self._s), _dp(U0), _dp(self.f), _dp(self.info)))
        self.t = 0.0
        self.nsteps = 0
        self.flags = 0
        self.omega = None

    def step(self, n=1, T=None, want_omega=False, abar=None):
        """Take n steps (stopping early once t reaches T, the last step clipped)."""
        g = np.empty_like(self.f)
        om = np.zeros(grid_shape(self.pb)) if want_omega else None
        ab = None if abar is None else np.ascontiguousarray(np.asarray(abar, dtype=np.float64))
        for _ in range(n):
            if T is not None and self.t >= T:
                break
            cap = (T - self.t) if T is not None else 0.0
            rc = _check(lib().orc_step(ctypes.byref(self._s), _dp(self.f), _dp(g), cap,
                                       None if ab is None else _dp(ab), _dp(self.info),
                                       None if om is None else _dp(om)))
            self.flags |= rc
            self.f, g = g, self.f
            self.t = T if (T is not None and self.info[2] == cap) else self.t + self.info[2]
            self.nsteps += 1
        if want_omega:
            self.omega = om
        return self

    def advance_to(self, T, max_steps=10**9):
        t = ctypes.c_double(self.t)
        ns = ctypes.c_long(0)
        rc = _check(lib().orc_advance(ctypes.byref(self._s), _dp(self.f), ctypes.byref(t),
                                      float(T), int(max_steps), ctypes.byref(ns)))
        self.flags |= rc
        self.t = t.value
        self.nsteps += ns.value
        return self

    def moments(self):
        return moments(self.pb, self.f)
