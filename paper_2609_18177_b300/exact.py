"""Exact solutions of textbook problems: they pin the oracle in the tests and
are the reference curves of the example figures (`figures.py`).

- Euler Riemann problem: exact solver built on the pressure function of the
  two-rarefaction/two-shock analysis (Toro, "Riemann Solvers and Numerical
  Methods for Fluid Dynamics", ch. 4), solved for p* by Newton iteration and
  sampled along x/t.
- Shallow-water dam break over a dry bed (Ritter's solution), used for
  Example 5.9.

Written from the textbook definitions; neither the oracle nor the CUDA path
uses it.
"""
import math

import numpy as np


def _pressure_fn(p, rho, pk, ck, gamma):
    if p > pk:  # shock
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        f = (p - pk) * math.sqrt(A / (p + B))
        df = math.sqrt(A / (B + p)) * (1.0 - (p - pk) / (2.0 * (B + p)))
    else:  # rarefaction
        f = 2.0 * ck / (gamma - 1.0) * ((p / pk) ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)
        df = 1.0 / (rho * ck) * (p / pk) ** (-(gamma + 1.0) / (2.0 * gamma))
    return f, df


def riemann_star(left, right, gamma=1.4):
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(gamma * pl / rl), math.sqrt(gamma * pr / rr)
    p = max(1e-10, 0.5 * (pl + pr))
    for _ in range(100):
        fl, dfl = _pressure_fn(p, rl, pl, cl, gamma)
        fr, dfr = _pressure_fn(p, rr, pr, cr, gamma)
        pn = p - (fl + fr + ur - ul) / (dfl + dfr)
        pn = max(pn, 1e-12)
        if abs(pn - p) <= 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _pressure_fn(p, rl, pl, cl, gamma)
    fr, _ = _pressure_fn(p, rr, pr, cr, gamma)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def riemann_sample(left, right, s, gamma=1.4):
    """Exact (rho, u, p) at similarity coordinate s = (x - x0)/t."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(gamma * pl / rl), math.sqrt(gamma * pr / rr)
    ps, us = riemann_star(left, right, gamma)
    g1 = (gamma - 1.0) / (gamma + 1.0)
    if s <= us:  # left of contact
        if ps > pl:  # left shock
            rs = rl * (ps / pl + g1) / (g1 * ps / pl + 1.0)
            sl = ul - cl * math.sqrt((gamma + 1.0) / (2 * gamma) * ps / pl + (gamma - 1.0) / (2 * gamma))
            return (rl, ul, pl) if s <= sl else (rs, us, ps)
        rs = rl * (ps / pl) ** (1.0 / gamma)
        cs = cl * (ps / pl) ** ((gamma - 1.0) / (2 * gamma))
        head, tail = ul - cl, us - cs
        if s <= head:
            return (rl, ul, pl)
        if s >= tail:
            return (rs, us, ps)
        u = 2.0 / (gamma + 1.0) * (cl + (gamma - 1.0) / 2.0 * ul + s)
        c = 2.0 / (gamma + 1.0) * (cl + (gamma - 1.0) / 2.0 * (ul - s))
        rho = rl * (c / cl) ** (2.0 / (gamma - 1.0))
        return (rho, u, pl * (c / cl) ** (2.0 * gamma / (gamma - 1.0)))
    if ps > pr:  # right shock
        rs = rr * (ps / pr + g1) / (g1 * ps / pr + 1.0)
        sr = ur + cr * math.sqrt((gamma + 1.0) / (2 * gamma) * ps / pr + (gamma - 1.0) / (2 * gamma))
        return (rr, ur, pr) if s >= sr else (rs, us, ps)
    rs = rr * (ps / pr) ** (1.0 / gamma)
    cs = cr * (ps / pr) ** ((gamma - 1.0) / (2 * gamma))
    head, tail = ur + cr, us + cs
    if s >= head:
        return (rr, ur, pr)
    if s <= tail:
        return (rs, us, ps)
    u = 2.0 / (gamma + 1.0) * (-cr + (gamma - 1.0) / 2.0 * ur + s)
    c = 2.0 / (gamma + 1.0) * (cr - (gamma - 1.0) / 2.0 * (ur - s))
    rho = rr * (c / cr) ** (2.0 / (gamma - 1.0))
    return (rho, u, pr * (c / cr) ** (2.0 * gamma / (gamma - 1.0)))


def riemann_profile(left, right, x, t, x0=0.5, gamma=1.4):
    out = np.array([riemann_sample(left, right, (xi - x0) / t, gamma) for xi in np.ravel(x)])
    return out[:, 0], out[:, 1], out[:, 2]


def ritter(x, t, h0=2.0, g=9.81, x0=0.0):
    """Dam break onto a dry bed: depth h0 for x <= x0 at t = 0, at rest."""
    c0 = math.sqrt(g * h0)
    s = (np.asarray(x, dtype=np.float64) - x0) / t
    h = np.where(s <= -c0, h0, np.where(s >= 2 * c0, 0.0, (2 * c0 - s) ** 2 / (9 * g)))
    u = np.where(s <= -c0, 0.0, np.where(s >= 2 * c0, 0.0, 2.0 / 3.0 * (s + c0)))
    return h, u


def total_variation(a):
    return float(np.sum(np.abs(np.diff(a))))
