"""Brute-force push-form stepper of Eq. (2.2) for tiny grids (test infrastructure).

A second, deliberately different implementation of one time step, used to pin
the oracle's pull-form organisation, indices and boundary handling:

  - it loops over nodes in pure Python, one node and one velocity at a time;
  - it PUSHES post-collision values from x to x + e_k exactly as (2.2) is
    written, instead of pulling from x - e_k;
  - it projects differences onto characteristic fields with closed-form
    primitive-variable decompositions (w_+-, entropy, shear, species
    amplitudes) instead of inverting the right-eigenvector matrix;
  - it solves the Arrhenius half-source with scipy's brentq.

The readings are the same as the oracle's (ghost extension of f by index
wrap/clamp, per-step abar, cell-centred nodes, eigenvector scaling).
"""
import math

import numpy as np
from scipy.optimize import brentq

ADVECTION, EULER, SWE, REACTIVE = 0, 1, 2, 3
G = 3


def _unpack(pb, U):
    d = pb.dim
    if pb.system in (EULER, REACTIVE):
        rho = U[0]
        u = U[1] / rho
        v = U[2] / rho if d == 2 else 0.0
        chem = pb.q * U[d + 2] if pb.system == REACTIVE else 0.0
        p = (pb.gamma - 1) * (U[d + 1] - 0.5 * rho * (u * u + v * v) - chem)
        Y = U[d + 2] / rho if pb.system == REACTIVE else 0.0
        return dict(rho=rho, u=u, v=v, p=p, Y=Y, c=math.sqrt(pb.gamma * p / rho))
    if pb.system == SWE:
        h = U[0]
        dry = h < pb.h_dry
        u = 0.0 if dry else U[1] / h
        v = 0.0 if (dry or d == 1) else U[2] / h
        return dict(h=h, u=u, v=v, c=math.sqrt(pb.g * max(h, 0.0)))
    return {}


def flux(pb, j, U):
    d = pb.dim
    if pb.system == ADVECTION:
        return [pb.adv[j] * U[0]]
    w = _unpack(pb, U)
    vn = w["u"] if j == 0 else w["v"]
    if pb.system == SWE:
        F = [w["h"] * vn, w["h"] * w["u"] * vn]
        if d == 2:
            F.append(w["h"] * w["v"] * vn)
        F[1 + j] += 0.5 * pb.g * w["h"] ** 2
        return F
    F = [w["rho"] * vn, w["rho"] * w["u"] * vn]
    if d == 2:
        F.append(w["rho"] * w["v"] * vn)
    F[1 + j] += w["p"]
    F.append(vn * (U[d + 1] + w["p"]))
    if pb.system == REACTIVE:
        F.append(U[d + 2] * vn)
    return F


def speed(pb, j, U):
    if pb.system == ADVECTION:
        return abs(pb.adv[j])
    w = _unpack(pb, U)
    return abs(w["u"] if j == 0 else w["v"]) + w["c"]


def char_amplitudes(pb, j, U, dU):
    """L_j(U) dU via the primitive-variable decomposition (list of m amplitudes)."""
    d = pb.dim
    if pb.system == ADVECTION:
        return [dU[0]]
    w = _unpack(pb, U)
    if pb.system == SWE:
        c = max(w["c"], math.sqrt(pb.g * pb.h_dry))
        un = w["u"] if j == 0 else w["v"]
        dmn = dU[1 + j] - un * dU[0]  # h d(u_n)
        out = [0.5 * (dU[0] - dmn / c)]
        if d == 2:
            ut = w["v"] if j == 0 else w["u"]
            out.append(dU[2 - j] - ut * dU[0])  # h d(u_t)
        out.append(0.5 * (dU[0] + dmn / c))
        return out
    rho, u, v, c = w["rho"], w["u"], w["v"], w["c"]
    un = u if j == 0 else v
    dm = [dU[1], dU[2] if d == 2 else 0.0]
    dp = (pb.gamma - 1) * (dU[d + 1] - u * dm[0] - v * dm[1] + 0.5 * (u * u + v * v) * dU[0]
                           - (pb.q * dU[d + 2] if pb.system == REACTIVE else 0.0))
    rdun = dm[j] - un * dU[0]  # rho d(u_n)
    out = [0.5 * (dp - c * rdun) / (c * c), dU[0] - dp / (c * c)]
    if d == 2:
        ut = v if j == 0 else u
        out.append(dm[1 - j] - ut * dU[0])  # rho d(u_t)
    if pb.system == REACTIVE:
        out.append(dU[d + 2] - w["Y"] * dU[0])  # rho dY
    out.append(0.5 * (dp + c * rdun) / (c * c))
    return out


def source(pb, U, x, y):
    m = len(U)
    S = [0.0] * m
    d = pb.dim
    if pb.system == SWE and pb.bed_amp != 0.0:
        rx, ry = x - pb.bed_xc, (y - pb.bed_yc) if d == 2 else 0.0
        b = pb.bed_amp * math.exp(-(rx * rx + ry * ry) / pb.bed_w2)
        S[1] = -pb.g * U[0] * (-2 * rx / pb.bed_w2 * b)
        if d == 2:
            S[2] = -pb.g * U[0] * (-2 * ry / pb.bed_w2 * b)
    if pb.system == REACTIVE and pb.K != 0.0:
        w = _unpack(pb, U)
        S[d + 2] = -pb.K * U[d + 2] * math.exp(-pb.Ti / (w["p"] / w["rho"]))
    return S


def velocities(d):
    if d == 1:
        return [(0, 0), (1, 0), (-1, 0)]
    return [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1)]


def step(pb, f):
    """One step; f is a numpy array (Q, m, ny, nx).  Returns (f_new, dt)."""
    Q, m, ny, nx = f.shape
    d = pb.dim
    dx = (pb.x1 - pb.x0) / nx
    evel = velocities(d)

    def mp(e, n, lo, hi):
        if e < 0:
            return e % n if lo == 0 else (-1 - e if lo == 2 else 0)
        if e >= n:
            return e % n if hi == 0 else (2 * n - 1 - e if hi == 2 else n - 1)
        return e

    def side(e, n, lo, hi):  # boundary type across which e lies, None inside
        return lo if e < 0 else (hi if e >= n else None)

    def src(ei, ej):
        i = mp(ei - G, nx, pb.bc[0], pb.bc[1])
        j = mp(ej - G, ny, pb.bc[2], pb.bc[3]) if d == 2 else 0
        return i, j

    def sides(p):
        sx = side(p[0], nx, pb.bc[0], pb.bc[1])
        sy = side(p[1], ny, pb.bc[2], pb.bc[3]) if d == 2 else None
        return sx, sy

    momentum = pb.system in (EULER, SWE, REACTIVE)
    jrange = range(-G, ny + G) if d == 2 else range(0, 1)
    Ue, fe = {}, {}
    for ej in jrange:
        for ei in range(-G, nx + G):
            i, j = src(ei + G, ej + G if d == 2 else G)
            vals = [[f[k, c, j, i] for c in range(m)] for k in range(Q)]
            # a reflecting ghost: velocity e mirrored across the wall, normal
            # momentum reversed
            for dirn, sd in enumerate(sides((ei, ej))[:d]):
                if sd != 2:
                    continue
                mirrored = []
                for k in range(Q):
                    e = list(evel[k])
                    e[dirn] = -e[dirn]
                    kk = evel.index(tuple(e))
                    row = list(vals[kk])
                    if momentum:
                        row[1 + dirn] = -row[1 + dirn]
                    mirrored.append(row)
                vals = mirrored
            fe[(ei, ej)] = vals
            Ue[(ei, ej)] = [sum(vals[k][c] for k in range(Q)) for c in range(m)]
    abar = [0.0, 0.0]
    for j in range(ny):
        for i in range(nx):
            for dirn in range(d):
                abar[dirn] = max(abar[dirn], speed(pb, dirn, Ue[(i, j)]))
    dt = pb.cfl * dx / sum(abar[:d])
    lam = dx / dt
    alpha = [abar[j] + pb.eps for j in range(d)]
    a = [1 - sum(alpha) / lam] + [alpha[j] / (2 * lam) for j in range(d)] * 2

    def equilibrium(U):
        Fs = [flux(pb, j, U) for j in range(d)]
        feq = [[(1 - sum(alpha) / lam) * U[c] for c in range(m)]]
        for j in range(d):
            feq.append([(alpha[j] * U[c] + Fs[j][c]) / (2 * lam) for c in range(m)])
        for j in range(d):
            feq.append([(alpha[j] * U[c] - Fs[j][c]) / (2 * lam) for c in range(m)])
        return feq

    # an inflow ghost holds the equilibrium of the fixed inflow state
    for p in list(fe.keys()):
        if 3 in sides(p):
            Uin = [float(v) for v in pb.u_in[:m]]
            fe[p] = equilibrium(Uin)
            Ue[p] = [sum(fe[p][k][c] for k in range(Q)) for c in range(m)]

    def nu_at(p):
        tot = 0.0
        for dirn in range(d):
            s = (1, 0) if dirn == 0 else (0, 1)
            U0 = Ue[p]
            Um = Ue[(p[0] - s[0], p[1] - s[1])]
            Up = Ue[(p[0] + s[0], p[1] + s[1])]
            wm = char_amplitudes(pb, dirn, U0, [U0[c] - Um[c] for c in range(m)])
            wp = char_amplitudes(pb, dirn, U0, [Up[c] - U0[c] for c in range(m)])
            for r in range(m):
                tot += abs(wp[r] - wm[r]) / (abs(wm[r]) + abs(wp[r]) + dx) + abs(wm[r]) + abs(wp[r])
        return tot

    def omega_at(p):
        if pb.omega_mode == 1:
            w = pb.omega_fixed
        else:
            box = [(bi, bj) for bi in (-1, 0, 1) for bj in ((-1, 0, 1) if d == 2 else (0,))]
            w = 1.0 + 1.0 / (1.0 + sum(nu_at((p[0] + bi, p[1] + bj)) for bi, bj in box))
        L = getattr(pb, "sponge_width", 0.0)
        if L > 0.0:
            r = (p[0] + 0.5) * dx / L
            sigma = 1.0 if r <= 0 else (0.0 if r >= 1 else 0.5 * (1 + math.cos(math.pi * r)))
            w = 1.0 + (w - 1.0) * (1.0 - sigma)
        return w

    def coords(p):
        i, j = src(p[0] + G, p[1] + G if d == 2 else G)
        sx, sy = sides(p)
        if sx == 2:
            i = p[0]
        if sy == 2:
            j = p[1]
        x = pb.x0 + (i + 0.5) * dx
        y = pb.y0 + (j + 0.5) * dx if d == 2 else 0.0
        return x, y

    # push every node within one layer of the domain to x + e_k
    arrived = {}
    for ej in (range(-1, ny + 1) if d == 2 else range(0, 1)):
        for ei in range(-1, nx + 1):
            p = (ei, ej)
            U = Ue[p]
            om = omega_at(p)
            feq = equilibrium(U)
            S = source(pb, U, *coords(p))
            for k in range(Q):
                tgt = (ei + evel[k][0], ej + evel[k][1])
                if not (0 <= tgt[0] < nx and 0 <= tgt[1] < ny):
                    continue
                fk = fe[p][k]
                arrived[(tgt, k)] = [fk[c] - om * (fk[c] - feq[k][c]) + 0.5 * dt * a[k] * S[c]
                                     for c in range(m)]
    fn = np.zeros_like(f)
    for j in range(ny):
        for i in range(nx):
            Fk = [arrived[((i, j), k)] for k in range(Q)]
            Ubar = [sum(Fk[k][c] for k in range(Q)) for c in range(m)]
            x, y = coords((i, j))
            Un = list(Ubar)
            if pb.system == SWE and pb.bed_amp != 0.0:
                S = source(pb, Ubar, x, y)  # no mass source: h^{n+1} = hbar
                for c in range(1, m):
                    Un[c] = Ubar[c] + 0.5 * dt * S[c]
            if pb.system == REACTIVE and pb.K != 0.0 and Ubar[d + 2] != 0.0:
                zb = Ubar[d + 2]

                def g(z):
                    V = list(Ubar)
                    V[d + 2] = z
                    return z - zb - 0.5 * dt * source(pb, V, x, y)[d + 2]

                lo, hi = (0.0, zb) if zb > 0 else (zb, 0.0)
                Un[d + 2] = brentq(g, lo, hi, xtol=1e-300, rtol=8.9e-16, maxiter=500)
            S = source(pb, Un, x, y)
            for k in range(Q):
                for c in range(m):
                    fn[k, c, j, i] = Fk[k][c] + 0.5 * dt * a[k] * S[c]
    return fn, dt
