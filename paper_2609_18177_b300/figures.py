"""Headless figures of Examples 5.5, 5.9 and 5.10: the adaptive scheme against
the fixed omega = 1 scheme (the paper's comparison) and the exact solution
where one exists, written as PNG files with a caption file beside each.

    python -m paper_2609_18177_b300.figures --out figs/

Example 5.5: Lax tube, N = 600, t = 0.14 - density, velocity, pressure, omega.
Example 5.9: dry-bed dam break, N = 600, t = 0.15 - depth, velocity, omega.
Example 5.10: circular dam break, 400 x 400, t = 0.07 - centreline depth and
velocity, depth field, omega field (no exact curve: the paper's radial
reference solution is not reproduced).
Colours: blue = adaptive omega (Eq. 2.16), red = omega = 1, black = exact.
The runs use the CUDA library in FP64; the figure also reports the L1 error
of each scheme against the exact solution (JSON on stdout).
"""
import argparse
import json
import os
import struct
import zlib

import numpy as np

from . import exact as X
from . import lbmh
from . import workloads as W

BLUE, RED, BLACK = (30, 80, 220), (220, 40, 40), (0, 0, 0)


def write_png(path, img):
    """RGB uint8 image (H, W, 3) as a PNG (zlib, filter 0 per row)."""
    h, w, _ = img.shape
    raw = b"".join(b"\x00" + img[r].tobytes() for r in range(h))

    def chunk(tag, data):
        return struct.pack(">I", len(data)) + tag + data + struct.pack(">I", zlib.crc32(tag + data) & 0xFFFFFFFF)

    with open(path, "wb") as fh:
        fh.write(b"\x89PNG\r\n\x1a\n" + chunk(b"IHDR", struct.pack(">IIBBBBB", w, h, 8, 2, 0, 0, 0))
                 + chunk(b"IDAT", zlib.compress(raw, 9)) + chunk(b"IEND", b""))


class Panel:
    """A plot area of a canvas with data limits; lines are drawn by dense
    sampling of each segment."""

    def __init__(self, img, x0, y0, w, h, xlim, ylim):
        self.img, self.x0, self.y0, self.w, self.h = img, x0, y0, w, h
        self.xlim, self.ylim = xlim, ylim
        img[y0, x0:x0 + w] = img[y0 + h - 1, x0:x0 + w] = 120
        img[y0:y0 + h, x0] = img[y0:y0 + h, x0 + w - 1] = 120

    def _px(self, x, y):
        (a, b), (c, d) = self.xlim, self.ylim
        px = self.x0 + (np.asarray(x) - a) / (b - a) * (self.w - 1)
        py = self.y0 + self.h - 1 - (np.asarray(y) - c) / (d - c) * (self.h - 1)
        return px, py

    def line(self, x, y, color, thick=1):
        px, py = self._px(x, y)
        for i in range(len(px) - 1):
            n = int(max(abs(px[i + 1] - px[i]), abs(py[i + 1] - py[i]))) + 2
            xs = np.linspace(px[i], px[i + 1], n)
            ys = np.linspace(py[i], py[i + 1], n)
            for o in range(-(thick // 2), thick // 2 + 1):
                xi = np.clip(np.round(xs).astype(int), self.x0, self.x0 + self.w - 1)
                yi = np.clip(np.round(ys).astype(int) + o, self.y0, self.y0 + self.h - 1)
                self.img[yi, xi] = color


def heat(img, x0, y0, field, lo, hi):
    """Grey-scale image of a 2D field (row 0 at the bottom)."""
    f = np.clip((field - lo) / (hi - lo), 0.0, 1.0)[::-1]
    v = (255 * (1.0 - f)).astype(np.uint8)
    img[y0:y0 + v.shape[0], x0:x0 + v.shape[1]] = v[..., None]


def limits(*arrays, pad=0.08):
    lo = min(float(np.nanmin(a)) for a in arrays)
    hi = max(float(np.nanmax(a)) for a in arrays)
    d = (hi - lo) or 1.0
    return lo - pad * d, hi + pad * d


def solve(pb, U0, T, omega_fixed):
    pb = pb.with_(omega_mode=1 if omega_fixed else 0, omega_fixed=1.0, precision=lbmh.FP64)
    s = lbmh.Solver(pb, precision=lbmh.FP64, kernel=lbmh.KERNEL_FUSED).set_state(U0)
    s.advance_to(T)
    U = s.moments()
    om = s.omega()
    t = s.t
    s.close()
    return U, om, t


def l1(a, b, dx):
    return float(np.sum(np.abs(a - b)) * dx)


def example_5_5(out, nx=600):
    pb, U0 = W.lax(nx)
    res = {}
    panels = {}
    for tag, fixed in (("adaptive", False), ("omega1", True)):
        U, om, t = solve(pb, U0, 0.14, fixed)
        rho = U[0, 0]
        u = U[1, 0] / rho
        p = 0.4 * (U[2, 0] - 0.5 * rho * u * u)
        panels[tag] = (rho, u, p, om[0], t)
    xs = W.cell_centres(pb)[0][0]
    t = panels["adaptive"][4]
    ex = X.riemann_profile((0.445, 0.698, 3.528), (0.5, 0.0, 0.571), xs, t, x0=0.5)
    for tag in panels:
        res[tag] = {name: l1(panels[tag][i], ex[i], pb.dx) for i, name in enumerate(("rho", "u", "p"))}
    img = np.full((2 * 260 + 30, 2 * 420 + 30, 3), 255, np.uint8)
    for k, (i, exv) in enumerate(((0, ex[0]), (1, ex[1]), (2, ex[2]), (3, None))):
        cur = [panels[tag][i] for tag in panels]
        yl = (0.9, 2.05) if i == 3 else limits(*cur, exv)
        P = Panel(img, 10 + (k % 2) * 430, 10 + (k // 2) * 270, 420, 260, (pb.x0, pb.x1), yl)
        if exv is not None:
            P.line(xs, exv, BLACK)
        P.line(xs, panels["omega1"][i], RED)
        P.line(xs, panels["adaptive"][i], BLUE)
    write_png(os.path.join(out, "example_5_5_lax.png"), img)
    caption = (f"Example 5.5, Lax tube, N = {nx}, t = {t:.4f}: density (top left), velocity (top right), "
               "pressure (bottom left), omega (bottom right, axis 0.9..2.05).  Blue: adaptive omega; red: "
               "omega = 1; black: exact.")
    return caption, res


def example_5_9(out, nx=600):
    pb, U0 = W.dry_dam_break_1d(nx)
    panels = {}
    for tag, fixed in (("adaptive", False), ("omega1", True)):
        U, om, t = solve(pb, U0, 0.15, fixed)
        h = U[0, 0]
        u = np.where(h > 1e-5, U[1, 0] / np.where(h > 0, h, 1.0), 0.0)
        panels[tag] = (h, u, om[0], t)
    xs = W.cell_centres(pb)[0][0]
    t = panels["adaptive"][3]
    hx, ux = X.ritter(xs, t)
    res = {tag: {"h": l1(panels[tag][0], hx, pb.dx), "u": l1(panels[tag][1], ux, pb.dx)} for tag in panels}
    img = np.full((260 + 20, 3 * 420 + 40, 3), 255, np.uint8)
    for k, (i, exv) in enumerate(((0, hx), (1, ux), (2, None))):
        cur = [panels[tag][i] for tag in panels]
        yl = (0.9, 2.05) if i == 2 else limits(*cur, exv)
        P = Panel(img, 10 + k * 430, 10, 420, 260, (pb.x0, pb.x1), yl)
        if exv is not None:
            P.line(xs, exv, BLACK)
        P.line(xs, panels["omega1"][i], RED)
        P.line(xs, panels["adaptive"][i], BLUE)
    write_png(os.path.join(out, "example_5_9_dry_dam_break.png"), img)
    caption = (f"Example 5.9, dam break over a dry bed, N = {nx}, t = {t:.4f}: depth, velocity, omega (axis "
               "0.9..2.05).  Blue: adaptive omega; red: omega = 1; black: Ritter's solution.")
    return caption, res


def example_5_10(out, n=400):
    pb, U0 = W.circular_dam_break(n)
    panels = {}
    for tag, fixed in (("adaptive", False), ("omega1", True)):
        U, om, t = solve(pb, U0, 0.07, fixed)
        panels[tag] = (U, om, t)
    xs = W.cell_centres(pb)[0][0]
    j = n // 2
    img = np.full((2 * 410 + 30, 2 * 410 + 30, 3), 255, np.uint8)
    cur_h = [panels[tag][0][0, j] for tag in panels]
    cur_u = [panels[tag][0][1, j] / panels[tag][0][0, j] for tag in panels]
    Ph = Panel(img, 10, 10, 400, 400, (pb.x0, pb.x1), limits(*cur_h))
    Pu = Panel(img, 420, 10, 400, 400, (pb.x0, pb.x1), limits(*cur_u))
    for tag, col in (("omega1", RED), ("adaptive", BLUE)):
        U = panels[tag][0]
        Ph.line(xs, U[0, j], col)
        Pu.line(xs, U[1, j] / U[0, j], col)
    U, om, t = panels["adaptive"]
    heat(img, 10 + (400 - n) // 2, 420 + (400 - n) // 2, U[0], 1.0, 2.0)
    heat(img, 420 + (400 - n) // 2, 420 + (400 - n) // 2, 2.0 - om, 0.0, 1.0)
    write_png(os.path.join(out, "example_5_10_circular_dam_break.png"), img)
    caption = (f"Example 5.10, circular dam break, {n} x {n}, t = {t:.4f}: centreline depth (top left) and "
               "velocity (top right), blue adaptive, red omega = 1; adaptive depth field (bottom left, white 1, "
               "black 2) and omega (bottom right, white 2, black 1).")
    res = {"omega_min": float(om.min()), "omega_max": float(om.max()),
           "centreline_depth_max_abs_diff_adaptive_vs_omega1":
               float(np.abs(panels["adaptive"][0][0, j] - panels["omega1"][0][0, j]).max())}
    return caption, res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="figures")
    args = ap.parse_args()
    os.makedirs(args.out, exist_ok=True)
    summary = {}
    for name, fn in (("5.5", example_5_5), ("5.9", example_5_9), ("5.10", example_5_10)):
        caption, res = fn(args.out)
        with open(os.path.join(args.out, f"example_{name.replace('.', '_')}.txt"), "w") as fh:
            fh.write(caption + "\n")
        summary[name] = res
    print(json.dumps(summary), flush=True)


if __name__ == "__main__":
    main()
