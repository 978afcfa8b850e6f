"""Example 5.13, the 2D stable cellular detonation, on the fused FP32 path.

    python -m paper_2609_18177_b300.detonation [--nx 1200 --ny 900 --t-end 268
                                                --sample-dt 0.5 --out detonation.npz]

Runs the reactive Euler lattice of `workloads.cellular_detonation` (reflecting
walls at y = +-15, fixed inflow of the unreacted state at x = 40, outflow and
a sponge at x = 0, ZND initial profile, transverse velocity perturbation) to
t_end, and records on the device the front-region peak pressure
p_peak(y, t) = max over 20 <= x <= 31 of p(x, y, t) every sample_dt (the
space-time diagnostic of the example), the leading-shock position, and at the
end the fields rho, u, T = p/rho, p, Y and the relaxation parameter omega.
Every step runs in the CUDA library; torch only reduces the sampled moments.
"""
import argparse
import json
import time

import numpy as np

from . import lbmh
from . import workloads as W


def pressure(U, gamma, q):
    """p of the conservative reactive state U[5, ny, nx] (a torch tensor)."""
    rho, mx, my, E, z = U[0], U[1], U[2], U[3], U[4]
    return (gamma - 1.0) * (E - 0.5 * (mx * mx + my * my) / rho - q * z)


def run(nx=1200, ny=900, t_end=268.0, sample_dt=0.5, precision=lbmh.FP32, window=(20.0, 31.0)):
    import torch
    pb, U0 = W.cellular_detonation(nx=nx, ny=ny)
    pb = pb.with_(precision=precision)
    c = W.DETONATION_5_13
    dev = torch.device("cuda", torch.cuda.current_device())
    xs = pb.x0 + (np.arange(nx) + 0.5) * pb.dx
    cols = np.nonzero((xs >= window[0]) & (xs <= window[1]))[0]
    c0, c1 = int(cols[0]), int(cols[-1]) + 1
    s = lbmh.Solver(pb, precision=precision, kernel=lbmh.KERNEL_FUSED)
    s.set_state(torch.from_numpy(U0).to(dev))
    U = torch.empty((5, ny, nx), dtype=torch.float64, device=dev)
    times, peaks, fronts = [], [], []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    k = 0
    while True:
        k += 1
        target = min(k * sample_dt, t_end)
        s.advance_to(target)
        s.moments(out=U)
        p = pressure(U, c["gamma"], c["q"])
        peaks.append(p[:, c0:c1].amax(dim=1).cpu().numpy())
        # leading shock: the last column (from the inflow side) whose mean
        # pressure exceeds twice the upstream value
        pm = p.mean(dim=0)
        hot = torch.nonzero(pm > 2.0)
        fronts.append(float(xs[int(hot.max())]) if hot.numel() else float("nan"))
        times.append(s.t)
        if s.t >= t_end or target >= t_end:
            break
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    steps = s.nsteps
    Uh = U.cpu().numpy()
    om = s.omega()
    s.close()
    rho = Uh[0]
    pf = pressure(torch.from_numpy(Uh), c["gamma"], c["q"]).numpy()
    fields = {"rho": rho, "u": Uh[1] / rho, "T": pf / rho, "p": pf, "Y": Uh[4] / rho, "omega": om.reshape(ny, nx)}
    return {"problem": pb, "t": np.array(times), "p_peak": np.array(peaks), "front_x": np.array(fronts),
            "fields": fields, "steps": steps, "wall_s": wall, "node_updates": steps * nx * ny}


def cells_across(p_peak, t, t_from):
    """Dominant transverse wavenumber of p_peak(y) over t >= t_from: the
    number of detonation cells across the 30-wide channel (each cell spans one
    period of the transverse pattern)."""
    sel = p_peak[t >= t_from]
    if not len(sel):
        return 0
    spec = np.abs(np.fft.rfft(sel - sel.mean(axis=1, keepdims=True), axis=1)).mean(axis=0)
    return int(np.argmax(spec[1:]) + 1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=1200)
    ap.add_argument("--ny", type=int, default=900)
    ap.add_argument("--t-end", type=float, default=268.0)
    ap.add_argument("--sample-dt", type=float, default=0.5)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--out", default=None, help="write t, p_peak, front_x and the final fields (.npz)")
    args = ap.parse_args()
    prec = lbmh.FP32 if args.precision == "fp32" else lbmh.FP64
    res = run(args.nx, args.ny, args.t_end, args.sample_dt, prec)
    t, pk = res["t"], res["p_peak"]
    late = t >= max(0.0, args.t_end - 20.0)
    summary = {
        "example": "5.13 cellular detonation", "nx": args.nx, "ny": args.ny, "t_end": float(t[-1]),
        "precision": args.precision, "steps": int(res["steps"]), "wall_s": res["wall_s"],
        "mlups": res["node_updates"] / res["wall_s"] / 1e6,
        "cells_across_last_20": cells_across(pk, t, args.t_end - 20.0),
        "front_x_last_20": [float(np.nanmin(res["front_x"][late])), float(np.nanmax(res["front_x"][late]))],
        "p_peak_last_20": [float(pk[late].min()), float(pk[late].max())],
        "omega_final": [float(res["fields"]["omega"].min()), float(res["fields"]["omega"].max())],
        "Y_min_final": float(res["fields"]["Y"].min()),
    }
    print(json.dumps(summary), flush=True)
    if args.out:
        np.savez_compressed(args.out, t=t, p_peak=pk, front_x=res["front_x"],
                            **{k: v.astype(np.float32) for k, v in res["fields"].items()})


if __name__ == "__main__":
    main()
