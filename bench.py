"""Benchmark of the collide-and-stream step on one B300 (or N replicas).

Workload (default): 2D Euler (gamma = 1.4) four-quadrant Riemann problem on
[0,1]^2 with quadrant states drawn from a seed (rho in [0.1,1.5], |u|,|v| <= 1.2,
p in [0.03,1.5]), zero-gradient outflow boundaries, one 8192 x 8192 grid,
FP32 distributions (D2Q5, m = 4: 5.37 GB per copy), CFL 0.9.  One bench step
is one time step of the whole lattice (all hot-path stages, one launch of the
fused kernel).  Inputs are far larger than L2 (126 MB), so no flush is needed
between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank runs its own replica
of the lattice (weak scaling, no data-path collective).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS & HBM GB/s vs 8 TB/s; batched/served solves/s, p50/p99 at stated L1 err"
UNIT = "MLUPS"
CSRC = os.path.join(ROOT, "paper_2609_18177_b300", "csrc")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--kernel", default="auto", choices=["auto", "fused", "unfused"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-n", type=int, default=384)
    return ap.parse_args()


KERNEL_SOURCES = ("common.cuh", "physics.cuh", "unfused.cuh", "fused.cuh")


def source_hash():
    """Hash of the sources that define the step kernels (not the host code)."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(CSRC, name), "rb") as fh:
            h.update(name.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def recorded_traffic(kernel_name):
    """dram bytes per launch from a committed ncu capture, valid only for the
    kernel source it was taken on."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    ent = d.get(kernel_name)
    if not ent or ent.get("source_hash") != source_hash():
        return None
    return ent.get("bytes_per_launch")


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def workload(n, seed, precision):
    from paper_2609_18177_b300 import workloads as W
    pb, U0 = W.riemann_2d_seeded(n, seed=seed, cfl=0.9)
    pb = pb.with_(precision=1 if precision == "fp32" else 0)
    return pb, U0


def cpu_baseline(args, seconds):
    """The FP64 oracle as it stands, on a bounded sample of the same workload."""
    import oracle
    n = args.ref_n
    pb, U0 = workload(n, args.seed, "fp64")
    r = oracle.Run(pb, U0)
    r.step(1)
    steps = 0
    t0 = time.perf_counter()
    while True:
        r.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds and steps >= 3:
            break
    mlups = pb.nodes * steps / el / 1e6
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": mlups, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n}x{n} grid of the same seeded 2D Riemann workload, FP64, {steps} steps "
                      f"({el:.1f} s), OpenMP over rows"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    n = args.ref_n
    pb, U0 = workload(n, args.seed, "fp64")
    r = oracle.Run(pb, U0)
    r.step(args.warmup)
    t0 = time.perf_counter()
    r.step(args.steps)
    el = time.perf_counter() - t0
    value = pb.nodes * args.steps / el / 1e6
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"2D Euler seeded 4-quadrant Riemann, oracle sample {n}x{n} of the "
                               f"{args.n}x{args.n} grid", "n": n, "seed": args.seed},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{n}x{n} grid, FP64, {args.steps} steps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    from paper_2609_18177_b300 import lbmh

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    pb, U0 = workload(args.n, args.seed, args.precision)
    kernel = {"auto": lbmh.KERNEL_AUTO, "fused": lbmh.KERNEL_FUSED, "unfused": lbmh.KERNEL_UNFUSED}[args.kernel]
    prec = lbmh.FP32 if args.precision == "fp32" else lbmh.FP64
    U0_dev = torch.from_numpy(U0).to(dev)
    solver = lbmh.Solver(pb, precision=prec, kernel=kernel)
    solver.set_state(U0_dev)
    stream = torch.cuda.current_stream()
    solver.step(args.warmup)
    torch.cuda.synchronize()

    info0 = solver.info()
    kernel_used = "fused" if info0["kernel"] == lbmh.KERNEL_FUSED else "unfused"
    launches_per_step = 1 if kernel_used == "fused" else 4

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    solver.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    if world > 1:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    info = solver.info()
    nodes = pb.nodes
    value = nodes * args.steps * world / (ms / 1e3) / 1e6
    elem = 4 if prec == lbmh.FP32 else 8
    Q, m = 2 * pb.dim + 1, pb.nfields
    bytes_per_launch = 2 * Q * m * elem * nodes
    ms_launch = ms / args.steps
    achieved = bytes_per_launch / (ms_launch / 1e3) / 1e9
    peak, peak_kind = measured_peaks()
    kname = f"step_{kernel_used}"

    e2e = None
    if not args.no_e2e:
        # the user's call sequence with host buffers: set_state from pinned host
        # memory, K steps, moments back to pinned host memory
        host_U = torch.from_numpy(U0).pin_memory()
        host_out = torch.empty_like(host_U).pin_memory()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.set_state(host_U)
        solver.step(args.steps)
        solver.moments(out=host_out, check=False)
        e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        ms_e2e = max(e0.elapsed_time(e1), wall * 1e3)
        if world > 1:
            t = torch.tensor([ms_e2e], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms_e2e = float(t.item())
        ubytes = U0.nbytes
        e2e = {"value": nodes * args.steps * world / (ms_e2e / 1e3) / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": ubytes / args.steps, "d2h_bytes_per_step": ubytes / args.steps,
               "note": "per solve: set_state from pinned host U0, K steps, moments to pinned host; "
                       "bytes are per step averaged over the K steps of one solve"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == lbmh.FP32 else "f64", "data": "synthetic",
            "config": {"workload": f"2D Euler seeded 4-quadrant Riemann {args.n}x{args.n}, outflow, "
                                   f"CFL 0.9, D2Q5 {args.precision} distributions",
                       "n": args.n, "seed": args.seed, "kernel": kernel_used,
                       "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (no flush needed)",
                       "hbm_gbs_step": achieved},
            "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": recorded_traffic(kname),
                         "algorithmic_bytes_per_launch": bytes_per_launch},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "status": info["status"],
            "sim_time": info["t"],
        }
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
