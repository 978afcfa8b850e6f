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
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the FP64 run that measures the FP32 result's error (outside the timed region)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-n", type=int, default=384)
    ap.add_argument("--workload", default="riemann2d",
                    choices=["riemann2d", "batched", "served", "lines1d", "cube3d", "slabs"])
    ap.add_argument("--lattice", default="riemann2d", choices=["riemann2d", "reactive", "dambreak"],
                    help="single-lattice line: the lattice stepped (default: the 2D Riemann roofline run)")
    ap.add_argument("--case", default=None,
                    help="lines1d: run one case only, NAME:N:DTYPE (e.g. sod:262144:f32)")
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--sample", type=int, default=16)
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--autotune", action="store_true",
                    help="served: let each system's batch time its kernel variants once it holds two lattices")
    ap.add_argument("--sweep-rates", default="16,8,4",
                    help="served: lower offered rates (req/s) of the load sweep, comma-separated")
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


def recorded_traffic(kernel_name, lattice, n, precision):
    """dram bytes per launch from a committed ncu capture, valid only for the
    kernel source, lattice, size and precision it was taken on."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    ent = d.get(kernel_name)
    if not ent or ent.get("source_hash") != source_hash():
        return None
    if (ent.get("lattice", "riemann2d"), ent.get("n", 8192), ent.get("precision", "fp32")) != (lattice, n, precision):
        return None
    return ent.get("bytes_per_launch")


def max_over_ranks(ms, world, device=None):
    """The slowest rank's time (all ranks get it); identity for one rank."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank, world, ms):
    """Whole-job MLUPS of `world` replicas that each updated units_per_rank
    nodes, timed by the slowest rank (weak scaling)."""
    return units_per_rank * world / (ms / 1e3) / 1e6


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


LATTICES = {
    "riemann2d": "2D Euler seeded 4-quadrant Riemann {n}x{n}, outflow, CFL 0.9",
    "reactive": "2D reactive Euler circle (Example 5.12 states and constants) {n}x{n}, outflow, CFL 0.9",
    "dambreak": "2D shallow-water dam break over a Gaussian bump {n}x{n}, outflow, CFL 0.4",
}


def workload(n, seed, precision, lattice="riemann2d"):
    from paper_2609_18177_b300 import workloads as W
    if lattice == "reactive":
        pb, U0 = W.reactive_circle(n)
    elif lattice == "dambreak":
        pb, U0 = W.dam_break_bump(n)
    else:
        pb, U0 = W.riemann_2d_seeded(n, seed=seed, cfl=0.9)
    pb = pb.with_(precision=1 if precision == "fp32" else 0)
    return pb, U0


def _time_oracle(pb, U0, seconds, min_steps=3):
    """Node updates per second of the oracle stepping (pb, U0) for ~seconds."""
    import oracle
    r = oracle.Run(pb, U0)
    r.step(1)
    steps = 0
    t0 = time.perf_counter()
    while True:
        r.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds and steps >= min_steps:
            break
    return pb.nodes * steps / el / 1e6, steps, el


def _native_oracle():
    """The oracle tuned for this host's CPU (-march=native, built here)."""
    import oracle
    if oracle._lib is None:
        oracle.use_native_build()
    return oracle


def cpu_baseline(args, seconds):
    """The FP64 oracle as it stands, on a bounded sample of the same workload:
    on all host cores (OpenMP over rows) and on one core."""
    oracle = _native_oracle()
    n = args.ref_n
    pb, U0 = workload(n, args.seed, "fp64", args.lattice)
    cores = oracle.set_threads(os.cpu_count() or 1)
    mlups, steps, el = _time_oracle(pb, U0, seconds)
    oracle.set_threads(1)
    n1 = max(64, n // 2)
    pb1, U1 = workload(n1, args.seed, "fp64", args.lattice)
    mlups1, steps1, el1 = _time_oracle(pb1, U1, seconds / 3)
    oracle.set_threads(cores)
    return {"value": mlups, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n}x{n} grid of the same workload ({args.lattice}), FP64, {steps} steps "
                      f"({el:.1f} s), OpenMP over rows on {cores} threads; oracle built -O3 -march=native "
                      "-ffp-contract=off on this host",
            "single_thread": {"value": mlups1, "unit": UNIT, "cores": 1,
                              "sample": f"{n1}x{n1} grid, {steps1} steps ({el1:.1f} s)"},
            "cpu": _cpu_model()}


def _cpu_model():
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    oracle = _native_oracle()
    oracle.set_threads(os.cpu_count() or 1)
    n = args.ref_n
    pb, U0 = workload(n, args.seed, "fp64", args.lattice)
    r = oracle.Run(pb, U0)
    r.step(args.warmup)
    t0 = time.perf_counter()
    r.step(args.steps)
    el = time.perf_counter() - t0
    value = pb.nodes * args.steps / el / 1e6
    cores = oracle.set_threads(0)
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


def headline_accuracy(solver, pb, U0_dev, steps, kernel):
    """Error of the FP32 lattice after `steps` steps from U0 (the timed step
    count, at most 200) against the FP64 fused path over the same steps, in the
    contract norm (paper_2609_18177_b300.accuracy).  Outside the timed region."""
    import torch
    from paper_2609_18177_b300 import accuracy as A
    from paper_2609_18177_b300 import lbmh
    u32 = torch.empty((pb.nfields,) + pb.shape(), dtype=torch.float64, device=U0_dev.device)
    solver.set_state(U0_dev).step(steps)
    solver.moments(out=u32, check=False)
    t32 = solver.info()["t"]
    with lbmh.Solver(pb.with_(precision=0), precision=lbmh.FP64, kernel=kernel) as s64:
        s64.set_state(U0_dev).step(steps)
        u64 = torch.empty_like(u32)
        s64.moments(out=u64, check=False)
        t64 = s64.info()["t"]
    err = A.contract_l1_torch(u32, u64, pb.system, pb.dim)
    del u32, u64
    return {"norm": "relative L1 per quantity, momentum as a vector per node", "steps": steps,
            "t_fp32": t32, "t_fp64": t64, "errors": err, "tolerance": A.tolerance(pb.system),
            "meets_tolerance": err["max"] <= A.tolerance(pb.system),
            "reference": "FP64 fused GPU path (oracle parity 1e-12)"}


def rel_l1_fields(a, b):
    """per field: sum|a-b| / sum|b|"""
    m = b.shape[0]
    a2, b2 = a.reshape(m, -1), b.reshape(m, -1)
    den = np.abs(b2).sum(axis=1)
    return [float(v) for v in np.abs(a2 - b2).sum(axis=1) / np.where(den > 0, den, 1.0)]


def rel_l1(a, b):
    """max over fields of sum|a-b| / sum|b|"""
    return max(rel_l1_fields(a, b))


def perturbed_input(U0, seed=12345):
    """U0 with every value moved by a relative 2^-24 (half an FP32 ulp) in a
    seeded random direction: the FP64 solve from it measures how far the
    problem itself moves under an FP32-sized input change (zeros stay zero)."""
    rng = np.random.default_rng(seed)
    return U0 * (1.0 + 2.0 ** -24 * rng.choice([-1.0, 1.0], size=U0.shape))


def fp64_per_grid(pb, U0, T=None, steps=None):
    """The plain per-grid FP64 GPU path: one fused FP64 handle per lattice."""
    import torch
    from paper_2609_18177_b300 import lbmh
    s = lbmh.Solver(pb.with_(precision=0), precision=lbmh.FP64, kernel=lbmh.KERNEL_FUSED)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.set_state(U0)
    if T is not None:
        s.advance_to(T)
    else:
        s.step(steps)
    U = s.moments(check=False)
    el = time.perf_counter() - t0
    nsteps = s.nsteps
    s.close()
    return U, el, nsteps


def run_batched(args):
    """Many shallow-water dam breaks over a bump (wet-dry, bed source) of uneven
    sizes n ~ U{64..1024}, each to T = 0.1, in one FP32 batch."""
    import torch
    from paper_2609_18177_b300 import lbmh
    from paper_2609_18177_b300 import workloads as W
    rng = np.random.default_rng(args.seed)
    sizes = [int(v) for v in rng.integers(64, 1025, args.instances)]
    T = 0.1
    cases = [W.dam_break_bump(n) for n in sizes]
    cap = sum(lbmh.Batch.footprint(pb, lbmh.FP32) for pb, _ in cases) + (64 << 20)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b = lbmh.Batch(W.SWE, precision=lbmh.FP32, capacity_bytes=cap, max_instances=len(cases))
    slots = [b.add(pb.with_(precision=1), U0, T=T) for pb, U0 in cases]
    t_admit = time.perf_counter() - t0
    b.autotune(steps_per_candidate=2)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    device_ms = 0.0
    while True:
        b.step(30)
        done, t, steps, status = b.poll()
        if all(done[s] == 1 for s in slots):
            break
    e1.record(stream)
    torch.cuda.synchronize()
    device_ms = e0.elapsed_time(e1)
    results = {s: b.moments(s) for s in slots}
    wall = time.perf_counter() - t0
    node_steps = sum(pb.nodes * int(steps[s]) for (pb, _), s in zip(cases, slots))
    info = b.info()
    b.close()
    # plain per-grid FP64 GPU path on a seeded sample, and FP32 accuracy against it
    from paper_2609_18177_b300 import accuracy as A
    pick = rng.choice(len(cases), size=min(args.sample, len(cases)), replace=False)
    t64, ns64, errs, floor = 0.0, 0, [], []
    for i in pick:
        pb, U0 = cases[i]
        U64, el, n64 = fp64_per_grid(pb, U0, T=T)
        t64 += el
        ns64 += pb.nodes * n64
        errs.append(A.contract_l1(results[slots[i]], U64, pb.system, pb.dim))
        # conditioning floor: the FP64 solve from an FP32-sized input perturbation
        U64r, _el, _n = fp64_per_grid(pb, perturbed_input(U0), T=T)
        floor.append(A.contract_l1(U64r, U64, pb.system, pb.dim))
    solves = len(cases) / wall
    # the per-grid FP64 path would need (node updates of all lattices) / (its measured rate)
    fp64_rate = ns64 / t64
    fp64_solves = len(cases) / (node_steps / fp64_rate)
    names = [k for k, _ in A.quantities(W.SWE, 2)]
    return {
        "metric": METRIC, "workload": "batched", "value": solves, "unit": "solves/s",
        "higher_is_better": True, "n_gpus": 1, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{len(cases)} shallow-water dam breaks over a Gaussian bump, n ~ U{{64..1024}} "
                               f"(seed {args.seed}), T = {T}, CFL 0.4, outflow, FP32 batch, one persistent launch "
                               "per step + 3-step CUDA graphs, autotuned", "instances": len(cases)},
        "wall_s": wall, "admission_s": t_admit, "device_s_stepping": device_ms / 1e3,
        "mlups_stepping": node_steps / (device_ms / 1e3) / 1e6,
        "hbm_gbs_stepping": node_steps * 2 * 15 * 4 / (device_ms / 1e3) / 1e9,
        "batch_variant": info["variant"], "grid": info["grid"],
        "fp64_per_grid_solves_per_s": fp64_solves, "fp64_per_grid_mlups": fp64_rate / 1e6,
        "fp64_sample": len(pick),
        "fp64_note": "one fused FP64 handle per lattice, run back to back; rate measured on the sample, "
                     "solves/s = lattices / (node updates of all lattices / rate)",
        "speedup_vs_fp64_per_grid": solves / fp64_solves,
        "l1_err_vs_fp64": {"norm": "relative L1 per quantity, momentum as a vector per node",
                           "quantities": names,
                           "max": float(max(e["max"] for e in errs)),
                           "per_quantity_max": {k: float(max(e[k] for e in errs)) for k in names},
                           "per_quantity_median": {k: float(np.median([e[k] for e in errs])) for k in names},
                           "floor_fp64_input_perturbed_2^-24_max": {k: float(max(e[k] for e in floor))
                                                                    for k in names},
                           "tolerance": A.tolerance(W.SWE),
                           "meets_tolerance": bool(max(e["max"] for e in errs) <= A.tolerance(W.SWE)),
                           "reference": "FP64 fused GPU path per lattice, from the same input to the same time "
                                        "(its parity with the CPU oracle, and the FP32 batch's at T on the "
                                        "n = 274 lattice, are GPU tests)"},
    }


def served_sample(trace, seed=0, budget=3e9):
    """Requests whose results are checked against FP64: per system the two
    smallest (node updates) and two drawn from the seed among those the FP64
    path finishes in seconds (at most `budget` node updates)."""
    rng = np.random.default_rng(seed)
    pick = []
    for kind in ("euler", "swe", "reactive"):
        reqs = sorted((r for r in trace if r.kind == kind), key=lambda r: r.n * r.n * r.steps)
        pick += reqs[:2]
        rest = [r for r in reqs[2:] if r.n * r.n * r.steps <= budget]
        if rest:
            pick += [rest[int(i)] for i in rng.choice(len(rest), size=min(2, len(rest)), replace=False)]
    return pick


def fp64_rate(kind, n, steps=40):
    """Node updates per second of the plain per-grid FP64 path (one fused FP64
    handle) on a lattice of the given kind and size."""
    import torch
    from paper_2609_18177_b300 import lbmh
    from paper_2609_18177_b300 import serve as S
    pb, U0 = S.make_problem(S.Request(0, kind, n, steps, 1, 0.0))
    with lbmh.Solver(pb.with_(precision=0), precision=lbmh.FP64, kernel=lbmh.KERNEL_FUSED) as s:
        s.set_state(U0).step(3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.step(steps)
        torch.cuda.synchronize()
        return pb.nodes * steps / (time.perf_counter() - t0)


def run_served(args):
    """Poisson arrivals of mixed solves (2D Euler Riemann, shallow-water dam
    break, reactive Euler circle), n ~ U{128..2048}, 200..5000 steps."""
    from paper_2609_18177_b300 import accuracy as A
    from paper_2609_18177_b300 import serve as S
    out = {}
    plan = [("offered", args.rate, args.requests)]
    plan += [(f"rate_{r:g}", r, max(8, int(round(4 * r)))) for r in
             (float(v) for v in args.sweep_rates.split(",") if v.strip())]
    for idx, (label, rate, nreq) in enumerate(plan):
        trace = S.poisson_trace(nreq, rate, seed=args.seed + idx)
        sample = served_sample(trace, seed=args.seed) if label == "offered" else []
        srv = S.Server(capacity_bytes=24 << 30, max_instances=256, chunk=32,
                       keep_results={r.rid for r in sample}, autotune=args.autotune)
        feed = S.InputPrefetcher(trace)  # the clients' inputs, built on host threads as they arrive
        results, stats = srv.run(trace, inputs=feed)
        feed.close()
        srv.close()
        stats["rate_req_per_s"] = rate
        print(f"served {label}: {json.dumps(stats)}", file=sys.stderr, flush=True)
        if label == "offered":
            by = {r.rid: r for r in results}
            errs = []
            for req in sample:
                pb, U0 = S.make_problem(req)
                U64, _el, _n = fp64_per_grid(pb, U0, steps=req.steps)
                e = {"kind": req.kind, "n": req.n, "steps": req.steps,
                     "l1_vs_fp64": A.contract_l1(by[req.rid].U, U64, pb.system, pb.dim)}
                # the scheme's own spread: FP64 from an FP32-sized change of its input
                U64r, _el, _n = fp64_per_grid(pb, perturbed_input(U0), steps=req.steps)
                e["floor_fp64_input_perturbed_2^-24"] = A.contract_l1(U64r, U64, pb.system, pb.dim)
                errs.append(e)
                print(f"served accuracy: {json.dumps(e)}", file=sys.stderr, flush=True)
            tol = {k: A.tolerance(S.KIND_SYSTEM[k]) for k in S.KINDS}
            stats["l1_err_vs_fp64"] = {
                "norm": "relative L1 per quantity, momentum as a vector per node, rho*Y against rho",
                "max_per_system": {k: float(max([e["l1_vs_fp64"]["max"] for e in errs if e["kind"] == k] or [0.0]))
                                   for k in S.KINDS},
                "tolerance": tol,
                "meets_tolerance": bool(all(e["l1_vs_fp64"]["max"] <= tol[e["kind"]] for e in errs)),
                "requests": errs}
            # the plain per-grid FP64 path serving the same trace back to back:
            # its rate per system on a lattice of the trace's mean size
            rate64 = {}
            for kind in ("euler", "swe", "reactive"):
                ns = [r.n for r in trace if r.kind == kind]
                if ns:
                    rate64[kind] = fp64_rate(kind, int(round(np.mean(ns))))
            t64 = sum(r.n * r.n * r.steps / rate64[r.kind] for r in trace)
            stats["fp64_per_grid_solves_per_s"] = len(trace) / t64
            stats["fp64_per_grid_mlups"] = {k: v / 1e6 for k, v in rate64.items()}
            stats["fp64_note"] = ("one fused FP64 handle per request, run back to back with no arrival gaps; "
                                  "rate per system measured over 40 steps on a lattice of the trace's mean size; "
                                  "time = sum of node updates / rate")
        out[label] = stats
    off = out["offered"]
    return {
        "metric": METRIC, "workload": "served", "value": off["solves_per_s"], "unit": "solves/s",
        "higher_is_better": True, "n_gpus": 1, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "Poisson arrivals of mixed 2D Euler Riemann / shallow-water dam break / reactive "
                               "Euler solves, n ~ U{128..2048}, steps ~ U{200..5000}, FP32, continuous batching "
                               "(one batch per system, admission by arena footprint)",
                   "requests": args.requests, "rate": args.rate},
        "p50_latency_s": off["p50_latency_s"], "p99_latency_s": off["p99_latency_s"],
        "fp64_per_grid_solves_per_s": off["fp64_per_grid_solves_per_s"],
        "speedup_vs_fp64_per_grid": off["solves_per_s"] / off["fp64_per_grid_solves_per_s"],
        "l1_err_vs_fp64": {k: off["l1_err_vs_fp64"][k] for k in ("norm", "max_per_system", "tolerance",
                                                                   "meets_tolerance")},
        "offered": off, "load_sweep": [v for k, v in out.items() if k != "offered"],
    }


def run_lines1d(args):
    """The 1D lattices: linear advection of a square pulse (N = 400, periodic,
    CFL 0.5, FP64, the 800 steps to T = 1) and the Sod and Shu-Osher shock tubes
    (CFL 0.3, N = 2^12 .. 2^18, FP64 and FP32 distributions).  They fit in L2
    (<= 18.9 MB per copy), so the bound is launch latency and L2 bandwidth, not
    HBM: each case reports MLUPS and the algorithmic bytes per second
    (2 Q m sizeof(real) per node update) as L2 GB/s."""
    import torch
    from paper_2609_18177_b300 import lbmh
    from paper_2609_18177_b300 import workloads as W
    cases = [("advection pulse", W.advection_1d(400, profile="pulse", cfl=0.5), lbmh.FP64, 800)]
    for n in (1 << 12, 1 << 14, 1 << 16, 1 << 18):
        for name, gen in (("sod", W.sod), ("shu-osher", W.shu_osher)):
            for prec in (lbmh.FP64, lbmh.FP32):
                cases.append((name, gen(n), prec, args.steps))
    if args.case:
        cname, cn, cdt = args.case.split(":")
        cases = [c for c in cases if c[0].startswith(cname) and c[1][0].nx == int(cn)
                 and (c[2] == lbmh.FP32) == (cdt == "f32")]
    out = []
    stream = torch.cuda.current_stream()
    for name, (pb, U0), prec, steps in cases:
        s = lbmh.Solver(pb.with_(precision=prec), precision=prec, kernel=lbmh.KERNEL_FUSED).set_state(U0)
        s.step(max(3, args.warmup))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        st = s.info()["status"]
        s.close()
        elem = 4 if prec == lbmh.FP32 else 8
        bytes_step = 2 * 3 * pb.nfields * elem * pb.nodes
        out.append({"case": name, "n": pb.nx, "dtype": "f32" if prec == lbmh.FP32 else "f64", "steps": steps,
                    "us_per_step": ms * 1e3 / steps, "mlups": pb.nodes * steps / (ms / 1e3) / 1e6,
                    "l2_gbs": bytes_step * steps / (ms / 1e3) / 1e9, "status": st})
    # accuracy at the examples' end times: the FP32 result against the FP64
    # path (pinned to the oracle by the GPU tests) in the contract's norm, every
    # size (the FP64 runs to T at 2^18 nodes take about two minutes)
    from paper_2609_18177_b300 import accuracy as A
    acc = []
    if not args.no_accuracy and not args.case:
        for n in (1 << 12, 1 << 14, 1 << 16, 1 << 18):
            for name, gen, T in (("sod", W.sod, 0.2), ("shu-osher", W.shu_osher, 1.8)):
                pb, U0 = gen(n)
                res = {}
                for prec in (lbmh.FP64, lbmh.FP32):
                    with lbmh.Solver(pb.with_(precision=prec), precision=prec, kernel=lbmh.KERNEL_FUSED) as s:
                        s.set_state(U0).advance_to(T)
                        res[prec] = (s.moments(), s.nsteps, s.t)
                e = A.contract_l1(res[lbmh.FP32][0], res[lbmh.FP64][0], pb.system, pb.dim)
                acc.append({"case": name, "n": n, "T": T, "steps_fp64": res[lbmh.FP64][1],
                            "steps_fp32": res[lbmh.FP32][1], "l1_fp32_vs_fp64": e,
                            "meets_tolerance": bool(e["max"] <= A.tolerance(pb.system))})
    # the FP64 oracle as it stands on a bounded sample (its OpenMP loop runs
    # over rows, and a 1D lattice has one: a single core)
    cpu = None
    if not args.no_cpu_baseline and not args.case:
        orc = _native_oracle()
        orc.set_threads(1)
        pb1, U1 = W.sod(1 << 14)
        mlups1, steps1, el1 = _time_oracle(pb1, U1, 8.0)
        orc.set_threads(os.cpu_count() or 1)
        cpu = {"value": mlups1, "unit": "MLUPS", "cores": 1, "kind": "oracle",
               "sample": f"Sod 2^14 nodes, FP64, {steps1} steps ({el1:.1f} s), one core (the oracle's OpenMP "
                         "loop is over rows; a 1D lattice has one); oracle built -O3 -march=native "
                         "-ffp-contract=off on this host",
               "cpu": _cpu_model()}
    head = ([c for c in out if c["case"] == "sod" and c["n"] == 1 << 18 and c["dtype"] == "f32"] or out)[0]
    return {
        "metric": METRIC, "workload": "lines1d", "value": head["mlups"], "unit": "MLUPS",
        "higher_is_better": True, "n_gpus": 1, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "1D lattices (D1Q3): advection pulse N=400 FP64 800 steps; Sod and Shu-Osher "
                               "N=2^12..2^18, CFL 0.3, FP64 and FP32; value = Sod 2^18 FP32",
                   "l2": "L2-resident (<= 18.9 MB per copy): reported as L2 GB/s, not an HBM fraction",
                   "launch": "one launch per step, runs of 24 steps replayed as a CUDA graph"},
        "cases": out,
        "l1_err_vs_fp64": {"norm": "relative L1 per quantity (contract norm)",
                           "reference": "FP64 fused GPU path to the same end time (oracle parity 1e-12 per step)",
                           "cases": acc},
        "cpu_baseline": cpu,
    }


def run_slabs(args):
    """The slab decomposition of one lattice along y (the multi-GPU form), with
    its slabs held side by side on this one GPU: each step the host takes the
    maximum of the slabs' speed bounds (a read and a write of d numbers per
    slab), steps every slab once, and copies each slab's three outermost rows
    into its neighbour's halo through device buffers.  The 8192^2 Riemann
    workload in FP32, 1, 2 and 4 slabs; the slabs' rows must equal the whole
    lattice bit for bit (checked on the rows next to every cut).  The line's
    `clocks` cover the whole run, host-side set-up included (the GPU idles
    there); `clocks_timed_4_slabs` the timed loop of 4 slabs."""
    import torch
    from paper_2609_18177_b300 import lbmh
    from paper_2609_18177_b300 import slab as S
    from paper_2609_18177_b300 import workloads as W
    n = args.n
    steps = max(4, min(args.steps, 600))
    pb, U0 = workload(n, args.seed, "fp32", "riemann2d")
    with lbmh.Solver(pb, precision=lbmh.FP32, kernel=lbmh.KERNEL_FUSED) as s:
        s.set_state(U0).step(max(3, args.warmup))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.step(steps)
        torch.cuda.synchronize()
        whole_ms = (time.perf_counter() - t0) * 1e3 / steps
        want = s.moments()
    cases = []
    timed = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))  # the timed loops only
    for world in (2, 4):
        rows = S.partition_rows(pb.ny, world)
        slabs = [lbmh.Slab(pb, b, e, precision=lbmh.FP32) for (b, e) in rows]
        nbr = [S.neighbours(r, world, pb.bc[2] == W.PERIODIC) for r in range(world)]
        local = [np.ascontiguousarray(U0[:, S.local_rows(pb.ny, b, e, sl.halo), :]) for (b, e), sl in zip(rows, slabs)]
        ab0 = np.max([sl.state_speed_bound(u) for sl, u in zip(slabs, local)], axis=0)
        for sl, u in zip(slabs, local):
            sl.set_state_bound(u, ab0)
        del local
        bufs = [[torch.empty(sl.halo_bytes, dtype=torch.uint8, device="cuda") for _ in range(2)] for sl in slabs]

        def one_step():
            ab = np.max([sl.get_speed_bound() for sl in slabs], axis=0)
            for sl in slabs:
                sl.set_speed_bound(ab).step(1)
            for r, sl in enumerate(slabs):
                for side in (0, 1):
                    if nbr[r][side] is not None:
                        sl.halo_get(side, bufs[r][side])
            for r, sl in enumerate(slabs):
                lo, hi = nbr[r]
                if lo is not None:
                    sl.halo_set(0, bufs[lo][1])
                if hi is not None:
                    sl.halo_set(1, bufs[hi][0])

        for _ in range(max(3, args.warmup)):
            one_step()
        torch.cuda.synchronize()
        if world == 4:
            timed.start()
        t0 = time.perf_counter()
        for _ in range(steps):
            one_step()
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3 / steps
        if world == 4:
            clocks_timed = timed.stop()
        same = True
        for (b, e), sl in zip(rows, slabs):
            U = sl.moments()
            mine = U[:, sl.halo[0]:U.shape[1] - sl.halo[1], :]
            for rr in sorted({0, 1, 2, e - b - 3, e - b - 2, e - b - 1}):
                same &= bool(np.array_equal(mine[:, rr, :], want[:, b + rr, :]))
            sl.close()
        cases.append({"slabs": world, "ms_per_step": ms, "mlups": pb.nodes / (ms / 1e3) / 1e6,
                      "overhead_vs_whole": ms / whole_ms - 1.0, "rows_next_to_cuts_bitwise_equal": same})
    return {
        "metric": METRIC, "workload": "slabs", "value": cases[0]["mlups"], "unit": "MLUPS",
        "higher_is_better": True, "n_gpus": 1, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"2D Euler seeded 4-quadrant Riemann {n}x{n}, FP32, decomposed along y into "
                               "slabs held on one GPU (host maximum of the speed bounds, device-buffer halo "
                               "copies); wall time per step", "steps": steps},
        "whole_lattice_ms_per_step": whole_ms, "cases": cases,
        "clocks_timed_4_slabs": clocks_timed,
    }


def run_cube3d(args):
    """The 3D (D3Q7) path: Euler on a periodic n^3 cube with a seeded random
    state (smooth fields plus a jump), FP32 and FP64, and reactive Euler (the
    Example 5.12 constants) in FP32; the default kernel choice (the fused
    z-marching kernel in FP32, the four-kernel path in FP64) unless --kernel
    names one, the kernel of each case reported.  value = Euler
    FP32 MLUPS; algorithmic bytes per node update 2 Q m sizeof(real) (Q = 7,
    m = 5: 280 B in FP32; reactive m = 6: 336 B)."""
    import torch
    from paper_2609_18177_b300 import lbmh
    from paper_2609_18177_b300 import workloads as W
    n = args.n if args.n != 8192 else 256
    out = []
    stream = torch.cuda.current_stream()
    peak, peak_kind = measured_peaks()
    for system, prec in ((W.EULER, lbmh.FP32), (W.EULER, lbmh.FP64), (W.REACTIVE, lbmh.FP32)):
        if system == W.EULER:
            pb = W.cube(W.EULER, n, cfl=0.8)
        else:  # the Example 5.12 constants on the seeded 3D state
            pb = W.cube(W.REACTIVE, n, cfl=0.8, gamma=1.2, K=2566.4, Ti=50.0, q=50.0)
        U0 = W.random_state(pb, seed=args.seed)
        kern = {"auto": lbmh.KERNEL_AUTO, "fused": lbmh.KERNEL_FUSED, "unfused": lbmh.KERNEL_UNFUSED}[args.kernel]
        s = lbmh.Solver(pb.with_(precision=prec), precision=prec, kernel=kern).set_state(U0)
        s.step(max(3, args.warmup))
        steps = min(args.steps, 200) if prec == lbmh.FP32 else min(args.steps, 20)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        st = s.info()["status"]
        kinfo = s.info()["kernel"]
        s.close()
        elem = 4 if prec == lbmh.FP32 else 8
        gbs = 2 * 7 * pb.nfields * elem * pb.nodes * steps / (ms / 1e3) / 1e9
        out.append({"system": "euler" if system == W.EULER else "reactive",
                    "kernel": "fused" if kinfo == lbmh.KERNEL_FUSED else "four-kernel",
                    "dtype": "f32" if prec == lbmh.FP32 else "f64", "n": n, "steps": steps,
                    "ms_per_step": ms / steps, "mlups": pb.nodes * steps / (ms / 1e3) / 1e6,
                    "hbm_gbs_algorithmic": gbs, "frac_of_peak": gbs / peak, "status": st})
    return {
        "metric": METRIC, "workload": "cube3d", "value": out[0]["mlups"], "unit": "MLUPS",
        "higher_is_better": True, "n_gpus": 1, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"3D Euler (D3Q7) periodic {n}^3, seeded random state, CFL 0.8",
                   "peak_gbs": peak, "peak_kind": peak_kind, "l2": "inputs larger than L2"},
        "cases": out,
    }


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ("batched", "served", "lines1d", "cube3d", "slabs"):
        sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
        sampler.start()
        line = {"batched": run_batched, "served": run_served, "lines1d": run_lines1d,
                "cube3d": run_cube3d, "slabs": run_slabs}[args.workload](args)
        line["clocks"] = sampler.stop()  # sampled over the whole run, reference solves included
        print(json.dumps(line), flush=True)
        return 0
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

    pb, U0 = workload(args.n, args.seed, args.precision, args.lattice)
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
    ms = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    info = solver.info()
    nodes = pb.nodes
    value = replica_throughput(nodes * args.steps, world, ms)
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
        ms_e2e = max_over_ranks(max(e0.elapsed_time(e1), wall * 1e3), world, dev)
        ubytes = U0.nbytes
        e2e = {"value": replica_throughput(nodes * args.steps, world, ms_e2e), "unit": UNIT,
               "h2d_bytes_per_step": ubytes / args.steps, "d2h_bytes_per_step": ubytes / args.steps,
               "note": "per solve: set_state from pinned host U0, K steps, moments to pinned host; "
                       "bytes are per step averaged over the K steps of one solve"}

    accuracy = None
    if rank == 0 and prec == lbmh.FP32 and not args.no_accuracy:
        accuracy = headline_accuracy(solver, pb, U0_dev, min(args.steps, 200), kernel)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == lbmh.FP32 else "f64", "data": "synthetic",
            "config": {"workload": LATTICES[args.lattice].format(n=args.n) + f", D2Q5 {args.precision} distributions",
                       "n": args.n, "seed": args.seed, "kernel": kernel_used,
                       "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (no flush needed)",
                       "hbm_gbs_step": achieved},
            "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": recorded_traffic(kname, args.lattice, args.n, args.precision),
                         "algorithmic_bytes_per_launch": bytes_per_launch},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "l1_err_vs_fp64": accuracy,
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
