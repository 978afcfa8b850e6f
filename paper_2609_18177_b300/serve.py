"""Continuous-batching solve server on top of the batch C ABI.

Requests of mixed systems (2D Euler Riemann, shallow-water dam break over a
bump, reactive Euler circle) and sizes arrive over time.  The server keeps one
batch per system, each on its own CUDA stream so the three persistent launches
overlap on the device.  A request is admitted as soon as it has arrived and its
lattice fits in its system's arena (first fit, by footprint); admitted lattices
stay resident on the device until they finish, and finished ones are harvested
(moments copied to the host) and removed between step chunks, which frees
space for the next admissions.  Latency = harvest time - arrival time.  A
request withdrawn by its client (cancel_at) leaves the queue at once, or, if
its lattice is resident, is removed at its batch's next harvest point.

The scheduling logic is plain host code; every step runs in the CUDA library.
"""
import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np

from . import lbmh
from . import workloads as W

KINDS = ("euler", "swe", "reactive")
KIND_SYSTEM = {"euler": W.EULER, "swe": W.SWE, "reactive": W.REACTIVE}


@dataclass
class Request:
    rid: int
    kind: str
    n: int
    steps: int
    seed: int
    arrival: float  # seconds after the start of the run
    cancel_at: Optional[float] = None  # seconds after the start: withdrawn by its client then


def make_problem(req: Request):
    """Problem and initial state of a request (seeded, synthetic)."""
    if req.kind == "euler":
        pb, U0 = W.riemann_2d_seeded(req.n, seed=req.seed, cfl=0.9)
    elif req.kind == "swe":
        pb, U0 = W.dam_break_bump(req.n)
    else:
        pb, U0 = W.reactive_circle(req.n)
    return pb.with_(precision=lbmh.FP32), U0


def poisson_trace(nreq, rate, seed=0, n_range=(128, 2048), steps_range=(200, 5000), kinds=KINDS):
    """Arrivals of a Poisson process of `rate` requests/s with seeded kinds,
    grid sizes (uniform in n_range) and step counts (uniform in steps_range)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(nreq):
        t += rng.exponential(1.0 / rate) if rate > 0 else 0.0
        kind = kinds[int(rng.integers(len(kinds)))]
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        out.append(Request(i, kind, n, steps, int(rng.integers(1 << 30)), t))
    return out


def request_footprint(req: Request) -> int:
    """Device bytes the request's lattice takes in its system's batch arena
    (from the problem's geometry alone: no input is built)."""
    pb = W.Problem(system=KIND_SYSTEM[req.kind], dim=2, nx=req.n, ny=req.n)
    return lbmh.Batch.footprint(pb, lbmh.FP32)


class InputPrefetcher:
    """Builds the requests' (problem, U0) on host threads ahead of their
    arrival order, so that the serving loop does not stop to build inputs
    (numpy releases the GIL in its array loops).  At most `lookahead` inputs are
    held at a time; an input is kept until the server releases it after the
    admission (a request that waits for room is not built twice).  Usable as
    the server's `inputs` mapping."""

    def __init__(self, trace, make=None, workers=4, lookahead=24):
        from concurrent.futures import ThreadPoolExecutor
        self.order = [r for r in sorted(trace, key=lambda r: r.arrival)]
        self.make = make or make_problem
        self.pool = ThreadPoolExecutor(max_workers=workers)
        self.lookahead = lookahead
        self.futures = {}
        self.next = 0
        self._fill()

    def _fill(self):
        while self.next < len(self.order) and len(self.futures) < self.lookahead:
            req = self.order[self.next]
            self.futures[req.rid] = self.pool.submit(self.make, req)
            self.next += 1

    def __bool__(self):
        return True

    def __contains__(self, rid):
        return True

    def __getitem__(self, rid):
        fut = self.futures.get(rid)
        if fut is None:  # beyond the window: built now, and kept until released
            from concurrent.futures import Future
            req = next(r for r in self.order if r.rid == rid)
            fut = Future()
            fut.set_result(self.make(req))
            self.futures[rid] = fut
        return fut.result()

    def release(self, rid):
        """The server has admitted the request: drop its input, build the next."""
        self.futures.pop(rid, None)
        self._fill()

    def close(self):
        self.pool.shutdown(wait=False, cancel_futures=True)


@dataclass
class Result:
    rid: int
    kind: str
    n: int
    steps: int
    arrival: float
    admitted: float
    finished: float
    U: Optional[np.ndarray] = None
    cancelled: bool = False  # withdrawn before it finished: steps = those done (admitted NaN if never)

    @property
    def latency(self):
        return self.finished - self.arrival


class Server:
    """One batch per system; requests are admitted by footprint and stepped
    together in chunks of `chunk` steps."""

    def __init__(self, capacity_bytes=8 << 30, max_instances=256, chunk=32, autotune=False, keep_results=False,
                 batches=None, new_event=None):
        """keep_results: True keeps every result's moments, a set keeps those of
        the request ids in it, False none.
        `batches` (one object per system with the lbmh.Batch methods add,
        step, poll, moments, remove, autotune) and `new_event` (a factory of
        objects with record(stream) and query()) replace the CUDA batches and
        events, e.g. to exercise the scheduling on a host without a GPU."""
        if batches is None:
            import torch
            self.streams = {k: torch.cuda.Stream() for k in KINDS}
            self.batches = {k: lbmh.Batch(KIND_SYSTEM[k], precision=lbmh.FP32, capacity_bytes=capacity_bytes,
                                          max_instances=max_instances, stream=self.streams[k].cuda_stream)
                            for k in KINDS}
            self.new_event = new_event or torch.cuda.Event
        else:
            self.streams = {k: None for k in KINDS}
            self.batches = batches
            self.new_event = new_event
        self.chunk = chunk
        self.autotune = autotune
        self.keep_results = keep_results
        self.tuned = set()

    def close(self):
        for b in self.batches.values():
            b.close()

    def _free_bytes(self, k):
        """Free arena bytes of system k's batch (None for batches without an arena)."""
        info = getattr(self.batches[k], "info", None)
        if info is None:
            return None
        d = info()
        return d["capacity_bytes"] - d["used_bytes"]

    def run(self, trace: List[Request], inputs: Optional[Dict[int, tuple]] = None, max_seconds=1e9):
        """Serve `trace` in real time; `inputs` may hold pre-built (problem, U0)
        per request id.  Returns the list of results and summary statistics.

        Each system's batch runs its own cycle: when its previous chunk of
        steps has finished on its stream (a CUDA event, polled without
        blocking), finished lattices are harvested and removed, waiting
        requests admitted, and the next chunk launched.  The batches do not
        wait for one another, so a system with heavier steps does not hold the
        others idle."""
        pending = sorted(trace, key=lambda r: r.arrival)
        queue: Dict[str, List[Request]] = {k: [] for k in KINDS}
        live: Dict[str, Dict[int, tuple]] = {k: {} for k in KINDS}  # slot -> (request, admitted time)
        inflight: Dict[str, Optional[object]] = {k: None for k in KINDS}  # event of the launched chunk
        results: List[Result] = []
        footprints: Dict[int, int] = {}
        node_steps = 0
        deferred = set()  # requests refused admission at least once (arena full)
        t0 = time.perf_counter()
        nxt = 0
        while True:
            now = time.perf_counter() - t0
            while nxt < len(pending) and pending[nxt].arrival <= now:
                queue[pending[nxt].kind].append(pending[nxt])
                nxt += 1
            progressed = False
            # withdrawn requests that were not admitted yet leave the queue
            for k in KINDS:
                keep = []
                for req in queue[k]:
                    if req.cancel_at is not None and req.cancel_at <= now:
                        results.append(Result(req.rid, k, req.n, 0, req.arrival, float("nan"), now, None, True))
                    else:
                        keep.append(req)
                queue[k] = keep
            for k in KINDS:
                ev = inflight[k]
                if ev is not None:
                    if not ev.query():
                        continue  # this batch is still stepping
                    inflight[k] = None
                    progressed = True
                    # harvest finished lattices
                    done, t, steps, status = self.batches[k].poll()
                    for slot in list(live[k].keys()):
                        req = live[k][slot][0]
                        withdrawn = req.cancel_at is not None and req.cancel_at <= time.perf_counter() - t0
                        if done[slot] == 1 or withdrawn:
                            req, adm = live[k].pop(slot)
                            U = self.batches[k].moments(slot) if done[slot] == 1 else None
                            fin = time.perf_counter() - t0
                            self.batches[k].remove(slot)
                            node_steps += req.n * req.n * int(steps[slot])
                            keep = self.keep_results is True or (self.keep_results and req.rid in self.keep_results)
                            results.append(Result(req.rid, k, req.n, int(steps[slot]), req.arrival, adm, fin,
                                                  U if keep else None, bool(done[slot] != 1)))
                # the batch is idle: admit (first fit by footprint, in arrival order);
                # a request whose lattice cannot fit in the free space is passed
                # over before its input is built
                kept = []
                free = self._free_bytes(k)
                for req in queue[k]:
                    if free is not None:
                        need = footprints.setdefault(req.rid, request_footprint(req))
                        if need > free:
                            kept.append(req)
                            deferred.add(req.rid)
                            continue
                    pb, U0 = inputs[req.rid] if inputs and req.rid in inputs else make_problem(req)
                    slot = self.batches[k].add(pb, U0, max_steps=req.steps)
                    if slot is None:
                        kept.append(req)
                        deferred.add(req.rid)
                    else:
                        live[k][slot] = (req, time.perf_counter() - t0)
                        progressed = True
                        if free is not None:
                            free -= footprints[req.rid]
                        if hasattr(inputs, "release"):
                            inputs.release(req.rid)
                queue[k] = kept
                if live[k]:
                    if self.autotune and k not in self.tuned and len(live[k]) >= 2:
                        self.batches[k].autotune(steps_per_candidate=2)
                        self.tuned.add(k)
                    self.batches[k].step(self.chunk)
                    ev = self.new_event()
                    ev.record(self.streams[k])
                    inflight[k] = ev
                    progressed = True
            if not any(live.values()) and all(e is None for e in inflight.values()):
                if nxt >= len(pending) and not any(queue.values()):
                    break
            if time.perf_counter() - t0 > max_seconds:
                break
            if not progressed:
                # nothing finished and nothing arrived: wait briefly
                wait = 0.0005
                if nxt < len(pending):
                    wait = min(wait, max(0.0, pending[nxt].arrival - (time.perf_counter() - t0)))
                time.sleep(wait)
        for k in KINDS:
            if inflight[k] is not None:
                inflight[k].synchronize()
        makespan = time.perf_counter() - t0
        served = [r for r in results if not r.cancelled]
        lat = np.array([r.latency for r in served]) if served else np.zeros(1)
        stats = {
            "completed": len(served),
            "cancelled": len(results) - len(served),
            "submitted": len(trace),
            "makespan_s": makespan,
            "solves_per_s": len(served) / makespan if makespan > 0 else 0.0,
            "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)),
            "node_updates_per_s": node_steps / makespan if makespan > 0 else 0.0,
            "deferred_admissions": len(deferred),
        }
        return results, stats


def run_alone(req: Request, pb, U0):
    """The request's lattice in a batch of its own (the reference for the
    alone-versus-mix identity)."""
    b = lbmh.Batch(pb.system, precision=lbmh.FP32, capacity_bytes=lbmh.Batch.footprint(pb, lbmh.FP32) + (1 << 20),
                   max_instances=1)
    slot = b.add(pb, U0, max_steps=req.steps)
    b.step(req.steps)
    U = b.moments(slot)
    b.close()
    return U
