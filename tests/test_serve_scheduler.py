"""Scheduling of the continuous-batching server, on the host: fake batches and
events stand in for the CUDA ones (the GPU path itself is covered in
test_gpu_serve.py).  Every request completes with its requested step count;
a full arena defers admission instead of failing; and a system whose chunks
take longer does not hold the other systems' batches idle."""
import numpy as np

from paper_2609_18177_b300 import serve as S


class FakeBatch:
    """Lattices advance by whole chunks; at most `slots` are resident."""

    def __init__(self, slots, max_instances=16):
        self.slots, self.max_instances = slots, max_instances
        self.live = {}  # slot -> [steps done, steps wanted]
        self.step_calls = 0

    def add(self, pb, U0, max_steps=0, T=0.0):
        if len(self.live) >= self.slots:
            return None
        slot = min(set(range(self.max_instances)) - set(self.live))
        self.live[slot] = [0, max_steps]
        return slot

    def step(self, n):
        self.step_calls += 1
        for v in self.live.values():
            v[0] = min(v[0] + n, v[1])

    def poll(self):
        done = np.full(self.max_instances, -1, dtype=np.int32)
        steps = np.zeros(self.max_instances, dtype=np.int64)
        for s, (k, want) in self.live.items():
            done[s] = 1 if k >= want else 0
            steps[s] = k
        return done, np.zeros(self.max_instances), steps, np.zeros(self.max_instances, dtype=np.uint32)

    def moments(self, slot):
        return np.array([float(slot)])

    def remove(self, slot):
        del self.live[slot]

    def autotune(self, steps_per_candidate=2):
        return 0.0


class FakeEvent:
    """Done after `polls` queries (a chunk that takes a while on the device)."""

    def __init__(self, polls=0):
        self.left = polls

    def record(self, stream):
        pass

    def query(self):
        self.left -= 1
        return self.left < 0

    def synchronize(self):
        self.left = -1


def requests(kinds_steps, arrival=0.0):
    return [S.Request(i, kind, 64, steps, i, arrival) for i, (kind, steps) in enumerate(kinds_steps)]


def dummy_inputs(trace):
    return {r.rid: (None, None) for r in trace}


def test_every_request_completes_with_its_steps():
    trace = requests([("euler", 96), ("swe", 40), ("reactive", 200), ("euler", 33), ("swe", 1)])
    srv = S.Server(chunk=32, batches={k: FakeBatch(slots=4) for k in S.KINDS}, new_event=FakeEvent,
                   keep_results=True)
    results, stats = srv.run(trace, inputs=dummy_inputs(trace), max_seconds=10.0)
    assert stats["completed"] == stats["submitted"] == len(trace)
    by = {r.rid: r for r in results}
    for req in trace:
        assert by[req.rid].steps == req.steps and by[req.rid].kind == req.kind
        assert by[req.rid].finished >= by[req.rid].admitted >= req.arrival
    assert stats["deferred_admissions"] == 0


def test_full_arena_defers_admission():
    trace = requests([("swe", 64)] * 6)
    batches = {k: FakeBatch(slots=2) for k in S.KINDS}
    srv = S.Server(chunk=32, batches=batches, new_event=FakeEvent)
    results, stats = srv.run(trace, inputs=dummy_inputs(trace), max_seconds=10.0)
    assert stats["completed"] == 6
    assert stats["deferred_admissions"] == 4  # two fit at first; the rest waited for removals
    assert not batches["swe"].live  # everything harvested and removed


def test_slow_system_does_not_hold_the_others():
    """Reactive chunks stay in flight for many polls; the Euler batch must keep
    stepping meanwhile (per-system cycles, no lockstep over the three)."""
    trace = requests([("reactive", 64), ("euler", 320)])
    batches = {k: FakeBatch(slots=4) for k in S.KINDS}
    # every reactive chunk stays in flight for 200 polls, the others for none
    events = {"reactive": lambda: FakeEvent(polls=200), "euler": lambda: FakeEvent(0), "swe": lambda: FakeEvent(0)}
    # route the factory by the batch being stepped: the server records the event
    # right after stepping a batch, so the last stepped batch names the stream
    last = {"k": None}
    for k, b in batches.items():
        orig = b.step

        def step(n, _k=k, _orig=orig):
            last["k"] = _k
            _orig(n)
        b.step = step
    srv = S.Server(chunk=32, batches=batches, new_event=lambda: events[last["k"]](), keep_results=True)
    results, stats = srv.run(trace, inputs=dummy_inputs(trace), max_seconds=20.0)
    by = {r.kind: r for r in results}
    assert stats["completed"] == 2
    # Euler needs 10 chunks, reactive 2; with a lockstep over systems Euler
    # could not finish before reactive, whose chunks each wait 200 polls
    assert by["euler"].finished < by["reactive"].finished
    assert batches["euler"].step_calls == 10 and batches["reactive"].step_calls == 2


def test_withdrawn_requests_leave_queue_and_batch():
    """A request withdrawn before admission leaves the queue; one withdrawn
    while resident is removed at its batch's next harvest point with the steps
    it had done; the others are served as usual."""
    trace = [S.Request(0, "swe", 64, 64, 0, 0.0),
             S.Request(1, "swe", 64, 64, 1, 0.0, cancel_at=0.0),      # waits for the single slot
             S.Request(2, "euler", 64, 3200, 2, 0.0, cancel_at=0.2)]  # 100 slow chunks (~1 s)
    batches = {"euler": FakeBatch(slots=4), "swe": FakeBatch(slots=1), "reactive": FakeBatch(slots=4)}
    last = {"k": None}
    for k, b in batches.items():
        orig = b.step

        def step(n, _k=k, _orig=orig):
            last["k"] = _k
            _orig(n)
        b.step = step
    events = {"euler": lambda: FakeEvent(polls=20), "swe": lambda: FakeEvent(0), "reactive": lambda: FakeEvent(0)}
    srv = S.Server(chunk=32, batches=batches, new_event=lambda: events[last["k"]](), keep_results=True)
    results, stats = srv.run(trace, inputs=dummy_inputs(trace), max_seconds=20.0)
    by = {r.rid: r for r in results}
    assert stats["completed"] == 1 and stats["cancelled"] == 2 and len(results) == 3
    assert not by[0].cancelled and by[0].steps == 64 and by[0].U is not None
    assert by[1].cancelled and by[1].steps == 0 and by[1].admitted != by[1].admitted  # never admitted (NaN)
    assert by[2].cancelled and 0 < by[2].steps < 3200 and by[2].steps % 32 == 0 and by[2].U is None
    assert by[2].finished >= 0.2
    assert all(not b.live for b in batches.values())


def test_input_prefetcher_builds_inputs_ahead_in_arrival_order():
    """The prefetcher hands the server each request's input once, built on
    host threads in arrival order, holding at most `lookahead` at a time."""
    import threading
    from paper_2609_18177_b300 import serve as S
    trace = S.poisson_trace(12, rate=50.0, seed=3)
    built = []
    lock = threading.Lock()

    def make(req):
        with lock:
            built.append(req.rid)
        return ("pb", req.rid)

    feed = S.InputPrefetcher(trace, make=make, workers=2, lookahead=4)
    assert len(feed.futures) <= 4
    for req in sorted(trace, key=lambda r: r.arrival):
        assert req.rid in feed
        assert feed[req.rid] == ("pb", req.rid)
        assert feed[req.rid] == ("pb", req.rid)  # asked again while it waits for room: not rebuilt
        feed.release(req.rid)
        assert len(feed.futures) <= 4
    feed.close()
    assert sorted(built) == sorted(r.rid for r in trace) and len(built) == len(trace)
