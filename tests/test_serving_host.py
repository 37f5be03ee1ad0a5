"""Host logic of the continuous-batching engine (no GPU): admission by footprint, FIFO order,
concurrency, completion and latency accounting, with a simulated backend on a virtual clock."""
import pytest

from paper_2003_12811_gb300.serve import ServingEngine, Request, percentile


class VClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += dt


class FakeShot:
    def __init__(self, clock, cost_per_step, dt, log, rid):
        self.clock, self.cost, self.dt, self.log, self.rid = clock, cost_per_step, dt, log, rid
        self.ready_at = 0.0
        self.steps = 0

    def launch(self, n):
        self.ready_at = max(self.ready_at, self.clock()) + n * self.cost
        self.steps += n
        self.log.append(("launch", self.rid, n))

    def busy(self):
        return self.clock() < self.ready_at

    def result(self):
        return self.steps

    def close(self):
        self.log.append(("close", self.rid))


class FakeBackend:
    def __init__(self, clock, sizes):
        self.clock, self.sizes, self.log = clock, sizes, []

    def footprint(self, problem):
        return self.sizes[problem]

    def create(self, problem, cfl, dt=None):
        self.log.append(("create", problem))
        return FakeShot(self.clock, 1e-3, 0.01, self.log, problem)


def _run(sizes, arrivals, nsteps, cap, max_active=8, tick=4):
    clk = VClock()
    be = FakeBackend(clk, sizes)
    eng = ServingEngine(cap, backend=be, tick_steps=tick, max_active=max_active, clock=clk, sleep=clk.sleep,
                        idle_sleep=1e-4)
    reqs = [Request(rid=i, arrival=a, problem=i, nsteps=n) for i, (a, n) in enumerate(zip(arrivals, nsteps))]
    return eng, be, eng.run(reqs)


def test_all_requests_complete_with_their_steps():
    eng, be, res = _run({i: 10 for i in range(6)}, [0.0, 0.001, 0.002, 0.01, 0.02, 0.5], [8, 12, 6, 4, 10, 2], cap=100)
    assert [r.rid for r in res] == list(range(6))
    assert [r.fields for r in res] == [8, 12, 6, 4, 10, 2]
    assert all(r.finished >= r.admitted >= r.arrival for r in res)


def test_footprint_cap_is_never_exceeded_and_admission_waits():
    sizes = {0: 60, 1: 50, 2: 30, 3: 70}
    eng, be, res = _run(sizes, [0.0, 0.0, 0.0, 0.0], [40, 40, 40, 40], cap=100)
    assert eng.peak_bytes <= 100
    # FIFO: request 1 (50) cannot join request 0 (60); it is admitted only after 0 finishes,
    # and request 2 is not admitted ahead of it
    order = [e[1] for e in be.log if e[0] == "create"]
    assert order == [0, 1, 2, 3]
    r = {x.rid: x for x in res}
    assert r[1].admitted >= r[0].finished - 1e-12


def test_work_overlaps_when_memory_allows():
    eng, be, res = _run({i: 10 for i in range(5)}, [0.0] * 5, [20] * 5, cap=100)
    assert eng.peak_active == 5
    # all five run concurrently: the last finishes long before 5 sequential runs would
    assert max(r.finished for r in res) < 5 * 20 * 1e-3


def test_max_active_limits_concurrency():
    eng, be, res = _run({i: 1 for i in range(6)}, [0.0] * 6, [8] * 6, cap=100, max_active=2)
    assert eng.peak_active == 2


def test_oversized_request_is_rejected():
    with pytest.raises(ValueError):
        _run({0: 500}, [0.0], [4], cap=100)


def test_odd_remainders_and_ticks():
    eng, be, res = _run({0: 1}, [0.0], [11], cap=10, tick=4)
    launches = [e[2] for e in be.log if e[0] == "launch"]
    assert launches == [4, 4, 3]


def test_percentile():
    assert percentile([1, 2, 3, 4], 50) == 2.5
    assert percentile([5], 99) == 5


# ------------------------------------------------------------------ the batch engine (persistent kernel)
class FakeBatchBackend:
    """A batch of slots on a virtual clock: a tick of k steps costs `cost` per step of the resident
    shots together (one launch serves all of them); each slot advances by its own remaining count."""

    def __init__(self, clock, sizes, max_shots=4, cost=1e-3):
        self.clock, self.sizes, self.cost = clock, sizes, cost
        self.rem = [-1] * max_shots
        self.steps = [0] * max_shots
        self.rid = [None] * max_shots
        self.log = []

    def footprint(self, problem):
        return self.sizes[problem]

    def admit(self, problem, nsteps, cfl, dt=None):
        slot = self.rem.index(-1)
        self.rem[slot], self.steps[slot], self.rid[slot] = nsteps, 0, problem
        self.log.append(("admit", problem, slot))
        return slot, 0.01

    def step(self, k):
        self.clock.t += k * self.cost
        for s in range(len(self.rem)):
            if self.rem[s] > 0:
                n = min(k, self.rem[s])
                self.rem[s] -= n
                self.steps[s] += n
        self.log.append(("step", k, tuple(r for r in self.rem)))

    def poll(self):
        return list(self.rem)

    def retire(self, slot):
        self.log.append(("retire", self.rid[slot], slot))
        out = self.steps[slot]
        self.rem[slot] = -1
        return out


def _run_batch(sizes, arrivals, nsteps, cap, max_active=4, tick=4):
    from paper_2003_12811_gb300.serve import BatchServingEngine
    clk = VClock()
    be = FakeBatchBackend(clk, sizes, max_shots=max_active)
    eng = BatchServingEngine(cap, backend=be, tick_steps=tick, max_active=max_active, clock=clk, sleep=clk.sleep)
    reqs = [Request(rid=i, arrival=a, problem=i, nsteps=n) for i, (a, n) in enumerate(zip(arrivals, nsteps))]
    return eng, be, eng.run(reqs)


def test_batch_engine_completes_every_request_with_its_steps():
    eng, be, res = _run_batch({i: 10 for i in range(7)}, [0.0, 0.0, 0.001, 0.002, 0.01, 0.05, 0.5],
                              [8, 13, 6, 4, 10, 2, 5], cap=100)
    assert [r.rid for r in res] == list(range(7))
    assert [r.fields for r in res] == [8, 13, 6, 4, 10, 2, 5]
    assert all(r.finished >= r.admitted >= r.arrival for r in res)


def test_batch_engine_shares_ticks_and_respects_slots_and_cap():
    sizes = {0: 40, 1: 40, 2: 40, 3: 10, 4: 10}
    eng, be, res = _run_batch(sizes, [0.0] * 5, [40, 40, 8, 8, 8], cap=90, max_active=4)
    assert eng.peak_bytes <= 90 and eng.peak_active <= 4
    # 0 and 1 are resident together (one tick advances both); 2 waits for memory (FIFO: 3 and 4
    # are not admitted ahead of it)
    admits = [e[1] for e in be.log if e[0] == "admit"]
    assert admits == [0, 1, 2, 3, 4]
    r = {x.rid: x for x in res}
    assert r[2].admitted >= r[0].finished - 1e-12
    first_step = next(e for e in be.log if e[0] == "step")
    assert sum(1 for x in first_step[2] if x >= 0) == 2


def test_batch_engine_admits_between_ticks_while_others_run():
    eng, be, res = _run_batch({0: 10, 1: 10}, [0.0, 0.0105], [40, 4], cap=100, tick=4)
    r = {x.rid: x for x in res}
    # request 1 joins while request 0 is still running and finishes first
    assert r[1].admitted < r[0].finished and r[1].finished < r[0].finished


def test_batch_engine_makes_a_callable_payload_once():
    """A request that waits for memory is looked at on several passes; its payload (a callable that
    builds the problem) is made once."""
    from paper_2003_12811_gb300.serve import BatchServingEngine
    clk = VClock()
    be = FakeBatchBackend(clk, {0: 80, 1: 80}, max_shots=2)
    calls = {0: 0, 1: 0}

    def make(i):
        calls[i] += 1
        return i

    eng = BatchServingEngine(100, backend=be, tick_steps=4, max_active=2, clock=clk, sleep=clk.sleep)
    reqs = [Request(rid=i, arrival=0.0, problem=(lambda i=i: make(i)), nsteps=20) for i in range(2)]
    res = eng.run(reqs)
    assert [r.fields for r in res] == [20, 20]
    assert calls == {0: 1, 1: 1}


class FakeAsyncBatchBackend(FakeBatchBackend):
    """Retirement in two halves, as the GPU backend does it: retire_async frees the slot and starts
    the read-back, collect (one poll later) returns the fields and releases the memory."""

    def __init__(self, *a, **k):
        super().__init__(*a, **k)
        self.open = 0

    def retire_async(self, slot):
        out = self.retire(slot)
        self.open += 1
        return out

    def collect(self, h):
        self.open -= 1
        self.log.append(("collect", h))
        return h


def test_batch_engine_asynchronous_retirement_matches_and_respects_the_cap():
    from paper_2003_12811_gb300.serve import BatchServingEngine
    sizes = {0: 40, 1: 40, 2: 40, 3: 10, 4: 10}
    arrivals, nsteps = [0.0] * 5, [40, 40, 8, 8, 8]
    clk = VClock()
    be = FakeAsyncBatchBackend(clk, sizes, max_shots=4)
    eng = BatchServingEngine(90, backend=be, tick_steps=4, max_active=4, clock=clk, sleep=clk.sleep)
    res = eng.run([Request(rid=i, arrival=a, problem=i, nsteps=n) for i, (a, n) in enumerate(zip(arrivals, nsteps))])
    assert [r.fields for r in res] == nsteps
    assert be.open == 0 and eng.peak_bytes <= 90
    # a shot's memory counts until its result is collected: request 2 (40) is admitted only after
    # one of the first two is collected
    first_collect = next(i for i, e in enumerate(be.log) if e[0] == "collect")
    admit2 = next(i for i, e in enumerate(be.log) if e[0] == "admit" and e[1] == 2)
    assert admit2 > first_collect
