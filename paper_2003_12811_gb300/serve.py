"""Continuous batching of independent forward solves ("shots") on one GPU.

Requests arrive over time (each with its own grid, material, sources and step count).  An
engine admits a waiting request as soon as a slot is free and its device footprint
(``sbp_grid_footprint``) fits under the HBM cap, keeps every admitted shot's wavefield resident,
and advances the active shots in ticks of ``tick_steps`` leapfrog steps; when a shot finishes,
its result is read back, its memory is released and the next request is admitted -- while the
others keep running.  Two engines:

* ``BatchServingEngine`` (the serving path): every active shot lives in one ``sbp_batch``; a
  tick is one CUDA-graph replay of ``tick_steps`` launches of the persistent tile-queue kernel,
  whose CTAs pull interior and boundary tiles of all resident shots from one device queue.
* ``ServingEngine``: each shot on its own CUDA stream, ticks replayed from a per-shot CUDA graph
  (``sbp_step_graph``); the kernels of different shots overlap through the streams.

All arithmetic is in libsbp; this module only schedules.  The scheduling logic is written
against small backend interfaces so that it can be exercised without a GPU.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Any, Callable, List, Optional


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float                 # seconds after the engine starts
    problem: Any                   # workloads.Problem, or a callable returning it (made on admission)
    nsteps: int
    dt: Optional[float] = None     # None: dt = suggest_dt(cfl) of the shot


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    nsteps: int
    dt: float
    fields: Any                    # final displacement per block (host arrays), or backend data

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class GpuBackend:
    """libsbp shots on CUDA streams (torch streams/events are used only as handles)."""

    def __init__(self, precision="fp32", autotune=True):
        import torch
        from .binding import Solver, footprint_bytes
        self.torch = torch
        self.Solver = Solver
        self.footprint_bytes = footprint_bytes
        self.precision = precision
        self.autotune = autotune
        self._tuned = {}

    def footprint(self, problem) -> int:
        return self.footprint_bytes(problem, self.precision)

    def create(self, problem, cfl, dt=None):
        import numpy as np
        torch = self.torch
        S = self.Solver(problem, self.precision)
        if dt is None:
            dt = S.suggest_dt(cfl)
        z = [np.zeros((2, b.N2, b.N1)) for b in problem.blocks]
        S.set_state(z, z, 0.0)
        if self.autotune:
            key = tuple((b.N1, b.N2) for b in problem.blocks) + (problem.order,)
            if key not in self._tuned:
                self._tuned[key] = S.sbp_autotune()
            else:
                S.sbp_set_tuning(*self._tuned[key])
        return _GpuShot(S, torch.cuda.Stream(), dt, torch)


class _GpuShot:
    def __init__(self, solver, stream, dt, torch):
        self.S = solver
        self.stream = stream
        self.dt = dt
        self.torch = torch
        self.event = None

    def launch(self, nsteps):
        h = self.stream.cuda_stream
        if nsteps % 2 == 0:
            self.S.sbp_step_graph(nsteps, self.dt, h)
        else:
            self.S.sbp_step(nsteps, self.dt, h)
        self.event = self.torch.cuda.Event()
        self.event.record(self.stream)

    def busy(self) -> bool:
        return self.event is not None and not self.event.query()

    def result(self):
        self.stream.synchronize()
        _, u = self.S.state()
        return u

    def close(self):
        self.S.close()


class ServingEngine:
    def __init__(self, hbm_cap_bytes: int, backend=None, tick_steps: int = 32, max_active: int = 16,
                 cfl: float = 0.3, clock: Callable[[], float] = time.perf_counter,
                 idle_sleep: float = 2e-4, sleep: Callable[[float], None] = time.sleep):
        if tick_steps < 2 or tick_steps % 2:
            raise ValueError("tick_steps must be an even number >= 2")
        self.cap = int(hbm_cap_bytes)
        self.backend = backend if backend is not None else GpuBackend()
        self.tick = tick_steps
        self.max_active = max_active
        self.cfl = cfl
        self.clock = clock
        self.idle_sleep = idle_sleep
        self.sleep = sleep
        self.peak_bytes = 0           # largest admitted footprint sum seen
        self.peak_active = 0
        self.trace: List[tuple] = []  # (time, event, rid) for inspection

    def run(self, requests: List[Request]) -> List[Result]:
        pending = collections.deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        waiting: collections.deque = collections.deque()
        active = []
        used = 0
        results = []
        t0 = self.clock()
        while pending or waiting or active:
            now = self.clock() - t0
            progressed = False
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            # admission: first come, first served, by device footprint
            while waiting and len(active) < self.max_active:
                req = waiting[0]
                prob = _problem_of(req)
                fp = self.backend.footprint(prob)
                if fp > self.cap:
                    raise ValueError(f"request {req.rid} needs {fp} bytes, more than the cap {self.cap}")
                if used + fp > self.cap:
                    break
                waiting.popleft()
                shot = self.backend.create(prob, self.cfl, req.dt)
                used += fp
                self.peak_bytes = max(self.peak_bytes, used)
                active.append(dict(req=req, shot=shot, fp=fp, done=0, admitted=self.clock() - t0))
                self.peak_active = max(self.peak_active, len(active))
                self.trace.append((self.clock() - t0, "admit", req.rid))
                progressed = True
            # progress every active shot whose previous tick has finished
            still = []
            for slot in active:
                shot, req = slot["shot"], slot["req"]
                if shot.busy():
                    still.append(slot)
                    continue
                if slot["done"] >= req.nsteps:
                    fields = shot.result()
                    shot.close()
                    used -= slot["fp"]
                    t = self.clock() - t0
                    results.append(Result(req.rid, req.arrival, slot["admitted"], t, req.nsteps, shot.dt, fields))
                    self.trace.append((t, "finish", req.rid))
                    progressed = True
                    continue
                n = min(self.tick, req.nsteps - slot["done"])
                shot.launch(n)
                slot["done"] += n
                still.append(slot)
                progressed = True
            active = still
            if not progressed:
                if pending and not waiting and not active:
                    # nothing resident: jump to the next arrival instead of spinning
                    wait = pending[0].arrival - (self.clock() - t0)
                    if wait > 0:
                        self.sleep(min(wait, 0.05))
                else:
                    self.sleep(self.idle_sleep)
        return sorted(results, key=lambda r: r.rid)


def _problem_of(req):
    """The request's problem; a callable payload is made once and kept with the request."""
    if callable(req.problem):
        req.problem = req.problem()
    return req.problem


class GpuBatchBackend:
    """Shots in one libsbp batch (persistent tile-queue kernel), stepped on one CUDA stream."""

    def __init__(self, order=6, max_shots=256, rows=0, precision="fp32"):
        import torch
        from .binding import Batch, Solver, footprint_bytes
        if precision != "fp32":
            raise ValueError("the batch kernel steps FP32 shots")
        self.torch = torch
        self.Solver = Solver
        self.footprint_bytes = footprint_bytes
        self.batch = Batch(order, max_shots)
        if rows:
            self.batch.sbp_batch_set_rows(rows)
        self.stream = torch.cuda.Stream()
        self.side = torch.cuda.Stream()
        self._ev0 = torch.cuda.Event(enable_timing=True)
        self._ev1 = torch.cuda.Event(enable_timing=True)
        self.max_shots = max_shots
        self.shots = {}

    def footprint(self, problem) -> int:
        return self.footprint_bytes(problem, "fp32")

    def admit(self, problem, nsteps, cfl, dt=None):
        # a new handle's state is zero at t = 0 (its buffers are cleared when allocated): a shot
        # that starts at rest needs no state upload
        S = self.Solver(problem, "fp32")
        if dt is None:
            dt = S.suggest_dt(cfl)
        slot = self.batch.sbp_batch_add(S, nsteps, dt)
        self.shots[slot] = S
        return slot, dt

    def step(self, k):
        self._ev0.record(self.stream)
        self.batch.sbp_batch_step(k, self.stream.cuda_stream)
        self._ev1.record(self.stream)

    def poll(self):
        return self.batch.sbp_batch_poll(self.stream.cuda_stream)

    def tick_seconds(self):
        """Device time of the last tick (valid after poll)."""
        return self._ev0.elapsed_time(self._ev1) / 1e3

    def retire(self, slot):
        return self.collect(self.retire_async(slot))

    def retire_async(self, slot):
        """Free the slot and start reading the shot's u^n back on a side stream (the next tick may
        already be queued on the batch stream; a finished shot no longer changes).  collect() waits
        for the copy, releases the handle and returns the fields."""
        from .binding import FIELD_CUR
        torch = self.torch
        self.batch.sbp_batch_remove(slot, self.stream.cuda_stream)
        S = self.shots.pop(slot)
        outs = []
        with torch.cuda.stream(self.side):
            for b, blk in enumerate(S.problem.blocks):
                pitch = (blk.N1 + 3) // 4 * 4                  # 16-byte rows
                dev = torch.empty((2, blk.N2, pitch), dtype=torch.float32, device="cuda")
                S.sbp_get_field_device(b, FIELD_CUR, dev.data_ptr(), pitch, self.side.cuda_stream)
                host = torch.empty(dev.shape, dtype=torch.float32, pin_memory=True)
                host.copy_(dev, non_blocking=True)
                outs.append((host, blk.N1, dev))
            ev = torch.cuda.Event()
            ev.record(self.side)
        return S, outs, ev

    def collect(self, pending):
        S, outs, ev = pending
        ev.synchronize()
        fields = [host[:, :, :n1].numpy().astype("float64") for host, n1, _ in outs]
        S.close()
        return fields

    def close(self):
        for S in self.shots.values():
            S.close()
        self.shots = {}
        self.batch.close()


class BatchServingEngine:
    """Continuous batching on the persistent tile-queue kernel (see the module docstring).

    The engine launches the next tick of every resident shot, admits waiting requests first come
    first served while slots and the HBM cap allow and while the tick runs (for about one tick's
    device time, at least one request: admission is host-side setup, so the GPU is kept busy), then
    waits for the tick and retires finished shots (reading their results).  Each shot advances by
    its own step count."""

    def __init__(self, hbm_cap_bytes: int, backend=None, tick_steps: int = 32, max_active: int = 256,
                 cfl: float = 0.3, clock: Callable[[], float] = time.perf_counter,
                 sleep: Callable[[float], None] = time.sleep, min_admit_budget: float = 2e-3):
        if tick_steps < 1:
            raise ValueError("tick_steps must be >= 1")
        self.cap = int(hbm_cap_bytes)
        self.backend = backend if backend is not None else GpuBatchBackend(max_shots=max_active)
        self.tick = tick_steps
        self.max_active = max_active
        self.cfl = cfl
        self.clock = clock
        self.sleep = sleep
        self.min_admit_budget = min_admit_budget
        self.peak_bytes = 0
        self.peak_active = 0
        self.ticks = 0
        # host time per phase of the loop: tick launch, admissions, waiting for the tick, retirement
        self.phase_s = {"launch": 0.0, "admit": 0.0, "poll": 0.0, "retire": 0.0}
        self.trace: List[tuple] = []

    def run(self, requests: List[Request]) -> List[Result]:
        pending = collections.deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        waiting: collections.deque = collections.deque()
        active = {}                       # slot -> dict(req, fp, admitted, dt)
        retiring = []                     # (info, backend handle) of results being read back
        asynchronous = hasattr(self.backend, "retire_async")
        used = 0
        results = []
        tick_est = 0.0                    # device time of the last tick
        t0 = self.clock()

        def finish(info, fields):
            nonlocal used
            used -= info["fp"]
            t = self.clock() - t0
            req = info["req"]
            results.append(Result(req.rid, req.arrival, info["admitted"], t, req.nsteps, info["dt"], fields))
            self.trace.append((t, "finish", req.rid))

        def collect():
            # release the shots retired at the previous poll: their read-back ran beside the
            # current tick; freeing their device memory waits for the device, as the poll does
            t_c = self.clock()
            for info, hnd in retiring:
                finish(info, self.backend.collect(hnd))
            retiring.clear()
            self.phase_s["retire"] += self.clock() - t_c

        while pending or waiting or active or retiring:
            now = self.clock() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            # the next tick of every resident shot goes to the GPU first; new shots are set up
            # while it runs (for about the tick's duration) and join at the following tick
            launched = bool(active)
            if launched:
                t_l = self.clock()
                self.backend.step(self.tick)
                self.ticks += 1
                self.phase_s["launch"] += self.clock() - t_l
            budget = max(self.min_admit_budget, tick_est if launched else 0.0)
            t_adm = self.clock()
            while waiting and len(active) < self.max_active:
                req = waiting[0]
                prob = _problem_of(req)
                fp = self.backend.footprint(prob)
                if fp > self.cap:
                    raise ValueError(f"request {req.rid} needs {fp} bytes, more than the cap {self.cap}")
                if used + fp > self.cap:
                    break
                waiting.popleft()
                slot, dt = self.backend.admit(prob, req.nsteps, self.cfl, req.dt)
                used += fp
                self.peak_bytes = max(self.peak_bytes, used)
                active[slot] = dict(req=req, fp=fp, admitted=self.clock() - t0, dt=dt)
                self.peak_active = max(self.peak_active, len(active))
                self.trace.append((self.clock() - t0, "admit", req.rid))
                if self.clock() - t_adm >= budget:
                    break
            self.phase_s["admit"] += self.clock() - t_adm
            collect()
            if launched:
                t_p = self.clock()
                rem = self.backend.poll()
                if hasattr(self.backend, "tick_seconds"):
                    tick_est = self.backend.tick_seconds()
                t_r = self.clock()
                self.phase_s["poll"] += t_r - t_p
                for slot in sorted(active):
                    if rem[slot] == 0:
                        info = active.pop(slot)
                        if asynchronous:
                            retiring.append((info, self.backend.retire_async(slot)))
                        else:
                            finish(info, self.backend.retire(slot))
                self.phase_s["retire"] += self.clock() - t_r
            elif not active and pending and not retiring:
                wait = pending[0].arrival - (self.clock() - t0)
                if wait > 0:
                    self.sleep(min(wait, 0.05))
        return sorted(results, key=lambda r: r.rid)


def percentile(values, q):
    v = sorted(values)
    if not v:
        return float("nan")
    k = (len(v) - 1) * q / 100.0
    lo, hi = int(k), min(int(k) + 1, len(v) - 1)
    return v[lo] + (v[hi] - v[lo]) * (k - lo)
