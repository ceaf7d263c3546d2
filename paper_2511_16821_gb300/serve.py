"""Continuous-batching server for hybrid solves.

Requests (a problem description and a number of time steps) arrive over time. The server admits
them as device memory (a fixed budget, counted from each problem's workspace size) and slots free
up, keeps their census banks, tallies and collided-flux state resident between steps, and on each
tick advances every resident problem by one step together: one batched MC-leg launch over all
their histories, then their collided solves and remaps as concurrent branches (``hyb.Batch`` in
eager mode, rebuilt when the resident set changes). Requests that arrive while others are on the
GPU join at the next tick, so their work overlaps on the device.

Step latency of a request's step k = completion time of that step minus the time it became
eligible (arrival for k = 0, completion of step k - 1 otherwise); p50/p99 are over all steps.
Each request's results are those of solving it alone (the batch is exact per problem).
"""
from __future__ import annotations

import math
import random
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import hyb
from . import workloads as W


@dataclass
class Request:
    rid: int
    spec: W.ProblemSpec
    steps: int
    t_arrival: float
    problem: object = None
    ws_bytes: int = 0
    done_steps: int = 0
    t_ready: float = 0.0
    t_admit: float = -1.0
    t_done: float = -1.0
    step_latency: list = field(default_factory=list)
    histories: int = 0
    flux: np.ndarray | None = None
    bank: dict | None = None


class Server:
    def __init__(self, budget_bytes: float = 120e9, max_active: int = 512, tuning: dict | None = None,
                 clock=None, keep_banks: bool = False):
        import torch
        self.torch = torch
        self.keep_banks = keep_banks      # copy each finished request's census bank to the host
        self.budget = float(budget_bytes)
        self.max_active = max_active
        self.tuning = dict(block=256, chunk=4096, streams=16, use_graph=0)
        if tuning:
            self.tuning.update(tuning)
            self.tuning["use_graph"] = 0
        self.clock = clock or time.perf_counter
        self.stream = torch.cuda.Stream()
        self.queue: list[Request] = []
        self.active: list[Request] = []
        self.finished: list[Request] = []
        self.used = 0.0
        self.batch = None
        self.members: tuple = ()
        self.ticks = 0
        self.peak_used = 0.0
        self.rebuilds = 0
        # problems are created by a worker thread on a stream of its own (device memory reserved at
        # admission), so creation stays off the step loop; ready problems join at the next tick
        self.async_create = True
        self.ready: list[Request] = []
        self.creating = 0
        self._cv = threading.Condition()
        self._stop = False
        self._create_stream = torch.cuda.Stream()
        self._creator = None

    # ---- admission --------------------------------------------------------------------------
    def submit(self, spec: W.ProblemSpec, steps: int, t_arrival: float | None = None, rid: int | None = None) -> Request:
        r = Request(rid=len(self.finished) + len(self.active) + len(self.queue) if rid is None else rid,
                    spec=spec, steps=int(steps), t_arrival=self.clock() if t_arrival is None else t_arrival)
        r.ws_bytes = hyb.workspace_size(spec)
        if r.ws_bytes > self.budget:
            raise ValueError(f"request {r.rid} needs {r.ws_bytes} bytes, above the whole budget")
        r.t_ready = r.t_arrival
        with self._cv:
            self.queue.append(r)
            self._cv.notify_all()
        return r

    def _admissible(self) -> bool:
        return bool(self.queue) and len(self.active) + len(self.ready) + self.creating < self.max_active and \
            self.used + self.queue[0].ws_bytes <= self.budget

    def _create_loop(self) -> None:
        torch = self.torch
        while True:
            with self._cv:
                while not self._stop and not self._admissible():
                    self._cv.wait(0.05)
                if self._stop:
                    return
                r = self.queue.pop(0)
                self.used += r.ws_bytes            # reserved before the problem exists
                self.peak_used = max(self.peak_used, self.used)
                self.creating += 1
            with torch.cuda.stream(self._create_stream):
                r.problem = hyb.Problem(r.spec, stream=self._create_stream)
            with self._cv:
                self.creating -= 1
                self.ready.append(r)

    def _admit(self) -> None:
        if self.async_create:
            if self._creator is None:
                self._creator = threading.Thread(target=self._create_loop, daemon=True)
                self._creator.start()
            with self._cv:
                ready, self.ready = self.ready, []
                self._cv.notify_all()
            t = self.clock()
            for r in ready:
                r.t_admit = t
                self.active.append(r)
            return
        while self._admissible():
            r = self.queue.pop(0)
            with self.torch.cuda.stream(self.stream):
                r.problem = hyb.Problem(r.spec, stream=self.stream)
            self.used += r.ws_bytes
            self.peak_used = max(self.peak_used, self.used)
            r.t_admit = self.clock()
            self.active.append(r)

    def _retire(self) -> None:
        keep = []
        for r in self.active:
            if r.done_steps >= r.steps:
                r.flux = r.problem.tally("flux")
                if self.keep_banks:
                    r.bank = r.problem.bank()
                r.problem.close()
                r.problem = None
                with self._cv:
                    self.used -= r.ws_bytes
                    self._cv.notify_all()
                r.t_done = self.clock()
                self.finished.append(r)
            else:
                keep.append(r)
        self.active = keep

    # ---- one tick: every resident problem advances one step ----------------------------------
    def tick(self) -> int:
        self._admit()
        if not self.active:
            return 0
        members = tuple(r.rid for r in self.active)
        if members != self.members:
            # the resident set changed: the batch keeps its streams and buffers, takes the new set
            if self.batch is None:
                self.batch = hyb.Batch([r.problem for r in self.active], stream=self.stream, tuning=self.tuning)
            else:
                self.batch.set_problems([r.problem for r in self.active])
            self.members = members
            self.rebuilds += 1
        stats = self.batch.step(1)
        t = self.clock()
        for r, s in zip(self.active, stats):
            r.step_latency.append(t - r.t_ready)
            r.t_ready = t
            r.done_steps += 1
            r.histories += s["histories"]
        self.ticks += 1
        n = len(self.active)
        self._retire()
        return n

    # ---- drivers ----------------------------------------------------------------------------
    def run_schedule(self, schedule: list[tuple[int, W.ProblemSpec, int]]) -> list[Request]:
        """Deterministic driver: schedule entries (tick, spec, steps) are submitted at that tick and
        admitted at once when memory allows (problems created on the step loop)."""
        self.async_create = False
        pending = sorted(enumerate(schedule), key=lambda e: e[1][0])
        k = 0
        tick = 0
        while k < len(pending) or self.queue or self.active:
            while k < len(pending) and pending[k][1][0] <= tick:
                i, (_, spec, steps) = pending[k]
                self.submit(spec, steps, rid=i)
                k += 1
            self.tick()
            tick += 1
        return sorted(self.finished, key=lambda r: r.rid)

    def run_poisson(self, lam: float, duration: float, seed: int = 0, max_side: int = 256,
                    hist_cap: int | None = None, drain: float = 30.0) -> dict:
        """Wall-clock driver: Poisson arrivals of rate lam for `duration` seconds, each request drawn
        from the batched distribution with 1..64 steps and dt in [0.05, 0.2] (`arrivals`); after the
        arrival window the server runs until drained or for at most `drain` more seconds. Latency
        statistics cover the steps completed; requests still queued or resident are counted."""
        arrivals = poisson_arrivals(lam, duration, seed, max_side, hist_cap)
        t0 = self.clock()
        k = 0
        while k < len(arrivals) or self.queue or self.active or self.ready or self.creating:
            now = self.clock() - t0
            if now > duration + drain:
                break
            while k < len(arrivals) and arrivals[k][0] <= now:
                ta, spec, steps = arrivals[k]
                self.submit(spec, steps, t_arrival=t0 + ta, rid=k)
                k += 1
            if not self.tick():
                time.sleep(0.0005 if (self.queue or self.creating) else
                           max(0.0, min(arrivals[k][0] - (self.clock() - t0), 0.01)) if k < len(arrivals) else 0.0)
        wall = self.clock() - t0
        return latency_summary(lam, duration, arrivals, self.finished, self.active + self.queue, wall,
                               ticks=self.ticks, rebuilds=self.rebuilds, peak_bytes=self.peak_used)

    def close(self) -> None:
        with self._cv:
            self._stop = True
            self._cv.notify_all()
        if self._creator is not None:
            self._creator.join()
            self._creator = None
        if self.batch is not None:
            self.batch.close()
            self.batch = None
        for r in self.active + self.queue + self.ready:
            if r.problem is not None:
                r.problem.close()


def poisson_arrivals(lam: float, duration: float, seed: int = 0, max_side: int = 256,
                     hist_cap: int | None = None) -> list:
    """(arrival time, problem, steps) of a Poisson stream of rate lam over `duration` seconds; each
    request from the batched distribution with 1..64 steps and dt in [0.05, 0.2]."""
    rng = random.Random(seed)
    arrivals = []
    t = 0.0
    i = 0
    while True:
        t += rng.expovariate(lam)
        if t > duration:
            break
        spec = W.random_batch_problem(seed, i, dt=rng.uniform(0.05, 0.2), max_side=max_side)
        if hist_cap:
            spec = spec.with_(n_hist=min(spec.n_hist, hist_cap))
        arrivals.append((t, spec.with_(sn_warm_start=1), rng.randint(1, 64)))
        i += 1
    return arrivals


def latency_summary(lam, duration, arrivals, finished, unfinished, wall, **extra) -> dict:
    lat = np.array([x for r in finished for x in r.step_latency] +
                   [x for r in unfinished for x in r.step_latency])
    hist = sum(r.histories for r in finished) + sum(r.histories for r in unfinished)
    out = {"lambda": lam, "arrival_s": duration, "arrived": len(arrivals), "requests_done": len(finished),
           "requests_unfinished": len(unfinished), "steps": int(lat.size), "wall_s": wall,
           "histories_per_s": hist / wall if wall > 0 else 0.0,
           "p50_ms": float(np.percentile(lat, 50) * 1e3) if lat.size else math.nan,
           "p99_ms": float(np.percentile(lat, 99) * 1e3) if lat.size else math.nan}
    out.update(extra)
    return out


def run_poisson_plain(lam: float, duration: float, seed: int = 0, max_side: int = 256,
                      hist_cap: int | None = None, drain: float = 30.0, clock=None) -> dict:
    """The plain single-problem path on the same request stream: requests served one at a time in
    arrival order, each problem created and stepped alone (hyb_step) -- the same results as in the
    batch, bit for bit. Step latency as for the server (eligibility to completion), so a request's
    first step includes its wait behind the earlier ones."""
    import torch
    clock = clock or time.perf_counter
    arrivals = poisson_arrivals(lam, duration, seed, max_side, hist_cap)
    stream = torch.cuda.Stream()
    done, t0 = [], clock()
    cur = None
    for k, (ta, spec, steps) in enumerate(arrivals):
        now = clock() - t0
        if now > duration + drain:
            break
        if ta > now:
            time.sleep(ta - now)
        r = Request(rid=k, spec=spec, steps=steps, t_arrival=t0 + ta)
        r.t_ready = r.t_arrival
        with torch.cuda.stream(stream):
            P = hyb.Problem(spec, stream=stream)
        r.t_admit = clock()
        cur = r
        for _ in range(steps):
            st = P.step(1)[0]
            t = clock()
            r.step_latency.append(t - r.t_ready)
            r.t_ready = t
            r.done_steps += 1
            r.histories += st["histories"]
            if t - t0 > duration + drain:
                break
        P.close()
        cur = None
        if r.done_steps == r.steps:
            done.append(r)
        else:
            return latency_summary(lam, duration, arrivals, done, [r], clock() - t0, path="plain")
    del cur
    return latency_summary(lam, duration, arrivals, done, [], clock() - t0, path="plain")
