"""Continuous-batching server for Swendsen-Wang chains.

A request asks for one Markov chain of the periodic 2D Ising model: side L,
inverse temperature beta, seed, start (hot or cold) and a number of sweeps;
its result is the per-sweep energy and magnetisation trace (§2.4's E and M
after every sweep) and, on request, the final spins. The chain a request
gets is the chain its parameters fix: the same bits whether it runs alone
or beside any other requests (every draw is keyed by the replica's own seed,
sweep counter and site, §2.1).

The server keeps one sw_batch. Each scheduling step it
  1. admits queued requests in arrival order while the device bytes of the
     admitted replicas (sw_batch_footprint) stay within the memory budget,
     each with a sweep limit equal to its request (sw_batch_set_limit);
  2. advances the whole batch by one chunk of sweeps (one replay of a
     captured CUDA graph, the same chunk every time); a replica that
     reaches its sweep limit inside a chunk idles for the rest of it (its
     tiles return at once), so every request stops exactly at its count
     while the others keep full chunks;
  3. reads back the traces of the replicas that reached their target and
     frees their slots.
A request that cannot be served (invalid parameters, larger than the whole
budget, a failed allocation) gets a result with ``error`` set; the others
go on. All arithmetic runs in libsw's kernels; this module schedules.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Callable, Iterable, Optional

import numpy as np

from . import (SW_INIT_HOT, SWError, sw_batch_add, sw_batch_create, sw_batch_destroy, sw_batch_footprint,
               sw_batch_get_sweep, sw_batch_info, sw_batch_observables, sw_batch_remove, sw_batch_set_limit,
               sw_batch_spins, sw_batch_sweep)


@dataclasses.dataclass
class Request:
    rid: int
    L: int
    beta: float
    seed: int
    sweeps: int
    init: int = SW_INIT_HOT
    arrival: float = 0.0          # seconds after the server's start
    want_spins: bool = False


@dataclasses.dataclass
class Result:
    rid: int
    E: Optional[np.ndarray] = None      # int64 [sweeps]
    M: Optional[np.ndarray] = None      # int64 [sweeps]
    spins: Optional[np.ndarray] = None  # int8 [L][L] after the last sweep
    error: Optional[str] = None
    arrival: float = 0.0
    admitted: float = float("nan")
    finished: float = float("nan")

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class BatchBackend:
    """The libsw batch calls the server uses (a seam for host-only tests)."""

    def __init__(self, shape: int = -1, stream: int | None = None):
        self.b = sw_batch_create([], [], [], shape=shape, stream=stream)

    def footprint(self, L, sweeps):
        return sw_batch_footprint(self.b, L, sweeps)

    def add(self, L, beta, seed, init):
        return sw_batch_add(self.b, L, beta, seed, init)

    def set_limit(self, slot, sweeps):
        sw_batch_set_limit(self.b, slot, sweeps)

    def sweep(self, n):
        sw_batch_sweep(self.b, n)

    def sweep_count(self, slot):
        return sw_batch_get_sweep(self.b, slot)

    def observables(self, slot, count):
        return sw_batch_observables(self.b, slot, 0, count)

    def spins(self, slot, L):
        return sw_batch_spins(self.b, slot, L)

    def remove(self, slot):
        sw_batch_remove(self.b, slot)

    def info(self):
        return sw_batch_info(self.b)

    def close(self):
        if self.b:
            sw_batch_destroy(self.b)
            self.b = None


@dataclasses.dataclass
class _Live:
    req: Request
    slot: int
    footprint: int
    admitted: float


class Server:
    # 128 x 64 tiles with 2-row strips: the sweep's own choice for L > 64,
    # which is where a serving mix spends its time.
    DEFAULT_SHAPE = 6

    def __init__(self, budget_bytes: int, chunk: int = 64, backend=None, shape: int = DEFAULT_SHAPE,
                 stream: int | None = None, clock: Callable[[], float] = time.perf_counter):
        if chunk < 1:
            raise ValueError("chunk must be >= 1")
        self.budget = int(budget_bytes)
        self.chunk = int(chunk)
        self.backend = backend if backend is not None else BatchBackend(shape=shape, stream=stream)
        self.clock = clock
        self.t0 = clock()
        self.queue: collections.deque[Request] = collections.deque()
        self.live: dict[int, _Live] = {}
        self.used = 0             # device bytes of the live replicas
        self.site_updates = 0
        self.steps = 0

    def now(self) -> float:
        return self.clock() - self.t0

    def close(self):
        self.backend.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---------------------------------------------------------------- steps
    def submit(self, req: Request) -> None:
        self.queue.append(req)

    def _fail(self, req: Request, msg: str) -> Result:
        t = self.now()
        return Result(req.rid, error=msg, arrival=req.arrival, admitted=t, finished=t)

    def admit(self) -> list[Result]:
        """Admit queued requests in order while they fit; failed ones return."""
        failed = []
        while self.queue:
            req = self.queue[0]
            if req.sweeps < 0:
                self.queue.popleft()
                failed.append(self._fail(req, "sweeps must be >= 0"))
                continue
            try:
                fp = self.backend.footprint(req.L, req.sweeps)
            except SWError as e:
                self.queue.popleft()
                failed.append(self._fail(req, str(e)))
                continue
            if fp > self.budget:
                self.queue.popleft()
                failed.append(self._fail(req, f"needs {fp} device bytes, budget is {self.budget}"))
                continue
            if self.used + fp > self.budget:
                break   # head of line waits for memory
            self.queue.popleft()
            try:
                slot = self.backend.add(req.L, req.beta, req.seed, req.init)
            except SWError as e:
                failed.append(self._fail(req, str(e)))
                continue
            self.backend.set_limit(slot, req.sweeps)
            self.live[slot] = _Live(req, slot, fp, self.now())
            self.used += fp
        return failed

    def advance(self) -> int:
        """Run one chunk over the live replicas; returns its length (0 if idle)."""
        left = {s: lv.req.sweeps - self.backend.sweep_count(s) for s, lv in self.live.items()}
        if not any(r > 0 for r in left.values()):
            return 0
        n = self.chunk
        self.backend.sweep(n)
        for s, lv in self.live.items():
            self.site_updates += min(n, max(left[s], 0)) * lv.req.L * lv.req.L
        self.steps += 1
        return n

    def collect(self) -> list[Result]:
        """Results of the replicas that reached their sweep count."""
        out = []
        for slot in [s for s, lv in self.live.items() if self.backend.sweep_count(s) >= lv.req.sweeps]:
            lv = self.live.pop(slot)
            req = lv.req
            res = Result(req.rid, arrival=req.arrival, admitted=lv.admitted)
            try:
                res.E, res.M = self.backend.observables(slot, req.sweeps)
                if req.want_spins:
                    res.spins = self.backend.spins(slot, req.L)
            except SWError as e:
                res.error = str(e)
            res.finished = self.now()
            self.backend.remove(slot)
            self.used -= lv.footprint
            out.append(res)
        return out

    def step(self) -> list[Result]:
        done = self.admit()
        self.advance()
        done += self.collect()
        return done

    # ------------------------------------------------------------- drivers
    def run(self, requests: Iterable[Request], realtime: bool = True) -> list[Result]:
        """Serve `requests` (sorted by arrival) to completion.

        With realtime, a request enters the queue once the wall clock since
        the server's start passes its arrival time; otherwise all requests
        are queued at once and arrivals only label the results.
        """
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        results: list[Result] = []
        self.t0 = self.clock()
        while pending or self.queue or self.live:
            now = self.now()
            while pending and (not realtime or pending[0].arrival <= now):
                self.submit(pending.popleft())
            results += self.step()
            if not self.live and not self.queue and pending and realtime:
                time.sleep(max(0.0, min(pending[0].arrival - self.now(), 0.05)))
        return results


def latency_summary(results: list[Result]) -> dict:
    ok = [r.latency for r in results if r.error is None]
    if not ok:
        return {"served": 0, "failed": len(results)}
    lat = np.asarray(ok)
    return {"served": len(ok), "failed": len(results) - len(ok),
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "max_s": float(lat.max())}
