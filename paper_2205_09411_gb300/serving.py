"""Serving loop: continuous batching of Poisson solves on resident trees.

A session is one fixed geometry (tree, level set, stencils, boundary
values): it stays resident in HBM while its right-hand sides change.  Each
resident session holds `slots` right-hand-side slots (gmg_set_num_rhs); a
request is a new right-hand side for a session, solved to `tol`.

Every tick of the loop:

1. requests whose arrival time has passed join their session's queue;
2. sessions with queued requests are made resident if the HBM budget allows
   (idle resident sessions, those with no request in a slot, are evicted
   least recently used first to make room);
3. queued requests take the free slots of their session
   (gmg_set_rhs_slots) and get their first residual (gmg_iterate_begin with
   residual_only), while the other slots keep their state;
4. every resident session with occupied slots runs one V-cycle (FP64) or
   defect-correction step (mixed) on those slots; the sessions' steps are
   enqueued on their own CUDA streams before any is waited for, so they
   overlap on the device;
5. slots that reached `tol` are read out and freed.

A request's latency is its completion time minus its arrival time (queueing
included).  Because a slot's arithmetic never mixes with another slot's and
a converged slot is frozen, a request's result and cycle count are those of
the same right-hand side solved alone.

The scheduler only needs the tree interface (workspace_bytes, bind,
set_rhs_slots, iterate_begin / iterate_end, solution_slots, close), so its
host logic can be exercised with a stand-in on machines without a GPU.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

__all__ = ["Session", "Request", "Server", "poisson_arrivals", "summarize"]


@dataclass
class Request:
    session: str
    rhs: object                 # leaf-ordered right-hand side, or callable(session) -> it
    arrival: float              # seconds after the start of the run
    id: int = -1
    start: float = float("nan")     # when it took a slot
    done: float = float("nan")      # when its solution was read out
    cycles: int = 0
    rel_l2: float = float("nan")
    result: object = None

    @property
    def latency(self):
        return self.done - self.arrival


@dataclass
class Session:
    name: str
    make: Callable[[int], object]   # slots -> set-up (unbound) tree with that many slots
    tree: object = None
    nbytes: int = 0
    stream: object = None
    slot_req: list = field(default_factory=list)
    active: Optional[np.ndarray] = None
    queue: deque = field(default_factory=deque)
    last_used: float = 0.0
    loads: int = 0
    ctx: dict = field(default_factory=dict)   # per-residency data (e.g. leaf centres on the device)

    @property
    def resident(self):
        return self.tree is not None

    def busy(self):
        return any(r is not None for r in self.slot_req)


def poisson_arrivals(rate: float, n: int, seed: int) -> np.ndarray:
    """n arrival times of a Poisson process of the given rate (per second)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


class Server:
    def __init__(self, sessions, budget_bytes, slots=8, precision=1, tol=1e-8, max_cycles=80, keep_results=True,
                 on_load=None, new_stream=None, clock=time.perf_counter, result_to=None, stream_context=None):
        self.sessions = {s.name: s for s in sessions}
        self.budget = int(budget_bytes)
        self.slots = int(slots)
        self.precision = precision
        self.tol = tol
        self.max_cycles = max_cycles
        self.keep_results = keep_results
        self.on_load = on_load            # callable(session) after bind (e.g. leaf centres to the device)
        self.new_stream = new_stream      # callable() -> stream object passed to the tree calls
        self.clock = clock
        self.result_to = result_to        # callable(session, slot) -> result (default: host copy)
        self.stream_context = stream_context  # callable(session) -> context for building a right-hand side
        self.pending = deque()
        self.completed = []
        self.t0 = None
        self.log = []
        self.peak_bytes = 0
        self.ticks = 0

    # -- memory ---------------------------------------------------------------
    def resident_bytes(self):
        return sum(s.nbytes for s in self.sessions.values() if s.resident)

    def _load(self, s: Session):
        tree = s.make(self.slots)
        nbytes = int(tree.workspace_bytes())
        if nbytes > self.budget:
            raise ValueError("session %s needs %d bytes, more than the whole budget" % (s.name, nbytes))
        while self.resident_bytes() + nbytes > self.budget:
            idle = [x for x in self.sessions.values() if x.resident and not x.busy() and x is not s]
            if not idle:
                tree.close()
                return False
            victim = min(idle, key=lambda x: x.last_used)
            self._evict(victim)
        tree.bind()
        s.tree, s.nbytes = tree, nbytes
        s.slot_req = [None] * self.slots
        s.active = np.zeros(self.slots, dtype=np.int32)
        s.stream = self.new_stream() if self.new_stream else None
        s.loads += 1
        s.last_used = self._now()
        if self.on_load:
            self.on_load(s)
        self.peak_bytes = max(self.peak_bytes, self.resident_bytes())
        self.log.append(("load", s.name, self._now()))
        return True

    def _evict(self, s: Session):
        s.tree.close()
        s.tree, s.nbytes, s.stream, s.ctx = None, 0, None, {}
        self.log.append(("evict", s.name, self._now()))

    # -- loop ----------------------------------------------------------------
    def _now(self):
        return self.clock() - self.t0 if self.t0 is not None else 0.0

    def submit(self, req: Request):
        if req.session not in self.sessions:
            raise KeyError(req.session)
        self.pending.append(req)

    def _arrivals(self, now):
        while self.pending and self.pending[0].arrival <= now:
            r = self.pending.popleft()
            self.sessions[r.session].queue.append(r)

    def _finish(self, s: Session, slot: int, rel: float):
        req = s.slot_req[slot]
        req.rel_l2 = rel
        if self.keep_results:
            req.result = (self.result_to(s, slot) if self.result_to
                          else s.tree.solution_slots(slot, 1, stream=s.stream)[0].copy())
        req.done = self._now()
        s.slot_req[slot] = None
        s.active[slot] = 0
        s.last_used = req.done
        self.completed.append(req)

    def tick(self):
        self.ticks += 1
        now = self._now()
        self._arrivals(now)
        # residency for sessions with queued work, oldest request first
        waiting = sorted((s for s in self.sessions.values() if s.queue and not s.resident),
                         key=lambda s: s.queue[0].arrival)
        for s in waiting:
            self._load(s)
        # new requests into free slots, first residual of each
        fresh = []
        for s in self.sessions.values():
            if not s.resident or not s.queue:
                continue
            new = np.zeros(self.slots, dtype=np.int32)
            for slot in range(self.slots):
                if s.slot_req[slot] is None and s.queue:
                    req = s.queue.popleft()
                    if callable(req.rhs):
                        if self.stream_context:
                            with self.stream_context(s):
                                g = req.rhs(s)
                        else:
                            g = req.rhs(s)
                    else:
                        g = req.rhs
                    s.tree.set_rhs_slots(slot, g, stream=s.stream)
                    req.start = self._now()
                    s.slot_req[slot] = req
                    new[slot] = 1
            if new.any():
                s.tree.iterate_begin(self.precision, new, residual_only=True, stream=s.stream)
                fresh.append((s, new))
        for s, new in fresh:
            rel, _ = s.tree.iterate_end()
            for slot in np.nonzero(new)[0]:
                if rel[slot] <= self.tol:
                    self._finish(s, int(slot), float(rel[slot]))
                else:
                    s.active[slot] = 1
        # one step on every session with occupied slots, all enqueued first
        stepping = []
        for s in self.sessions.values():
            if s.resident and s.active.any():
                s.tree.iterate_begin(self.precision, s.active, stream=s.stream)
                stepping.append(s)
        for s in stepping:
            rel, _ = s.tree.iterate_end()
            s.last_used = self._now()
            for slot in np.nonzero(s.active)[0]:
                req = s.slot_req[slot]
                req.cycles += 1
                if rel[slot] <= self.tol:
                    self._finish(s, int(slot), float(rel[slot]))
                elif req.cycles >= self.max_cycles or not np.isfinite(rel[slot]):
                    raise RuntimeError("request %d did not converge (rel %.3e after %d cycles)"
                                       % (req.id, rel[slot], req.cycles))
        return bool(stepping or fresh)

    def run(self, requests, idle_sleep=0.0):
        """Serve the requests (arrival times relative to the start); returns
        them completed, in completion order."""
        self.completed = []
        for i, r in enumerate(sorted(requests, key=lambda r: r.arrival)):
            if r.id < 0:
                r.id = i
            self.submit(r)
        self.t0 = self.clock()
        n = len(self.pending)
        while len(self.completed) < n:
            worked = self.tick()
            if not worked and self.pending:
                # nothing on the device: wait for the next arrival
                wait = self.pending[0].arrival - self._now()
                if wait > 0 and idle_sleep is not None:
                    time.sleep(min(wait, 0.05) if idle_sleep == 0.0 else idle_sleep)
        return list(self.completed)

    def close(self):
        for s in self.sessions.values():
            if s.resident:
                self._evict(s)


def summarize(done):
    lat = np.array([r.latency for r in done]) * 1e3
    span = max(r.done for r in done) - min(r.arrival for r in done)
    return {"requests": len(done), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "solves_per_s": len(done) / span, "span_s": span,
            "cycles_mean": float(np.mean([r.cycles for r in done]))}
