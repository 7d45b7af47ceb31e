"""Continuous-batching service for projection solves of different grid sizes.

Requests (a grid size and a problem) arrive over time.  The scheduler admits a
request as soon as a *slot* can take it: a slot is a resident multigrid
hierarchy for one grid size (plus its working buffers and its own CUDA stream).
A request uses an idle slot of its size, or a new slot when the device-memory
budget still has room for one, or -- when the budget is full -- the space of the
least recently used idle slot of another size, which is evicted.  Otherwise it
waits in FIFO order.  Admitted solves run on their slot's stream from a worker
thread (the library call releases the GIL and synchronises only that stream),
so requests arriving while others are on the GPU are admitted as slots and
memory free up, and their kernels overlap on the device.

The scheduling core (``Scheduler``) holds no CUDA state: it is driven by a
``backend`` object that creates slots, reports their size in bytes and runs a
request on a slot.  ``GpuBackend`` is the real one (library handles on CUDA
streams); the tests also drive the scheduler with a host-only backend.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    n: int
    arrival: float                     # seconds, relative to the stream start
    payload: object = None             # backend-specific problem description
    admitted: float = float("nan")
    finished: float = float("nan")
    result: object = None
    status: object = None
    keep: bool = False                 # keep the projected velocity in ``result``

    @property
    def latency(self):
        return self.finished - self.arrival


class Slot:
    def __init__(self, n, nbytes, state):
        self.n = n
        self.nbytes = nbytes
        self.state = state
        self.busy = False
        self.last_used = 0.0


class Scheduler:
    """Admission by device-memory budget, FIFO queue, slot reuse and LRU eviction.

    backend must provide: ``slot_bytes(n)``, ``make_slot(n) -> state``,
    ``free_slot(state)`` and ``run(state, request) -> (result, status)``.
    ``run`` is called from a worker thread.
    """

    def __init__(self, backend, budget_bytes, max_inflight=16, clock=time.perf_counter):
        self.backend = backend
        self.budget = int(budget_bytes)
        self.max_inflight = int(max_inflight)
        self.clock = clock
        self.slots = []
        self.queue = collections.deque()
        self.done = []
        self.inflight = 0
        self.lock = threading.Condition()
        self.t0 = None
        self.evictions = 0
        self.created = 0
        self.errors = []

    # -- bookkeeping (called with the lock held) --------------------------------
    def used_bytes(self):
        return sum(s.nbytes for s in self.slots)

    def _pick_slot(self, n):
        for s in self.slots:
            if s.n == n and not s.busy:
                return s
        need = self.backend.slot_bytes(n)
        if need > self.budget:
            raise ValueError(f"a {n}^3 slot needs {need} bytes, more than the whole budget {self.budget}")
        if self.used_bytes() + need <= self.budget:
            s = Slot(n, need, self.backend.make_slot(n))
            self.slots.append(s)
            self.created += 1
            return s
        # evict least recently used idle slots of other sizes until the new one fits
        idle = sorted((s for s in self.slots if not s.busy and s.n != n), key=lambda s: s.last_used)
        freed, victims = 0, []
        for s in idle:
            victims.append(s)
            freed += s.nbytes
            if self.used_bytes() - freed + need <= self.budget:
                for v in victims:
                    self.slots.remove(v)
                    self.backend.free_slot(v.state)
                    self.evictions += 1
                s2 = Slot(n, need, self.backend.make_slot(n))
                self.slots.append(s2)
                self.created += 1
                return s2
        return None

    def _admit(self):
        """Admit queued requests in FIFO order while slots can be had."""
        started = []
        while self.queue and self.inflight < self.max_inflight:
            req = self.queue[0]
            slot = self._pick_slot(req.n)
            if slot is None:
                break  # FIFO: the head waits for memory or a slot; nothing overtakes it
            self.queue.popleft()
            slot.busy = True
            self.inflight += 1
            req.admitted = self.clock() - self.t0
            started.append((slot, req))
        return started

    def _worker(self, slot, req):
        try:
            res, st = self.backend.run(slot.state, req)
            req.result, req.status = res, st
        except Exception as e:  # a failing request fails alone; the rest of the mix continues
            req.status = e
            self.errors.append((req.rid, repr(e)))
        with self.lock:
            req.finished = self.clock() - self.t0
            slot.busy = False
            slot.last_used = req.finished
            self.inflight -= 1
            self.done.append(req)
            started = self._admit()
            self.lock.notify_all()
        self._start(started)

    def _start(self, started):
        for slot, req in started:
            threading.Thread(target=self._worker, args=(slot, req), daemon=True).start()

    # -- driving ------------------------------------------------------------------
    def run_stream(self, requests, timeout=600.0):
        """Feed requests at their arrival times; return them when all are done."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        self.t0 = self.clock()
        i = 0
        deadline = self.t0 + timeout
        while True:
            now = self.clock() - self.t0
            arrived = []
            while i < len(reqs) and reqs[i].arrival <= now:
                arrived.append(reqs[i])
                i += 1
            with self.lock:
                self.queue.extend(arrived)
                started = self._admit()
                finished = len(self.done) == len(reqs)
            self._start(started)
            if finished:
                break
            if self.clock() > deadline:
                raise TimeoutError(f"serving stream did not finish within {timeout} s")
            wait = (reqs[i].arrival - now) if i < len(reqs) else 0.05
            with self.lock:
                if len(self.done) < len(reqs):
                    self.lock.wait(timeout=max(min(wait, 0.05), 0.0005))
        return reqs

    def close(self):
        for s in self.slots:
            self.backend.free_slot(s.state)
        self.slots = []


def latency_stats(reqs):
    lat = np.array([r.latency for r in reqs]) * 1e3
    span = max(r.finished for r in reqs) - min(r.arrival for r in reqs)
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "solves_per_s": len(reqs) / span, "count": len(reqs)}


class GpuBackend:
    """Slots are mixed-precision MAC projection hierarchies on their own streams.

    problems: dict n -> list of device-resident problems (dicts of tensors from
    ``device_problem``); a request's payload is (n, index into that list).
    """

    def __init__(self, problems, device="cuda:0", tol=1e-10, prec="mixed"):
        import torch

        from . import native as N
        from .solver import ProjectionSolver
        self.torch, self.N, self.ProjectionSolver = torch, N, ProjectionSolver
        self.problems = problems
        self.device = torch.device(device)
        self.tol = tol
        self.prec = prec
        self._bytes = {}

    def slot_bytes(self, n):
        if n not in self._bytes:
            N = self.N
            geom = self.problems[n][0]["geom"]
            g = N.mg_geometry(3, (n, n, n), tuple(geom["h"]), N.MG_LOC_CELL)
            bc = N.mg_bc(tuple(N.BC[b] for b in geom["bclo"]), tuple(N.BC[b] for b in geom["bchi"]))
            opt = N.mg_default_options()
            opt.prec = N.MG_PREC_MIXED if self.prec == "mixed" else N.MG_PREC_FP64
            hier = N.mg_hierarchy_bytes(g, bc, opt)
            work = 8 * (3 * (n + 1) * n * n + n ** 3)   # U faces and phi of the slot
            self._bytes[n] = hier + work
        return self._bytes[n]

    def make_slot(self, n):
        torch = self.torch
        p0 = self.problems[n][0]
        stream = torch.cuda.Stream(device=self.device)
        with torch.cuda.stream(stream):
            solver = self.ProjectionSolver(p0["geom"], p0["sigma"], loc="cell", prec=self.prec, stream=stream,
                                           flags=self.N.MG_FLAG_ZERO_GUESS | self.N.MG_FLAG_AUTOTUNE)
            U = [torch.empty_like(u) for u in p0["U"]]
            phi = torch.empty_like(p0["sigma"])
        stream.synchronize()
        return {"solver": solver, "stream": stream, "U": U, "phi": phi}

    def free_slot(self, state):
        state["solver"].close()

    def run(self, state, req):
        torch = self.torch
        n, k = req.payload
        p = self.problems[n][k]
        s = state["solver"]
        with torch.cuda.stream(state["stream"]):
            s.update_coeff(p["sigma"])
            for a, b in zip(state["U"], p["U"]):
                a.copy_(b)
            st = s.project(state["U"], p["beta0"], p["S"], beta0_face=p["beta0_face"], phi=state["phi"],
                           tol=self.tol, allow_not_converged=True)
            out = [u.clone() for u in state["U"]] if req.keep else None
        state["stream"].synchronize()
        return out, st


def device_problem(p, device):
    """Move one generated problem (inputs.polytrope_star / stratified) to the device."""
    import torch
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
    return {"geom": p["geom"], "sigma": T(p["sigma"]), "beta0": T(p["beta0"]), "S": T(p["S"]),
            "beta0_face": [T(b) for b in p["beta0_face"]], "U": [T(u) for u in p["U_mac"]]}


def shard(requests, rank, world):
    """Requests of one rank when independent solves are spread over ranks (one GPU each)."""
    return [r for r in requests if r.rid % world == rank]


def make_requests(arrivals, sizes, problems_per_size=1, seed=5):
    """Requests from arrival times and sizes; problem index drawn from a seeded stream."""
    rng = np.random.default_rng(seed)
    return [Request(i, int(n), float(t), (int(n), int(rng.integers(problems_per_size))))
            for i, (t, n) in enumerate(zip(arrivals, sizes))]
