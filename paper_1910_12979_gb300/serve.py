"""Continuous-batching service for projection solves of different grid sizes.

Requests (a grid size and a problem) arrive over time.  The scheduler admits a
request as soon as a *slot* can take it: a slot is a resident multigrid
hierarchy for one grid size (plus its working buffers and its own CUDA stream).
A request uses an idle slot of its size, or a new slot when the device-memory
budget still has room for one, or -- when the budget is full -- the space of the
least recently used idle slot of another size, which is evicted.  Otherwise it
waits in FIFO order.  Admitted solves run on their slot's stream from a worker
thread (the library call releases the GIL and synchronises only those streams),
so requests arriving while others are on the GPU are admitted as slots and
memory free up, and their kernels overlap on the device.  Requests admitted
together (several were waiting when a slot freed up, or arrived together) are
run as one batch when the backend offers ``run_batch``: on the GPU their
elliptic solves share one graph launch (mg_project_batch).

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
        self.batches = []   # size of every group of requests started together

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

    def _batch_worker(self, started):
        try:
            outs = self.backend.run_batch([slot.state for slot, _ in started], [req for _, req in started])
            for (_, req), (res, st) in zip(started, outs):
                req.result, req.status = res, st
        except Exception as e:  # the batch fails as a whole; the rest of the stream continues
            for _, req in started:
                req.status = e
                self.errors.append((req.rid, repr(e)))
        with self.lock:
            now = self.clock() - self.t0
            for slot, req in started:
                req.finished = now
                slot.busy = False
                slot.last_used = now
                self.inflight -= 1
                self.done.append(req)
            nxt = self._admit()
            self.lock.notify_all()
        self._start(nxt)

    def _start(self, started):
        if not started:
            return
        with self.lock:
            self.batches.append(len(started))
        if len(started) > 1 and getattr(self.backend, "run_batch", None) is not None:
            threading.Thread(target=self._batch_worker, args=(started,), daemon=True).start()
            return
        for slot, req in started:
            threading.Thread(target=self._worker, args=(slot, req), daemon=True).start()

    # -- driving ------------------------------------------------------------------
    def run_stream(self, requests, timeout=600.0):
        """Feed requests at their arrival times; return them when all are done.
        The slots (resident hierarchies) stay from one stream to the next; the
        per-stream counters (done, batches, evictions) start again."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        with self.lock:
            self.done = []
            self.batches = []
            self.evictions = 0
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

    problems: dict n -> list of host-resident problems (pinned tensors, from
    ``host_problem``); a request's payload is (n, index into that list).  Every
    request uploads its problem (sigma, beta0 at cells and faces, S, U) from
    pinned host memory on its slot's stream, rebuilds the hierarchy's
    coefficients from that sigma, projects, and reads the projected velocity
    back into the slot's pinned host buffers, so its latency includes both
    transfers.  ``run_batch`` runs several requests with their solves in one
    graph launch (mg_project_batch).
    """

    def __init__(self, problems, device="cuda:0", tol=1e-10, prec="mixed"):
        import torch

        from . import native as N
        from .solver import ProjectionSolver, project_batch
        self.torch, self.N, self.ProjectionSolver, self.project_batch = torch, N, ProjectionSolver, project_batch
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
            # device inputs (sigma, beta0, S on cells; beta0 and U on faces) and phi
            work = 8 * (6 * (n + 1) * n * n + 4 * n ** 3)
            self._bytes[n] = hier + work
        return self._bytes[n]

    def make_slot(self, n):
        torch = self.torch
        p0 = self.problems[n][0]
        stream = torch.cuda.Stream(device=self.device)
        dev = lambda t: torch.empty(t.shape, dtype=t.dtype, device=self.device)
        with torch.cuda.stream(stream):
            d = {"sigma": dev(p0["sigma"]), "beta0": dev(p0["beta0"]), "S": dev(p0["S"]),
                 "beta0_face": [dev(b) for b in p0["beta0_face"]], "U": [dev(u) for u in p0["U"]]}
            d["sigma"].copy_(p0["sigma"], non_blocking=True)
            solver = self.ProjectionSolver(p0["geom"], d["sigma"], loc="cell", prec=self.prec, stream=stream,
                                           flags=self.N.MG_FLAG_ZERO_GUESS | self.N.MG_FLAG_AUTOTUNE)
            phi = torch.empty_like(d["sigma"])
        host_U = [torch.empty(u.shape, dtype=u.dtype).pin_memory() for u in p0["U"]]
        stream.synchronize()
        return {"solver": solver, "stream": stream, "d": d, "phi": phi, "host_U": host_U}

    def free_slot(self, state):
        state["solver"].close()

    def _stage(self, state, req):
        """Upload the request's problem and rebuild the coefficients (asynchronous)."""
        torch = self.torch
        n, k = req.payload
        p, d = self.problems[n][k], state["d"]
        with torch.cuda.stream(state["stream"]):
            for name in ("sigma", "beta0", "S"):
                d[name].copy_(p[name], non_blocking=True)
            for a, b in zip(d["beta0_face"] + d["U"], p["beta0_face"] + p["U"]):
                a.copy_(b, non_blocking=True)
            state["solver"].update_coeff(d["sigma"])

    def _finish(self, state, req):
        """Read the projected velocity back to the slot's pinned host buffers."""
        torch = self.torch
        with torch.cuda.stream(state["stream"]):
            for h, u in zip(state["host_U"], state["d"]["U"]):
                h.copy_(u, non_blocking=True)
        state["stream"].synchronize()
        return [h.clone() for h in state["host_U"]] if req.keep else None

    def run(self, state, req):
        self._stage(state, req)
        d = state["d"]
        with self.torch.cuda.stream(state["stream"]):
            st = state["solver"].project(d["U"], d["beta0"], d["S"], beta0_face=d["beta0_face"], phi=state["phi"],
                                         tol=self.tol, allow_not_converged=True)
        return self._finish(state, req), st

    def run_batch(self, states, reqs):
        for st_, req in zip(states, reqs):
            self._stage(st_, req)
        ds = [s["d"] for s in states]
        sts = self.project_batch([s["solver"] for s in states], [d["U"] for d in ds], [d["beta0"] for d in ds],
                                 [d["S"] for d in ds], beta0_face=[d["beta0_face"] for d in ds],
                                 phi=[s["phi"] for s in states], tols=[self.tol] * len(states),
                                 allow_not_converged=True)
        return [(self._finish(s, r), st) for s, r, st in zip(states, reqs, sts)]


def host_problem(p):
    """One generated problem (inputs.polytrope_star / stratified) in pinned host memory."""
    import torch
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
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
