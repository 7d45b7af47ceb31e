"""Host-side tests of the continuous-batching scheduler (no GPU): the backend is
a host-only stand-in whose 'solve' sleeps for a time proportional to the grid."""
import os
import threading
import time

import pytest

from paper_1910_12979_gb300.serve import Request, Scheduler, latency_stats, make_requests, shard


class FakeBackend:
    def __init__(self, per_cell_s=2e-8, fail=()):
        self.per_cell_s = per_cell_s
        self.fail = set(fail)
        self.lock = threading.Lock()
        self.live_bytes = 0
        self.max_live = 0
        self.active = 0
        self.max_active = 0
        self.made = []

    def slot_bytes(self, n):
        return n ** 3 * 100

    def make_slot(self, n):
        with self.lock:
            self.live_bytes += self.slot_bytes(n)
            self.max_live = max(self.max_live, self.live_bytes)
            self.made.append(n)
        return {"n": n}

    def free_slot(self, st):
        with self.lock:
            self.live_bytes -= self.slot_bytes(st["n"])

    def run(self, st, req):
        assert st["n"] == req.n
        with self.lock:
            self.active += 1
            self.max_active = max(self.max_active, self.active)
        time.sleep(self.per_cell_s * req.n ** 3)
        with self.lock:
            self.active -= 1
        if req.rid in self.fail:
            raise RuntimeError("poisoned request")
        return req.rid, 0


def stream(count=40, rate=400.0, sizes=(32, 64, 96)):
    import numpy as np
    rng = np.random.default_rng(0)
    t = np.cumsum(rng.exponential(1 / rate, size=count))
    ns = rng.choice(sizes, size=count)
    return make_requests(t - t[0], ns)


def test_all_served_budget_respected_fifo():
    be = FakeBackend()
    budget = 2 * 96 ** 3 * 100 + 64 ** 3 * 100
    sch = Scheduler(be, budget, max_inflight=8)
    reqs = sch.run_stream(stream())
    assert all(r.finished >= r.admitted >= r.arrival - 1e-9 for r in reqs)
    assert be.max_live <= budget
    # FIFO: admission times are non-decreasing in arrival order
    adm = [r.admitted for r in sorted(reqs, key=lambda r: r.arrival)]
    assert all(b >= a - 1e-9 for a, b in zip(adm, adm[1:]))
    st = latency_stats(reqs)
    assert st["count"] == 40 and st["p99_ms"] >= st["p50_ms"] > 0
    sch.close()
    assert be.live_bytes == 0


def test_slots_are_reused_and_evicted():
    be = FakeBackend(per_cell_s=1e-9)
    budget = 96 ** 3 * 100 + 10   # room for a single 96^3 slot (or a few small ones)
    sch = Scheduler(be, budget, max_inflight=4)
    reqs = sch.run_stream(stream(count=30))
    assert len(reqs) == 30 and all(r.status == 0 for r in reqs)
    assert sch.evictions > 0 and be.max_live <= budget
    assert len(be.made) < 30      # slots are reused between requests of the same size
    sch.close()


def test_poisoned_request_fails_alone():
    be = FakeBackend(fail={3, 7})
    sch = Scheduler(be, 10 ** 9, max_inflight=4)
    reqs = sch.run_stream(stream(count=12))
    bad = {r.rid for r in reqs if isinstance(r.status, Exception)}
    assert bad == {3, 7}
    assert all(r.status == 0 for r in reqs if r.rid not in bad)
    sch.close()


def test_overlap_shortens_the_stream():
    """Requests that arrive together run concurrently when slots allow it."""
    reqs1 = [Request(i, 64, 0.0, (64, 0)) for i in range(8)]
    reqs2 = [Request(i, 64, 0.0, (64, 0)) for i in range(8)]
    be1, be2 = FakeBackend(per_cell_s=1e-7), FakeBackend(per_cell_s=1e-7)
    s1 = Scheduler(be1, 10 ** 9, max_inflight=1)
    s8 = Scheduler(be2, 10 ** 9, max_inflight=8)
    t1 = max(r.finished for r in s1.run_stream(reqs1))
    t8 = max(r.finished for r in s8.run_stream(reqs2))
    assert be2.max_active > 1 and t8 < 0.5 * t1


def test_shard_partitions_requests():
    reqs = stream(count=21)
    parts = [shard(reqs, r, 4) for r in range(4)]
    ids = sorted(x.rid for p in parts for x in p)
    assert ids == list(range(21))


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    reqs = shard(stream(count=24), rank, world)
    sch = Scheduler(FakeBackend(per_cell_s=1e-9), 10 ** 9, max_inflight=4)
    done = sch.run_stream(reqs)
    stats = [None] * world
    dist.all_gather_object(stats, {"rank": rank, "ids": [r.rid for r in done]})
    if rank == 0:
        out.put(stats)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_serving_covers_the_stream():
    import multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    stats = q.get(timeout=120)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    ids = sorted(i for s in stats for i in s["ids"])
    assert ids == list(range(24))
