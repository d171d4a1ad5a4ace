"""Host logic of the serving loop on the CPU: the arena allocator and the
scheduler (admission under an HBM budget, FIFO order, slots, rejection,
cancellation, round-robin iteration issue) driven by a fake executor."""
import itertools
import random

import pytest

from paper_1803_10045_b300.serving import ALIGN, Arena, Server, summarize


def test_arena_first_fit_and_coalescing():
    a = Arena(10 * ALIGN)
    x = a.alloc(3 * ALIGN)
    y = a.alloc(1)                      # rounded up to ALIGN
    z = a.alloc(4 * ALIGN)
    assert (x, y, z) == (0, 3 * ALIGN, 4 * ALIGN)
    assert a.alloc(3 * ALIGN) is None   # 2 blocks left
    a.free(y)
    assert a.alloc(2 * ALIGN) == 8 * ALIGN
    a.free(x)
    a.free(z)                           # x, y, z ranges merge into one
    assert a.free_list == [(0, 8 * ALIGN)]
    assert a.alloc(8 * ALIGN) == 0 and a.used == 10 * ALIGN


def test_arena_random_never_overlaps():
    rng = random.Random(0)
    a = Arena(1 << 20)
    live = {}
    for _ in range(3000):
        if live and rng.random() < 0.45:
            off = rng.choice(list(live))
            a.free(off)
            del live[off]
        else:
            n = rng.randrange(1, 40000)
            off = a.alloc(n)
            if off is not None:
                live[off] = -(-n // ALIGN) * ALIGN
        spans = sorted(live.items())
        for (o1, n1), (o2, _) in zip(spans, spans[1:]):
            assert o1 + n1 <= o2
        assert sum(live.values()) == a.used <= a.size
    for off in list(live):
        a.free(off)
    assert a.free_list == [(0, a.size)]


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 0.001
        return self.t


class FakeReq:
    def __init__(self, rid, arrival, size, n_iter):
        self.rid, self.arrival, self.size, self.n_iter = rid, arrival, size, n_iter


class FakeExecutor:
    """Each issued iteration takes `lag` polls to finish; logs the issue order."""

    def __init__(self, lag=2):
        self.lag = lag
        self.log = []
        self.concurrent = 0
        self.max_concurrent = 0

    def footprint(self, r):
        return r.size

    def admit(self, r, off, slot):
        self.concurrent += 1
        self.max_concurrent = max(self.max_concurrent, self.concurrent)
        return {"r": r, "left": self.lag, "slot": slot, "off": off}

    def issue(self, job):
        self.log.append(job["r"].rid)
        job["left"] = self.lag

    def ready(self, job):
        job["left"] -= 1
        return job["left"] < 0

    def finish(self, job):
        job["left"] = self.lag

    def result(self, job):
        return ("maps", job["r"].rid)

    def release(self, job):
        self.concurrent -= 1


def test_all_finish_within_budget_and_slots():
    ex = FakeExecutor()
    reqs = [FakeReq(i, 0.002 * i, (1 + i % 3) * 1000 * ALIGN, 3 + i % 4) for i in range(30)]
    srv = Server(ex, budget_bytes=4000 * ALIGN, max_active=3, clock=FakeClock(), idle_sleep=0)
    recs = srv.run(reqs)
    assert all(r.status == "done" and r.iterations == q.n_iter for r, q in zip(recs, reqs))
    assert all(r.result == ("maps", r.rid) for r in recs)
    assert srv.arena.peak <= 4000 * ALIGN and srv.arena.used == 0
    assert ex.max_concurrent <= 3
    # FIFO admission: admission times are non-decreasing in arrival order
    adm = [r.admitted for r in recs]
    assert adm == sorted(adm)
    s = summarize(recs)
    assert s["completed"] == 30 and s["p99_s"] >= s["p50_s"] > 0


def test_budget_binds_and_round_robin_interleaves():
    ex = FakeExecutor(lag=1)
    reqs = [FakeReq(i, 0.0, 1000 * ALIGN, 4) for i in range(6)]
    srv = Server(ex, budget_bytes=2000 * ALIGN, max_active=8, clock=FakeClock(), idle_sleep=0)
    srv.run(reqs)
    assert ex.max_concurrent == 2       # the budget, not the slots, limits concurrency
    # the first two studies alternate iteration by iteration
    first = [rid for rid in ex.log if rid in (0, 1)]
    assert first[:4] in ([0, 1, 0, 1], [1, 0, 1, 0])


def test_oversized_request_is_rejected_others_served():
    ex = FakeExecutor()
    reqs = [FakeReq(0, 0.0, 500 * ALIGN, 2), FakeReq(1, 0.0, 5000 * ALIGN, 2),
            FakeReq(2, 0.0, 500 * ALIGN, 2)]
    recs = Server(ex, 1000 * ALIGN, clock=FakeClock(), idle_sleep=0).run(reqs)
    assert [r.status for r in recs] == ["done", "rejected", "done"]


def test_cancel_queued_and_active():
    ex = FakeExecutor(lag=3)
    reqs = [FakeReq(i, 0.0, 1000 * ALIGN, 50) for i in range(3)]
    srv = Server(ex, 1000 * ALIGN, clock=FakeClock(), idle_sleep=0)   # one at a time
    ticks = itertools.count()

    def on_tick(server, now):
        k = next(ticks)
        if k == 5:
            server.cancel(2)            # still queued
        if k == 40:
            server.cancel(0)            # active, mid-run
    recs = srv.run(reqs, on_tick=on_tick)
    assert [r.status for r in recs] == ["cancelled", "done", "cancelled"]
    assert 0 < recs[0].iterations < 50 and recs[2].iterations == 0
    assert srv.arena.used == 0 and ex.concurrent == 0


def test_backfill_admits_small_behind_a_blocked_large_one():
    ex = FakeExecutor(lag=2)
    # a resident large study, then a large one that must wait, then small ones
    reqs = [FakeReq(0, 0.0, 700 * ALIGN, 40), FakeReq(1, 0.0005, 700 * ALIGN, 5)] + \
        [FakeReq(2 + i, 0.0006, 100 * ALIGN, 3) for i in range(4)]
    fifo = Server(FakeExecutor(lag=2), 1000 * ALIGN, clock=FakeClock(), idle_sleep=0).run(reqs)
    back = Server(ex, 1000 * ALIGN, clock=FakeClock(), idle_sleep=0, policy="backfill").run(reqs)
    assert all(r.status == "done" for r in fifo + back)
    # FIFO: the small studies wait for the blocked large one; backfill: they run
    # beside the first large study and finish before the second is admitted
    assert all(f.done > fifo[1].admitted for f in fifo[2:])
    assert all(b.done < back[1].admitted for b in back[2:])


def test_backfill_does_not_starve_the_oldest():
    reqs = [FakeReq(0, 0.0, 600 * ALIGN, 30), FakeReq(1, 0.0005, 600 * ALIGN, 2)] + \
        [FakeReq(2 + i, 0.0006 + 0.0001 * i, 300 * ALIGN, 2) for i in range(60)]
    srv = Server(FakeExecutor(lag=1), 1000 * ALIGN, clock=FakeClock(), idle_sleep=0,
                 policy="backfill", max_bypass=5)
    recs = srv.run(reqs)
    assert all(r.status == "done" for r in recs)
    bypassers = [r for r in recs[2:] if r.admitted < recs[1].admitted]
    assert len(bypassers) <= 5
