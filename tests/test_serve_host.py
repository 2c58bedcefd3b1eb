"""Scheduler logic of the serving loop, with a fake executor (no GPU):
budget accounting, arrival-order admission, no drops, batching limits."""
import threading
import time

import numpy as np
import pytest

from paper_1210_3165_gb300.serve import Rejected, Request, Server, request_bytes


class Ev:
    """Completes once the executor's clock (one tick per query) reaches `due`."""

    def __init__(self, ex, polls):
        self.ex, self.due = ex, ex.now + polls

    def query(self):
        self.ex.now += 1
        return self.ex.now > self.due


class FakeExecutor:
    def __init__(self, h2d_polls=1, run_polls=2, d2h_polls=1, streams=2):
        self.polls = (h2d_polls, run_polls, d2h_polls)
        self.live = {}
        self.order = []            # admission order (request ids)
        self.launches = []         # list of request-id lists
        self.inflight = [None] * streams
        self.rr = 0
        self.peak_live = 0
        self.now = 0

    def alloc(self, req):
        slot = dict(req=req)
        self.live[id(slot)] = req.nbytes
        self.peak_live = max(self.peak_live, sum(self.live.values()))
        self.order.append(req.rid)
        return slot

    def h2d(self, slot, req):
        return Ev(self, self.polls[0])

    def done(self, ev):
        return ev.query()

    def can_launch(self):
        e = self.inflight[self.rr]
        return e is None or self.now > e.due

    def launch(self, slots):
        ev = Ev(self, self.polls[1])
        self.inflight[self.rr] = ev
        self.rr = (self.rr + 1) % len(self.inflight)
        self.launches.append([s["req"].rid for s in slots])
        for s in slots:
            s["out"] = (s["req"].image > 127).astype(np.uint8)
        return ev, None

    def d2h(self, slot):
        return Ev(self, self.polls[2]), slot["out"]

    def release(self, slot):
        del self.live[id(slot)]


def req(rid, h, w, ch=1, W=15, packed=False):
    rng = np.random.default_rng(rid)
    img = rng.integers(0, 256, (h, w) if ch == 1 else (h, w, 3), dtype=np.uint8)
    r = Request(image=img, W=W, packed=packed)
    r.rid = rid
    return r


def drive(server, limit=100000):
    n = 0
    while server.pending():
        server.step()
        n += 1
        assert n < limit, "scheduler made no progress"
    return n


def test_request_bytes():
    assert request_bytes(10, 100, 1) == 10 * (112 + 112)
    assert request_bytes(10, 100, 3) == 10 * (304 + 112)
    assert request_bytes(3, 100, 1, packed=True) == 3 * (112 + 16)


def test_all_complete_in_budget_and_in_arrival_order():
    ex = FakeExecutor()
    reqs = [req(i, 20 + 7 * (i % 5), 30 + 11 * (i % 3), ch=1 + 2 * (i % 2)) for i in range(40)]
    budget = 3 * max(request_bytes(*r.shape[:2], 1 if r.image.ndim == 2 else 3) for r in reqs)
    srv = Server(ex, budget_bytes=budget, max_batch=4)
    futs = [srv.submit(r) for r in reqs]
    drive(srv)
    assert [f.done() for f in futs] == [True] * 40
    for r, f in zip(reqs, futs):
        np.testing.assert_array_equal(f.result(), (r.image > 127).astype(np.uint8))
    assert ex.order == list(range(40))            # FIFO admission, none skipped ahead
    assert srv.high_water <= budget and ex.peak_live <= budget
    assert srv.reserved == 0 and not ex.live      # everything released
    assert all(len(b) <= 4 for b in ex.launches)
    assert sorted(sum(ex.launches, [])) == list(range(40))  # each page launched exactly once
    st = srv.stats()
    assert st["completed"] == 40 and st["p99_ms"] >= st["p50_ms"] >= 0


def test_large_request_waits_for_memory_and_blocks_later_ones():
    ex = FakeExecutor(run_polls=5)
    small = request_bytes(16, 16, 1)
    srv = Server(ex, budget_bytes=small * 4)
    a = [req(i, 16, 16) for i in range(3)]
    big = req(10, 16, 16 * 3)        # needs more than what three small pages leave free
    b = req(11, 16, 16)
    for r in a + [big, b]:
        srv.submit(r)
    srv.step()
    assert ex.order == [0, 1, 2]     # big does not fit yet; b must not overtake it
    drive(srv)
    assert ex.order == [0, 1, 2, 10, 11]


def test_oversized_request_is_rejected_not_queued():
    srv = Server(FakeExecutor(), budget_bytes=1000)
    f = srv.submit(req(0, 100, 100))
    with pytest.raises(Rejected):
        f.result(timeout=0)
    assert srv.pending() == 0


def test_continuous_batching_uses_pages_that_arrive_while_others_run():
    ex = FakeExecutor(run_polls=3, streams=1)
    srv = Server(ex, budget_bytes=1 << 30, max_batch=64)
    for i in range(4):
        srv.submit(req(i, 8, 8))
    srv.step(); srv.step()            # first step launched over the first pages
    for i in range(4, 8):
        srv.submit(req(i, 8, 8))
    drive(srv)
    assert len(ex.launches) >= 2
    assert ex.launches[0] == [0, 1, 2, 3]
    assert sorted(sum(ex.launches, [])) == list(range(8))


def test_threaded_server_drains_concurrent_submitters():
    ex = FakeExecutor()
    lock = threading.Lock()

    srv = Server(ex, budget_bytes=request_bytes(32, 32, 3) * 5, poll_s=1e-5).start()
    futs = []

    def client(base):
        for i in range(25):
            f = srv.submit(req(base + i, 32, 32, ch=3 if i % 2 else 1))
            with lock:
                futs.append(f)
            time.sleep(1e-4)

    ts = [threading.Thread(target=client, args=(100 * t,)) for t in range(3)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    srv.stop(drain=True, timeout=30)
    assert len(futs) == 75 and all(f.done() and f.exception() is None for f in futs)
    assert srv.completed == 75 and srv.reserved == 0


class PoolExecutor(FakeExecutor):
    """Fake GPU side whose buffers come from the native pool over a fake range."""

    def __init__(self, budget, **kw):
        import paper_1210_3165_gb300 as bnz
        super().__init__(**kw)
        self.pool = bnz.Pool(1 << 40, budget)
        self.budget_bytes = budget

    def alloc(self, req):
        ptr = self.pool.alloc(req.nbytes)
        if ptr is None:
            return None
        slot = super().alloc(req)
        slot["ptr"] = ptr
        return slot

    def release(self, slot):
        self.pool.free(slot["ptr"])
        super().release(slot)


def test_pool_backed_admission_waits_on_fragmentation_and_injected_failures():
    unit = request_bytes(16, 16, 1)          # 512 bytes: two 256-byte pool units
    ex = PoolExecutor(budget=unit * 6, run_polls=4)
    srv = Server(ex, max_batch=2)            # budget taken from the executor
    assert srv.budget == unit * 6
    ex.pool.fail_next(3)
    reqs = [req(i, 16, 16 * (1 + i % 3)) for i in range(30)]
    futs = [srv.submit(r) for r in reqs]
    drive(srv)
    assert all(f.result() is not None for f in futs)
    assert ex.order == list(range(30))
    assert srv.alloc_waits >= 3              # the injected failures deferred admission, dropped nothing
    st = ex.pool.stats()
    assert st["used"] == 0 and st["largest_free"] == unit * 6 and st["high_water"] <= unit * 6


def test_cancelled_and_timed_out_requests_do_not_run():
    ex = FakeExecutor(run_polls=50)
    unit = request_bytes(8, 8, 1)
    srv = Server(ex, budget_bytes=unit)      # one request at a time
    a, b, c = req(0, 8, 8), req(1, 8, 8), req(2, 8, 8)
    c.timeout_s = 0.0
    fa, fb, fc = srv.submit(a), srv.submit(b), srv.submit(c)
    srv.step()                               # a admitted; b and c wait
    assert fb.cancel()
    assert not fa.cancel()                   # running: too late to cancel
    time.sleep(0.01)
    drive(srv)
    assert fa.result() is not None and fb.cancelled()
    with pytest.raises(TimeoutError):
        fc.result(timeout=0)
    assert ex.order == [0] and srv.cancelled == 1 and srv.timed_out == 1 and srv.pending() == 0


@pytest.mark.parametrize("bad", [
    dict(image=np.zeros((0, 5), np.uint8)), dict(image=np.zeros((4, 0, 3), np.uint8)),
    dict(image=np.zeros((4, 5, 2), np.uint8)), dict(image=np.zeros((4, 5), np.float32)),
    dict(W=0), dict(W=256), dict(W=15.0), dict(rule="otsu"), dict(R=0.0)])
def test_malformed_requests_fail_their_future_not_the_loop(bad):
    ex = FakeExecutor()
    srv = Server(ex, budget_bytes=1 << 20)
    kw = dict(image=np.zeros((4, 5), np.uint8), W=3)
    kw.update(bad)
    f = srv.submit(Request(**kw))
    with pytest.raises(ValueError):
        f.result(timeout=0)
    good = req(1, 4, 5)
    g = srv.submit(good)
    drive(srv)
    assert g.result() is not None and ex.order == [1]


def test_each_step_runs_one_kernel_instance_oldest_first():
    """Launches never mix kernel instances (channels, rule, W mod 8); the oldest ready page picks the next one."""
    from paper_1210_3165_gb300.serve import instance_key
    ex = FakeExecutor(run_polls=1, streams=1)
    srv = Server(ex, budget_bytes=1 << 30, max_batch=64)
    specs = [(15, "sauvola", 1), (23, "sauvola", 1), (17, "sauvola", 1), (15, "niblack", 1), (31, "sauvola", 3),
             (7, "sauvola", 1), (15, "sauvola", 1)]
    reqs = []
    for i, (W, rule, ch) in enumerate(specs):
        r = req(i, 8, 8, ch=ch, W=W)
        r.rule = rule
        reqs.append(r)
        srv.submit(r)
    drive(srv)
    by_id = {r.rid: r for r in reqs}
    for launch in ex.launches:
        assert len({instance_key(by_id[i]) for i in launch}) == 1
    assert ex.launches[0] == [0, 1, 5, 6]      # W 15, 23, 7, 15: gray Sauvola, W mod 8 = 7
    assert sorted(sum(ex.launches, [])) == list(range(len(specs)))


def test_host_arena_blocks_live_as_long_as_any_view():
    """Result arrays are views of one pinned arena; a block returns to the pool only when the last array
    viewing it is gone (here over plain memory: the bookkeeping never touches the bytes)."""
    import gc
    import paper_1210_3165_gb300 as bnz
    from paper_1210_3165_gb300.serve import _Block
    buf = np.zeros(1 << 16, np.uint8)
    base = buf.ctypes.data + ((-buf.ctypes.data) % 256)
    pool = bnz.Pool(base, (1 << 16) - 512)
    a = np.asarray(_Block(pool, pool.alloc(100 * 50), 100, 50))
    a[:] = 7
    part = a[10:20]
    del a
    gc.collect()
    assert pool.stats()["live"] == 1 and int(part.sum()) == 7 * 10 * 50
    del part
    gc.collect()
    assert pool.stats()["live"] == 0


def test_mask_copies_wait_for_host_memory_without_stalling_the_loop():
    """When the host arena has no room for a mask, the request keeps its place and is retried; the loop
    goes on delivering (which frees host memory) instead of blocking."""
    class TightHost(FakeExecutor):
        def __init__(self):
            super().__init__()
            self.refusals = 0

        def d2h(self, slot):
            if self.refusals < 5:   # the first attempts find the host arena full
                self.refusals += 1
                return None
            return super().d2h(slot)

    ex = TightHost()
    srv = Server(ex, budget_bytes=1 << 30, max_batch=4)
    futs = [srv.submit(req(i, 8, 8)) for i in range(12)]
    drive(srv)
    assert all(f.result() is not None for f in futs) and ex.refusals == 5
