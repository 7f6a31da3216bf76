"""Host-side bookkeeping of the serving loop, with the device replaced by a
stub: admission in arrival order within the slots and the memory budget,
retirement returning memory and slots, rejection, latency summary."""
import collections

import pytest

torch = pytest.importorskip("torch")
from paper_2207_13848_gb300 import serve  # noqa: E402


class _Ev:
    def __init__(self):
        self.fired = False

    def query(self):
        return self.fired


class StubServer(serve.Server):
    """Server without a GPU: launches record an event the test fires by hand.
    `rows` gives each operand's row count (for the small-request test); an
    operand missing from it is never merged."""

    def __init__(self, slots, budget, sizes, rows=None, batch_rows=0, max_batch=64):
        self.streams = [None] * slots
        self.free_slots = collections.deque(range(slots))
        self.budget = budget
        self.batch_rows = batch_rows
        self.max_batch = max_batch
        self.used = 0
        self.wait_small = collections.deque()
        self.wait_large = collections.deque()
        self.inflight = {}
        self.finished = []
        self.failed = []
        self.pool = collections.defaultdict(list)
        self.bpool = collections.defaultdict(list)
        self.staging_pool = collections.defaultdict(list)
        self.stats = serve._Stats()
        self._next_id = 0
        self._next_launch = 0
        self.sizes = sizes
        self.rows = rows or {}
        self.launched = []
        self.fail_next = False

    def request_bytes(self, A, B):
        return self.sizes[A]

    def _small(self, r):
        return self.batch_rows > 0 and not r.solo and self.rows.get(r.A, 1 << 40) <= self.batch_rows

    def _begin(self, ln):
        ln.event = _Ev()
        self.inflight[self._next_launch] = ln
        self._next_launch += 1
        self.used += ln.nbytes
        self.stats.admitted += len(ln.requests)
        self.stats.peak_inflight = max(self.stats.peak_inflight, sum(len(x.requests) for x in self.inflight.values()))
        self.stats.peak_bytes = max(self.stats.peak_bytes, self.used)
        self.launched.append([r.rid for r in ln.requests])

    def _launch_many(self, group, nbytes):
        slot = self.free_slots.popleft()
        if self.fail_next:  # the first request's call is rejected: it fails, the rest wait again
            self.fail_next = False
            for r in reversed(group[1:]):
                self.wait_large.appendleft(r)
            self._fail(serve._Launch(group[:1], slot, group[0].nbytes), None, "rejected by the stub")
            return
        for r in group:
            r.slot = slot
        self._begin(serve._Launch(group, slot, nbytes))

    def _launch_batch(self, group, nbytes):
        slot = self.free_slots.popleft()
        for r in group:
            r.slot, r.batched = slot, True
        self._begin(serve._Launch(group, slot, nbytes, batch=True))

    def _retire(self, ln):
        self.used -= ln.nbytes
        self.free_slots.append(ln.slot)
        self.finished.extend(ln.requests)
        self.stats.finished += len(ln.requests)
        return len(ln.requests)


def fire(srv, *reqs):
    for ln in srv.inflight.values():
        if any(r in ln.requests for r in reqs):
            ln.event.fired = True


def test_admission_follows_arrival_order_slots_and_budget():
    srv = StubServer(slots=2, budget=100, sizes={"a": 60, "b": 30, "c": 50, "huge": 101})
    ra = srv.submit("a", None, None, arrival=0.0)
    rb = srv.submit("b", None, None, arrival=0.1)
    rc = srv.submit("c", None, None, arrival=0.2)
    assert srv.submit("huge", None, None) is None and srv.stats.rejected == 1
    srv.poll()
    # requests that wait together go out in one launch while they fit: 90 bytes <= 100
    assert srv.launched == [[ra.rid, rb.rid]]
    assert srv.used == 90 and list(srv.waiting) == [rc]
    fire(srv, ra)
    srv.poll()                                   # a and b retire: 90 bytes back; c (50) fits
    assert srv.launched == [[ra.rid, rb.rid], [rc.rid]]
    assert srv.used == 50 and srv.stats.peak_bytes <= 100
    fire(srv, rc)
    srv.poll()
    assert srv.used == 0 and not srv.inflight and srv.stats.finished == 3


def test_head_of_line_waits_for_memory():
    srv = StubServer(slots=4, budget=100, sizes={"x": 70, "y": 40, "z": 10})
    rx = srv.submit("x", None, None)
    ry = srv.submit("y", None, None)
    rz = srv.submit("z", None, None)
    srv.poll()
    # y does not fit beside x; admission is in arrival order, so z waits behind y
    assert srv.launched == [[rx.rid]] and list(srv.waiting) == [ry, rz]
    fire(srv, rx)
    srv.poll()
    assert srv.launched == [[rx.rid], [ry.rid, rz.rid]]


def test_small_requests_waiting_together_share_one_launch():
    # continuous batching: small requests at the head of the queue are merged,
    # in arrival order, into one launch on one slot; a large one goes alone
    srv = StubServer(slots=2, budget=1000, sizes={"s": 10, "L": 100}, rows={"s": 64, "L": 10 ** 6},
                     batch_rows=1024)
    rs = [srv.submit(k, None, None) for k in ("s", "s", "s", "L", "s", "s")]
    srv.poll()
    # the small requests are merged whatever large one arrived between them;
    # the large one goes alone on the other slot
    assert srv.launched == [[0, 1, 2, 4, 5], [3]] and not srv.waiting
    assert all(r.batched for r in rs if r.A == "s") and not rs[3].batched
    fire(srv, rs[0])
    srv.poll()
    assert srv.stats.finished == 5 and srv.used == 100
    rl = srv.submit("L", None, None)
    rsm = srv.submit("s", None, None)
    srv.poll()                                   # the freed slot takes the earlier arrival: the large one
    assert srv.launched[-1] == [rl.rid] and srv.waiting == [rsm]
    fire(srv, *rs, rl)
    srv.poll()
    assert srv.launched[-1] == [rsm.rid]
    fire(srv, rsm)
    srv.poll()
    assert srv.stats.finished == 8 and srv.used == 0


def test_batches_respect_max_batch_and_the_budget():
    srv = StubServer(slots=3, budget=35, sizes={"s": 10}, rows={"s": 1}, batch_rows=8, max_batch=2)
    rs = [srv.submit("s", None, None) for _ in range(5)]
    srv.poll()
    # at most two per launch, and 35 bytes hold three requests at once
    assert srv.launched == [[0, 1], [2]] and srv.used == 30
    fire(srv, *rs)
    srv.poll()
    assert srv.launched[2:] == [[3, 4]]


def test_a_rejected_launch_does_not_stop_the_loop():
    srv = StubServer(slots=1, budget=100, sizes={"a": 10, "b": 10})
    srv.fail_next = True
    ra = srv.submit("a", None, None)
    rb = srv.submit("b", None, None)
    srv.poll()
    # a's call was rejected: it is marked failed, its slot and memory are back,
    # and b was admitted again on the same poll
    assert ra.error and srv.failed == [ra] and srv.stats.failed == 1 and srv.stats.rejected == 1
    assert srv.launched == [[rb.rid]] and srv.used == 10
    fire(srv, rb)
    srv.poll()
    assert srv.finished == [rb] and srv.used == 0 and len(srv.free_slots) == 1


def test_latency_summary():
    rs = []
    for i, (a, d) in enumerate([(0.0, 1.0), (0.5, 2.5), (1.0, 1.5), (2.0, 6.0)]):
        r = serve.Request(None, None, None, rid=i, arrival=a)
        r.done = d
        rs.append(r)
    s = serve.latency_summary(rs)
    assert s["n"] == 4 and s["span"] == 6.0
    assert s["p50"] == pytest.approx(1.5) and s["mean"] == pytest.approx((1 + 2 + 0.5 + 4) / 4)


def test_size_classes():
    assert serve._size_class(1) == 1 << 20
    assert serve._size_class((1 << 20) + 1) == 1 << 21
    assert serve._size_class(3 << 20) == 1 << 22


class _AutoServer(StubServer):
    """Every launch completes at the next poll; records whether Python's cyclic
    collector was on while the loop ran, and can raise from a poll."""

    def __init__(self, raise_at=None):
        super().__init__(slots=2, budget=100, sizes={"a": 10, "b": 20})
        self.gc_seen = set()
        self.polls = 0
        self.raise_at = raise_at

    def poll(self):
        import gc
        self.gc_seen.add(gc.isenabled())
        self.polls += 1
        if self.raise_at is not None and self.polls == self.raise_at:
            raise RuntimeError("poll failed")
        for ln in self.inflight.values():
            ln.event.fired = True
        return super().poll()


def test_run_poisson_pauses_the_cyclic_collector_and_restores_it():
    import gc
    assert gc.isenabled()
    srv = _AutoServer()
    done, _ = serve.run_poisson(srv, [("a", "a"), ("b", "b")], rate=0, n_requests=20, seed=3)
    assert len(done) == 20 and [r.index for r in done] == list(range(20))
    assert srv.gc_seen == {False}  # off while serving
    assert gc.isenabled()          # on again afterwards
    srv = _AutoServer()
    serve.run_poisson(srv, [("a", "a")], rate=0, n_requests=5, pause_gc=False)
    assert srv.gc_seen == {True} and gc.isenabled()


def test_run_poisson_restores_the_collector_when_the_loop_raises():
    import gc
    srv = _AutoServer(raise_at=1)
    with pytest.raises(RuntimeError):
        serve.run_poisson(srv, [("a", "a")], rate=0, n_requests=10)
    assert gc.isenabled()
    # a caller that had switched the collector off keeps it off
    gc.disable()
    try:
        serve.run_poisson(_AutoServer(), [("a", "a")], rate=0, n_requests=3)
        assert not gc.isenabled()
    finally:
        gc.enable()
