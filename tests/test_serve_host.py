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
    """Server without a GPU: launches record an event the test fires by hand."""

    def __init__(self, slots, budget, sizes):
        self.streams = [None] * slots
        self.free_slots = collections.deque(range(slots))
        self.budget = budget
        self.used = 0
        self.waiting = collections.deque()
        self.inflight = {}
        self.finished = []
        self.pool = collections.defaultdict(list)
        self.stats = serve._Stats()
        self._next_id = 0
        self.sizes = sizes
        self.launched = []

    def request_bytes(self, A, B):
        return self.sizes[A]

    def _launch(self, r):
        r.slot = self.free_slots.popleft()
        self.used += r.nbytes
        r._event = _Ev()
        self.inflight[r.rid] = r
        self.launched.append(r.rid)
        self.stats.admitted += 1
        self.stats.peak_inflight = max(self.stats.peak_inflight, len(self.inflight))
        self.stats.peak_bytes = max(self.stats.peak_bytes, self.used)

    def _retire(self, r):
        self.used -= r.nbytes
        self.free_slots.append(r.slot)
        self.finished.append(r)
        self.stats.finished += 1


def test_admission_follows_arrival_order_slots_and_budget():
    srv = StubServer(slots=2, budget=100, sizes={"a": 60, "b": 30, "c": 50, "huge": 101})
    ra = srv.submit("a", None, None, arrival=0.0)
    rb = srv.submit("b", None, None, arrival=0.1)
    rc = srv.submit("c", None, None, arrival=0.2)
    assert srv.submit("huge", None, None) is None and srv.stats.rejected == 1
    srv.poll()
    assert srv.launched == [ra.rid, rb.rid]      # two slots, 90 bytes <= 100
    assert srv.used == 90 and list(srv.waiting) == [rc]
    ra._event.fired = True
    srv.poll()                                   # a retires: slot and 60 bytes back; c (50) fits
    assert srv.launched == [ra.rid, rb.rid, rc.rid]
    assert srv.used == 80 and srv.stats.peak_bytes <= 100
    rb._event.fired = rc._event.fired = True
    srv.poll()
    assert srv.used == 0 and not srv.inflight and srv.stats.finished == 3


def test_head_of_line_waits_for_memory():
    srv = StubServer(slots=4, budget=100, sizes={"x": 70, "y": 40, "z": 10})
    rx = srv.submit("x", None, None)
    ry = srv.submit("y", None, None)
    rz = srv.submit("z", None, None)
    srv.poll()
    # y does not fit beside x; admission is in arrival order, so z waits behind y
    assert srv.launched == [rx.rid] and list(srv.waiting) == [ry, rz]
    rx._event.fired = True
    srv.poll()
    assert srv.launched == [rx.rid, ry.rid, rz.rid]


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
