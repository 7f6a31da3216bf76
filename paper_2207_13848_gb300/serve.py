"""Serving loop for structure predictions: requests are admitted continuously
into device slots, by free slots and by device memory, and run concurrently.

A request is one prediction (Eq. 4 of the paper, the spgemm_predict_structure
call) on operands that are already resident on the device.  The server owns
`slots` CUDA streams and a device-memory budget.  Every `poll()`:

  1. retires the requests whose completion event has fired: their outputs
     (pred, offsets, the result record) stay with the request, their memory goes
     back to the budget and their workspace back to the pool;
  2. admits waiting requests in arrival order while a slot is free and the
     request's bytes (workspace + outputs) fit what is left of the budget, and
     launches each one at once on its slot's stream.

So a request that arrives while others are on the GPU starts as soon as a slot
and memory free up, and its kernel overlaps theirs on the device (small
predictions occupy a few SMs each).  Results do not depend on the mix: every
output is an exact integer fixed by the operands and the sampling seed.

Workspaces are pooled by size class (powers of two); a workspace is zero-filled
when created and every call that ends without an error status leaves it clean,
so a pooled workspace is reused as is (after an error it is zeroed again).
Everything here is host-side marshalling and bookkeeping on top of the C ABI.
"""
import collections
import time
from dataclasses import dataclass

from . import (Workspace, _outputs, _torch, config, new_result, spgemm_predict_structure,
               spgemm_status_string, workspace_size, OK, RESULT_BYTES, STATUS_ERR_BAD_INPUT,
               STATUS_ERR_TIMEOUT)


@dataclass
class Request:
    """One prediction: device operands A, B (DeviceCSR) and its sampling config."""
    A: object
    B: object
    cfg: object
    rid: int = -1
    arrival: float = 0.0       # host time (perf_counter) the request arrived
    admitted: float = 0.0      # host time it was launched
    done: float = 0.0          # host time its completion was observed
    pred: object = None        # int32[M] device tensor
    offsets: object = None     # int64[M+1] device tensor
    res: object = None         # device result record (6 x int64)
    res_host: object = None    # pinned host copy of the record, valid once done
    nbytes: int = 0
    slot: int = -1
    _ws: object = None
    _event: object = None

    @property
    def latency(self):
        return self.done - self.arrival


def _size_class(nbytes):
    c = 1 << 20
    while c < nbytes:
        c <<= 1
    return c


@dataclass
class _Stats:
    submitted: int = 0
    admitted: int = 0
    finished: int = 0
    rejected: int = 0
    peak_inflight: int = 0
    peak_bytes: int = 0


class Server:
    """Continuous admission of predictions into `slots` streams within
    `memory_budget` bytes of device memory (workspaces + outputs)."""

    def __init__(self, slots=8, memory_budget=8 << 30, device="cuda"):
        torch = _torch()
        if slots < 1:
            raise ValueError("slots must be >= 1")
        self.device = torch.device(device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(slots)]
        self.free_slots = collections.deque(range(slots))
        self.budget = int(memory_budget)
        self.used = 0
        self.waiting = collections.deque()
        self.inflight = {}
        self.finished = []
        self.pool = collections.defaultdict(list)
        self.stats = _Stats()
        self._next_id = 0

    # ---- requests
    def request_bytes(self, A, B):
        ws = workspace_size(A, B)
        return _size_class(ws) + 4 * max(A.rows, 0) + 8 * (A.rows + 1) + RESULT_BYTES

    def submit(self, A, B, cfg, arrival=None):
        """Queue a request; returns it (or None when it can never fit the budget)."""
        r = Request(A, B, cfg, rid=self._next_id, arrival=time.perf_counter() if arrival is None else arrival)
        self._next_id += 1
        r.nbytes = self.request_bytes(A, B)
        self.stats.submitted += 1
        if r.nbytes > self.budget:
            self.stats.rejected += 1
            return None
        self.waiting.append(r)
        return r

    # ---- the loop
    def poll(self):
        """Retire finished requests, admit waiting ones; returns the number retired."""
        retired = 0
        for rid in [rid for rid, r in self.inflight.items() if r._event.query()]:
            r = self.inflight.pop(rid)
            r.done = time.perf_counter()
            self._retire(r)
            retired += 1
        while self.waiting and self.free_slots and self.used + self.waiting[0].nbytes <= self.budget:
            self._launch(self.waiting.popleft())
        return retired

    def drain(self, timeout=60.0):
        """Poll until nothing is waiting or running."""
        t0 = time.perf_counter()
        while self.waiting or self.inflight:
            self.poll()
            if time.perf_counter() - t0 > timeout:
                raise TimeoutError(f"{len(self.waiting)} waiting, {len(self.inflight)} running after {timeout} s")

    # ---- internals
    def _workspace(self, nbytes, st):
        """A clean workspace usable on stream st: from the pool (st waits for
        its last use or reset) or new (zero-filled on st itself)."""
        torch = _torch()
        cls = _size_class(nbytes)
        lst = self.pool[cls]
        if lst:
            ws = lst.pop()
            st.wait_event(ws.event)
            return ws
        with torch.cuda.stream(st):
            ws = Workspace(cls, self.device)
        ws.event = torch.cuda.Event()
        return ws

    def _launch(self, r):
        torch = _torch()
        slot = self.free_slots.popleft()
        st = self.streams[slot]
        r.slot = slot
        self.used += r.nbytes
        with torch.cuda.stream(st):
            r.pred, r.offsets, _ = _outputs(r.A.rows, self.device, False)
            r.res = new_result(self.device)
        r.res_host = torch.empty(RESULT_BYTES // 8, dtype=torch.int64, pin_memory=True)
        r._ws = self._workspace(workspace_size(r.A, r.B), st)
        rc = spgemm_predict_structure(r.A, r.B, r.cfg, r.pred, r.offsets, None, r.res, r._ws, st)
        if rc != OK:
            self.used -= r.nbytes
            self.free_slots.append(slot)
            raise RuntimeError(f"request {r.rid}: {spgemm_status_string(rc)} ({rc})")
        with torch.cuda.stream(st):
            r.res_host.copy_(r.res, non_blocking=True)
        r._event = torch.cuda.Event()
        r._event.record(st)
        r.admitted = time.perf_counter()
        self.inflight[r.rid] = r
        self.stats.admitted += 1
        self.stats.peak_inflight = max(self.stats.peak_inflight, len(self.inflight))
        self.stats.peak_bytes = max(self.stats.peak_bytes, self.used)

    def _retire(self, r):
        # the workspace is clean unless the call ended with an error status
        # (read from the pinned copy, already complete: no device sync here)
        torch = _torch()
        status = int(r.res_host[5]) & 0xFFFFFFFF
        if status & (STATUS_ERR_BAD_INPUT | STATUS_ERR_TIMEOUT):
            st = self.streams[r.slot]
            with torch.cuda.stream(st):
                r._ws.reset()
        r._ws.event.record(self.streams[r.slot])
        self.pool[r._ws.nbytes].append(r._ws)
        r._ws = None
        self.used -= r.nbytes
        self.free_slots.append(r.slot)
        self.finished.append(r)
        self.stats.finished += 1


def latency_summary(requests):
    """p50 / p99 / mean latency (seconds) and the span from first arrival to last completion."""
    import numpy as np
    lat = np.array([r.latency for r in requests])
    span = max(r.done for r in requests) - min(r.arrival for r in requests)
    return {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
            "mean": float(lat.mean()), "span": float(span), "n": len(requests)}


def run_poisson(server, pool, rate, n_requests, seed=0, ratio=0.01):
    """Offer n_requests predictions with Poisson arrivals at `rate` per second,
    each on an operand pair drawn uniformly from `pool` (a list of (A, B) device
    pairs) with its own sampling seed; returns the finished requests in id order."""
    import numpy as np
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=n_requests) if rate > 0 else np.zeros(n_requests)
    arrivals = np.cumsum(gaps)
    picks = rng.integers(0, len(pool), size=n_requests)
    T = int(ratio * (1 << 32))
    server.finished = []
    t0 = time.perf_counter()
    i = 0
    while i < n_requests or server.waiting or server.inflight:
        now = time.perf_counter() - t0
        while i < n_requests and arrivals[i] <= now:
            A, B = pool[picks[i]]
            server.submit(A, B, config(threshold=T, seed=int(i)), arrival=t0 + arrivals[i])
            i += 1
        server.poll()
    return sorted(server.finished, key=lambda r: r.rid), picks
