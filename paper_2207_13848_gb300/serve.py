"""Serving loop for structure predictions: continuous batching.  Requests are
admitted continuously into device slots, by free slots and by device memory,
and run concurrently.

A request is one prediction (Eq. 4 of the paper: the spgemm_predict_structure
result) on operands that are already resident on the device.  The server owns
`slots` CUDA streams and a device-memory budget.  Every `poll()`:

  1. retires the launches whose completion event has fired: their requests'
     outputs (pred, offsets, the result record) stay with the requests, their
     memory goes back to the budget and their workspaces back to the pools;
  2. admits waiting requests in arrival order while a slot is free and the
     memory fits.  Small requests (A.rows <= batch_rows) that are waiting
     together are merged, up to max_batch of them, into ONE batched launch
     (spgemm_predict_batch: every case's outputs are bit-identical to its own
     spgemm_predict_structure call) that occupies one slot; a larger request
     gets its own single-launch call.

So a request that arrives while others are on the GPU starts as soon as a slot
and memory free up, small ones share launches instead of each paying its own,
and launches on different slots overlap on the device.  Results do not depend
on the mix: every output is an exact integer fixed by the operands and the
sampling seed.

Workspaces are pooled by size class (powers of two); a workspace is
zero-filled when created and every call that ends without an error status
leaves it clean, so a pooled workspace is reused as is (after an error it is
zeroed again).  A launch the library rejects does not stop the loop: its
requests are marked failed and counted as rejected.  Everything here is
host-side marshalling and bookkeeping on top of the C ABI.
"""
import collections
import ctypes
import time
from dataclasses import dataclass

from . import (BatchItemStruct, PlanStruct, Workspace, _torch, config, spgemm_batch_prepare,
               spgemm_batch_staging_size, spgemm_batch_workspace_size, spgemm_predict_batch,
               spgemm_predict_many, spgemm_status_string, workspace_size, OK, RESULT_BYTES,
               STATUS_ERR_BAD_INPUT, STATUS_ERR_TIMEOUT)


@dataclass
class Request:
    """One prediction: device operands A, B (DeviceCSR) and its sampling config."""
    A: object
    B: object
    cfg: object
    rid: int = -1
    index: int = -1            # position in the stream that offered it (run_poisson), else -1
    arrival: float = 0.0       # host time (perf_counter) the request arrived
    admitted: float = 0.0      # host time it was launched
    done: float = 0.0          # host time its completion was observed
    pred: object = None        # int32[M] device tensor
    offsets: object = None     # int64[M+1] device tensor
    res: object = None         # device result record (6 x int64)
    res_host: object = None    # pinned host copy of the record, valid once done
    nbytes: int = 0
    slot: int = -1
    batched: bool = False      # served by a batched launch
    solo: bool = False         # never merged (set when a batch it was in was rejected)
    error: str = ""            # why the library rejected its launch (then res is unset)

    @property
    def latency(self):
        return self.done - self.arrival


@dataclass
class _Launch:
    """One launch on one slot: a single request or a merged batch."""
    requests: list
    slot: int
    nbytes: int
    ws: object = None          # the batch's workspace (batch)
    wss: list = None           # one workspace per request (single predictions)
    batch: bool = False
    staging: object = None     # pinned plan staging (batch), reused once the launch completed
    event: object = None
    res_all: object = None     # [n, 6] device result records (batch)
    res_host: object = None    # [n, 6] pinned copy (batch)


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
    failed: int = 0
    peak_inflight: int = 0
    peak_bytes: int = 0
    launches: int = 0
    batched_launches: int = 0
    batched_requests: int = 0


class Server:
    """Continuous batching of predictions into `slots` streams within
    `memory_budget` bytes of device memory (workspaces + outputs).  Requests
    with A.rows <= batch_rows that wait together are merged into one batched
    launch of at most max_batch cases (batch_rows = 0: never merge)."""

    def __init__(self, slots=3, memory_budget=8 << 30, device="cuda", batch_rows=1 << 18, max_batch=128,
                 streams=1):
        torch = _torch()
        if slots < 1:
            raise ValueError("slots must be >= 1")
        self.device = torch.device(device)
        # `slots` launches may be in flight at once; they run on `streams` CUDA
        # streams, slot s on stream s mod streams (None: one per slot).  One
        # stream is the default: a large prediction is a cooperative launch
        # that needs every SM, so launches on several streams only wait for
        # one another, while on one stream they run back to back and the host
        # prepares the next ones meanwhile
        ns = slots if streams is None else max(1, min(int(streams), slots))
        own = [torch.cuda.Stream(device=self.device) for _ in range(ns)]
        self.streams = [own[i % ns] for i in range(slots)]
        self.free_slots = collections.deque(range(slots))
        self.budget = int(memory_budget)
        self.batch_rows = int(batch_rows)
        self.max_batch = max(1, int(max_batch))
        self.used = 0
        self.wait_small = collections.deque()  # requests that may be merged, in arrival order
        self.wait_large = collections.deque()  # requests launched alone, in arrival order
        self.inflight = {}         # launch id -> _Launch
        self.finished = []
        self.failed = []
        # workspaces by size class: single-call and batch workspaces have
        # different layouts, so each kind is reused only as its own kind
        self.pool = collections.defaultdict(list)
        self.bpool = collections.defaultdict(list)
        self.staging_pool = collections.defaultdict(list)  # pinned plan buffers by size class
        self.host_pool = collections.defaultdict(list)     # pinned result-record copies by count
        self.events = []                                   # idle completion events
        self.stats = _Stats()
        self._next_id = 0
        self._next_launch = 0

    # ---- requests
    def request_bytes(self, A, B):
        # kept on the operand A, per B (held, so that its id stays its own)
        cache = getattr(A, "_serve_bytes", None)
        if cache is None:
            cache = A._serve_bytes = {}
        hit = cache.get(id(B))
        if hit is not None and hit[0] is B:
            return hit[1]
        nb = _size_class(workspace_size(A, B)) + 4 * max(A.rows, 0) + 8 * (A.rows + 1) + RESULT_BYTES
        cache[id(B)] = (B, nb)
        return nb

    def submit(self, A, B, cfg, arrival=None, index=-1):
        """Queue a request; returns it (or None when it can never fit the budget)."""
        r = Request(A, B, cfg, rid=self._next_id, index=index,
                    arrival=time.perf_counter() if arrival is None else arrival)
        self._next_id += 1
        r.nbytes = self.request_bytes(A, B)
        self.stats.submitted += 1
        if r.nbytes > self.budget:
            self.stats.rejected += 1
            return None
        (self.wait_small if self._small(r) else self.wait_large).append(r)
        return r

    @property
    def waiting(self):
        """The requests not yet launched, in arrival order."""
        return sorted(list(self.wait_small) + list(self.wait_large), key=lambda r: r.rid)

    def _small(self, r):
        return self.batch_rows > 0 and not r.solo and r.A.rows <= self.batch_rows

    # ---- the loop
    def poll(self):
        """Retire finished launches, admit waiting requests; returns the number of
        requests retired."""
        retired = 0
        for lid in [lid for lid, ln in self.inflight.items() if ln.event.query()]:
            ln = self.inflight.pop(lid)
            retired += self._retire(ln)
        # the queue whose head arrived first goes first; small requests are
        # merged, up to max_batch, whatever large ones arrived between them
        while self.free_slots and (self.wait_small or self.wait_large):
            hs = self.wait_small[0] if self.wait_small else None
            hl = self.wait_large[0] if self.wait_large else None
            if hs is not None and (hl is None or hs.rid < hl.rid):
                if self.used + hs.nbytes > self.budget:
                    break
                group, nbytes = [], 0
                while (self.wait_small and len(group) < self.max_batch
                       and self.used + nbytes + self.wait_small[0].nbytes <= self.budget):
                    r = self.wait_small.popleft()
                    group.append(r)
                    nbytes += r.nbytes
                if len(group) == 1:
                    self._launch_single(group[0])
                else:
                    self._launch_batch(group, nbytes)
            else:
                # large requests that wait together go out by one host call
                # (each still its own prediction, on one stream, in order)
                group, nbytes = [], 0
                while (self.wait_large and len(group) < self.max_batch
                       and self.used + nbytes + self.wait_large[0].nbytes <= self.budget
                       and not (self.wait_small and self.wait_small[0].rid < self.wait_large[0].rid)):
                    r = self.wait_large.popleft()
                    group.append(r)
                    nbytes += r.nbytes
                if not group:
                    break
                self._launch_many(group, nbytes)
        return retired

    def drain(self, timeout=60.0):
        """Poll until nothing is waiting or running."""
        t0 = time.perf_counter()
        while self.wait_small or self.wait_large or self.inflight:
            self.poll()
            if time.perf_counter() - t0 > timeout:
                raise TimeoutError(f"{len(self.waiting)} waiting, {len(self.inflight)} running after {timeout} s")

    # ---- internals
    def _workspace(self, nbytes, st, batch=False):
        """A clean workspace usable on stream st: from the pool of its kind (st
        waits for its last use or reset) or new (zero-filled on st itself)."""
        torch = _torch()
        cls = _size_class(nbytes)
        lst = (self.bpool if batch else self.pool)[cls]
        if lst:
            ws = lst.pop()
            st.wait_event(ws.event)
            return ws
        with torch.cuda.stream(st):
            ws = Workspace(cls, self.device)
        ws.event = torch.cuda.Event()
        return ws

    def _staging(self, nbytes):
        torch = _torch()
        cls = _size_class(max(nbytes, 1))
        lst = self.staging_pool[cls]
        return lst.pop() if lst else torch.empty(cls, dtype=torch.uint8, pin_memory=True)

    def _start(self, ln, st):
        torch = _torch()
        ln.event = self.events.pop() if self.events else torch.cuda.Event()
        ln.event.record(st)
        now = time.perf_counter()
        for r in ln.requests:
            r.admitted = now
        self.inflight[self._next_launch] = ln
        self._next_launch += 1
        self.used += ln.nbytes
        self.stats.admitted += len(ln.requests)
        self.stats.launches += 1
        self.stats.peak_inflight = max(self.stats.peak_inflight, sum(len(x.requests) for x in self.inflight.values()))
        self.stats.peak_bytes = max(self.stats.peak_bytes, self.used)

    def _fail(self, ln, st, msg):
        """The library rejected the launch: give back its slot and workspace
        (zeroed again on the slot's stream), mark its requests failed, go on."""
        torch = _torch()
        if ln.ws is not None:
            with torch.cuda.stream(st):
                ln.ws.reset()
            ln.ws.event.record(st)
            (self.bpool if ln.batch else self.pool)[ln.ws.nbytes].append(ln.ws)
        for ws in ln.wss or []:
            ws.event.record(st)
            self.pool[ws.nbytes].append(ws)
        if ln.staging is not None:
            self.staging_pool[ln.staging.numel()].append(ln.staging)
        if ln.res_host is not None:
            self.host_pool[ln.res_host.shape[0]].append(ln.res_host)
        self.free_slots.append(ln.slot)
        now = time.perf_counter()
        for r in ln.requests:
            r.error, r.done = msg, now
            self.failed.append(r)
        self.stats.failed += len(ln.requests)
        self.stats.rejected += len(ln.requests)

    def _requeue(self, ln, requests, solo, keep_launch=False):
        """Put a rejected batch's requests back at the head of the queue, in
        order (solo: launched one by one from now on); unless keep_launch, give
        back the launch's slot."""
        for r in reversed(requests):
            r.batched, r.slot, r.solo = False, -1, r.solo or solo
            r.pred = r.offsets = r.res = r.res_host = None
            (self.wait_large if r.solo else self.wait_small).appendleft(r)
        if not keep_launch:
            self.free_slots.append(ln.slot)
            if ln.res_host is not None:
                self.host_pool[ln.res_host.shape[0]].append(ln.res_host)

    def _outputs_for(self, ln, requests, st):
        """pred, offsets and result records of a launch's requests: views of one
        allocation each (the library writes every record whole, so none is
        initialised), and a pinned host buffer for the records."""
        torch = _torch()
        rows = [max(r.A.rows, 0) for r in requests]
        n = len(requests)
        with torch.cuda.stream(st):
            preds = torch.empty(max(sum(rows), 1), dtype=torch.int32, device=self.device)
            offs = torch.empty(sum(rows) + n, dtype=torch.int64, device=self.device)
            ln.res_all = torch.empty((n, RESULT_BYTES // 8), dtype=torch.int64, device=self.device)
        hp = self.host_pool[n]
        ln.res_host = hp.pop() if hp else torch.empty((n, RESULT_BYTES // 8), dtype=torch.int64, pin_memory=True)
        a = b = 0
        for i, (r, m) in enumerate(zip(requests, rows)):
            r.pred = preds[a:a + m]
            r.offsets = offs[b:b + m + 1]
            r.res = ln.res_all[i]
            r.res_host = ln.res_host[i]
            a += m
            b += m + 1

    def _launch_single(self, r):
        self._launch_many([r], r.nbytes)

    def _launch_many(self, group, nbytes):
        """Single predictions of the requests in `group`, queued on one slot's
        stream by one library call (spgemm_predict_many)."""
        slot = self.free_slots.popleft()
        st = self.streams[slot]
        n = len(group)
        ln = _Launch(group, slot, nbytes, wss=[])
        self._outputs_for(ln, group, st)
        items = (BatchItemStruct * n)()
        ptrs = (ctypes.c_void_p * n)()
        sizes = (ctypes.c_size_t * n)()
        for i, r in enumerate(group):
            r.slot = slot
            it = items[i]
            it.A, it.B, it.cfg = _csr_struct(r.A), _csr_struct(r.B), r.cfg
            it.pred_row = r.pred.data_ptr() if r.A.rows > 0 else None
            it.offsets = r.offsets.data_ptr()
            it.flop_row = None
            it.res = r.res.data_ptr()
            ws = self._workspace(workspace_size(r.A, r.B), st)
            ln.wss.append(ws)
            ptrs[i] = ws.view.data_ptr()
            sizes[i] = ws.nbytes
        bad = ctypes.c_int32(-1)
        rc = spgemm_predict_many(items, n, ptrs, sizes, bad, st)
        if rc != OK:
            b = bad.value if 0 <= bad.value < n else 0
            # the calls before the culprit were queued and run; it fails alone;
            # the ones after it wait again at the head of their queue
            for r in reversed(group[b + 1:]):
                r.slot = -1
                r.pred = r.offsets = r.res = r.res_host = None
                self.wait_large.appendleft(r)
            for ws in ln.wss[b + 1:]:
                self.pool[ws.nbytes].append(ws)  # untouched: clean as they came
            culprit, culprit_ws = group[b], ln.wss[b]
            culprit_ws.event.record(st)
            self.pool[culprit_ws.nbytes].append(culprit_ws)  # its call was rejected before any work
            culprit.error, culprit.done = f"{spgemm_status_string(rc)} ({rc})", time.perf_counter()
            self.failed.append(culprit)
            self.stats.failed += 1
            self.stats.rejected += 1
            ln.requests, ln.wss = group[:b], ln.wss[:b]
            ln.nbytes = sum(r.nbytes for r in ln.requests)
            if not ln.requests:
                self.host_pool[ln.res_host.shape[0]].append(ln.res_host)
                self.free_slots.append(slot)
                return
        self._copy_back(ln, st)
        self._start(ln, st)

    def _copy_back(self, ln, st):
        torch = _torch()
        with torch.cuda.stream(st):
            ln.res_host.copy_(ln.res_all, non_blocking=True)

    def _launch_batch(self, group, nbytes):
        slot = self.free_slots.popleft()
        st = self.streams[slot]
        n = len(group)
        ln = _Launch(group, slot, nbytes, batch=True)
        self._outputs_for(ln, group, st)
        items = (BatchItemStruct * n)()
        for i, r in enumerate(group):
            r.slot, r.batched = slot, True
            it = items[i]
            it.A, it.B, it.cfg = _csr_struct(r.A), _csr_struct(r.B), r.cfg
            it.pred_row = r.pred.data_ptr() if r.A.rows > 0 else None
            it.offsets = r.offsets.data_ptr()
            it.flop_row = None
            it.res = r.res.data_ptr()
        wbytes = spgemm_batch_workspace_size(items, n)
        if wbytes == 0:  # some case is invalid: each request goes on alone
            self._requeue(ln, group, solo=True)
            return
        ln.ws = self._workspace(wbytes, st, batch=True)
        ln.staging = self._staging(spgemm_batch_staging_size(items, n))
        plan, bad = PlanStruct(), ctypes.c_int32(-1)
        rc = spgemm_batch_prepare(items, n, None, plan, ln.ws, ln.staging, bad, st)
        if rc != OK and 0 <= bad.value < n:
            # one case is at fault: it fails alone, the others wait again at the
            # head of the queue (they are merged again on this same poll)
            culprit = group[bad.value]
            self._requeue(ln, [r for r in group if r is not culprit], solo=False, keep_launch=True)
            ln.requests = [culprit]
            self._fail(ln, st, f"{spgemm_status_string(rc)} ({rc})")
            return
        if rc == OK:
            rc = spgemm_predict_batch(plan, ln.ws, st)
        if rc != OK:
            self._fail(ln, st, f"{spgemm_status_string(rc)} ({rc})")
            return
        self._copy_back(ln, st)
        self.stats.batched_launches += 1
        self.stats.batched_requests += n
        self._start(ln, st)

    def _retire(self, ln):
        # the workspace is clean unless a call ended with an error status (read
        # from the pinned copies, already complete: no device sync here)
        torch = _torch()
        st = self.streams[ln.slot]
        now = time.perf_counter()
        status = [(v & 0xFFFFFFFF) & (STATUS_ERR_BAD_INPUT | STATUS_ERR_TIMEOUT) for v in ln.res_host[:, 5].tolist()]
        wss = [ln.ws] * len(ln.requests) if ln.batch else ln.wss
        for ws, bad in zip(wss, status):
            if bad:
                with torch.cuda.stream(st):
                    ws.reset()
        for ws in ([ln.ws] if ln.batch else ln.wss):
            ws.event.record(st)
            (self.bpool if ln.batch else self.pool)[ws.nbytes].append(ws)
        if ln.staging is not None:
            self.staging_pool[ln.staging.numel()].append(ln.staging)
        for r in ln.requests:
            r.done = now
            r.res_host = r.res_host.clone()  # its own copy: the pinned buffer goes back to the pool
        self.host_pool[ln.res_host.shape[0]].append(ln.res_host)
        self.events.append(ln.event)
        self.used -= ln.nbytes
        self.free_slots.append(ln.slot)
        self.finished.extend(ln.requests)
        self.stats.finished += len(ln.requests)
        return len(ln.requests)


def _csr_struct(m):
    """The CsrStruct of a DeviceCSR, built once per operand."""
    s = getattr(m, "_serve_struct", None)
    if s is None:
        s = m.struct()
        m._serve_struct = s
    return s


def latency_summary(requests):
    """p50 / p99 / mean latency (seconds) and the span from first arrival to last completion."""
    import numpy as np
    lat = np.array([r.latency for r in requests])
    span = max(r.done for r in requests) - min(r.arrival for r in requests)
    return {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
            "mean": float(lat.mean()), "span": float(span), "n": len(requests)}


def run_poisson(server, pool, rate, n_requests, seed=0, ratio=0.01, pause_gc=True):
    """Offer n_requests predictions with Poisson arrivals at `rate` per second,
    each on an operand pair drawn uniformly from `pool` (a list of (A, B) device
    pairs) with its own sampling seed; returns the finished requests in id order.
    pause_gc: Python's cyclic garbage collector is off while the requests are
    served (and back on afterwards).  The loop's objects hold no reference
    cycles, so reference counting frees them, and a full collection over the
    run's tens of thousands of live objects would stall the host loop, and with
    it every request waiting or arriving meanwhile, for tens of milliseconds."""
    import gc
    import numpy as np
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=n_requests) if rate > 0 else np.zeros(n_requests)
    arrivals = np.cumsum(gaps)
    picks = rng.integers(0, len(pool), size=n_requests)
    T = int(ratio * (1 << 32))
    server.finished = []
    gc_on = gc.isenabled()
    if pause_gc:
        gc.disable()
    try:
        t0 = time.perf_counter()
        i = 0
        while i < n_requests or server.wait_small or server.wait_large or server.inflight:
            now = time.perf_counter() - t0
            while i < n_requests and arrivals[i] <= now:
                A, B = pool[picks[i]]
                server.submit(A, B, config(threshold=T, seed=int(i)), arrival=t0 + arrivals[i], index=int(i))
                i += 1
            server.poll()
    finally:
        if pause_gc and gc_on:
            gc.enable()
    return sorted(server.finished, key=lambda r: r.index), picks
