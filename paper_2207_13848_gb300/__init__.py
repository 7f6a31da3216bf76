"""GB300 output-structure predictor for SpGEMM C = A*B (sampled compression ratio,
Du et al., arXiv 2207.13848).

A thin binding over the C ABI declared in ``include/spgemm_predict.h``: the
functions named ``spgemm_*`` take the same arguments as their C counterparts,
with torch CUDA tensors standing in for device pointers, and return the C return
code.  Every step of the computation runs in the CUDA library; importing this
package does not load it, but the first call does, and fails loudly when the
library has not been built (``paper_2207_13848_gb300.build.build()``) or no GPU
is present.  PyTorch is used for device memory and streams only.

Convenience wrappers (``DeviceCSR``, ``Workspace``, ``predict_structure`` ...)
allocate the outputs with torch and call the C ABI.
"""
import ctypes
import os
from dataclasses import dataclass
from typing import Optional

from . import build as _build

# ---- constants mirrored from the header --------------------------------------
OK = 0
ERR_INVALID_ARG = -1
ERR_DIM_MISMATCH = -2
ERR_WORKSPACE = -3
ERR_CUDA = -4
ERR_TOO_LARGE = -5
ERR_STATIC_CAPACITY = -6
STATIC_MAX_ROWS = 1 << 21
STATUS_WARN_EMPTY_SAMPLE = 0x1
STATUS_WARN_SATURATED = 0x2
STATUS_WARN_UNSORTED = 0x4
STATUS_ERR_BAD_INPUT = 0x100
STATUS_ERR_TIMEOUT = 0x200
SAMPLE_BERNOULLI = 0
SAMPLE_PAPER_DRAW = 1
TWO32 = 1 << 32


class CsrStruct(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("cols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("rpt", ctypes.c_void_p), ("col", ctypes.c_void_p)]


class ConfigStruct(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("threshold", ctypes.c_uint64), ("sample_num", ctypes.c_int64),
                ("seed", ctypes.c_uint64)]


RESULT_BYTES = 48  # spgemm_result_t: 5 x int64 + 2 x int32
BATCH_MAX_CASES = 1 << 20


class BatchItemStruct(ctypes.Structure):
    _fields_ = [("A", CsrStruct), ("B", CsrStruct), ("cfg", ConfigStruct),
                ("pred_row", ctypes.c_void_p), ("offsets", ctypes.c_void_p),
                ("flop_row", ctypes.c_void_p), ("res", ctypes.c_void_p)]


class TuningStruct(ctypes.Structure):
    _fields_ = [("tile_items", ctypes.c_int32), ("warp_table", ctypes.c_int32),
                ("heavy_threshold", ctypes.c_int32), ("sample_chunk", ctypes.c_int32),
                ("flop_blocks_per_sm", ctypes.c_int32), ("launches", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]

    def as_dict(self):
        return {k: getattr(self, k) for k in ("tile_items", "warp_table", "heavy_threshold",
                                               "sample_chunk", "flop_blocks_per_sm", "launches")}


class PlanStruct(ctypes.Structure):
    _fields_ = [("n_cases", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("total_rows", ctypes.c_int64), ("total_candidates", ctypes.c_int64),
                ("total_tiles", ctypes.c_int64), ("total_chunks", ctypes.c_int64),
                ("total_table_blocks", ctypes.c_int64), ("ws_bytes", ctypes.c_uint64),
                ("tuning", TuningStruct)]


def tuning(**kw):
    """A TuningStruct; unnamed fields are 0 (the library's defaults)."""
    t = TuningStruct()
    for k, v in kw.items():
        setattr(t, k, int(v))
    return t

_lib = None


def library_path():
    return str(_build.LIB)


def load():
    """Load the CUDA library (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing "
                           "(run paper_2207_13848_gb300.build.build())")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    C = ctypes.POINTER(CsrStruct)
    G = ctypes.POINTER(ConfigStruct)
    sz = ctypes.c_size_t
    lib.spgemm_workspace_size.restype = sz
    lib.spgemm_workspace_size.argtypes = [C, C]
    lib.spgemm_flop_per_row.argtypes = [C, C, P, P, P, sz, P]
    lib.spgemm_predict_cr.argtypes = [C, C, G, P, P, sz, P]
    lib.spgemm_predict_structure.argtypes = [C, C, G, P, P, P, P, P, sz, P]
    lib.spgemm_predict_reference.argtypes = [C, C, G, P, P, P, P, P, sz, P]
    lib.spgemm_symbolic_exact.argtypes = [C, C, P, P, P, P, sz, P]
    lib.spgemm_sample_rows.argtypes = [ctypes.c_int64, G, P, ctypes.c_int64, P, P, sz, P]
    lib.spgemm_validate_csr.argtypes = [C, P, P, sz, P]
    lib.spgemm_predict_structure_static.argtypes = [C, C, G, P, P, P, P, P]
    lib.spgemm_predict_structure_static.restype = ctypes.c_int
    lib.spgemm_set_profile_events.argtypes = [P, P]
    lib.spgemm_set_profile_events.restype = ctypes.c_int
    lib.spgemm_predict_many.argtypes = [ctypes.POINTER(BatchItemStruct), ctypes.c_int32, ctypes.POINTER(P),
                                        ctypes.POINTER(sz), ctypes.POINTER(ctypes.c_int32), P]
    lib.spgemm_predict_many.restype = ctypes.c_int
    lib.spgemm_lookup_probe.argtypes = [P, ctypes.c_int64, P, ctypes.c_int64, P, P]
    lib.spgemm_lookup_probe.restype = ctypes.c_int
    I = ctypes.POINTER(BatchItemStruct)
    T = ctypes.POINTER(TuningStruct)
    PL = ctypes.POINTER(PlanStruct)
    i32 = ctypes.c_int32
    lib.spgemm_batch_workspace_size.restype = sz
    lib.spgemm_batch_workspace_size.argtypes = [I, i32]
    lib.spgemm_batch_staging_size.restype = sz
    lib.spgemm_batch_staging_size.argtypes = [I, i32]
    lib.spgemm_batch_prepare.argtypes = [I, i32, T, PL, P, sz, P, sz, ctypes.POINTER(i32), P]
    lib.spgemm_predict_batch.argtypes = [PL, P, sz, P]
    lib.spgemm_batch_autotune.argtypes = [I, i32, P, sz, i32, T, ctypes.POINTER(ctypes.c_float), PL, P]
    for fn in (lib.spgemm_batch_prepare, lib.spgemm_predict_batch, lib.spgemm_batch_autotune):
        fn.restype = ctypes.c_int
    lib.spgemm_status_string.restype = ctypes.c_char_p
    lib.spgemm_status_string.argtypes = [ctypes.c_int]
    i64 = ctypes.c_int64
    lib.spgemm_numeric_into.argtypes = [C, P, C, P, P, P, P, i64, P, P, P, P, sz, P]
    lib.spgemm_numeric_compact.argtypes = [C, P, C, P, P, P, i64, P, P, P, P, P, i64, P, P, sz, P]
    lib.spgemm_numeric_into.restype = ctypes.c_int
    lib.spgemm_numeric_compact.restype = ctypes.c_int
    for fn in (lib.spgemm_flop_per_row, lib.spgemm_predict_cr, lib.spgemm_predict_structure,
               lib.spgemm_predict_reference, lib.spgemm_symbolic_exact, lib.spgemm_sample_rows,
               lib.spgemm_validate_csr):
        fn.restype = ctypes.c_int
    _lib = lib
    return lib


def _torch():
    import torch
    return torch


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check(rc, what):
    if rc != OK:
        msg = load().spgemm_status_string(rc).decode()
        raise RuntimeError(f"{what} failed: {msg} ({rc})")
    return rc


# ---- device-side operands -----------------------------------------------------
class DeviceCSR:
    """A CSR matrix whose int32 rpt/col arrays live in CUDA memory (torch tensors)."""

    def __init__(self, rows, cols, rpt, col):
        self.rows, self.cols = int(rows), int(cols)
        self.rpt, self.col = rpt, col
        self.nnz = int(col.numel())

    @classmethod
    def from_host(cls, m, device="cuda", non_blocking=False):
        """Copy a host CSR (numpy rpt/col; e.g. workloads.CSR) to the device."""
        torch = _torch()
        rpt = torch.from_numpy(m.rpt).to(device, non_blocking=non_blocking)
        col = torch.from_numpy(m.col).to(device, non_blocking=non_blocking)
        if col.numel() == 0:
            col = torch.zeros(1, dtype=torch.int32, device=device)[:0]
        return cls(m.rows, m.cols, rpt, col)

    def struct(self):
        return CsrStruct(self.rows, self.cols, self.nnz, self.rpt.data_ptr(),
                         self.col.data_ptr() if self.nnz else 0)


def config(mode=SAMPLE_BERNOULLI, ratio=None, threshold=None, sample_num=0, seed=0):
    """Sampling configuration; ``ratio`` in [0, 1] maps to threshold floor(ratio * 2^32)."""
    if threshold is None:
        threshold = 0 if ratio is None else min(TWO32, int(ratio * TWO32))
    return ConfigStruct(int(mode), 0, int(threshold), int(sample_num), int(seed) & (2**64 - 1))


def workspace_size(A, B=None):
    a = A.struct()
    b = B.struct() if B is not None else None
    return int(load().spgemm_workspace_size(ctypes.byref(a), ctypes.byref(b) if b else None))


class Workspace:
    """Zero-filled device workspace, reusable across calls on one stream."""

    def __init__(self, nbytes, device="cuda"):
        torch = _torch()
        self.nbytes = int(nbytes)
        self.buf = torch.zeros(self.nbytes + 256, dtype=torch.uint8, device=device)
        off = (-self.buf.data_ptr()) % 256
        self.view = self.buf[off: off + self.nbytes]

    @classmethod
    def for_operands(cls, A, B=None, device="cuda"):
        return cls(workspace_size(A, B), device)

    def ptr(self):
        return ctypes.c_void_p(self.view.data_ptr())

    def reset(self):
        self.buf.zero_()


def new_result(device="cuda"):
    torch = _torch()
    return torch.zeros(RESULT_BYTES // 8, dtype=torch.int64, device=device)


def read_result(res):
    """Host copy of a device result record as a dict."""
    v = res.cpu().tolist()
    status = v[5] & 0xFFFFFFFF
    return dict(flop_total=v[0], flop_s=v[1], nnz_s=v[2], n_sampled=v[3], pred_total=v[4],
                status=status)


NUMERIC_RESULT_BYTES = 40


def new_numeric_result(device="cuda"):
    torch = _torch()
    return torch.zeros(NUMERIC_RESULT_BYTES // 8, dtype=torch.int64, device=device)


def read_numeric_result(res):
    """Host copy of a device numeric result record as a dict."""
    v = res.cpu().tolist()
    return dict(nnz_total=v[0], overflow_rows=v[1], overflow_nnz=v[2], alloc_total=v[3],
                status=v[4] & 0xFFFFFFFF)


# ---- the C ABI, same names and argument order -----------------------------------
def spgemm_flop_per_row(A, B, flop_row, res, ws, stream=None):
    a, b = A.struct(), B.struct()
    return load().spgemm_flop_per_row(ctypes.byref(a), ctypes.byref(b), _ptr(flop_row), _ptr(res),
                                      ws.ptr(), ws.nbytes, _stream(stream))


def spgemm_predict_cr(A, B, cfg, res, ws, stream=None):
    a, b = A.struct(), B.struct()
    return load().spgemm_predict_cr(ctypes.byref(a), ctypes.byref(b), ctypes.byref(cfg), _ptr(res),
                                    ws.ptr(), ws.nbytes, _stream(stream))


def spgemm_predict_structure(A, B, cfg, pred_row, offsets, flop_row, res, ws, stream=None):
    a, b = A.struct(), B.struct()
    return load().spgemm_predict_structure(ctypes.byref(a), ctypes.byref(b), ctypes.byref(cfg),
                                           _ptr(pred_row), _ptr(offsets), _ptr(flop_row), _ptr(res),
                                           ws.ptr(), ws.nbytes, _stream(stream))


def spgemm_predict_reference(A, B, cfg, pred_row, offsets, flop_row, res, ws, stream=None):
    a, b = A.struct(), B.struct()
    return load().spgemm_predict_reference(ctypes.byref(a), ctypes.byref(b), ctypes.byref(cfg),
                                           _ptr(pred_row), _ptr(offsets), _ptr(flop_row), _ptr(res),
                                           ws.ptr(), ws.nbytes, _stream(stream))


def spgemm_predict_structure_static(A, B, cfg, pred_row, offsets, flop_row, res, stream=None):
    """spgemm_predict_structure with the library's own fixed scratch array instead
    of a workspace, for callers that cannot allocate device memory (no
    allocation happens inside; the first call per device must precede any
    stream capture, and overlapping calls race)."""
    a, b = A.struct(), B.struct()
    return load().spgemm_predict_structure_static(ctypes.byref(a), ctypes.byref(b), ctypes.byref(cfg),
                                                  _ptr(pred_row), _ptr(offsets), _ptr(flop_row),
                                                  _ptr(res), _stream(stream))


def spgemm_symbolic_exact(A, B, nnz_row, offsets, res, ws, stream=None):
    a, b = A.struct(), B.struct()
    return load().spgemm_symbolic_exact(ctypes.byref(a), ctypes.byref(b), _ptr(nnz_row), _ptr(offsets),
                                        _ptr(res), ws.ptr(), ws.nbytes, _stream(stream))


def spgemm_sample_rows(rows, cfg, ids, capacity, res, ws, stream=None):
    return load().spgemm_sample_rows(int(rows), ctypes.byref(cfg), _ptr(ids), int(capacity), _ptr(res),
                                     ws.ptr(), ws.nbytes, _stream(stream))


def spgemm_validate_csr(A, res, ws, stream=None):
    a = A.struct()
    return load().spgemm_validate_csr(ctypes.byref(a), _ptr(res), ws.ptr(), ws.nbytes, _stream(stream))


def spgemm_set_profile_events(before, after):
    """Record torch.cuda.Event `before`/`after` around the main kernel of later calls
    (None, None turns it off)."""
    b = None if before is None else ctypes.c_void_p(before.cuda_event)
    a = None if after is None else ctypes.c_void_p(after.cuda_event)
    return load().spgemm_set_profile_events(b, a)


def spgemm_predict_many(items, n, ws_ptrs, ws_bytes, bad_item, stream=None):
    """items: ctypes array of BatchItemStruct; ws_ptrs: ctypes array of c_void_p;
    ws_bytes: ctypes array of c_size_t; bad_item: ctypes.c_int32 or None."""
    return load().spgemm_predict_many(items, int(n), ws_ptrs, ws_bytes,
                                      ctypes.byref(bad_item) if bad_item is not None else None, _stream(stream))


def spgemm_lookup_probe(col, table, out, stream=None):
    """Stream col (int32) with one lookup into table (uint8) per id; the sum of the
    bytes read goes to out (int64/uint64 tensor of one element)."""
    return load().spgemm_lookup_probe(_ptr(col), int(col.numel()), _ptr(table), int(table.numel()), _ptr(out),
                                      _stream(stream))


def _numel(t):
    return 0 if t is None else int(t.numel())


def spgemm_numeric_into(A, a_val, B, b_val, alloc_offsets, c_col, c_val, row_start, nnz_row, res, ws, stream=None):
    """C = A*B into per-row shares (alloc_offsets) or one pool (alloc_offsets None)."""
    a, b = A.struct(), B.struct()
    cap = min(_numel(c_col), _numel(c_val))
    return load().spgemm_numeric_into(ctypes.byref(a), _ptr(a_val), ctypes.byref(b), _ptr(b_val),
                                      _ptr(alloc_offsets), _ptr(c_col), _ptr(c_val), cap, _ptr(row_start),
                                      _ptr(nnz_row), _ptr(res), ws.ptr(), ws.nbytes, _stream(stream))


def spgemm_numeric_compact(A, a_val, B, b_val, c_col, c_val, row_start, nnz_row, out_rpt, out_col, out_val, res,
                           ws, stream=None):
    """The exact CSR of C from spgemm_numeric_into's output."""
    a, b = A.struct(), B.struct()
    cap = min(_numel(c_col), _numel(c_val))
    out_cap = min(_numel(out_col), _numel(out_val))
    return load().spgemm_numeric_compact(ctypes.byref(a), _ptr(a_val), ctypes.byref(b), _ptr(b_val),
                                         _ptr(c_col), _ptr(c_val), cap, _ptr(row_start), _ptr(nnz_row),
                                         _ptr(out_rpt), _ptr(out_col), _ptr(out_val), out_cap, _ptr(res),
                                         ws.ptr(), ws.nbytes, _stream(stream))


def spgemm_status_string(code):
    return load().spgemm_status_string(int(code)).decode()


def spgemm_batch_workspace_size(items, n):
    return int(load().spgemm_batch_workspace_size(items, int(n)))


def spgemm_batch_staging_size(items, n):
    return int(load().spgemm_batch_staging_size(items, int(n)))


def spgemm_batch_prepare(items, n, tuning_, plan, ws, host_staging, bad_item, stream=None):
    """items: ctypes array of BatchItemStruct; tuning_: TuningStruct or None;
    plan: PlanStruct (written); host_staging: pinned torch CPU tensor or None;
    bad_item: ctypes.c_int32 or None."""
    hs = None if host_staging is None else ctypes.c_void_p(host_staging.data_ptr())
    hb = 0 if host_staging is None else host_staging.numel() * host_staging.element_size()
    return load().spgemm_batch_prepare(items, int(n), ctypes.byref(tuning_) if tuning_ is not None else None,
                                       ctypes.byref(plan), ws.ptr(), ws.nbytes, hs, hb,
                                       ctypes.byref(bad_item) if bad_item is not None else None,
                                       _stream(stream))


def spgemm_predict_batch(plan, ws, stream=None):
    return load().spgemm_predict_batch(ctypes.byref(plan), ws.ptr(), ws.nbytes, _stream(stream))


def spgemm_batch_autotune(items, n, ws, reps, best, best_ms, plan, stream=None):
    """best: TuningStruct (written); best_ms: ctypes.c_float or None; plan: PlanStruct (written)."""
    return load().spgemm_batch_autotune(items, int(n), ws.ptr(), ws.nbytes, int(reps), ctypes.byref(best),
                                        ctypes.byref(best_ms) if best_ms is not None else None,
                                        ctypes.byref(plan), _stream(stream))


# ---- convenience wrappers -------------------------------------------------------
@dataclass
class Prediction:
    pred: "object"             # int32[M] predicted nnz per row (or exact nnz for symbolic)
    offsets: "object"          # int64[M+1]
    flop: Optional["object"]   # int32[M] FLOP per row when requested
    res: "object"              # device result record


def _outputs(M, device, want_flop):
    torch = _torch()
    pred = torch.empty(max(M, 0), dtype=torch.int32, device=device)
    offsets = torch.empty(M + 1, dtype=torch.int64, device=device)
    flop = torch.empty(max(M, 0), dtype=torch.int32, device=device) if want_flop else None
    return pred, offsets, flop


def predict_structure(A, B, cfg, ws=None, want_flop=False, reference=False, stream=None):
    """Run the proposed method (or the reference design) and return device tensors."""
    ws = ws or Workspace.for_operands(A, B)
    pred, offsets, flop = _outputs(A.rows, A.rpt.device, want_flop)
    res = new_result(A.rpt.device)
    fn = spgemm_predict_reference if reference else spgemm_predict_structure
    _check(fn(A, B, cfg, pred, offsets, flop, res, ws, stream), fn.__name__)
    return Prediction(pred, offsets, flop, res)


def symbolic_exact(A, B, ws=None, stream=None):
    ws = ws or Workspace.for_operands(A, B)
    nnz, offsets, _ = _outputs(A.rows, A.rpt.device, False)
    res = new_result(A.rpt.device)
    _check(spgemm_symbolic_exact(A, B, nnz, offsets, res, ws, stream), "spgemm_symbolic_exact")
    return Prediction(nnz, offsets, None, res)


def flop_per_row(A, B, ws=None, stream=None):
    torch = _torch()
    ws = ws or Workspace.for_operands(A, B)
    flop = torch.empty(max(A.rows, 0), dtype=torch.int32, device=A.rpt.device)
    res = new_result(A.rpt.device)
    _check(spgemm_flop_per_row(A, B, flop, res, ws, stream), "spgemm_flop_per_row")
    return flop, res


def predict_cr(A, B, cfg, ws=None, stream=None):
    ws = ws or Workspace.for_operands(A, B)
    res = new_result(A.rpt.device)
    _check(spgemm_predict_cr(A, B, cfg, res, ws, stream), "spgemm_predict_cr")
    return res


def sample_rows(rows, cfg, capacity=None, ws=None, device="cuda", stream=None):
    torch = _torch()
    # |S| <= rows in both modes (the library takes at most `rows` draws), so a
    # buffer of `rows` ids always holds the sample
    cap = max(rows, 1) if capacity is None else capacity
    ws = ws or Workspace(_build_ws_bytes(rows), device)
    ids = torch.full((max(cap, 1),), -1, dtype=torch.int32, device=device)
    res = new_result(device)
    _check(spgemm_sample_rows(rows, cfg, ids, cap, res, ws, stream), "spgemm_sample_rows")
    return ids, res


def _build_ws_bytes(rows):
    a = CsrStruct(rows, 0, 0, 0, 0)
    return int(load().spgemm_workspace_size(ctypes.byref(a), None))


def validate_csr(A, ws=None, stream=None):
    ws = ws or Workspace.for_operands(A)
    res = new_result(A.rpt.device)
    _check(spgemm_validate_csr(A, res, ws, stream), "spgemm_validate_csr")
    return res


def predict_structure_host(A_host, B_host, cfg, ws=None, device="cuda", stream=None, same=False):
    """End-to-end call on host operands: host->device copies of the CSR arrays,
    the prediction, and device->host copies of pred/offsets and the result.
    Returns host numpy arrays and the result dict."""
    torch = _torch()
    A = DeviceCSR.from_host(A_host, device, non_blocking=True)
    B = A if same else DeviceCSR.from_host(B_host, device, non_blocking=True)
    p = predict_structure(A, B, cfg, ws=ws, stream=stream)
    pred = p.pred.to("cpu", non_blocking=True)
    offsets = p.offsets.to("cpu", non_blocking=True)
    res = p.res.to("cpu", non_blocking=True)
    torch.cuda.current_stream().synchronize()
    return pred.numpy(), offsets.numpy(), read_result(res)


class Batch:
    """Many predictions in one batched run (spgemm_predict_batch).

    ``cases`` is a list of (A, B, cfg) with DeviceCSR operands.  Outputs are
    allocated per case (pred, offsets, optional flop) and the result records of
    all cases share one int64 tensor [n, 6], so one copy reads them all."""

    def __init__(self, cases, want_flop=False, device="cuda", tuning_=None, pinned=True):
        torch = _torch()
        self.cases = list(cases)
        self.n = len(self.cases)
        self.device = device
        self.res = torch.zeros((self.n, RESULT_BYTES // 8), dtype=torch.int64, device=device)
        self.outputs = [_outputs(A.rows, device, want_flop) for A, _, _ in self.cases]
        self.items = (BatchItemStruct * self.n)()
        for i, ((A, B, cfg), (pred, offs, flop)) in enumerate(zip(self.cases, self.outputs)):
            it = self.items[i]
            it.A, it.B, it.cfg = A.struct(), B.struct(), cfg
            it.pred_row = pred.data_ptr() if A.rows > 0 else None
            it.offsets = offs.data_ptr()
            it.flop_row = flop.data_ptr() if (flop is not None and A.rows > 0) else None
            it.res = self.res[i].data_ptr()
        nbytes = spgemm_batch_workspace_size(self.items, self.n)
        if nbytes == 0:
            raise RuntimeError("spgemm_batch_workspace_size rejected the batch")
        self.ws = Workspace(nbytes, device)
        sbytes = spgemm_batch_staging_size(self.items, self.n)
        self.staging = torch.empty(sbytes, dtype=torch.uint8, pin_memory=pinned) if sbytes else None
        self.plan = PlanStruct()
        self.prepare(tuning_)

    def prepare(self, tuning_=None, stream=None):
        bad = ctypes.c_int32(-1)
        rc = spgemm_batch_prepare(self.items, self.n, tuning_, self.plan, self.ws, self.staging, bad, stream)
        if rc != OK:
            raise RuntimeError(f"spgemm_batch_prepare failed on case {bad.value}: "
                               f"{spgemm_status_string(rc)} ({rc})")
        return self.plan

    def run(self, stream=None):
        _check(spgemm_predict_batch(self.plan, self.ws, stream), "spgemm_predict_batch")

    def autotune(self, reps=3, stream=None):
        best, ms = TuningStruct(), ctypes.c_float(0)
        _check(spgemm_batch_autotune(self.items, self.n, self.ws, reps, best, ms, self.plan, stream),
               "spgemm_batch_autotune")
        return best, ms.value

    def results(self):
        """Host list of result dicts, one per case."""
        rows = self.res.cpu().tolist()
        return [dict(flop_total=v[0], flop_s=v[1], nnz_s=v[2], n_sampled=v[3], pred_total=v[4],
                     status=v[5] & 0xFFFFFFFF) for v in rows]

    def prediction(self, i):
        pred, offs, flop = self.outputs[i]
        return Prediction(pred, offs, flop, self.res[i])



# ---- the consumer: numeric product allocated by the prediction ------------------
@dataclass
class NumericProduct:
    rpt: "object"      # int64[M + 1] exact offsets (device), or (row_start, nnz_row) without compaction
    col: "object"      # int32[NNZ(C)] (device; column order within a row is free)
    val: "object"      # float32[NNZ(C)] (device)
    info: dict         # prediction and numeric result records, allocation sizes


def numeric_product(A, a_val, B, b_val, cfg, ws=None, stream=None, compact=True, pool=True, slack=0.0):
    """C = A*B the way the prediction is meant to be used: predict the structure,
    allocate C by the prediction, compute every row into that allocation, then
    build the exact CSR (rows that were written are moved, rows that overflowed
    are computed again).  pool=True allocates the predicted total (times 1 +
    slack) as one pool; pool=False gives each row its predicted share.  One host
    read of the numeric result sizes the exact arrays.  With compact=False,
    returns (row_start, nnz_row) as the row layout, without the compaction (a
    complete product only when no row overflowed)."""
    import math
    torch = _torch()
    dev = A.rpt.device
    ws = ws or Workspace.for_operands(A, B)
    pred = predict_structure(A, B, cfg, ws=ws, stream=stream)
    presult = read_result(pred.res)
    total = max(presult["pred_total"], 0)
    cap = int(math.ceil(total * (1.0 + slack))) if pool else total
    c_col = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)[:cap]
    c_val = torch.empty(max(cap, 1), dtype=torch.float32, device=dev)[:cap]
    row_start = torch.empty(max(A.rows, 0), dtype=torch.int64, device=dev)
    nnz_row = torch.empty(max(A.rows, 0), dtype=torch.int32, device=dev)
    nres = new_numeric_result(dev)
    _check(spgemm_numeric_into(A, a_val, B, b_val, None if pool else pred.offsets, c_col, c_val, row_start, nnz_row,
                               nres, ws, stream), "spgemm_numeric_into")
    info = {"prediction": presult, "numeric": read_numeric_result(nres), "pool": pool}
    if not compact:
        return NumericProduct((row_start, nnz_row), c_col, c_val, info)
    Z = info["numeric"]["nnz_total"]
    out_rpt = torch.empty(A.rows + 1, dtype=torch.int64, device=dev)
    out_col = torch.empty(max(Z, 1), dtype=torch.int32, device=dev)[:Z]
    out_val = torch.empty(max(Z, 1), dtype=torch.float32, device=dev)[:Z]
    _check(spgemm_numeric_compact(A, a_val, B, b_val, c_col, c_val, row_start, nnz_row, out_rpt, out_col, out_val,
                                  nres, ws, stream), "spgemm_numeric_compact")
    info["numeric"]["status"] = read_numeric_result(nres)["status"]
    return NumericProduct(out_rpt, out_col, out_val, info)
