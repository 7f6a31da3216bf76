"""Host-side checks of the C ABI that need no GPU: the library builds, loads and
exports every function include/*.h declares; host-detected errors come back as
the documented negative codes before anything touches the device."""
import ctypes
import glob
import os
import re
import shutil

import pytest

import paper_2207_13848_gb300 as sp
from paper_2207_13848_gb300 import build as spbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \*]*?\b(spgemm_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(spbuild.LIB) and shutil.which("nvcc") is None:
        pytest.skip("no nvcc and no prebuilt library")
    spbuild.build()
    return sp.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("spgemm_flop_per_row", "spgemm_predict_cr", "spgemm_predict_structure",
              "spgemm_predict_reference", "spgemm_symbolic_exact", "spgemm_workspace_size",
              "spgemm_status_string", "spgemm_sample_rows", "spgemm_validate_csr"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert names
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(lib):
    for code in (0, -1, -2, -3, -4, -5, 1, 2, 4, 0x100, 0x200, 0x101, 0x3):
        s = sp.spgemm_status_string(code)
        assert isinstance(s, str) and s and s != "unknown code"


def test_struct_layouts_match_header():
    # the library asserts the same sizes at compile time
    assert ctypes.sizeof(sp.CsrStruct) == 40
    assert ctypes.sizeof(sp.ConfigStruct) == 32
    assert sp.RESULT_BYTES == 48
    assert ctypes.sizeof(sp.BatchItemStruct) == 144
    assert ctypes.sizeof(sp.TuningStruct) == 32
    assert ctypes.sizeof(sp.PlanStruct) == 88


def test_workspace_size_grows_with_rows(lib):
    a = sp.CsrStruct(0, 5, 0, 0, 0)
    s0 = lib.spgemm_workspace_size(ctypes.byref(a), None)
    a = sp.CsrStruct(1 << 20, 5, 0, 0, 0)
    s1 = lib.spgemm_workspace_size(ctypes.byref(a), None)
    assert s0 > 0 and s1 >= s0 + 8 * (1 << 20) - 4096
    assert lib.spgemm_workspace_size(None, None) == 0


class _Fake:
    """Operands with non-null fake device addresses: host checks must reject the
    call before any pointer is used."""

    def __init__(self, rows, cols, nnz):
        self.rows, self.cols, self.nnz = rows, cols, nnz

    def struct(self):
        return sp.CsrStruct(self.rows, self.cols, self.nnz, 0x1000, 0x2000 if self.nnz else 0)


def _call_predict(lib, A, B, cfg, ws_bytes, res=0x3000, ws=0x10000, pred=0x4000, offs=0x5000):
    a, b = A.struct(), B.struct()
    return lib.spgemm_predict_structure(ctypes.byref(a), ctypes.byref(b), ctypes.byref(cfg), pred, offs,
                                        None, res, ws, ws_bytes, None)


def test_host_errors(lib):
    A, B = _Fake(100, 50, 300), _Fake(50, 70, 200)
    cfg = sp.config(ratio=0.01)
    a, b = A.struct(), B.struct()
    ws = lib.spgemm_workspace_size(ctypes.byref(a), ctypes.byref(b))
    assert ws > lib.spgemm_workspace_size(ctypes.byref(sp.CsrStruct(100, 50, 0, 0, 0)),
                                          ctypes.byref(sp.CsrStruct(50, 0, 0, 0, 0)))  # B.cols counts
    assert _call_predict(lib, A, _Fake(51, 70, 200), cfg, ws) == sp.ERR_DIM_MISMATCH
    assert _call_predict(lib, A, B, cfg, ws - 1) == sp.ERR_WORKSPACE
    assert _call_predict(lib, A, B, cfg, ws, ws=0x10010) == sp.ERR_WORKSPACE  # misaligned
    assert _call_predict(lib, A, B, cfg, ws, res=0) == sp.ERR_INVALID_ARG
    assert _call_predict(lib, A, B, cfg, ws, pred=0) == sp.ERR_INVALID_ARG
    assert _call_predict(lib, _Fake(-1, 50, 0), B, cfg, ws) == sp.ERR_INVALID_ARG
    assert _call_predict(lib, _Fake(1 << 31, 50, 0), B, cfg, 1 << 40) == sp.ERR_TOO_LARGE
    bad = sp.config(threshold=(1 << 32) + 1)
    assert _call_predict(lib, A, B, bad, ws) == sp.ERR_INVALID_ARG
    bad = sp.config(mode=7, ratio=0.1)
    assert _call_predict(lib, A, B, bad, ws) == sp.ERR_INVALID_ARG
    bad = sp.config(mode=sp.SAMPLE_PAPER_DRAW, sample_num=101)  # more draws than rows
    assert _call_predict(lib, A, B, bad, ws) == sp.ERR_INVALID_ARG
    bad = sp.config(ratio=0.1)
    bad.reserved0 = 3
    assert _call_predict(lib, A, B, bad, ws) == sp.ERR_INVALID_ARG
    a, b = A.struct(), B.struct()
    assert lib.spgemm_flop_per_row(ctypes.byref(a), ctypes.byref(b), None, 0x3000, 0x10000, ws, None) \
        == sp.ERR_INVALID_ARG
    assert lib.spgemm_symbolic_exact(ctypes.byref(a), ctypes.byref(b), 0x4000, None, 0x3000, 0x10000, ws,
                                     None) == sp.ERR_INVALID_ARG
    cfgd = sp.config(mode=sp.SAMPLE_PAPER_DRAW, sample_num=10)
    assert lib.spgemm_sample_rows(100, ctypes.byref(cfgd), 0x4000, 5, 0x3000, 0x10000, ws, None) \
        == sp.ERR_INVALID_ARG


def _items(lib, shapes, cfg=None):
    """Batch items with fake device addresses (never dereferenced by host checks)."""
    items = (sp.BatchItemStruct * len(shapes))()
    for i, (a, b) in enumerate(shapes):
        items[i].A, items[i].B = _Fake(*a).struct(), _Fake(*b).struct()
        items[i].cfg = cfg or sp.config(ratio=0.01)
        items[i].pred_row, items[i].offsets, items[i].res = 0x4000, 0x5000, 0x3000
    return items


class _FakeWs:
    def __init__(self, addr, nbytes):
        self.addr, self.nbytes = addr, nbytes

    def ptr(self):
        return ctypes.c_void_p(self.addr)


def _prepare(lib, items, n, tuning, plan, ws, staging, bad):
    assert staging is None
    return lib.spgemm_batch_prepare(items, n, ctypes.byref(tuning) if tuning is not None else None,
                                    ctypes.byref(plan), ws.ptr(), ws.nbytes, None, 0,
                                    ctypes.byref(bad) if bad is not None else None, None)


def test_batch_workspace_and_staging_sizes(lib):
    one = _items(lib, [((100, 50, 300), (50, 70, 200))])
    two = _items(lib, [((100, 50, 300), (50, 70, 200)), ((1 << 20, 1 << 20, 1 << 24), ((1 << 20), 9, 5))])
    s1, s2 = sp.spgemm_batch_workspace_size(one, 1), sp.spgemm_batch_workspace_size(two, 2)
    assert s1 > 0 and s2 > s1 + 4 * (1 << 20) + (1 << 20)
    assert sp.spgemm_batch_staging_size(two, 2) >= 64 * 2
    assert sp.spgemm_batch_workspace_size(one, 0) == 0
    assert sp.spgemm_batch_workspace_size(_items(lib, [((100, 50, 300), (51, 70, 200))]), 1) == 0


def test_batch_host_errors(lib):
    shapes = [((100, 50, 300), (50, 70, 200))] * 2 + [((100, 50, 300), (51, 70, 200))]
    items = _items(lib, shapes)
    good = _items(lib, shapes[:2])
    need = sp.spgemm_batch_workspace_size(good, 2)
    ws = _FakeWs(0x100000, need)
    plan, bad = sp.PlanStruct(), ctypes.c_int32(-1)
    assert _prepare(lib, items, 3, None, plan, ws, None, bad) == sp.ERR_DIM_MISMATCH and bad.value == 2
    assert _prepare(lib, items, 0, None, plan, ws, None, None) == sp.ERR_INVALID_ARG
    assert _prepare(lib, good, 2, None, plan, _FakeWs(0x100010, need), None, None) == sp.ERR_WORKSPACE
    assert _prepare(lib, good, 2, None, plan, _FakeWs(0x100000, need - 256), None, None) \
        == sp.ERR_WORKSPACE
    for bad_tuning in (dict(warp_table=300), dict(warp_table=512, heavy_threshold=257),
                       dict(heavy_threshold=16), dict(tile_items=1000), dict(sample_chunk=5000),
                       dict(flop_blocks_per_sm=-1)):
        assert _prepare(lib, good, 2, sp.tuning(**bad_tuning), plan, ws, None, None) \
            == sp.ERR_INVALID_ARG, bad_tuning
    t = sp.tuning()
    t.reserved[1] = 1
    assert _prepare(lib, good, 2, t, plan, ws, None, None) == sp.ERR_INVALID_ARG
    for bad_launches in (dict(launches=2), dict(launches=3)):
        assert _prepare(lib, good, 2, sp.tuning(**bad_launches), plan, ws, None, None) == sp.ERR_INVALID_ARG
    nopred = _items(lib, shapes[:1])
    nopred[0].pred_row = None
    assert _prepare(lib, nopred, 1, None, plan, ws, None, bad) == sp.ERR_INVALID_ARG
    draws = _items(lib, shapes[:1], sp.config(mode=sp.SAMPLE_PAPER_DRAW, sample_num=101))
    assert _prepare(lib, draws, 1, None, plan, ws, None, bad) == sp.ERR_INVALID_ARG
    assert lib.spgemm_predict_batch(None, ws.ptr(), need, None) == sp.ERR_INVALID_ARG


def _call_numeric(lib, A, B, ws_bytes, compact=False, a_val=0x6000, b_val=0x7000, alloc=0x8000, c_col=0x9000,
                  c_val=0xA000, cap=1000, row_start=0xB000, nnz_row=0xC000, res=0xD000, ws=0x10000,
                  out_rpt=0xE000, out_col=0xF000, out_val=0xF800, out_cap=1000):
    a, b = A.struct(), B.struct()
    if compact:
        return lib.spgemm_numeric_compact(ctypes.byref(a), a_val, ctypes.byref(b), b_val, c_col, c_val, cap,
                                          row_start, nnz_row, out_rpt, out_col, out_val, out_cap, res, ws,
                                          ws_bytes, None)
    return lib.spgemm_numeric_into(ctypes.byref(a), a_val, ctypes.byref(b), b_val, alloc, c_col, c_val, cap,
                                   row_start, nnz_row, res, ws, ws_bytes, None)


@pytest.mark.parametrize("compact", [False, True])
def test_numeric_host_errors(lib, compact):
    # every argument the numeric calls check on the host, one at a time; the
    # good call itself is never made (it would touch the device)
    A, B = _Fake(100, 50, 300), _Fake(50, 70, 200)
    a, b = A.struct(), B.struct()
    ws = lib.spgemm_workspace_size(ctypes.byref(a), ctypes.byref(b))

    def call(**kw):
        return _call_numeric(lib, kw.pop("A", A), kw.pop("B", B), kw.pop("ws_bytes", ws), compact, **kw)

    assert call(B=_Fake(51, 70, 200)) == sp.ERR_DIM_MISMATCH
    assert call(A=_Fake(1 << 31, 50, 0), ws_bytes=1 << 40) == sp.ERR_TOO_LARGE
    assert call(A=_Fake(-1, 50, 0)) == sp.ERR_INVALID_ARG
    for arg in ("res", "ws", "a_val", "b_val", "row_start", "nnz_row", "c_col", "c_val"):
        assert call(**{arg: None}) == sp.ERR_INVALID_ARG, arg
    assert call(cap=-1) == sp.ERR_INVALID_ARG
    # no values are needed for operands without nonzeros, and no C arrays for
    # a zero capacity; the other checks still apply
    assert call(A=_Fake(100, 50, 0), a_val=None, cap=0, c_col=None, c_val=None, ws_bytes=ws - 1) \
        == sp.ERR_WORKSPACE
    assert call(ws_bytes=ws - 1) == sp.ERR_WORKSPACE
    assert call(ws=0x10010) == sp.ERR_WORKSPACE  # misaligned
    if compact:
        assert call(out_rpt=None) == sp.ERR_INVALID_ARG
        assert call(out_cap=-1) == sp.ERR_INVALID_ARG
        assert call(out_col=None) == sp.ERR_INVALID_ARG
        assert call(out_val=None) == sp.ERR_INVALID_ARG


def test_product_path_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(sp, "_lib", None)
    monkeypatch.setattr(sp, "library_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        sp.load()


def _call_static(lib, A, B, cfg, pred=0x4000, offs=0x5000, res=0x3000):
    a, b = A.struct(), B.struct()
    return lib.spgemm_predict_structure_static(ctypes.byref(a), ctypes.byref(b),
                                               ctypes.byref(cfg) if cfg is not None else None,
                                               pred, offs, None, res, None)


def test_static_entry_point_host_errors(lib):
    # The entry point without a workspace checks everything on the host before
    # it touches the device: a rejected call returns its code with nothing queued
    # (these calls never reach a CUDA call, so they run without a GPU).
    A, B = _Fake(100, 50, 300), _Fake(50, 70, 200)
    cfg = sp.config(ratio=0.01)
    assert _call_static(lib, A, _Fake(51, 70, 200), cfg) == sp.ERR_DIM_MISMATCH
    assert _call_static(lib, A, B, cfg, res=0) == sp.ERR_INVALID_ARG
    assert _call_static(lib, A, B, cfg, pred=0) == sp.ERR_INVALID_ARG
    assert _call_static(lib, A, B, cfg, offs=0) == sp.ERR_INVALID_ARG
    assert _call_static(lib, A, B, None) == sp.ERR_INVALID_ARG
    assert _call_static(lib, _Fake(-1, 50, 0), B, cfg) == sp.ERR_INVALID_ARG
    assert _call_static(lib, A, B, sp.config(threshold=(1 << 32) + 1)) == sp.ERR_INVALID_ARG
    assert _call_static(lib, A, B, sp.config(mode=7, ratio=0.1)) == sp.ERR_INVALID_ARG
    assert _call_static(lib, A, B, sp.config(mode=sp.SAMPLE_PAPER_DRAW, sample_num=101)) == sp.ERR_INVALID_ARG
    assert _call_static(lib, _Fake(1 << 31, 50, 0), B, cfg) == sp.ERR_TOO_LARGE
    big = sp.STATIC_MAX_ROWS + 1
    # any one of A.rows, A.cols, B.cols above the limit
    assert _call_static(lib, _Fake(big, 50, 0), B, cfg) == sp.ERR_STATIC_CAPACITY
    assert _call_static(lib, _Fake(100, big, 0), _Fake(big, 70, 0), cfg) == sp.ERR_STATIC_CAPACITY
    assert _call_static(lib, A, _Fake(50, big, 0), cfg) == sp.ERR_STATIC_CAPACITY


def test_lookup_probe_host_errors(lib):
    assert lib.spgemm_lookup_probe(0x1000, -1, 0x2000, 10, 0x3000, None) == sp.ERR_INVALID_ARG
    assert lib.spgemm_lookup_probe(0x1000, 10, 0x2000, 10, None, None) == sp.ERR_INVALID_ARG
    assert lib.spgemm_lookup_probe(0x1004, 10, 0x2000, 10, 0x3000, None) == sp.ERR_INVALID_ARG  # unaligned ids
    assert lib.spgemm_lookup_probe(None, 10, 0x2000, 10, 0x3000, None) == sp.ERR_INVALID_ARG
    assert lib.spgemm_lookup_probe(0x1000, 10, None, 10, 0x3000, None) == sp.ERR_INVALID_ARG
