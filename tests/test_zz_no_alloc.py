"""The entry point for callers that cannot allocate device memory
(spgemm_predict_structure_static) must give exactly the results of
spgemm_predict_structure, call after call, while using the library's own fixed
scratch array instead of a workspace.

Kept in a file that pytest collects last, so that a run stopping at the first
failure has already run every other test; it passes alone in a fresh process
and after the rest of the suite."""
import ctypes

import numpy as np
import pytest

import paper_2207_13848_gb300 as sp
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _outputs(M):
    return (torch.empty(M, dtype=torch.int32, device="cuda"),
            torch.empty(M + 1, dtype=torch.int64, device="cuda"),
            torch.empty(M, dtype=torch.int32, device="cuda"),
            sp.new_result("cuda"))


@pytest.mark.parametrize("case", ["er", "rmat", "lap2d"])
def test_static_scratch_matches_workspace_path_twice(case):
    if case == "er":
        A, T = W.erdos_renyi(1 << 17, 16, 41), int(0.01 * sp.TWO32)
    elif case == "rmat":
        A, T = W.rmat(16, 16, seed=42), int(0.005 * sp.TWO32)
    else:
        A, T = W.laplacian_2d(64), int(0.01 * sp.TWO32)
    dA = sp.DeviceCSR.from_host(A)
    M = A.rows
    # the existing entry point, with its own workspace
    ref = sp.predict_structure(dA, dA, sp.config(threshold=T, seed=3), want_flop=True)
    torch.cuda.synchronize()
    want = (ref.pred.cpu().numpy(), ref.offsets.cpu().numpy(), ref.flop.cpu().numpy(), sp.read_result(ref.res))
    pred, offs, flop, res = _outputs(M)
    for call in range(2):
        pred.fill_(-7)
        offs.fill_(-7)
        flop.fill_(-7)
        res.zero_()
        rc = sp.spgemm_predict_structure_static(dA, dA, sp.config(threshold=T, seed=3), pred, offs, flop, res)
        assert rc == sp.OK, sp.spgemm_status_string(rc)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(pred.cpu().numpy(), want[0], err_msg=f"pred, call {call}")
        np.testing.assert_array_equal(offs.cpu().numpy(), want[1], err_msg=f"offsets, call {call}")
        np.testing.assert_array_equal(flop.cpu().numpy(), want[2], err_msg=f"flop, call {call}")
        assert sp.read_result(res) == want[3], f"result record, call {call}"


def test_static_scratch_rejects_oversized_problems():
    big = sp.CsrStruct(sp.STATIC_MAX_ROWS + 1, 10, 0, 0x1000, 0)
    small = sp.CsrStruct(10, 10, 0, 0x1000, 0)
    cfg = sp.config(ratio=0.01)
    rc = sp.load().spgemm_predict_structure_static(ctypes.byref(big), ctypes.byref(small), ctypes.byref(cfg),
                                                   0x2000, 0x3000, None, 0x4000, None)
    assert rc == sp.ERR_STATIC_CAPACITY
    assert "static scratch" in sp.spgemm_status_string(rc)


def test_static_scratch_rectangular_product():
    # A(n x n/2) * B(n/2 x n) by the reshape rule: the static scratch is sized
    # from A.rows, A.cols and B.cols separately
    n = 1 << 15
    A = W.keep_left_columns(W.erdos_renyi(n, 12, 51), n // 2)
    B = W.keep_top_rows(W.erdos_renyi(n, 12, 52), n // 2)
    dA, dB = sp.DeviceCSR.from_host(A), sp.DeviceCSR.from_host(B)
    cfg = sp.config(ratio=0.02, seed=5)
    ref = sp.predict_structure(dA, dB, cfg, want_flop=True)
    torch.cuda.synchronize()
    pred, offs, flop, res = _outputs(A.rows)
    for call in range(2):
        rc = sp.spgemm_predict_structure_static(dA, dB, cfg, pred, offs, flop, res)
        assert rc == sp.OK, sp.spgemm_status_string(rc)
        torch.cuda.synchronize()
        assert torch.equal(pred, ref.pred) and torch.equal(offs, ref.offsets) and torch.equal(flop, ref.flop)
        assert sp.read_result(res) == sp.read_result(ref.res), f"call {call}"


def test_static_scratch_recovers_after_a_bad_input_and_handles_empty_b():
    # A column id out of range is reported in the status (the scratch may be
    # left dirty); the next call starts from a cleared scratch and is exact again.
    A = W.erdos_renyi(4096, 8, 61)
    badA = W.CSR(A.rows, A.cols, A.rpt.copy(), A.col.copy())
    badA.col[100] = A.cols + 5
    dA, dBad = sp.DeviceCSR.from_host(A), sp.DeviceCSR.from_host(badA)
    cfg = sp.config(ratio=0.05, seed=2)
    pred, offs, flop, res = _outputs(A.rows)
    rc = sp.spgemm_predict_structure_static(dBad, dA, cfg, pred, offs, flop, res)
    assert rc == sp.OK
    torch.cuda.synchronize()
    assert sp.read_result(res)["status"] & sp.STATUS_ERR_BAD_INPUT
    ref = sp.predict_structure(dA, dA, cfg, want_flop=True)
    rc = sp.spgemm_predict_structure_static(dA, dA, cfg, pred, offs, flop, res)
    assert rc == sp.OK
    torch.cuda.synchronize()
    assert torch.equal(pred, ref.pred) and torch.equal(offs, ref.offsets)
    assert sp.read_result(res) == sp.read_result(ref.res)
    # B with no columns: every product is empty; no split-row slots exist
    E = W.CSR(A.cols, 0, np.zeros(A.cols + 1, dtype=np.int32), np.zeros(0, dtype=np.int32))
    dE = sp.DeviceCSR.from_host(E)
    rc = sp.spgemm_predict_structure_static(dA, dE, cfg, pred, offs, flop, res)
    assert rc == sp.OK, sp.spgemm_status_string(rc)
    torch.cuda.synchronize()
    r = sp.read_result(res)
    assert r["flop_total"] == 0 and r["pred_total"] == 0 and r["status"] == sp.STATUS_WARN_EMPTY_SAMPLE
    assert int(offs.abs().sum()) == 0
    # and the library call after it still works (no stale CUDA error)
    ref2 = sp.predict_structure(dA, dA, cfg, want_flop=True)
    torch.cuda.synchronize()
    assert torch.equal(ref2.pred, ref.pred)
