"""GPU paths that the other parity tests do not reach.

- B with 2^23 columns or more: the single-launch predictor packs (row, column)
  keys of the sampled rows into 32 bits only while the column id fits 23 bits;
  wider B makes each warp count its sampled rows alone (the per-warp path),
  and heavy rows then take column bitmaps in several column passes.  Compared
  with the oracle bit for bit, both designs.
- A bounded wait that runs out: every wait between thread blocks gives up
  after about a second with SPGEMM_STATUS_ERR_TIMEOUT instead of hanging.  A
  workspace whose heavy-row count says three rows are queued, while no entry
  was ever written, makes the waits for those rows run out (no GPU fault: the
  wait loops are bounded and return).  The call must come back with the
  status bit set, and a re-zeroed workspace must then give exact results.
"""
import numpy as np
import pytest

import oracle
import paper_2207_13848_gb300 as sp
import workloads as W
from tests.gpu_helpers import TWO32, assert_prediction_equal, gpu_predict, oracle_predict, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

WIDE_N = (1 << 23) + 5


def _wide_operands():
    """A (3000 x 2048): rows of 6 entries, and 4 hub rows of 120 entries;
    B (2048 x (2^23 + 5)): rows of 8 entries over all columns, the last
    column included, so that hub rows have ~960 products spread over 2^23
    columns."""
    rng = np.random.default_rng(77)
    M, K = 3000, 2048
    rows = [np.repeat(np.arange(4), 120), np.repeat(np.arange(4, M), 6)]
    cols = [np.concatenate([rng.choice(K, 120, replace=False) for _ in range(4)]),
            rng.integers(0, K, 6 * (M - 4))]
    A = W.from_coo(M, K, np.concatenate(rows), np.concatenate(cols))
    rb = np.repeat(np.arange(K), 8)
    cb = rng.integers(0, WIDE_N, K * 8)
    cb[:5] = WIDE_N - 1 - np.arange(5)  # the top columns
    cb[5:8] = (1 << 23) + np.arange(3)  # ids above 2^23
    B = W.from_coo(K, WIDE_N, rb, cb)
    return A, B


@pytest.mark.parametrize("reference", [False, True])
def test_wide_b_per_warp_sampling(reference):
    A, B = _wide_operands()
    assert B.cols >= 1 << 23
    dA, dB = to_dev(A), to_dev(B)
    ws = sp.Workspace.for_operands(dA, dB)
    for seed, ratio in ((0, 0.05), (1, 0.5), (2, 1.0)):
        T = min(int(ratio * TWO32), TWO32)
        g = gpu_predict(A, B, sp.SAMPLE_BERNOULLI, seed, T, reference=reference, ws=ws, dA=dA, dB=dB)
        o = oracle_predict(A, B, oracle.BERNOULLI, seed, T, reference=reference)
        assert_prediction_equal(g, o, f"wide B seed {seed} ratio {ratio}")
    g = gpu_predict(A, B, sp.SAMPLE_PAPER_DRAW, 3, sample_num=700, reference=reference, ws=ws, dA=dA, dB=dB)
    o = oracle_predict(A, B, oracle.PAPER_DRAW, 3, sample_num=700, reference=reference)
    assert_prediction_equal(g, o, "wide B paper draws")


def test_wait_runs_out_and_reports_timeout():
    A = W.erdos_renyi(1 << 14, 8, 91)
    dA = to_dev(A)
    ws = sp.Workspace.for_operands(dA, dA)
    T = int(0.05 * TWO32)
    # the header's heavy-row count (a 32-bit word after the four 64-bit
    # accumulators) claims three queued rows; the queue itself stays empty
    ws.view[32:36].copy_(torch.tensor([3, 0, 0, 0], dtype=torch.uint8))
    cfg = sp.config(threshold=T, seed=4)
    p = sp.predict_structure(dA, dA, cfg, ws=ws, want_flop=True)
    torch.cuda.synchronize()  # returns: the waits are bounded
    r = sp.read_result(p.res)
    assert r["status"] & sp.STATUS_ERR_TIMEOUT, r
    # after an error the workspace is zeroed again; the next call is exact
    ws.reset()
    g = gpu_predict(A, A, sp.SAMPLE_BERNOULLI, 4, T, ws=ws, dA=dA, dB=dA)
    o = oracle_predict(A, A, oracle.BERNOULLI, 4, T)
    assert_prediction_equal(g, o, "after the timeout")


def test_lookup_probe_sums_the_bytes_it_reads():
    # the roofline calibration reads table[col[j]] for every j (ids outside the
    # table count as zero); its checksum is that sum
    rng = np.random.default_rng(5)
    n, K = (1 << 16) * 3 + 77, 5000
    col = rng.integers(-3, K + 3, n).astype(np.int32)
    tab = rng.integers(0, 256, K).astype(np.uint8)
    want = int(tab[col[(col >= 0) & (col < K)]].astype(np.int64).sum())
    dcol, dtab = torch.from_numpy(col).cuda(), torch.from_numpy(tab).cuda()
    out = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    assert sp.spgemm_lookup_probe(dcol, dtab, out) == sp.OK
    torch.cuda.synchronize()
    assert int(out.item()) == want


def test_predict_many_equals_single_calls_and_stops_at_a_rejected_item():
    # spgemm_predict_many queues the single-case calls of many items by one
    # host call: outputs bit-identical to spgemm_predict_structure; a call
    # rejected on the host stops it there (the calls before it were queued)
    import ctypes
    mats = [W.erdos_renyi(3000, 7, 1), W.rmat(12, 8, seed=2), W.laplacian_2d(40)]
    dev = [to_dev(m) for m in mats]
    T = int(0.05 * TWO32)
    n = 4
    items = (sp.BatchItemStruct * n)()
    outs, wss = [], []
    ptrs, sizes = (ctypes.c_void_p * n)(), (ctypes.c_size_t * n)()
    for i in range(n):
        dA = dev[i % 3]
        cfg = sp.config(threshold=T, seed=i) if i != 2 else sp.config(threshold=(1 << 32) + 1)
        pred, offs, res = (torch.empty(dA.rows, dtype=torch.int32, device="cuda"),
                           torch.empty(dA.rows + 1, dtype=torch.int64, device="cuda"), sp.new_result("cuda"))
        outs.append((pred, offs, res))
        it = items[i]
        it.A, it.B, it.cfg = dA.struct(), dA.struct(), cfg
        it.pred_row, it.offsets, it.flop_row, it.res = pred.data_ptr(), offs.data_ptr(), None, res.data_ptr()
        ws = sp.Workspace.for_operands(dA, dA)
        wss.append(ws)
        ptrs[i], sizes[i] = ws.view.data_ptr(), ws.nbytes
    bad = ctypes.c_int32(-1)
    rc = sp.spgemm_predict_many(items, n, ptrs, sizes, bad)
    torch.cuda.synchronize()
    assert rc == sp.ERR_INVALID_ARG and bad.value == 2
    for i in range(2):
        o = oracle_predict(mats[i], mats[i], oracle.BERNOULLI, i, T)
        g = dict(pred=outs[i][0].cpu().numpy(), offsets=outs[i][1].cpu().numpy(), flop=o["flop"],
                 **sp.read_result(outs[i][2]))
        assert_prediction_equal(g, o, f"item {i}")
