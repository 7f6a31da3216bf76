"""Parity of the CUDA path (through the C ABI) with the CPU oracle on seeded
synthetic inputs.  Every quantity is an integer with one correct value, so the
bar is bit-exact equality: FLOP per row, F, the sample, f*, z*, |S|, the
per-row predictions, the offsets, the exact nnz per row and the status."""
import numpy as np
import pytest

import oracle
import paper_2207_13848_gb300 as sp
import workloads as W
from tests.gpu_helpers import (TWO32, assert_prediction_equal, gpu_predict, gpu_symbolic,
                               oracle_predict, to_dev)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _small_cases():
    cases = {
        "lap2d-64": (W.laplacian_2d(64), None),
        "lap2d-torus-33": (W.laplacian_2d(33, periodic=True), None),
        "er-16k": (W.erdos_renyi(1 << 14, 16, 11), None),
        "er-ragged-12345": (W.erdos_renyi(12345, 7, 12), None),
        "rmat-14": (W.rmat(14, 16, seed=13), None),
        "st27-16x16x8": (W.stencil_3d_27(16, 16, 8), None),
        "blockdiag-4096": (W.block_diagonal(4096, 32, 0.3, 14), None),
        "dense-blocks-64": (W.dense_blocks(4096, 64), None),
        "rect-er": (W.keep_left_columns(W.erdos_renyi(8192, 12, 15), 4096),
                    W.keep_top_rows(W.erdos_renyi(8192, 12, 16), 4096)),
        "rect-rmat": (W.keep_left_columns(W.rmat(13, 8, seed=17), 4096),
                      W.keep_top_rows(W.rmat(13, 8, seed=18), 4096)),
    }
    return cases


CASES = _small_cases()


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("reference", [False, True])
def test_predict_small_bernoulli(name, reference):
    A, B = CASES[name]
    B = A if B is None else B
    dA = to_dev(A)
    dB = dA if B is A else to_dev(B)
    ws = sp.Workspace.for_operands(dA, dB)
    for seed in range(4):
        for ratio in (0.01, 0.1):
            T = int(ratio * TWO32)
            g = gpu_predict(A, B, sp.SAMPLE_BERNOULLI, seed, T, reference=reference, ws=ws, dA=dA, dB=dB)
            o = oracle_predict(A, B, oracle.BERNOULLI, seed, T, reference=reference)
            assert_prediction_equal(g, o, f"{name} seed {seed} ratio {ratio}")


@pytest.mark.parametrize("name", sorted(CASES))
def test_predict_small_paper_draw(name):
    A, B = CASES[name]
    B = A if B is None else B
    for seed in range(3):
        for s in (0, 7, 300):
            g = gpu_predict(A, B, sp.SAMPLE_PAPER_DRAW, seed, sample_num=s)
            o = oracle_predict(A, B, oracle.PAPER_DRAW, seed, sample_num=s)
            assert_prediction_equal(g, o, f"{name} seed {seed} draws {s}")
            r = gpu_predict(A, B, sp.SAMPLE_PAPER_DRAW, seed, sample_num=s, reference=True)
            o = oracle_predict(A, B, oracle.PAPER_DRAW, seed, sample_num=s, reference=True)
            assert_prediction_equal(r, o, f"{name} reference seed {seed} draws {s}")


@pytest.mark.parametrize("name", sorted(CASES))
def test_symbolic_exact_small(name):
    A, B = CASES[name]
    B = A if B is None else B
    nnz, offs, res = gpu_symbolic(A, B)
    onnz, ooffs, Z = oracle.symbolic_exact(A, B)
    _, F = oracle.flop_per_row(A, B)
    np.testing.assert_array_equal(nnz.astype(np.int64), onnz)
    np.testing.assert_array_equal(offs, ooffs)
    assert res["pred_total"] == Z and res["flop_total"] == F and res["status"] == 0


@pytest.mark.parametrize("name", sorted(CASES))
def test_flop_per_row_small(name):
    A, B = CASES[name]
    B = A if B is None else B
    dA = to_dev(A)
    dB = dA if B is A else to_dev(B)
    flop, res = sp.flop_per_row(dA, dB)
    of, F = oracle.flop_per_row(A, B)
    np.testing.assert_array_equal(flop.cpu().numpy().astype(np.int64), of)
    r = sp.read_result(res)
    assert r["flop_total"] == F and r["status"] == 0


def test_predict_cr_matches_oracle():
    A = W.rmat(13, 16, seed=21)
    dA = to_dev(A)
    for seed in range(5):
        T = int(0.02 * TWO32)
        r = sp.read_result(sp.predict_cr(dA, dA, sp.config(threshold=T, seed=seed)))
        o = oracle.predict(A, A, oracle.BERNOULLI, seed, T)
        assert (r["flop_s"], r["nnz_s"], r["n_sampled"]) == (o["flop_s"], o["nnz_s"], o["n_sampled"])
        assert r["status"] == o["status"]


@pytest.mark.parametrize("M", [1, 31, 4096, 100003, 1 << 20])
def test_sample_rows_known_answers(M):
    for seed in (0, 1, 12345):
        for ratio in (0.0, 0.005, 0.01, 0.5, 1.0):
            T = min(TWO32, int(ratio * TWO32))
            ids, res = sp.sample_rows(M, sp.config(threshold=T, seed=seed))
            r = sp.read_result(res)
            o = oracle.sample(M, oracle.BERNOULLI, seed, T)
            assert r["n_sampled"] == len(o)
            np.testing.assert_array_equal(ids.cpu().numpy()[: len(o)], o)
        ids, res = sp.sample_rows(M, sp.config(mode=sp.SAMPLE_PAPER_DRAW, seed=seed))
        o = oracle.sample(M, oracle.PAPER_DRAW, seed)
        np.testing.assert_array_equal(ids.cpu().numpy()[: len(o)], o)


# ---------------------------------------------------------------- edge cases
def test_empty_and_degenerate_matrices():
    empty = W.CSR(0, 7, np.zeros(1, np.int32), np.zeros(0, np.int32))
    B = W.erdos_renyi(7, 3, 1, ncols=9)
    g = gpu_predict(empty, B, sp.SAMPLE_BERNOULLI, 0, int(0.5 * TWO32))
    assert g["offsets"].tolist() == [0] and g["pred_total"] == 0
    no_nnz = W.CSR(50, 40, np.zeros(51, np.int32), np.zeros(0, np.int32))
    B = W.erdos_renyi(40, 5, 2, ncols=60)
    for ref in (False, True):
        g = gpu_predict(no_nnz, B, sp.SAMPLE_BERNOULLI, 0, int(0.5 * TWO32), reference=ref)
        o = oracle_predict(no_nnz, B, oracle.BERNOULLI, 0, int(0.5 * TWO32), reference=ref)
        assert_prediction_equal(g, o, "no nonzeros")
    one = W.erdos_renyi(1, 20, 3, ncols=30)
    B = W.erdos_renyi(30, 6, 4, ncols=30)
    for T in (0, TWO32):
        g = gpu_predict(one, B, sp.SAMPLE_BERNOULLI, 0, T)
        assert_prediction_equal(g, oracle_predict(one, B, oracle.BERNOULLI, 0, T), f"single row T={T}")


@pytest.mark.parametrize("rows", [(1 << 20) - 3, (1 << 21) + 12345, 3 << 20])
def test_tall_sparse_many_rows_per_block(rows):
    # about one nonzero per row: each block of the prediction holds from about
    # 8 thousand to over 20 thousand rows, i.e. one to six 4096-row chunks in
    # the per-block scan (scanned before or after the wait on the blocks
    # before it), with ragged ends
    A = W.erdos_renyi(rows, 1, 41 + rows % 7, ncols=1 << 15)
    B = W.erdos_renyi(1 << 15, 3, 42, ncols=5000)
    dA, dB = to_dev(A), to_dev(B)
    ws = sp.Workspace.for_operands(dA, dB)
    for ref in (False, True):
        for seed, ratio in ((5, 0.01), (6, 0.3)):
            T = int(ratio * TWO32)
            g = gpu_predict(A, B, sp.SAMPLE_BERNOULLI, seed, T, reference=ref, ws=ws, dA=dA, dB=dB)
            o = oracle_predict(A, B, oracle.BERNOULLI, seed, T, reference=ref)
            assert_prediction_equal(g, o, f"rows {rows} ref {ref} seed {seed}")


def test_empty_sample_and_full_sample():
    A = W.erdos_renyi(5000, 9, 5)
    for T in (0, TWO32):
        for ref in (False, True):
            g = gpu_predict(A, A, sp.SAMPLE_BERNOULLI, 3, T, reference=ref)
            o = oracle_predict(A, A, oracle.BERNOULLI, 3, T, reference=ref)
            assert_prediction_equal(g, o, f"T={T} ref={ref}")
    g = gpu_predict(A, A, sp.SAMPLE_BERNOULLI, 3, 0)
    assert g["status"] == sp.STATUS_WARN_EMPTY_SAMPLE
    np.testing.assert_array_equal(g["pred"], g["flop"])


def _row_with_products(K, N, per_entry, n_entries, seed):
    """B: K rows, row k has per_entry[k] distinct columns; A: one row using the
    first n_entries rows of B.  Column ids overlap across B rows, so the row has
    duplicates to remove."""
    rng = np.random.default_rng(seed)
    rr, cc = [], []
    for k in range(K):
        cols = rng.choice(N, size=per_entry[k], replace=False) if per_entry[k] else []
        rr += [k] * len(cols)
        cc += list(cols)
    B = W.from_coo(K, N, rr, cc)
    A = W.from_coo(1, K, [0] * n_entries, list(range(n_entries)))
    return A, B


@pytest.mark.parametrize("target", [31, 32, 33, 1023, 1024, 1025, 16383, 16384, 16385, 70000])
def test_path_boundaries(target):
    # one output row whose FLOP is exactly `target`, with <= 32 or > 32 entries
    for n_entries in (8, 40):
        per = [target // n_entries + (1 if k < target % n_entries else 0) for k in range(n_entries)]
        N = max(64, target // 3)
        A, B = _row_with_products(n_entries, N, per, n_entries, seed=target + n_entries)
        for T in (TWO32,):
            g = gpu_predict(A, B, sp.SAMPLE_BERNOULLI, 0, T)
            o = oracle_predict(A, B, oracle.BERNOULLI, 0, T)
            assert g["flop_total"] == target
            assert_prediction_equal(g, o, f"flop {target} entries {n_entries}")
        nnz, offs, res = gpu_symbolic(A, B)
        assert nnz[0] == oracle.row_nnz(A, B)[0]


def test_bitmap_column_ranges():
    # N larger than one shared-memory bitmap: the heavy pass splits the columns
    N = 1 << 21
    rng = np.random.default_rng(7)
    K = 64
    rr = np.repeat(np.arange(K), 3000)
    cc = rng.integers(0, N, rr.shape[0])
    B = W.from_coo(K, N, rr, cc)
    A = W.from_coo(3, K, [0] * K + [1] * 10 + [2] * 3, list(range(K)) + list(range(10)) + [5, 6, 7])
    for T in (TWO32,):
        g = gpu_predict(A, B, sp.SAMPLE_BERNOULLI, 0, T)
        assert_prediction_equal(g, oracle_predict(A, B, oracle.BERNOULLI, 0, T), "bitmap ranges")
    nnz, _, _ = gpu_symbolic(A, B)
    np.testing.assert_array_equal(nnz.astype(np.int64), oracle.row_nnz(A, B))


def test_bad_column_id_is_reported_not_faulted():
    A = W.erdos_renyi(300, 5, 9)
    col = A.col.copy()
    col[17] = A.cols  # one past the end: the kernels' range checks must catch it
    bad = W.CSR(A.rows, A.cols, A.rpt, col)
    dA = to_dev(bad)
    dB = to_dev(A)
    res = sp.read_result(sp.validate_csr(dA))
    assert res["status"] & sp.STATUS_ERR_BAD_INPUT
    p = sp.predict_structure(dA, dB, sp.config(ratio=0.5), want_flop=True)
    assert sp.read_result(p.res)["status"] & sp.STATUS_ERR_BAD_INPUT
    ok = sp.read_result(sp.validate_csr(to_dev(A)))
    assert ok["status"] == 0


def test_workspace_reuse_and_many_calls():
    A = W.erdos_renyi(20000, 10, 31)
    dA = to_dev(A)
    ws = sp.Workspace.for_operands(dA, dA)
    o = oracle_predict(A, A, oracle.BERNOULLI, 5, int(0.01 * TWO32))
    for it in range(30):
        g = gpu_predict(A, A, sp.SAMPLE_BERNOULLI, 5, int(0.01 * TWO32), ws=ws, dA=dA, dB=dA)
        assert_prediction_equal(g, o, f"iteration {it}")
        if it % 10 == 0:
            nnz, offs, res = gpu_symbolic(A, A, ws=ws)
            assert res["status"] == 0
