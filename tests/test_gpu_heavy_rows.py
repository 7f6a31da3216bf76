"""Sampled rows with very many products go through the heavy-row path: hub
rows of 400-500 thousand products are counted by a whole thread block with a
column bitmap (over several column passes when B is wider than one bitmap);
rows of more than 2^20 products are split by their entries into parts that
several blocks count at once (more such rows than split slots: the rest are
counted whole).  FLOP, f*, z*, |S|, the predictions and the offsets must equal
the oracle's, with several hub rows at once, for the reference design, and call
after call on one workspace."""
import numpy as np
import pytest

import oracle
import paper_2207_13848_gb300 as sp
import workloads as W
from tests.gpu_helpers import TWO32, assert_prediction_equal, gpu_predict, oracle_predict, wide_hubs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _hubs(n, hubs, hub_len, row_len, seed):
    """n x n pattern: rows 0..hubs-1 have hub_len entries (columns spread over
    [0, n)), the other rows row_len entries; C = A*A then has hub rows of about
    hub_len * row_len products."""
    rng = np.random.default_rng(seed)
    r, c = [], []
    for i in range(n):
        k = hub_len if i < hubs else row_len
        cols = rng.choice(n, size=min(k, n), replace=False)
        r.append(np.full(cols.shape[0], i))
        c.append(cols)
    return W.from_coo(n, n, np.concatenate(r), np.concatenate(c))


def _wide(M, K, N, hub_len, row_len, seed):
    """A (M x K) with one hub row over hub_len columns; B (K x N) with row_len
    entries per row spread over all N columns."""
    rng = np.random.default_rng(seed)
    ra = np.concatenate([np.zeros(hub_len, np.int64), np.repeat(np.arange(1, M), 3)])
    ca = np.concatenate([rng.choice(K, size=hub_len, replace=False), rng.integers(0, K, size=3 * (M - 1))])
    A = W.from_coo(M, K, ra, ca)
    rb = np.repeat(np.arange(K), row_len)
    cb = rng.integers(0, N, size=K * row_len)
    return A, W.from_coo(K, N, rb, cb)


@pytest.mark.parametrize("hubs", [2, 12])
def test_hub_rows_match_the_oracle(hubs):
    A = _hubs(6000, hubs, 2500, 180, seed=hubs)   # hub rows ~450k products (> 2^18)
    for seed, T in ((0, TWO32), (1, int(0.5 * TWO32))):
        g = gpu_predict(A, A, sp.SAMPLE_BERNOULLI, seed, T)
        o = oracle_predict(A, A, oracle.BERNOULLI, seed, T)
        assert_prediction_equal(g, o, f"hubs {hubs} seed {seed}")


def test_hub_rows_with_several_column_passes():
    A, B = _wide(300, 3000, (1 << 21) + 37, 2000, 250, seed=7)  # hub row ~500k products over 2^21+ columns
    g = gpu_predict(A, B, sp.SAMPLE_BERNOULLI, 3, TWO32)
    o = oracle_predict(A, B, oracle.BERNOULLI, 3, TWO32)
    assert_prediction_equal(g, o, "wide B")


def test_hub_rows_reference_design():
    A = _hubs(5000, 5, 2200, 200, seed=21)
    g = gpu_predict(A, A, sp.SAMPLE_BERNOULLI, 4, TWO32, reference=True)
    o = oracle_predict(A, A, oracle.BERNOULLI, 4, TWO32, reference=True)
    assert_prediction_equal(g, o, "reference design")


def test_hub_rows_repeated_calls_reuse_the_workspace():
    A = _hubs(4000, 9, 2000, 160, seed=5)
    dA = sp.DeviceCSR.from_host(A)
    ws = sp.Workspace.for_operands(dA, dA)
    o = oracle_predict(A, A, oracle.BERNOULLI, 2, TWO32)
    for _ in range(3):
        g = gpu_predict(A, A, sp.SAMPLE_BERNOULLI, 2, TWO32, ws=ws, dA=dA, dB=dA)
        assert_prediction_equal(g, o, "repeat")


@pytest.mark.parametrize("n_hubs", [3, 12])
def test_split_rows_match_the_oracle(n_hubs):
    # hub rows of about 2500 * 600 = 1.5 M products (> 2^20): split; with 12 of
    # them the 8 split slots run out and some are counted whole
    A, B = wide_hubs(300, 3000, 1 << 20, n_hubs, 2500, 600, seed=31 + n_hubs)
    for seed, T in ((0, TWO32), (1, int(0.5 * TWO32))):
        g = gpu_predict(A, B, sp.SAMPLE_BERNOULLI, seed, T)
        o = oracle_predict(A, B, oracle.BERNOULLI, seed, T)
        assert_prediction_equal(g, o, f"split hubs {n_hubs} seed {seed}")


def test_split_rows_with_several_column_passes_and_reference_design():
    A, B = wide_hubs(200, 2800, (1 << 21) + 37, 2, 2600, 500, seed=41)  # 1.3 M products, 3 column passes
    for ref in (False, True):
        g = gpu_predict(A, B, sp.SAMPLE_BERNOULLI, 5, TWO32, reference=ref)
        o = oracle_predict(A, B, oracle.BERNOULLI, 5, TWO32, reference=ref)
        assert_prediction_equal(g, o, f"split, wide B, reference {ref}")


def test_split_rows_repeated_calls_reuse_the_workspace():
    A, B = wide_hubs(300, 3000, 1 << 20, 5, 2400, 550, seed=51)
    dA, dB = sp.DeviceCSR.from_host(A), sp.DeviceCSR.from_host(B)
    ws = sp.Workspace.for_operands(dA, dB)
    o = oracle_predict(A, B, oracle.BERNOULLI, 6, TWO32)
    for _ in range(3):
        g = gpu_predict(A, B, sp.SAMPLE_BERNOULLI, 6, TWO32, ws=ws, dA=dA, dB=dB)
        assert_prediction_equal(g, o, "split, repeat")
