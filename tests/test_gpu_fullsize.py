"""Parity at the full workload sizes (n = 2^20), in the launch configuration the
benchmark times.  The oracle computes FLOP for every row and the exact nnz of
every sampled row, so the prediction is compared element by element; the exact
symbolic phase is compared on every row for the Erdos-Renyi input and on a
sample of rows (plus the heaviest rows) for R-MAT, where the full oracle count
would take minutes."""
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


@pytest.fixture(scope="module")
def er():
    return W.erdos_renyi(1 << 20, 16, 2000)


@pytest.fixture(scope="module")
def rmat():
    return W.rmat(20, 16, seed=3000)


def test_er_full_prediction(er):
    dA = to_dev(er)
    ws = sp.Workspace.for_operands(dA, dA)
    T = int(0.01 * TWO32)
    for seed in (0, 1):
        for ref in (False, True):
            g = gpu_predict(er, er, sp.SAMPLE_BERNOULLI, seed, T, reference=ref, ws=ws, dA=dA, dB=dA)
            o = oracle_predict(er, er, oracle.BERNOULLI, seed, T, reference=ref)
            assert_prediction_equal(g, o, f"ER seed {seed} ref {ref}")


def test_er_full_symbolic(er):
    dA = to_dev(er)
    p = sp.symbolic_exact(dA, dA)
    nnz, offs = p.pred.cpu().numpy(), p.offsets.cpu().numpy()
    onnz, ooffs, Z = oracle.symbolic_exact(er, er)
    np.testing.assert_array_equal(nnz.astype(np.int64), onnz)
    np.testing.assert_array_equal(offs, ooffs)
    assert sp.read_result(p.res)["pred_total"] == Z


def test_rmat_full_prediction(rmat):
    dA = to_dev(rmat)
    ws = sp.Workspace.for_operands(dA, dA)
    T = int(0.005 * TWO32)
    for seed in (0, 1):
        g = gpu_predict(rmat, rmat, sp.SAMPLE_BERNOULLI, seed, T, ws=ws, dA=dA, dB=dA)
        o = oracle_predict(rmat, rmat, oracle.BERNOULLI, seed, T)
        assert_prediction_equal(g, o, f"RMAT seed {seed}")
    g = gpu_predict(rmat, rmat, sp.SAMPLE_BERNOULLI, 0, T, reference=True, ws=ws, dA=dA, dB=dA)
    o = oracle_predict(rmat, rmat, oracle.BERNOULLI, 0, T, reference=True)
    assert_prediction_equal(g, o, "RMAT reference")
    g = gpu_predict(rmat, rmat, sp.SAMPLE_PAPER_DRAW, 4, ws=ws, dA=dA, dB=dA)
    o = oracle_predict(rmat, rmat, oracle.PAPER_DRAW, 4)
    assert_prediction_equal(g, o, "RMAT paper draws")


def test_rmat_full_symbolic_sampled_rows(rmat):
    dA = to_dev(rmat)
    p = sp.symbolic_exact(dA, dA)
    nnz, offs = p.pred.cpu().numpy().astype(np.int64), p.offsets.cpu().numpy()
    res = sp.read_result(p.res)
    flop, F = oracle.flop_per_row(rmat, rmat)
    assert res["flop_total"] == F and res["status"] == 0
    assert offs[0] == 0 and np.array_equal(np.diff(offs), nnz) and offs[-1] == res["pred_total"]
    assert np.all(nnz <= flop) and np.all((nnz == 0) == (flop == 0))
    rng = np.random.default_rng(99)
    rows = np.unique(np.concatenate([rng.integers(0, rmat.rows, 3000), np.argsort(flop)[-64:]]))
    np.testing.assert_array_equal(nnz[rows], oracle.row_nnz(rmat, rmat, rows=rows))
