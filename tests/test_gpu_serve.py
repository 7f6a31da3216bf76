"""The serving loop (paper_2207_13848_gb300.serve): every served result equals
the oracle's prediction for its request, and the result the same request gets
alone, whether it ran by itself or merged into a batched launch while others
ran; memory admission never exceeds the budget, and requests that can never
fit are rejected.  Every output is an exact integer, so "the same" means
bit-equal."""
import numpy as np
import pytest

import oracle
import paper_2207_13848_gb300 as sp
from paper_2207_13848_gb300 import serve
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def pool_host():
    """(A, B) host pairs: the five family structures at three small sizes, and
    two at n = 2^18 (launched alone: above the server's merge limit)."""
    out = []
    for s in W.STRUCTURES:
        for n, v in ((1 << 12, 3), (1 << 13, 10), (1 << 14, 17)):
            A, B, _ = W.family_case(s, n, v)
            out.append((A, B))
    for s, v in (("rmat", 8), ("er", 15)):
        A, B, _ = W.family_case(s, 1 << 18, v)
        out.append((A, B))
    return out


@pytest.fixture(scope="module")
def pool(pool_host):
    out = []
    for A, B in pool_host:
        dA = sp.DeviceCSR.from_host(A)
        dB = dA if B is A else sp.DeviceCSR.from_host(B)
        out.append((dA, dB))
    return out


def _solo(A, B, cfg):
    p = sp.predict_structure(A, B, cfg)
    torch.cuda.synchronize()
    return p.pred.cpu().numpy(), p.offsets.cpu().numpy(), sp.read_result(p.res)


def _check_same(done, pool, picks, ratio=0.01):
    T = int(ratio * sp.TWO32)
    for r in done:
        A, B = pool[picks[r.index]]
        want = _solo(A, B, sp.config(threshold=T, seed=r.index))
        np.testing.assert_array_equal(r.pred.cpu().numpy(), want[0], err_msg=f"pred, request {r.index}")
        np.testing.assert_array_equal(r.offsets.cpu().numpy(), want[1], err_msg=f"offsets, request {r.rid}")
        assert sp.read_result(r.res) == want[2], f"result record, request {r.rid}"


def _check_oracle(done, pool_host, picks, ratio=0.01):
    T = int(ratio * sp.TWO32)
    for r in done:
        A, B = pool_host[picks[r.index]]
        o = oracle.predict(A, B, oracle.BERNOULLI, r.index, T)
        np.testing.assert_array_equal(r.pred.cpu().numpy().astype(np.int64), o["pred"], err_msg=f"request {r.rid}")
        np.testing.assert_array_equal(r.offsets.cpu().numpy(), o["offsets"], err_msg=f"request {r.rid}")
        got = sp.read_result(r.res)
        for k in ("flop_total", "flop_s", "nnz_s", "n_sampled", "pred_total", "status"):
            assert got[k] == o[k], (k, r.rid, got[k], o[k])


def test_served_results_equal_the_oracle(pool, pool_host):
    # merge limit 2^16 rows: the two 2^18 entries go alone, the rest are merged
    srv = serve.Server(slots=8, memory_budget=4 << 30, batch_rows=1 << 16, max_batch=32)
    done, picks = serve.run_poisson(srv, pool, rate=0, n_requests=240, seed=5)  # all at once: maximal overlap
    assert len(done) == 240 and srv.stats.rejected == 0
    assert srv.stats.peak_inflight > 1, "requests never overlapped"
    assert srv.stats.batched_launches > 0, "no request was merged into a batched launch"
    assert any(r.batched for r in done) and any(not r.batched for r in done)
    _check_oracle(done, pool_host, picks)


def test_results_in_the_mix_equal_results_alone(pool):
    srv = serve.Server(slots=8, memory_budget=4 << 30)
    done, picks = serve.run_poisson(srv, pool, rate=0, n_requests=160, seed=6)
    assert len(done) == 160
    _check_same(done, pool, picks)


def test_without_merging_the_results_are_the_same(pool, pool_host):
    srv = serve.Server(slots=8, memory_budget=4 << 30, batch_rows=0)
    done, picks = serve.run_poisson(srv, pool, rate=0, n_requests=80, seed=8)
    assert srv.stats.batched_launches == 0 and len(done) == 80
    _check_oracle(done[::3], pool_host, picks)


def test_poisson_arrivals_and_latency_order(pool):
    srv = serve.Server(slots=4, memory_budget=4 << 30)
    done, picks = serve.run_poisson(srv, pool, rate=20000.0, n_requests=200, seed=9)
    assert len(done) == 200
    for r in done:
        assert r.arrival <= r.admitted <= r.done
    summ = serve.latency_summary(done)
    assert 0 < summ["p50"] <= summ["p99"]
    _check_same(done[::7], pool, picks)


def test_a_rejected_request_leaves_the_others_served(pool, pool_host):
    # a request whose configuration the library rejects (threshold above 2^32)
    # fails alone, merged or not; every other request is served exactly
    srv = serve.Server(slots=4, memory_budget=4 << 30)
    T = int(0.01 * sp.TWO32)
    small = [i for i, (A, _) in enumerate(pool) if A.rows <= srv.batch_rows][:6]
    reqs = []
    for k, i in enumerate(small):
        A, B = pool[i]
        cfg = sp.config(threshold=(1 << 32) + 1) if k == 2 else sp.config(threshold=T, seed=k)
        reqs.append((i, srv.submit(A, B, cfg)))
    srv.drain()
    bad = reqs[2][1]
    assert bad.error and srv.failed == [bad] and srv.stats.failed == 1
    for k, (i, r) in enumerate(reqs):
        if k == 2:
            continue
        A, B = pool_host[i]
        o = oracle.predict(A, B, oracle.BERNOULLI, k, T)
        np.testing.assert_array_equal(r.offsets.cpu().numpy(), o["offsets"], err_msg=f"request {k}")


def test_memory_admission_respects_the_budget(pool):
    big = max(pool, key=lambda ab: ab[0].rows)
    one = serve.Server(slots=8).request_bytes(*big)
    srv = serve.Server(slots=8, memory_budget=int(one * 1.5))  # room for one such request at a time
    done, picks = serve.run_poisson(srv, [big], rate=0, n_requests=12, seed=2)
    assert len(done) == 12
    assert srv.stats.peak_bytes <= srv.budget
    assert srv.stats.peak_inflight == 1
    _check_same(done, [big], picks)


def test_requests_that_can_never_fit_are_rejected(pool):
    A, B = pool[0]
    srv = serve.Server(slots=2, memory_budget=1024)
    assert srv.submit(A, B, sp.config(ratio=0.01)) is None
    assert srv.stats.rejected == 1
    srv.drain()
