"""The serving loop (paper_2207_13848_gb300.serve): requests admitted while
others run on the GPU give exactly the results they give alone, memory
admission never exceeds the budget, and requests that can never fit are
rejected.  Every output is an exact integer, so "the same" means bit-equal."""
import numpy as np
import pytest

import paper_2207_13848_gb300 as sp
from paper_2207_13848_gb300 import serve
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def pool():
    out = []
    for s in W.STRUCTURES:
        for n, v in ((1 << 12, 3), (1 << 13, 10), (1 << 14, 17)):
            A, B, _ = W.family_case(s, n, v)
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
        A, B = pool[picks[r.rid]]
        want = _solo(A, B, sp.config(threshold=T, seed=r.rid))
        np.testing.assert_array_equal(r.pred.cpu().numpy(), want[0], err_msg=f"pred, request {r.rid}")
        np.testing.assert_array_equal(r.offsets.cpu().numpy(), want[1], err_msg=f"offsets, request {r.rid}")
        assert sp.read_result(r.res) == want[2], f"result record, request {r.rid}"


def test_results_in_the_mix_equal_results_alone(pool):
    srv = serve.Server(slots=8, memory_budget=2 << 30)
    done, picks = serve.run_poisson(srv, pool, rate=0, n_requests=240, seed=5)  # all at once: maximal overlap
    assert len(done) == 240 and srv.stats.rejected == 0
    assert srv.stats.peak_inflight > 1, "requests never overlapped"
    _check_same(done, pool, picks)


def test_poisson_arrivals_and_latency_order(pool):
    srv = serve.Server(slots=4, memory_budget=2 << 30)
    done, picks = serve.run_poisson(srv, pool, rate=20000.0, n_requests=200, seed=9)
    assert len(done) == 200
    for r in done:
        assert r.arrival <= r.admitted <= r.done
    summ = serve.latency_summary(done)
    assert 0 < summ["p50"] <= summ["p99"]
    _check_same(done[::7], pool, picks)


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
