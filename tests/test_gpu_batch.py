"""Parity of the batched predictor (spgemm_predict_batch) with the oracle and
with one spgemm_predict_structure call per case: every case's FLOP per row,
predictions, offsets and result record are the same integers, whatever the
batch's composition, the tuning, repeated runs or graph replay."""
import ctypes

import numpy as np
import pytest

import paper_2207_13848_gb300 as sp
import workloads as W
from tests.gpu_helpers import TWO32, assert_prediction_equal, oracle_predict, wide_hubs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _case(A, B, mode=sp.SAMPLE_BERNOULLI, ratio=0.01, seed=0, sample_num=0, threshold=None):
    T = int(ratio * TWO32) if threshold is None else threshold
    return dict(A=A, B=B, mode=mode, threshold=T, seed=seed, sample_num=sample_num)


def _device_cases(cases):
    out = []
    for c in cases:
        dA = sp.DeviceCSR.from_host(c["A"])
        dB = dA if c["B"] is c["A"] else sp.DeviceCSR.from_host(c["B"])
        cfg = sp.config(mode=c["mode"], threshold=c["threshold"], sample_num=c["sample_num"], seed=c["seed"])
        out.append((dA, dB, cfg))
    return out


def _batch_outputs(batch):
    torch.cuda.synchronize()
    res = batch.results()
    outs = []
    for i in range(batch.n):
        pred, offs, flop = batch.outputs[i]
        outs.append(dict(pred=pred.cpu().numpy(), offsets=offs.cpu().numpy(), flop=flop.cpu().numpy(), **res[i]))
    return outs


def _family(sizes, variants, structures=W.STRUCTURES):
    cases = []
    for s in structures:
        for n in sizes:
            for v in variants:
                A, B, name = W.family_case(s, n, v)
                cases.append(dict(_case(A, B, seed=v), name=name))
    return cases


@pytest.fixture(scope="module")
def small_family():
    cases = _family([1 << 12], [0, 1, 6, 13, 24]) + _family([1 << 14], [3, 20], ("er", "rmat", "st27"))
    return cases


def test_batch_matches_oracle_on_family_cases(small_family):
    dev = _device_cases(small_family)
    batch = sp.Batch(dev, want_flop=True)
    batch.run()
    got = _batch_outputs(batch)
    for c, g in zip(small_family, got):
        o = oracle_predict(c["A"], c["B"], c["mode"], c["seed"], c["threshold"], c["sample_num"])
        assert_prediction_equal(g, o, c["name"])


def test_batch_matches_single_case_calls(small_family):
    dev = _device_cases(small_family)
    batch = sp.Batch(dev, want_flop=True)
    batch.run()
    got = _batch_outputs(batch)
    for (dA, dB, cfg), g, c in zip(dev, got, small_family):
        p = sp.predict_structure(dA, dB, cfg, want_flop=True)
        torch.cuda.synchronize()
        one = dict(pred=p.pred.cpu().numpy(), offsets=p.offsets.cpu().numpy(), flop=p.flop.cpu().numpy(),
                   **sp.read_result(p.res))
        for k in ("pred", "offsets", "flop"):
            np.testing.assert_array_equal(g[k], one[k], err_msg=f"{k} {c['name']}")
        for k in ("flop_total", "flop_s", "nnz_s", "n_sampled", "pred_total", "status"):
            assert g[k] == one[k], (k, c["name"])


def _edge_cases():
    er = W.erdos_renyi(5000, 9, 5)
    rm = W.rmat(13, 16, seed=21)  # hub rows: block hash and bitmap paths
    empty = W.CSR(0, 7, np.zeros(1, np.int32), np.zeros(0, np.int32))
    b7 = W.erdos_renyi(7, 3, 1, ncols=9)
    wide = W.erdos_renyi(300, 5, 9)
    return [
        dict(_case(er, er, seed=1), name="er"),
        dict(_case(rm, rm, ratio=0.05, seed=2), name="rmat-hubs"),
        dict(_case(empty, b7, seed=3), name="empty-A"),
        dict(_case(er, er, threshold=0, seed=4), name="empty-sample"),
        dict(_case(wide, wide, mode=sp.SAMPLE_PAPER_DRAW, seed=5), name="paper-draw-default"),
        dict(_case(er, er, mode=sp.SAMPLE_PAPER_DRAW, sample_num=777, seed=6), name="paper-draw-777"),
        dict(_case(rm, rm, threshold=TWO32, seed=7), name="all-rows"),
        dict(_case(W.laplacian_2d(64), W.laplacian_2d(64), seed=8), name="lap2d-64"),
    ]


@pytest.mark.parametrize("launches", [1, 4])
def test_batch_edge_cases_match_oracle(launches):
    # empty A, an empty sample, the paper's draws, ... in both forms (the
    # single launch's grid barriers also pass with no work in a phase)
    cases = _edge_cases()
    batch = sp.Batch(_device_cases(cases), want_flop=True, tuning_=sp.tuning(launches=launches))
    batch.run()
    for c, g in zip(cases, _batch_outputs(batch)):
        o = oracle_predict(c["A"], c["B"], c["mode"], c["seed"], c["threshold"], c["sample_num"])
        assert_prediction_equal(g, o, c["name"])



@pytest.mark.parametrize("launches", [1, 4])
def test_batch_with_phases_that_have_no_work(launches):
    # a batch of one 0 x 0 A (no rows, no B rows: no table, sample or heavy
    # work, one FLOP tile that writes offsets[0]), and the same with a case
    # whose sample is empty: every phase that has nothing to do must still
    # pass its barrier and leave exact results
    none = W.CSR(0, 0, np.zeros(1, np.int32), np.zeros(0, np.int32))
    b5 = W.CSR(0, 5, np.zeros(1, np.int32), np.zeros(0, np.int32))
    er = W.erdos_renyi(100, 2, 3)
    for cases in ([dict(_case(none, b5, seed=1), name="0x0")],
                  [dict(_case(none, b5, seed=1), name="0x0"), dict(_case(er, er, threshold=0, seed=2), name="no-sample")]):
        batch = sp.Batch(_device_cases(cases), want_flop=True, tuning_=sp.tuning(launches=launches))
        for _ in range(2):  # twice: the first run leaves the workspace clean for the next
            batch.run()
            for c, g in zip(cases, _batch_outputs(batch)):
                o = oracle_predict(c["A"], c["B"], c["mode"], c["seed"], c["threshold"], c["sample_num"])
                assert_prediction_equal(g, o, c["name"])

def test_batch_split_rows_match_oracle():
    # sampled hub rows of 1.3-1.5 M products (a whole block each, over B's
    # columns in a shared-memory bitmap): 12 + 4 + 2 of them, one case with B
    # wider than one bitmap pass, one with few columns (many duplicate
    # products), among ordinary cases; run after run on one workspace
    cases = [
        dict(_case(W.erdos_renyi(4096, 8, 71), None, ratio=0.05, seed=1), name="er 4096"),
        dict(_case(*wide_hubs(300, 3000, 1 << 20, 12, 2500, 600, seed=61), threshold=TWO32, seed=2),
             name="12 hubs, N 2^20"),
        dict(_case(W.rmat(13, 16, seed=72), None, seed=3), name="rmat 2^13"),
        dict(_case(*wide_hubs(300, 3000, 5000, 4, 2500, 600, seed=62), threshold=TWO32, seed=4),
             name="4 hubs, N 5000"),
        dict(_case(*wide_hubs(200, 2800, (1 << 21) + 37, 2, 2600, 500, seed=63), threshold=TWO32, seed=5),
             name="2 hubs, N 2^21 + 37"),
    ]
    for c in cases:
        if c["B"] is None:
            c["B"] = c["A"]
    batch = sp.Batch(_device_cases(cases), want_flop=True)
    want = [oracle_predict(c["A"], c["B"], c["mode"], c["seed"], c["threshold"], c["sample_num"]) for c in cases]
    for rep in range(3):
        batch.run()
        for c, g, o in zip(cases, _batch_outputs(batch), want):
            assert_prediction_equal(g, o, f"{c['name']} run {rep}")


TUNINGS = [
    dict(),  # four launches
    dict(launches=1),
    dict(tile_items=4096, sample_chunk=4096),
    dict(tile_items=4096, sample_chunk=4096, launches=4),
    dict(warp_table=512, heavy_threshold=32, tile_items=65536),
    dict(warp_table=512, heavy_threshold=32, tile_items=65536, launches=4),
    dict(warp_table=2048, heavy_threshold=1024, sample_chunk=131072, tile_items=8192),
    dict(warp_table=2048, heavy_threshold=1024, sample_chunk=131072, tile_items=8192, launches=4),
    dict(warp_table=1024, heavy_threshold=64, flop_blocks_per_sm=1, launches=4),
]


def test_tuning_never_changes_results():
    cases = _edge_cases() + _family([1 << 12], [2, 9], ("rmat", "blockdiag"))
    batch = sp.Batch(_device_cases(cases), want_flop=True)
    ref = None
    for tu in TUNINGS:
        batch.prepare(sp.tuning(**tu))
        batch.run()
        got = _batch_outputs(batch)
        if ref is None:
            ref = got
            continue
        for i, (a, b) in enumerate(zip(ref, got)):
            for k in ("pred", "offsets", "flop"):
                np.testing.assert_array_equal(a[k], b[k], err_msg=f"{k} case {i} tuning {tu}")
            for k in ("flop_total", "flop_s", "nnz_s", "n_sampled", "pred_total", "status"):
                assert a[k] == b[k], (k, i, tu)


@pytest.mark.parametrize("launches", [1, 4])
def test_repeated_runs_and_graph_replay(launches):
    cases = _edge_cases()
    batch = sp.Batch(_device_cases(cases), want_flop=True, tuning_=sp.tuning(launches=launches))
    assert batch.plan.tuning.launches == launches
    batch.run()
    first = _batch_outputs(batch)
    for _ in range(3):
        for p in batch.outputs:
            p[0].fill_(-1)
            p[1].fill_(-1)
        batch.res.zero_()
        batch.run()
    again = _batch_outputs(batch)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        batch.run(stream=s)  # warm-up on the capture stream
        s.synchronize()
        with torch.cuda.graph(g, stream=s):
            batch.run(stream=s)
    for p in batch.outputs:
        p[0].fill_(-1)
        p[1].fill_(-1)
    batch.res.zero_()
    for _ in range(3):
        g.replay()
    replay = _batch_outputs(batch)
    for run in (again, replay):
        for a, b in zip(first, run):
            for k in ("pred", "offsets", "flop"):
                np.testing.assert_array_equal(a[k], b[k])
            assert {k: a[k] for k in a if k not in ("pred", "offsets", "flop")} == \
                   {k: b[k] for k in b if k not in ("pred", "offsets", "flop")}


def test_new_batch_on_the_same_workspace():
    big = _family([1 << 12], [0, 5, 11], ("er", "rmat", "lap2d"))
    small = _edge_cases()[:3]
    b1 = sp.Batch(_device_cases(big), want_flop=True)
    b1.run()
    # re-plan another batch into the first one's workspace
    b2 = sp.Batch(_device_cases(small), want_flop=True)
    b2.ws = b1.ws
    b2.prepare()
    b2.run()
    for c, g in zip(small, _batch_outputs(b2)):
        o = oracle_predict(c["A"], c["B"], c["mode"], c["seed"], c["threshold"], c["sample_num"])
        assert_prediction_equal(g, o, c["name"])


def test_bad_column_id_is_reported_for_its_case_only():
    good = W.erdos_renyi(3000, 8, 31)
    bad = W.erdos_renyi(3000, 8, 32)
    col = bad.col.copy()
    col[len(col) // 2] = bad.cols + 5  # out of range: counted as zero, flagged
    bad = W.CSR(bad.rows, bad.cols, bad.rpt.copy(), col)
    cases = [dict(_case(good, good, seed=1), name="good"), dict(_case(bad, good, threshold=TWO32, seed=2), name="bad"),
             dict(_case(good, good, seed=3), name="good2")]
    batch = sp.Batch(_device_cases(cases), want_flop=True)
    batch.run()
    res = batch.results()
    assert res[0]["status"] == 0 and res[2]["status"] == 0
    assert res[1]["status"] & sp.STATUS_ERR_BAD_INPUT


def test_autotune_picks_a_valid_tuning_with_identical_results(small_family):
    cases = small_family[:12]
    batch = sp.Batch(_device_cases(cases), want_flop=True)
    batch.run()
    ref = _batch_outputs(batch)
    best, ms = batch.autotune(reps=2)
    assert ms > 0
    t = best.as_dict()
    assert t["warp_table"] in (512, 1024, 2048) and 32 <= t["heavy_threshold"] <= t["warp_table"] // 2
    assert 4096 <= t["tile_items"] and t["sample_chunk"] % 256 == 0 and t["flop_blocks_per_sm"] >= 1
    assert t["launches"] in (1, 4)
    assert batch.plan.tuning.as_dict() == t
    for p in batch.outputs:
        p[0].fill_(-1)
    batch.run()
    for a, b in zip(ref, _batch_outputs(batch)):
        for k in ("pred", "offsets", "flop"):
            np.testing.assert_array_equal(a[k], b[k])


def test_batch_with_full_size_cases_matches_oracle():
    # cases of the family at n = 2^20 (R-MAT with its hub rows, ER, a
    # rectangular block-diagonal product) among small ones, as in the 625-case
    # batch: every case bit-exact against the oracle
    cases = []
    for st, n, v in (("rmat", 1 << 20, 12), ("er", 1 << 20, 9), ("blockdiag", 1 << 20, 7), ("lap2d", 1 << 12, 3),
                     ("st27", 1 << 14, 20)):
        A, B, name = W.family_case(st, n, v)
        cases.append(dict(_case(A, B, seed=v), name=name))
    batch = sp.Batch(_device_cases(cases), want_flop=True)
    batch.run()
    for c, g in zip(cases, _batch_outputs(batch)):
        o = oracle_predict(c["A"], c["B"], c["mode"], c["seed"], c["threshold"], c["sample_num"])
        assert_prediction_equal(g, o, c["name"])


def test_one_launch_and_four_launches_agree_on_full_size_cases():
    # the single persistent launch (grid barriers between the phases) and the
    # four launches give the same integers on large, uneven cases
    cases = []
    for st, n, v in (("rmat", 1 << 18, 20), ("er", 1 << 18, 3), ("st27", 1 << 16, 9), ("lap2d", 1 << 12, 1)):
        A, B, name = W.family_case(st, n, v)
        cases.append(dict(_case(A, B, seed=v), name=name))
    dev = _device_cases(cases)
    outs = []
    for launches in (1, 4):
        batch = sp.Batch(dev, want_flop=True, tuning_=sp.tuning(launches=launches))
        batch.run()
        outs.append(_batch_outputs(batch))
    for c, a, b in zip(cases, *outs):
        for k in ("pred", "offsets", "flop"):
            np.testing.assert_array_equal(a[k], b[k], err_msg=f"{k} {c['name']}")
        assert {k: a[k] for k in a if k not in ("pred", "offsets", "flop")} == \
               {k: b[k] for k in b if k not in ("pred", "offsets", "flop")}, c["name"]


@pytest.mark.parametrize("launches", [1, 4])
def test_batch_of_more_cases_than_the_case_cache(launches):
    # above 1024 cases the heavy pass finds a queued row's case by a search in
    # global memory instead of the shared-memory copy of the cases' first rows:
    # 1100 small cases, with hub rows (queued as heavy) in cases on both sides
    # of case 1024, each compared with the oracle
    rng = np.random.default_rng(1100)
    hosts = []
    for i in range(1100):
        if i % 97 == 5 or i in (1023, 1024, 1099):
            # hub rows of ~2400 products; every row sampled, so both are queued
            A, B = wide_hubs(300, 200, 900, 2, 60, 40, seed=i)
            hosts.append(_case(A, B, seed=i, threshold=TWO32))
        else:
            A = W.erdos_renyi(int(rng.integers(1, 120)), 4, 5000 + i)
            hosts.append(_case(A, A, ratio=0.5, seed=i))
    dev = _device_cases(hosts)
    batch = sp.Batch(dev, want_flop=True, tuning_=sp.tuning(launches=launches))
    batch.run()
    got = _batch_outputs(batch)
    hub_cases = [i for i in range(1100) if i % 97 == 5 or i in (1023, 1024, 1099)]
    for i in range(1100):
        c = hosts[i]
        if i not in hub_cases and i % 37:
            continue  # every hub case, and a sample of the others
        o = oracle_predict(c["A"], c["B"], c["mode"], c["seed"], c["threshold"])
        assert_prediction_equal(got[i], o, f"case {i}")
