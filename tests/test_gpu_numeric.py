"""The consumer of the prediction: the numeric product C = A*B computed into the
allocation the predicted offsets give, with the overflow fallback, against the
oracle's double-precision product.

The structure must match exactly (offsets, and the set of columns of every
row; the kernels leave the column order within a row free).  Values are single
precision summed in no fixed order: each must lie within (terms + 1) * 2^-24 *
sum |a_ik * b_kc| of the oracle's exact-product double sum, the bound of any
order of single-precision summation of single-precision-rounded products."""
import numpy as np
import pytest

import oracle
import paper_2207_13848_gb300 as sp
import workloads as W
from tests.gpu_helpers import TWO32, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

EPS32 = 2.0 ** -24


def _values(m, seed):
    return np.random.default_rng(seed).uniform(-1.0, 1.0, m.nnz).astype(np.float32)


def _hub_pair(seed):
    """A with a few rows of 100-300 entries over B rows of 150-250 columns in a
    60000-wide B: rows of 15k-75k products (dense passes of the block path)."""
    rng = np.random.default_rng(seed)
    K, N = 400, 60000
    rr, cc = [], []
    for k in range(K):
        cols = rng.choice(N, size=int(rng.integers(150, 250)), replace=False)
        rr += [k] * len(cols)
        cc += cols.tolist()
    B = W.from_coo(K, N, rr, cc)
    ra, ca = [], []
    for i in range(40):
        n = int(rng.integers(100, 300)) if i % 8 == 0 else int(rng.integers(0, 20))
        ks = rng.choice(K, size=n, replace=False)
        ra += [i] * n
        ca += ks.tolist()
    A = W.from_coo(40, K, ra, ca)
    return A, B


def _entry_counts(seed):
    """Rows of 0 to 170 entries (31, 32, 33, 63, 64, 65 among them) over B rows
    of 1-3 columns: every row has at most 510 products, so every row takes the
    warp path, which keeps a row's first 32 entries from its FLOP loop and
    reads the later ones again."""
    rng = np.random.default_rng(seed)
    K, N = 3000, 5000
    rb, cb = [], []
    for k in range(K):
        n = int(rng.integers(1, 4))
        rb += [k] * n
        cb += rng.choice(N, size=n, replace=False).tolist()
    B = W.from_coo(K, N, rb, cb)
    counts = [0, 1, 31, 32, 33, 63, 64, 65, 96, 100, 150, 170] * 20
    ra, ca = [], []
    for i, e in enumerate(counts):
        ra += [i] * e
        ca += rng.choice(K, size=e, replace=False).tolist()
    return W.from_coo(len(counts), K, ra, ca), B


def _cases():
    er = W.erdos_renyi(1 << 14, 16, 11)
    return {
        "lap2d-64": (W.laplacian_2d(64), None),
        "er-16k": (er, None),
        "er-ragged-12345": (W.erdos_renyi(12345, 7, 12), None),
        "rmat-14": (W.rmat(14, 16, seed=13), None),
        "rmat-12": (W.rmat(12, 16, seed=19), None),
        "dense-blocks-64": (W.dense_blocks(4096, 64), None),
        "blockdiag-4096": (W.block_diagonal(4096, 32, 0.3, 14), None),
        "rect-er": (W.keep_left_columns(W.erdos_renyi(8192, 12, 15), 4096),
                    W.keep_top_rows(W.erdos_renyi(8192, 12, 16), 4096)),
        "hubs": _hub_pair(17),
        "entry-counts": _entry_counts(18),
    }


CASES = _cases()


def _check_against_oracle(A, B, av, bv, rpt, col, val, what):
    o_rpt, o_col, o_val, o_abs, o_terms = oracle.numeric(A, av, B, bv)
    rpt = rpt.cpu().numpy()
    col = col.cpu().numpy()
    val = val.cpu().numpy().astype(np.float64)
    assert np.array_equal(rpt, o_rpt), f"offsets {what}"
    M = A.rows
    # per row: sort the GPU entries by column, then compare entry by entry
    rows = np.repeat(np.arange(M), np.diff(rpt))
    order = np.lexsort((col, rows))
    col, val = col[order], val[order]
    assert np.array_equal(col, o_col), f"columns {what}"
    bound = (o_terms + 1) * EPS32 * o_abs
    err = np.abs(val - o_val)
    bad = np.nonzero(err > bound)[0]
    assert bad.size == 0, f"values {what}: {bad.size} outside the bound, first at {bad[:3]}: " \
                          f"gpu {val[bad[:3]]} oracle {o_val[bad[:3]]} bound {bound[bad[:3]]}"
    return o_rpt


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("pool", [False, True])
def test_numeric_product_matches_oracle(name, pool):
    A, B = CASES[name]
    B = A if B is None else B
    av = _values(A, 1)
    bv = av if B is A else _values(B, 2)
    dA = to_dev(A)
    dB = dA if B is A else to_dev(B)
    dav = torch.from_numpy(av).cuda()
    dbv = dav if B is A else torch.from_numpy(bv).cuda()
    ws = sp.Workspace.for_operands(dA, dB)
    for seed, ratio in ((0, 0.01), (1, 0.1)):
        cfg = sp.config(threshold=int(ratio * TWO32), seed=seed)
        p = sp.numeric_product(dA, dav, dB, dbv, cfg, ws=ws, pool=pool)
        o_rpt = _check_against_oracle(A, B, av, bv, p.rpt, p.col, p.val, f"{name} seed {seed} pool {pool}")
        info = p.info["numeric"]
        assert info["status"] == 0
        assert info["nnz_total"] == o_rpt[-1]
        pred = sp.predict_structure(dA, dB, cfg, ws=ws)
        exact = np.diff(o_rpt)
        assert info["alloc_total"] == int(pred.offsets[-1].item())
        if not pool:  # overflow rows: exact nnz above the predicted share
            share = np.diff(pred.offsets.cpu().numpy())
            assert info["overflow_rows"] == int(np.sum(exact > share))
            assert info["overflow_nnz"] == int(exact[exact > share].sum())
        elif o_rpt[-1] <= info["alloc_total"]:  # a pool of at least NNZ(C) may still be cut by its stripes
            assert info["overflow_nnz"] <= o_rpt[-1]


def _into(dA, dav, dB, dbv, alloc, ws, cap=None):
    """Numeric pass into per-row shares (alloc) or, with alloc None, a pool of cap entries."""
    cap = int(alloc[-1].item()) if cap is None else cap
    c_col = torch.full((max(cap, 1),), -7, dtype=torch.int32, device="cuda")[:cap]
    c_val = torch.zeros(max(cap, 1), dtype=torch.float32, device="cuda")[:cap]
    row_start = torch.empty(dA.rows, dtype=torch.int64, device="cuda")
    nnz_row = torch.empty(dA.rows, dtype=torch.int32, device="cuda")
    res = sp.new_numeric_result()
    assert sp.spgemm_numeric_into(dA, dav, dB, dbv, alloc, c_col, c_val, row_start, nnz_row, res, ws) == sp.OK
    return c_col, c_val, row_start, nnz_row, res


def _compact(dA, dav, dB, dbv, c_col, c_val, row_start, nnz_row, res, ws, Z):
    out_rpt = torch.empty(dA.rows + 1, dtype=torch.int64, device="cuda")
    out_col = torch.empty(max(Z, 1), dtype=torch.int32, device="cuda")[:Z]
    out_val = torch.empty(max(Z, 1), dtype=torch.float32, device="cuda")[:Z]
    assert sp.spgemm_numeric_compact(dA, dav, dB, dbv, c_col, c_val, row_start, nnz_row, out_rpt, out_col, out_val,
                                     res, ws) == sp.OK
    return out_rpt, out_col, out_val


@pytest.mark.parametrize("name", ["er-16k", "rmat-12", "dense-blocks-64", "hubs"])
@pytest.mark.parametrize("shrink", ["exact", "half", "minus-one", "zero", "flop"])
def test_overflow_fallback(name, shrink):
    """Allocations from exact (no overflow) to none at all (every row overflows):
    the compaction always yields the exact product."""
    A, B = CASES[name]
    B = A if B is None else B
    av = _values(A, 3)
    bv = av if B is A else _values(B, 4)
    dA = to_dev(A)
    dB = dA if B is A else to_dev(B)
    dav = torch.from_numpy(av).cuda()
    dbv = dav if B is A else torch.from_numpy(bv).cuda()
    ws = sp.Workspace.for_operands(dA, dB)
    exact = oracle.symbolic_exact(A, B)[0]
    share = {"exact": exact, "half": exact // 2, "minus-one": np.maximum(exact - 1, 0),
             "zero": np.zeros_like(exact), "flop": oracle.flop_per_row(A, B)[0]}[shrink]
    alloc_h = np.zeros(A.rows + 1, dtype=np.int64)
    np.cumsum(share, out=alloc_h[1:])
    alloc = torch.from_numpy(alloc_h).cuda()
    c_col, c_val, row_start, nnz_row, res = _into(dA, dav, dB, dbv, alloc, ws)
    info = sp.read_numeric_result(res)
    assert np.array_equal(nnz_row.cpu().numpy(), exact)
    assert info["nnz_total"] == int(exact.sum()) and info["status"] == 0
    over = exact > share
    assert info["overflow_rows"] == int(over.sum()) and info["overflow_nnz"] == int(exact[over].sum())
    rs = row_start.cpu().numpy()
    assert np.array_equal(rs < 0, over) and np.array_equal(rs[~over], alloc_h[:-1][~over])
    if shrink in ("exact", "flop"):
        assert info["overflow_rows"] == 0
    if shrink == "exact":  # the layout is the exact CSR already
        _check_against_oracle(A, B, av, bv, alloc, c_col, c_val, f"{name} padded")
    out = _compact(dA, dav, dB, dbv, c_col, c_val, row_start, nnz_row, res, ws, int(exact.sum()))
    _check_against_oracle(A, B, av, bv, *out, f"{name} {shrink}")
    assert sp.read_numeric_result(res)["status"] == 0


@pytest.mark.parametrize("name", ["er-16k", "rmat-12", "dense-blocks-64", "hubs"])
@pytest.mark.parametrize("fill", [0.0, 0.3, 0.9, 1.0, 1.5])
def test_pool_mode(name, fill):
    """One pool of fill * NNZ(C) entries: rows take exactly their size while a
    stripe has room; the rows written are disjoint, inside the pool, and hold
    their exact entries; the others overflow; the compaction gives the exact
    product every time."""
    A, B = CASES[name]
    B = A if B is None else B
    av = _values(A, 11)
    bv = av if B is A else _values(B, 12)
    dA = to_dev(A)
    dB = dA if B is A else to_dev(B)
    dav = torch.from_numpy(av).cuda()
    dbv = dav if B is A else torch.from_numpy(bv).cuda()
    ws = sp.Workspace.for_operands(dA, dB)
    exact = oracle.symbolic_exact(A, B)[0]
    Z = int(exact.sum())
    cap = int(fill * Z)
    c_col, c_val, row_start, nnz_row, res = _into(dA, dav, dB, dbv, None, ws, cap=cap)
    info = sp.read_numeric_result(res)
    assert info["status"] == 0 and info["nnz_total"] == Z and info["alloc_total"] == cap
    assert np.array_equal(nnz_row.cpu().numpy(), exact)
    rs = row_start.cpu().numpy()
    written = (rs >= 0) & (exact > 0)
    assert info["overflow_rows"] == int(np.sum(rs < 0))
    assert info["overflow_nnz"] == int(exact[rs < 0].sum())
    assert np.all(rs[written] + exact[written] <= cap)
    order = np.argsort(rs[written])
    ends = (rs[written] + exact[written])[order]
    assert np.all(ends[:-1] <= rs[written][order][1:])  # disjoint
    if fill == 0.0:
        assert np.all(rs[exact > 0] < 0)
    # the written rows hold their exact entries
    o_rpt, o_col, o_val, o_abs, o_terms = oracle.numeric(A, av, B, bv)
    cc = c_col.cpu().numpy()
    vv = c_val.cpu().numpy().astype(np.float64)
    for i in np.nonzero(written)[0][:200]:
        got = np.sort(cc[rs[i]:rs[i] + exact[i]])
        assert np.array_equal(got, o_col[o_rpt[i]:o_rpt[i + 1]]), f"row {i}"
    out = _compact(dA, dav, dB, dbv, c_col, c_val, row_start, nnz_row, res, ws, Z)
    _check_against_oracle(A, B, av, bv, *out, f"{name} pool {fill}")
    assert sp.read_numeric_result(res)["status"] == 0


def test_short_arrays_make_rows_overflow_not_writes():
    """c_capacity below alloc[M]: rows past the arrays count as overflows (nothing
    is written out of bounds) and the compaction still gives the exact product."""
    A, _ = CASES["er-16k"]
    av = _values(A, 5)
    dA = to_dev(A)
    dav = torch.from_numpy(av).cuda()
    ws = sp.Workspace.for_operands(dA, dA)
    exact = oracle.symbolic_exact(A, A)[0]
    alloc_h = np.zeros(A.rows + 1, dtype=np.int64)
    np.cumsum(exact, out=alloc_h[1:])
    alloc = torch.from_numpy(alloc_h).cuda()
    cap = int(alloc_h[-1] // 3)
    guard = 4096
    big_col = torch.full((cap + guard,), -7, dtype=torch.int32, device="cuda")
    big_val = torch.full((cap + guard,), 123.0, dtype=torch.float32, device="cuda")
    row_start = torch.empty(A.rows, dtype=torch.int64, device="cuda")
    nnz_row = torch.empty(A.rows, dtype=torch.int32, device="cuda")
    res = sp.new_numeric_result()
    assert sp.spgemm_numeric_into(dA, dav, dA, dav, alloc, big_col[:cap], big_val[:cap], row_start, nnz_row, res,
                                  ws) == sp.OK
    info = sp.read_numeric_result(res)
    fits = alloc_h[1:] <= cap
    assert info["overflow_rows"] == int((~fits & (exact > 0)).sum())
    assert np.all(big_col[cap:].cpu().numpy() == -7) and np.all(big_val[cap:].cpu().numpy() == 123.0)
    out = _compact(dA, dav, dA, dav, big_col[:cap], big_val[:cap], row_start, nnz_row, res, ws, int(exact.sum()))
    _check_against_oracle(A, A, av, av, *out, "short arrays")


def test_empty_and_degenerate():
    ws_dev = "cuda"
    # no rows
    empty = W.CSR(0, 7, np.zeros(1, np.int32), np.zeros(0, np.int32))
    B = W.erdos_renyi(7, 3, 1, ncols=9)
    dE, dB = to_dev(empty), to_dev(B)
    bv = torch.from_numpy(_values(B, 6)).cuda()
    ev = torch.zeros(0, dtype=torch.float32, device=ws_dev)
    p = sp.numeric_product(dE, ev, dB, bv, sp.config(ratio=0.5), ws=sp.Workspace.for_operands(dE, dB))
    assert p.rpt.cpu().tolist() == [0] and p.col.numel() == 0 and p.info["numeric"]["status"] == 0
    # rows without entries, B rows without entries
    A = W.from_coo(50, 40, [3, 3, 10, 49], [0, 39, 5, 5])
    B = W.from_coo(40, 60, [0, 0, 5, 39], [1, 59, 2, 2])
    av, bv = _values(A, 7), _values(B, 8)
    dA, dB = to_dev(A), to_dev(B)
    p = sp.numeric_product(dA, torch.from_numpy(av).cuda(), dB, torch.from_numpy(bv).cuda(), sp.config(ratio=1.0),
                           ws=sp.Workspace.for_operands(dA, dB))
    _check_against_oracle(A, B, av, bv, p.rpt, p.col, p.val, "sparse rows")
    # an id out of range is reported, not followed
    Abad = W.CSR(2, 4, np.array([0, 2, 3], np.int32), np.array([1, 9, 2], np.int32))
    Bok = W.erdos_renyi(4, 3, 9, ncols=5)
    dA, dB = to_dev(Abad), to_dev(Bok)
    ws = sp.Workspace.for_operands(dA, dB)
    alloc = torch.tensor([0, 8, 16], dtype=torch.int64, device="cuda")
    c_col, c_val, row_start, nnz_row, res = _into(dA, torch.ones(3, device="cuda"), dB,
                                                  torch.ones(Bok.nnz, device="cuda"), alloc, ws)
    assert sp.read_numeric_result(res)["status"] & sp.STATUS_ERR_BAD_INPUT


def test_repeated_calls_reuse_the_workspace():
    A, _ = CASES["rmat-12"]
    av = _values(A, 10)
    dA = to_dev(A)
    dav = torch.from_numpy(av).cuda()
    ws = sp.Workspace.for_operands(dA, dA)
    first = None
    for k in range(4):
        p = sp.numeric_product(dA, dav, dA, dav, sp.config(ratio=0.02, seed=k % 2), ws=ws, pool=k % 2 == 0)
        rows = np.repeat(np.arange(A.rows), np.diff(p.rpt.cpu().numpy()))
        key = np.lexsort((p.col.cpu().numpy(), rows))
        got = (p.rpt.cpu().numpy(), p.col.cpu().numpy()[key])
        if first is None:
            first = got
            _check_against_oracle(A, A, av, av, p.rpt, p.col, p.val, "repeat")
        assert np.array_equal(got[0], first[0]) and np.array_equal(got[1], first[1])
