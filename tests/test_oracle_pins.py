"""Pins for the CPU oracle: each check ties the oracle to something other than itself.

- published known-answer vectors of the random generator the sample uses;
- brute-force dense products and a library sparse product on small inputs;
- closed forms of stencil matrices derived from geometry, not from CSR loops;
- the paper's printed numbers (Table III, the Sec. I worked example, sample_num);
- identities that hold exactly (Eq. 5, FLOP = sum_k colcount_A(k) * rowlen_B(k)).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads as W

TWO32 = 2**32


# ---------------------------------------------------------------- random numbers
def test_splitmix64_known_answers(golden):
    for seed, k, out in golden("splitmix64_kat.txt"):
        assert oracle.splitmix64(int(seed), int(k)) == int(out, 0)


def test_h32_is_high_half_of_next_output():
    for seed in (0, 1, 7, 2**40 + 3):
        for x in (0, 1, 2, 1000, 2**31 + 5):
            assert oracle.h32(seed, x) == oracle.splitmix64(seed, x + 1) >> 32


def test_bernoulli_sample_size_is_binomial():
    M = 1 << 20
    for seed, ratio in ((0, 0.01), (3, 0.005), (11, 0.25)):
        T = int(ratio * TWO32)
        ids = oracle.sample(M, oracle.BERNOULLI, seed, T)
        p = T / TWO32
        mu, sd = M * p, math.sqrt(M * p * (1 - p))
        assert abs(len(ids) - mu) < 6 * sd
        assert np.all(np.diff(ids) > 0)


def test_bernoulli_threshold_extremes():
    M = 5000
    assert len(oracle.sample(M, oracle.BERNOULLI, 1, 0)) == 0
    assert np.array_equal(oracle.sample(M, oracle.BERNOULLI, 1, TWO32), np.arange(M))


def test_bernoulli_membership_matches_hash():
    M = 3000
    T = int(0.1 * TWO32)
    ids = set(oracle.sample(M, oracle.BERNOULLI, 42, T).tolist())
    for i in range(M):
        assert (i in ids) == (oracle.h32(42, i) < T)


def test_bernoulli_threshold_is_strict():
    # Sampling probability T / 2^32 for a uniform 32-bit hash means the rule is
    # h < T: raising T by one adds exactly the rows whose hash equals T, so a
    # row whose hash is the threshold itself is not yet sampled.
    M, seed = 4000, 9
    for i0 in (0, 17, 2500, M - 1):
        T = oracle.h32(seed, i0)
        lo = set(oracle.sample(M, oracle.BERNOULLI, seed, T).tolist())
        hi = set(oracle.sample(M, oracle.BERNOULLI, seed, T + 1).tolist())
        assert i0 not in lo and i0 in hi and lo <= hi
        assert hi - lo == {i for i in range(M) if oracle.h32(seed, i) == T}

def test_paper_sample_num(golden):
    for M, s in golden("paper_sample_num.txt"):
        assert oracle.paper_sample_num(int(M)) == int(s)
    assert oracle.paper_sample_num(100) == 1  # clamped to one draw
    assert oracle.paper_sample_num(0) == 0


def test_paper_draw_rows_in_range():
    for M in (1, 7, 46835, 1 << 20):
        ids = oracle.sample(M, oracle.PAPER_DRAW, 5)
        assert len(ids) == oracle.paper_sample_num(M)
        assert ids.min() >= 0 and ids.max() < M
        for r in range(min(len(ids), 20)):
            assert ids[r] == (oracle.h32(5, r) * M) >> 32



def test_paper_draw_mapping_covers_rows_in_order():
    # Algorithm 2 scales a uniform number in [0, 1) by M (rid = M * rand): the
    # row id is monotone in the draw's hash, reaches the whole range [0, M) and
    # is uniform over it.  A mapping onto part of the rows (M/2, say) misses the
    # top of the range; one that wraps (h mod M) breaks the order.
    M, n = 1 << 20, 4000
    for seed in range(5):
        ids = oracle.sample(M, oracle.PAPER_DRAW, seed, sample_num=n).astype(np.int64)
        assert len(ids) == n and ids.min() >= 0 and ids.max() < M
        assert ids.max() > 0.99 * M and ids.min() < 0.01 * M
        sd = M / math.sqrt(12 * n)  # standard deviation of the mean of n uniform draws
        assert abs(ids.mean() - (M - 1) / 2) < 6 * sd
        # 16 equal bins: counts within 6 sigma of n/16 each
        cnt = np.bincount(ids * 16 // M, minlength=16)
        assert np.all(np.abs(cnt - n / 16) < 6 * math.sqrt(n / 16))
        h = np.array([oracle.h32(seed, r) for r in range(n)], dtype=np.int64)
        order = np.argsort(h, kind="stable")
        assert np.all(np.diff(ids[order]) >= 0)

# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("shape", [(1, 1, 1), (5, 3, 7), (17, 33, 9), (40, 64, 64), (64, 20, 50)])
@pytest.mark.parametrize("density", [0.05, 0.3, 0.9])
def test_flop_and_nnz_against_dense_product(shape, density):
    M, K, N = shape
    A, B, da, db = W.tiny_random(M, K, N, density, seed=M * 1000 + K * 10 + N)
    ai, bi = da.astype(np.int64), db.astype(np.int64)
    # number of products per row: sum_k A_ik * |B_k*|
    flop_ref = ai @ db.sum(axis=1).astype(np.int64)
    # structural nonzeros of the integer product (all terms positive: no cancellation)
    nnz_ref = np.count_nonzero(ai @ bi, axis=1)
    flop, F = oracle.flop_per_row(A, B)
    assert np.array_equal(flop, flop_ref) and F == flop_ref.sum()
    assert np.array_equal(oracle.row_nnz(A, B), nnz_ref)
    nnz, offs, Z = oracle.symbolic_exact(A, B)
    assert np.array_equal(nnz, nnz_ref) and Z == nnz_ref.sum()
    assert offs[0] == 0 and np.array_equal(np.diff(offs), nnz_ref)


def test_empty_rows_and_columns():
    A = W.from_coo(6, 5, [0, 0, 3], [1, 4, 4])
    B = W.from_coo(5, 8, [1, 1, 4], [0, 7, 7])
    flop, F = oracle.flop_per_row(A, B)
    assert flop.tolist() == [3, 0, 0, 1, 0, 0] and F == 4
    assert oracle.row_nnz(A, B).tolist() == [2, 0, 0, 1, 0, 0]


def test_flop_total_identity_and_library_product():
    scipy_sparse = pytest.importorskip("scipy.sparse")
    for seed, (n, k, avg) in enumerate([(4096, 4096, 8), (3000, 1500, 5), (2000, 5000, 12)]):
        A = W.erdos_renyi(n, avg, 100 + seed, ncols=k)
        B = W.erdos_renyi(k, avg, 200 + seed, ncols=n)
        flop, F = oracle.flop_per_row(A, B)
        colcount = np.bincount(A.col, minlength=k).astype(np.int64)
        assert F == int(colcount @ np.diff(B.rpt).astype(np.int64))
        sa = scipy_sparse.csr_matrix((np.ones(A.nnz), A.col, A.rpt), shape=(n, k))
        sb = scipy_sparse.csr_matrix((np.ones(B.nnz), B.col, B.rpt), shape=(k, n))
        sc = (sa @ sb).tocsr()
        sc.sum_duplicates()
        assert np.array_equal(oracle.row_nnz(A, B), np.diff(sc.indptr))
        # the number of products of row i equals the sum of the integer product's row
        assert np.array_equal(flop, np.asarray(sc.sum(axis=1)).ravel().astype(np.int64))


# ---------------------------------------------------------------- closed forms
def _lap2d_geometry(N):
    """Per-row FLOP and nnz of A*A for the N x N 5-point stencil, from grid geometry:
    nnz_i = grid points within Manhattan distance 2; flop_i = sum of the stencil
    sizes of i's stencil points."""
    deg = np.zeros((N, N), dtype=np.int64)
    for x in range(N):
        for y in range(N):
            deg[x, y] = 1 + (x > 0) + (x < N - 1) + (y > 0) + (y < N - 1)
    flop = np.zeros(N * N, dtype=np.int64)
    nnz = np.zeros(N * N, dtype=np.int64)
    for x in range(N):
        for y in range(N):
            f = deg[x, y]
            for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                if 0 <= x + dx < N and 0 <= y + dy < N:
                    f += deg[x + dx, y + dy]
            c = 0
            for dx in range(-2, 3):
                for dy in range(-2, 3):
                    if abs(dx) + abs(dy) <= 2 and 0 <= x + dx < N and 0 <= y + dy < N:
                        c += 1
            flop[x + N * y] = f
            nnz[x + N * y] = c
    return flop, nnz


@pytest.mark.parametrize("N", [3, 4, 5, 9, 64])
def test_laplacian_2d_closed_form(N):
    A = W.laplacian_2d(N)
    flop, F = oracle.flop_per_row(A, A)
    nnz = oracle.row_nnz(A, A)
    gf, gn = _lap2d_geometry(N)
    assert np.array_equal(flop, gf) and np.array_equal(nnz, gn)
    # totals by counting ordered pairs per offset / squared stencil sizes
    Z = N * N + 4 * N * (N - 1) + 4 * N * (N - 2) + 4 * (N - 1) ** 2
    Fc = 25 * (N - 2) ** 2 + 64 * (N - 2) + 36
    assert int(nnz.sum()) == Z and F == Fc
    if N == 64:
        assert (A.nnz, F, Z) == (20224, 100104, 51972)


def test_periodic_laplacian_uniform_rows():
    for N in (5, 8, 33):
        A = W.laplacian_2d(N, periodic=True)
        flop, _ = oracle.flop_per_row(A, A)
        assert np.all(flop == 25) and np.all(oracle.row_nnz(A, A) == 13)
        for seed in (0, 1, 2):
            r = oracle.predict(A, A, oracle.BERNOULLI, seed, int(0.2 * TWO32))
            assert r["status"] == 0 and np.all(r["pred"] == 13)
            # the allocation offsets of rows of 13: 0, 13, 26, ...
            assert np.array_equal(r["offsets"], 13 * np.arange(A.rows + 1))


@pytest.mark.parametrize("dims", [(3, 3, 3), (4, 5, 6), (8, 8, 8), (16, 4, 9)])
def test_stencil_27_closed_form(dims):
    A = W.stencil_3d_27(*dims)
    flop, F = oracle.flop_per_row(A, A)
    nnz = oracle.row_nnz(A, A)
    # tensor-product structure: per axis, stencil size 3 inside and 2 at the ends
    assert F == math.prod(9 * n - 10 for n in dims)
    assert int(nnz.sum()) == math.prod(5 * n - 6 for n in dims)
    nx, ny, nz = dims
    for z in range(2, nz - 2):
        for y in range(2, ny - 2):
            for x in range(2, nx - 2):
                i = x + nx * (y + ny * z)
                assert flop[i] == 729 and nnz[i] == 125


@pytest.mark.parametrize("b", [1, 2, 7, 32])
def test_dense_blocks(b):
    A = W.dense_blocks(64 * b, b)
    flop, _ = oracle.flop_per_row(A, A)
    assert np.all(flop == b * b) and np.all(oracle.row_nnz(A, A) == b)
    r = oracle.predict(A, A, oracle.BERNOULLI, 3, int(0.3 * TWO32))
    assert np.all(r["pred"] == b) and Fraction(r["flop_s"], r["nnz_s"]) == b



def test_reference_design_uniform_rows():
    # Eq. 2 on a matrix whose output rows all have the same FLOP f and nnz z:
    # any non-empty sample gives z* = z |S| and F = f M, so Z1* = z* M / |S| =
    # z M = Z exactly, and every row's prediction flop_i / CR1 = f z M / F is z.
    # Torus 5-point stencil: f = 25, z = 13; dense b x b blocks: f = b^2, z = b.
    cases = [(W.laplacian_2d(N, periodic=True), 13) for N in (5, 8, 33)]
    cases += [(W.dense_blocks(64 * b, b), b) for b in (2, 7, 32)]
    for A, z in cases:
        M = A.rows
        runs = [(oracle.BERNOULLI, seed, int(ratio * TWO32), 0)
                for seed in range(3) for ratio in (0.2, 0.5)]
        runs += [(oracle.PAPER_DRAW, seed, 0, s) for seed in range(3) for s in (7, min(40, M))]
        for mode, seed, T, s in runs:
            r = oracle.predict_reference(A, A, mode, seed, T, s)
            if r["n_sampled"] < 2:
                continue
            assert r["status"] == 0, (mode, seed)
            assert np.all(r["pred"] == z), (mode, seed, np.unique(r["pred"]))
            assert r["pred_total"] == z * M and r["offsets"][-1] == z * M
            e = oracle.estimates(r["flop_total"], z * M, r["flop_s"], r["nnz_s"], M, r["n_sampled"])
            assert e["Z1"] == z * M and e["eps1"] == 0


def test_rounding_up_worked_example():
    # Hand-worked case for the rounding of flop_i / r*: three dense 2 x 2 blocks
    # and two dense 3 x 3 blocks (12 rows).  Six rows have flop 4 and nnz 2, six
    # have flop 9 and nnz 3, so with every row sampled z* = 30 and f* = 78, and
    # r* = 78 / 30 = 2.6.  A row of flop 4 predicts 4 / 2.6 = 1.54 -> 2 and a row
    # of flop 9 predicts 9 / 2.6 = 3.46 -> 4 (rounded up; down would give 1 and 3).
    # The reference design (p = 1, F = f*) gives the same.
    rows, cols = [], []
    starts = [(0, 2), (2, 2), (4, 2), (6, 3), (9, 3)]
    for s0, b in starts:
        for i in range(b):
            for j in range(b):
                rows.append(s0 + i)
                cols.append(s0 + j)
    A = W.from_coo(12, 12, np.array(rows), np.array(cols))
    want = [2] * 6 + [4] * 6
    for fn in (oracle.predict, oracle.predict_reference):
        r = fn(A, A, oracle.BERNOULLI, 0, TWO32)
        assert (r["flop_s"], r["nnz_s"], r["n_sampled"]) == (78, 30, 12)
        assert r["pred"].tolist() == want and r["pred_total"] == 36

# ---------------------------------------------------------------- the method
def _cases():
    yield "lap64", W.laplacian_2d(64), None
    yield "er", W.erdos_renyi(3000, 9, 7), None
    yield "rmat", W.rmat(11, 8, seed=5), None
    yield "rect", W.keep_left_columns(W.erdos_renyi(2048, 12, 8), 1024), \
        W.keep_top_rows(W.erdos_renyi(2048, 12, 9), 1024)


@pytest.mark.parametrize("name", ["lap64", "er", "rmat", "rect"])
def test_all_rows_sampled_gives_exact_totals(name):
    A, B = next((a, b) for n, a, b in _cases() if n == name)
    B = A if B is None else B
    nnz, _, Z = oracle.symbolic_exact(A, B)
    for ref in (False, True):
        fn = oracle.predict_reference if ref else oracle.predict
        r = fn(A, B, oracle.BERNOULLI, 0, TWO32)
        assert r["n_sampled"] == A.rows and r["flop_s"] == r["flop_total"] and r["nnz_s"] == Z
        e = oracle.estimates(r["flop_total"], Z, r["flop_s"], r["nnz_s"], A.rows, r["n_sampled"])
        assert e["Z1"] == Z and e["Z2"] == Z and e["eps1"] == 0 and e["eps2"] == 0


@pytest.mark.parametrize("name", ["lap64", "er", "rmat", "rect"])
@pytest.mark.parametrize("mode", [oracle.BERNOULLI, oracle.PAPER_DRAW])
def test_prediction_invariants(name, mode):
    A, B = next((a, b) for n, a, b in _cases() if n == name)
    B = A if B is None else B
    nnz_all = oracle.row_nnz(A, B)
    for seed in range(3):
        r = oracle.predict(A, B, mode, seed, int(0.05 * TWO32))
        ids = r["ids"]
        flop, pred, off = r["flop"], r["pred"], r["offsets"]
        # f* and z* are the sums over the sample (with multiplicity) of pinned per-row values
        assert r["flop_s"] == int(flop[ids].sum())
        assert r["nnz_s"] == int(nnz_all[ids].sum())
        assert r["nnz_s"] <= r["flop_s"]
        assert off[0] == 0 and np.array_equal(np.diff(off), pred) and off[-1] == r["pred_total"]
        if r["flop_s"]:
            assert np.all(pred <= flop) and np.all((pred >= 1) == (flop >= 1))
            # ceil(flop * z / f): the smallest integer q with q * f >= flop * z
            f, z = r["flop_s"], r["nnz_s"]
            for i in range(0, A.rows, max(1, A.rows // 97)):
                q = int(pred[i])
                assert q * f >= int(flop[i]) * z and (q - 1) * f < int(flop[i]) * z
        rr = oracle.predict_reference(A, B, mode, seed, int(0.05 * TWO32))
        assert rr["nnz_s"] == r["nnz_s"] and rr["n_sampled"] == r["n_sampled"]
        F, S, M = rr["flop_total"], rr["n_sampled"], A.rows
        for i in range(0, A.rows, max(1, A.rows // 97)):
            q = int(rr["pred"][i])
            num = int(flop[i]) * r["nnz_s"] * M
            if flop[i] == 0:
                assert q == 0
            elif q < 2**31 - 1:
                assert q * F * S >= num and (q - 1) * F * S < num


def test_eq5_identity_exact():
    A = W.rmat(12, 8, seed=9)
    nnz, _, Z = oracle.symbolic_exact(A, A)
    seen = 0
    for seed in range(20):
        r = oracle.predict(A, A, oracle.BERNOULLI, seed, int(0.01 * TWO32))
        if not r["flop_s"]:
            continue
        e = oracle.estimates(r["flop_total"], Z, r["flop_s"], r["nnz_s"], A.rows, r["n_sampled"])
        assert e["eps2"] == (e["eps1"] - e["eps_f"]) / (1 + e["eps_f"])
        seen += 1
    assert seen >= 15


def test_table3_rows_satisfy_eq5(golden):
    # Rebuild each printed case from its own numbers and recompute eps_2 with the
    # oracle's estimator formulas; it must agree with the printed eps_2 to rounding.
    for _, s, cr, nnzc, e1, ef, e2 in golden("table3_relative_errors.txt"):
        Z = Fraction(int(nnzc))
        F = Z * Fraction(cr)
        M, S = Fraction(100000), Fraction(int(s))
        p = S / M
        z = (1 + Fraction(e1) / 100) * p * Z
        f = (1 + Fraction(ef) / 100) * p * F
        e = oracle.estimates(F, Z, f, z, M, S)
        assert abs(float(e["eps1"]) * 100 - float(e1)) < 1e-9
        assert abs(float(e["eps_f"]) * 100 - float(ef)) < 1e-9
        # eps_1, eps_f and eps_2 are printed to 0.01 pp (each off by at most 0.005 pp):
        # propagate the input rounding through Eq. 5 and add the output rounding.
        a, b = float(e1) / 100, float(ef) / 100
        tol = 0.005 / (1 + b) + 0.005 * (1 + a) / (1 + b) ** 2 + 0.005 + 1e-9
        assert abs(float(e["eps2"]) * 100 - float(e2)) <= tol


def test_intro_worked_example():
    # Sec. I: sampled FLOP 25 % and sampled NNZ 30 % above expectation give a
    # predicted compression ratio 3.85 % off.
    F, Z, M, S = 10000, 5000, 100, 1
    f = Fraction(125, 100) * F * S / M
    z = Fraction(130, 100) * Z * S / M
    e = oracle.estimates(F, Z, f, z, M, S)
    assert round(abs(float(e["r_star"] / e["CR"] - 1)) * 100, 2) == 3.85
    assert e["eps2"] == Fraction(4, 100)


def test_empty_sample_falls_back_to_flop():
    A = W.erdos_renyi(500, 6, 1)
    r = oracle.predict(A, A, oracle.BERNOULLI, 0, 0)
    assert r["status"] == oracle.WARN_EMPTY_SAMPLE and r["n_sampled"] == 0
    assert np.array_equal(r["pred"], r["flop"])
    rr = oracle.predict_reference(A, A, oracle.BERNOULLI, 0, 0)
    assert rr["status"] == oracle.WARN_EMPTY_SAMPLE and np.array_equal(rr["pred"], rr["flop"])


def test_paper_draw_counts_repeats():
    A = W.erdos_renyi(50, 4, 2)
    ids = np.array([3, 3, 7], dtype=np.int32)
    r = oracle.predict_with_ids(A, A, ids)
    nnz = oracle.row_nnz(A, A)
    assert r["flop_s"] == 2 * r["flop"][3] + r["flop"][7]
    assert r["nnz_s"] == 2 * nnz[3] + nnz[7] and r["n_sampled"] == 3


def test_rectangular_reshape_rule():
    A = W.erdos_renyi(300, 10, 3)
    B = W.erdos_renyi(300, 10, 4)
    A2, B2 = W.keep_left_columns(A, 120), W.keep_top_rows(B, 120)
    assert (A2.rows, A2.cols, B2.rows, B2.cols) == (300, 120, 120, 300)
    dA = np.zeros((300, 300), dtype=np.int64)
    dB = np.zeros((300, 300), dtype=np.int64)
    dA[np.repeat(np.arange(300), np.diff(A.rpt)), A.col] = 1
    dB[np.repeat(np.arange(300), np.diff(B.rpt)), B.col] = 1
    ref = np.count_nonzero(dA[:, :120] @ dB[:120, :], axis=1)
    assert np.array_equal(oracle.row_nnz(A2, B2), ref)


# ---------------------------------------------------------------- numeric product
def _signed_values(m, seed):
    """Seeded single-precision values in [-1, 1) for every nonzero (cancellation possible)."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, m.nnz).astype(np.float32)


def _dense(m, val):
    d = np.zeros((m.rows, m.cols), dtype=np.float64)
    rows = np.repeat(np.arange(m.rows), np.diff(m.rpt))
    d[rows, m.col] = val.astype(np.float64)
    return d


@pytest.mark.parametrize("shape", [(1, 1, 1), (5, 3, 7), (17, 33, 9), (40, 64, 64)])
@pytest.mark.parametrize("density", [0.1, 0.5])
def test_numeric_against_dense_product(shape, density):
    M, K, N = shape
    A, B, da, db = W.tiny_random(M, K, N, density, seed=M * 7 + K * 3 + N)
    av, bv = _signed_values(A, 1), _signed_values(B, 2)
    Ad, Bd = _dense(A, av), _dense(B, bv)
    offs, col, val, abs_sum, terms = oracle.numeric(A, av, B, bv)
    # structure: the boolean product (no cancellation in a count of paths)
    paths = da.astype(np.int64) @ db.astype(np.int64)
    assert np.array_equal(np.diff(offs), np.count_nonzero(paths, axis=1))
    rows = np.repeat(np.arange(M), np.diff(offs))
    assert np.array_equal(paths[rows, col], terms)
    for i in range(M):  # ascending columns within each row
        assert np.all(np.diff(col[offs[i]:offs[i + 1]]) > 0)
    # values: the dense double product (products of single-precision values are exact in double)
    ref = Ad @ Bd
    np.testing.assert_allclose(val, ref[rows, col], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(abs_sum, (np.abs(Ad) @ np.abs(Bd))[rows, col], rtol=1e-12, atol=1e-12)
    # and nothing outside the structure
    mask = np.zeros((M, N), dtype=bool)
    mask[rows, col] = True
    assert np.all(ref[~mask] == 0.0)


@pytest.mark.parametrize("N", [5, 8, 13])
def test_numeric_laplacian_squared_closed_form(N):
    # A = 4 I - (sum of the four grid shifts), Dirichlet: (A^2)_ij by geometry:
    # i = j: 16 + deg(i); one step apart: -8; diagonal neighbours: 2 (two paths);
    # two steps in a line: 1 (one path through the middle node)
    A = W.laplacian_2d(N, values="laplace")
    av = A.val.astype(np.float32)
    offs, col, val, _, _ = oracle.numeric(A, av, A, av)
    for i in range(N * N):
        x, y = i % N, i // N
        deg = sum(1 for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)) if 0 <= x + dx < N and 0 <= y + dy < N)
        want = {i: 16.0 + deg}
        for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            if 0 <= x + dx < N and 0 <= y + dy < N:
                want[(x + dx) + N * (y + dy)] = -8.0
            if 0 <= x + 2 * dx < N and 0 <= y + 2 * dy < N:
                want[(x + 2 * dx) + N * (y + 2 * dy)] = 1.0
        for dx, dy in ((1, 1), (1, -1), (-1, 1), (-1, -1)):
            if 0 <= x + dx < N and 0 <= y + dy < N:
                want[(x + dx) + N * (y + dy)] = 2.0
        got = dict(zip(col[offs[i]:offs[i + 1]].tolist(), val[offs[i]:offs[i + 1]].tolist()))
        assert got == want, (i, got, want)


def test_numeric_sum_identity():
    # sum of all entries of A*B = sum_k (column sum k of A) * (row sum k of B)
    A = W.erdos_renyi(300, 6, 21, ncols=200)
    B = W.erdos_renyi(200, 5, 22, ncols=250)
    av, bv = _signed_values(A, 3), _signed_values(B, 4)
    _, _, val, _, _ = oracle.numeric(A, av, B, bv)
    colsum_a = np.bincount(A.col, weights=av.astype(np.float64), minlength=A.cols)
    rowsum_b = np.add.reduceat(bv.astype(np.float64), B.rpt[:-1]) * (np.diff(B.rpt) > 0)
    assert math.isclose(val.sum(), float(colsum_a @ rowsum_b), rel_tol=1e-9, abs_tol=1e-9)
