"""CPU oracle for the sampled-compression-ratio SpGEMM structure predictor.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the GPU library: the arithmetic lives in ``oracle.c`` (plain C, exact
integers) and this module only marshals numpy arrays into it.  The reported
real-valued estimates (Eq. 2, 3, 4 and the relative errors of Sec. VI-A) are
formed here from exact rationals and rounded once to double.

A matrix is any object with attributes ``rows``, ``cols``, ``rpt`` (int32,
rows+1) and ``col`` (int32, nnz), in canonical CSR (Sec. II-B).
"""
import ctypes
from fractions import Fraction

import numpy as np

from . import build as _build

WARN_EMPTY_SAMPLE = 1
WARN_SATURATED = 2

BERNOULLI = 0
PAPER_DRAW = 1

_lib = None

_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_p = ctypes.c_void_p


def _bind(path):
    lib = ctypes.CDLL(str(path))
    lib.orc_splitmix64.restype = _u64
    lib.orc_splitmix64.argtypes = [_u64, _u64]
    lib.orc_h32.restype = ctypes.c_uint32
    lib.orc_h32.argtypes = [_u64, _u64]
    lib.orc_flop_per_row.restype = _i64
    lib.orc_flop_per_row.argtypes = [_i64, _p, _p, _p, _p]
    lib.orc_row_nnz.restype = _i64
    lib.orc_row_nnz.argtypes = [_i64, _p, _p, _p, _p, _p, _i64, _p]
    lib.orc_sample_bernoulli.restype = _i64
    lib.orc_sample_bernoulli.argtypes = [_i64, _u64, _u64, _p]
    lib.orc_paper_sample_num.restype = _i64
    lib.orc_paper_sample_num.argtypes = [_i64]
    lib.orc_sample_paper_draw.restype = _i64
    lib.orc_sample_paper_draw.argtypes = [_i64, _u64, _i64, _p]
    for fn in (lib.orc_predict, lib.orc_predict_reference):
        fn.restype = ctypes.c_int
        fn.argtypes = [_i64, _i64, _p, _p, _p, _p, _p, _i64, _p, _p, _p, _p]
    lib.orc_symbolic_exact.restype = _i64
    lib.orc_symbolic_exact.argtypes = [_i64, _i64, _p, _p, _p, _p, _p, _p]
    lib.orc_spgemm_numeric.restype = _i64
    lib.orc_spgemm_numeric.argtypes = [_i64, _i64] + [_p] * 11
    lib.orc_num_threads.restype = ctypes.c_int
    lib.orc_set_num_threads.argtypes = [ctypes.c_int]
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(_build.build())
    return _lib


def use_library(path):
    """Swap in another build of oracle.c (the mutation tests use this); returns the
    previous handle, which ``restore_library`` puts back."""
    global _lib
    prev = _lib
    _lib = _bind(path)
    return prev


def restore_library(prev):
    global _lib
    _lib = prev


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a.size else None


def _csr(m):
    rpt = np.ascontiguousarray(m.rpt, dtype=np.int32)
    col = np.ascontiguousarray(m.col, dtype=np.int32)
    if rpt.shape[0] != m.rows + 1:
        raise ValueError("rpt must have rows+1 entries")
    return rpt, col


def num_threads():
    return _load().orc_num_threads()


def set_num_threads(n):
    _load().orc_set_num_threads(int(n))


def splitmix64(seed, k):
    """k-th output (k >= 1) of SplitMix64 started at state ``seed``."""
    return int(_load().orc_splitmix64(seed & (2**64 - 1), k & (2**64 - 1)))


def h32(seed, x):
    """High 32 bits of output x+1 of SplitMix64 seeded with ``seed``."""
    return int(_load().orc_h32(seed & (2**64 - 1), x & (2**64 - 1)))


def flop_per_row(A, B):
    """Algorithm 1: (flop int64[M], total_flop)."""
    if A.cols != B.rows:
        raise ValueError("A.cols != B.rows")
    a_rpt, a_col = _csr(A)
    b_rpt, _ = _csr(B)
    flop = np.zeros(A.rows, dtype=np.int64)
    F = _load().orc_flop_per_row(A.rows, _ptr(a_rpt), _ptr(a_col), _ptr(b_rpt), _ptr(flop))
    return flop, int(F)


def row_nnz(A, B, rows=None):
    """Exact nnz of the listed output rows (all rows if ``rows`` is None)."""
    if A.cols != B.rows:
        raise ValueError("A.cols != B.rows")
    a_rpt, a_col = _csr(A)
    b_rpt, b_col = _csr(B)
    if rows is None:
        n = A.rows
        ids = None
    else:
        ids = np.ascontiguousarray(rows, dtype=np.int32)
        n = ids.shape[0]
    out = np.zeros(n, dtype=np.int64)
    tot = _load().orc_row_nnz(B.cols, _ptr(a_rpt), _ptr(a_col), _ptr(b_rpt), _ptr(b_col),
                              None if ids is None else _ptr(ids), n, _ptr(out))
    if tot < 0:
        raise MemoryError("oracle marker allocation failed")
    return out


def paper_sample_num(M):
    return int(_load().orc_paper_sample_num(M))


def sample(M, mode=BERNOULLI, seed=0, threshold=0, sample_num=0):
    """The sampled row ids: Bernoulli(threshold / 2^32) or the paper's draws."""
    lib = _load()
    if mode == BERNOULLI:
        if not 0 <= threshold <= 2**32:
            raise ValueError("threshold must be in [0, 2^32]")
        ids = np.zeros(max(M, 1), dtype=np.int32)
        n = lib.orc_sample_bernoulli(M, seed & (2**64 - 1), threshold, _ptr(ids))
        return ids[:n].copy()
    if mode == PAPER_DRAW:
        s = sample_num if sample_num > 0 else paper_sample_num(M)
        ids = np.zeros(max(s, 1), dtype=np.int32)
        lib.orc_sample_paper_draw(M, seed & (2**64 - 1), s, _ptr(ids))
        return ids[:s].copy()
    raise ValueError("unknown sampling mode")


def _run(fn, A, B, ids):
    if A.cols != B.rows:
        raise ValueError("A.cols != B.rows")
    a_rpt, a_col = _csr(A)
    b_rpt, b_col = _csr(B)
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    M = A.rows
    flop = np.zeros(M, dtype=np.int64)
    pred = np.zeros(M, dtype=np.int64)
    offsets = np.zeros(M + 1, dtype=np.int64)
    sc = np.zeros(6, dtype=np.int64)
    rc = fn(M, B.cols, _ptr(a_rpt), _ptr(a_col), _ptr(b_rpt), _ptr(b_col), _ptr(ids),
            ids.shape[0], _ptr(flop), _ptr(pred), _ptr(offsets), _ptr(sc))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return dict(flop=flop, pred=pred, offsets=offsets, ids=ids, flop_total=int(sc[0]),
                flop_s=int(sc[1]), nnz_s=int(sc[2]), n_sampled=int(sc[3]),
                pred_total=int(sc[4]), status=int(sc[5]))


def predict(A, B, mode=BERNOULLI, seed=0, threshold=0, sample_num=0):
    """The proposed method (Eq. 4, Algorithm 2) on the seed-determined sample."""
    ids = sample(A.rows, mode, seed, threshold, sample_num)
    return _run(_load().orc_predict, A, B, ids)


def predict_reference(A, B, mode=BERNOULLI, seed=0, threshold=0, sample_num=0):
    """The reference design (Eq. 2) on the same sample."""
    ids = sample(A.rows, mode, seed, threshold, sample_num)
    return _run(_load().orc_predict_reference, A, B, ids)


def predict_with_ids(A, B, ids, reference=False):
    """Either design on an explicit sample (repeats allowed)."""
    lib = _load()
    return _run(lib.orc_predict_reference if reference else lib.orc_predict, A, B, ids)


def symbolic_exact(A, B):
    """Exact nnz per output row, offsets and Z = NNZ(C)."""
    if A.cols != B.rows:
        raise ValueError("A.cols != B.rows")
    a_rpt, a_col = _csr(A)
    b_rpt, b_col = _csr(B)
    nnz = np.zeros(A.rows, dtype=np.int64)
    offsets = np.zeros(A.rows + 1, dtype=np.int64)
    Z = _load().orc_symbolic_exact(A.rows, B.cols, _ptr(a_rpt), _ptr(a_col), _ptr(b_rpt),
                                   _ptr(b_col), _ptr(nnz), _ptr(offsets))
    if Z < 0:
        raise MemoryError("oracle marker allocation failed")
    return nnz, offsets, int(Z)


def numeric(A, a_val, B, b_val):
    """C = A*B with values (the numeric phase the prediction allocates for):
    returns (offsets int64[M+1], col int32, val float64, abs_sum float64,
    terms int32), columns ascending within each row; abs_sum and terms are the
    sum of |products| and the number of products behind each entry."""
    if A.cols != B.rows:
        raise ValueError("A.cols != B.rows")
    a_rpt, a_col = _csr(A)
    b_rpt, b_col = _csr(B)
    a_val = np.ascontiguousarray(a_val, dtype=np.float32)
    b_val = np.ascontiguousarray(b_val, dtype=np.float32)
    if a_val.shape[0] != a_col.shape[0] or b_val.shape[0] != b_col.shape[0]:
        raise ValueError("one value per nonzero")
    _, offsets, Z = symbolic_exact(A, B)
    col = np.zeros(Z, dtype=np.int32)
    val = np.zeros(Z, dtype=np.float64)
    abs_sum = np.zeros(Z, dtype=np.float64)
    terms = np.zeros(Z, dtype=np.int32)
    n = _load().orc_spgemm_numeric(A.rows, B.cols, _ptr(a_rpt), _ptr(a_col), _ptr(a_val), _ptr(b_rpt),
                                   _ptr(b_col), _ptr(b_val), _ptr(offsets), _ptr(col), _ptr(val),
                                   _ptr(abs_sum), _ptr(terms))
    if n < 0:
        raise MemoryError("oracle accumulator allocation failed")
    return offsets, col, val, abs_sum, terms


def estimates(F, Z, f, z, M, S):
    """Sec. IV and VI-A quantities as exact rationals (None where undefined).

    Z1* = z / p (Eq. 2), F* = f / p (Eq. 3), Z2* = F z / f (Eq. 4), p = S / M;
    eps1 = (Z1* - Z)/Z, eps_f = (F* - F)/F, eps2 = (Z2* - Z)/Z; r* = f / z.
    """
    out = {}
    out["Z1"] = Fraction(z * M, S) if S else None
    out["F_star"] = Fraction(f * M, S) if S else None
    out["Z2"] = Fraction(F * z, f) if f else None
    out["r_star"] = Fraction(f, z) if z else None
    out["CR"] = Fraction(F, Z) if Z else None
    out["eps1"] = (out["Z1"] - Z) / Z if (S and Z) else None
    out["eps_f"] = (out["F_star"] - F) / F if (S and F) else None
    out["eps2"] = (out["Z2"] - Z) / Z if (f and Z) else None
    return out


def estimates_float(F, Z, f, z, M, S):
    """``estimates`` with every rational rounded once to the nearest double."""
    return {k: (None if v is None else float(v)) for k, v in estimates(F, Z, f, z, M, S).items()}
