"""Seeded synthetic sparse matrices for the SpGEMM structure-prediction workloads.

This module only builds inputs.  It holds none of the prediction method's
arithmetic (no FLOP counts, no nnz counts, no sampling), so both the CUDA
library and the CPU oracle can be fed from it.  All matrices are canonical CSR
(Sec. II-B of the paper): int32 row offsets ``rpt`` (rows+1 entries) and int32
column ids ``col``, sorted and unique within each row.  Values are produced only
on request: the method never reads them.

Stand-ins for the paper's SuiteSparse inputs (Sec. VI, Table II), which are not
used here: 2D 5-point and 3D 27-point stencils, Erdos-Renyi matrices with
Poisson row lengths, R-MAT power-law matrices, random block-diagonal matrices,
and the rectangular reshape rule of Sec. VI-A (keep the left columns of the
first operand, the top rows of the second).
"""
from dataclasses import dataclass
from typing import Optional

import numpy as np


@dataclass
class CSR:
    rows: int
    cols: int
    rpt: np.ndarray  # int32[rows + 1]
    col: np.ndarray  # int32[nnz]
    val: Optional[np.ndarray] = None

    @property
    def nnz(self):
        return int(self.col.shape[0])


def from_coo(rows, cols, r, c, val=None, dedup=True):
    """Canonical CSR from coordinate lists (duplicates merged when ``dedup``)."""
    r = np.asarray(r, dtype=np.int64)
    c = np.asarray(c, dtype=np.int64)
    key = r * np.int64(cols) + c
    if dedup:
        key = np.sort(key, kind="stable")
        if key.shape[0]:
            keep = np.empty(key.shape[0], dtype=bool)
            keep[0] = True
            np.not_equal(key[1:], key[:-1], out=keep[1:])
            key = key[keep]
        val = None if val is None else np.ones(key.shape[0], dtype=np.asarray(val).dtype)
    else:
        order = np.argsort(key, kind="stable")
        key = key[order]
        val = None if val is None else np.asarray(val)[order]
    rr = key // cols
    cc = (key - rr * cols).astype(np.int32)
    counts = np.bincount(rr, minlength=rows).astype(np.int64)
    rpt = np.zeros(rows + 1, dtype=np.int64)
    np.cumsum(counts, out=rpt[1:])
    if rpt[-1] >= 2**31:
        raise ValueError("nnz does not fit int32 offsets")
    return CSR(rows, cols, rpt.astype(np.int32), cc, val)


def _with_values(m, kind, rng=None):
    if kind is None:
        return m
    if kind == "laplace":
        # 4 on the diagonal, -1 elsewhere (fp64), as in the 2D 5-point config.
        rows = np.repeat(np.arange(m.rows), np.diff(m.rpt))
        m.val = np.where(m.col == rows, 4.0, -1.0)
    elif kind == "uniform":
        rng = rng or np.random.default_rng(0)
        m.val = rng.random(m.nnz, dtype=np.float32)
    return m


def laplacian_2d(N, periodic=False, values=None, Ny=None):
    """5-point stencil on an N x Ny grid (Ny = N by default; row id = x + N*y),
    Dirichlet or periodic boundaries."""
    Ny = N if Ny is None else Ny
    n = N * Ny
    idx = np.arange(n, dtype=np.int64)
    x, y = idx % N, idx // N
    rs, cs = [idx], [idx]
    for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
        xx, yy = x + dx, y + dy
        if periodic:
            xx %= N
            yy %= Ny
            ok = np.ones(n, dtype=bool)
        else:
            ok = (xx >= 0) & (xx < N) & (yy >= 0) & (yy < Ny)
        rs.append(idx[ok])
        cs.append((xx + N * yy)[ok])
    m = from_coo(n, n, np.concatenate(rs), np.concatenate(cs))
    return _with_values(m, "laplace" if values else None)


def grid_2d(n):
    """Grid sides (N, Ny) with N*Ny == n, as square as a power of two allows."""
    e = int(round(np.log2(n)))
    if 2**e != n:
        raise ValueError("n must be a power of two")
    return 2 ** ((e + 1) // 2), 2 ** (e // 2)


def stencil_3d_27(nx, ny, nz, values=None, seed=0):
    """27-point stencil on an nx x ny x nz box (Dirichlet; row id = x + nx*(y + ny*z))."""
    n = nx * ny * nz
    idx = np.arange(n, dtype=np.int64)
    x = idx % nx
    y = (idx // nx) % ny
    z = idx // (nx * ny)
    rs, cs = [], []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                xx, yy, zz = x + dx, y + dy, z + dz
                ok = (xx >= 0) & (xx < nx) & (yy >= 0) & (yy < ny) & (zz >= 0) & (zz < nz)
                rs.append(idx[ok])
                cs.append((xx + nx * (yy + ny * zz))[ok])
    m = from_coo(n, n, np.concatenate(rs), np.concatenate(cs))
    return _with_values(m, "uniform" if values else None, np.random.default_rng(seed))


def erdos_renyi(n, avg, seed, ncols=None, values=None):
    """Uniform random matrix: Poisson(avg) entries drawn per row, uniform columns, merged."""
    ncols = n if ncols is None else ncols
    rng = np.random.default_rng(seed)
    lens = rng.poisson(avg, n).astype(np.int64)
    r = np.repeat(np.arange(n, dtype=np.int64), lens)
    c = rng.integers(0, ncols, r.shape[0], dtype=np.int64)
    m = from_coo(n, ncols, r, c)
    return _with_values(m, "uniform" if values else None, rng)


def rmat(scale, edge_factor, abcd=(0.57, 0.19, 0.19, 0.05), seed=0, values=None):
    """R-MAT graph (Chakrabarti, Zhan, Faloutsos 2004): edge_factor * 2^scale edges,
    each placed by ``scale`` recursive quadrant choices with probabilities (a, b, c, d);
    no vertex permutation; duplicate edges merged."""
    n = 1 << scale
    E = edge_factor * n
    a, b, c, _ = abcd
    rng = np.random.default_rng(seed)
    r = np.zeros(E, dtype=np.int64)
    cc = np.zeros(E, dtype=np.int64)
    t1, t2, t3 = a, a + b, a + b + c
    for level in range(scale):
        u = rng.random(E, dtype=np.float32)
        bit = np.int64(1) << (scale - 1 - level)
        rbit = u >= t2                       # quadrants c, d: lower half
        cbit = ((u >= t1) & (u < t2)) | (u >= t3)  # quadrants b, d: right half
        r += rbit * bit
        cc += cbit * bit
    m = from_coo(n, n, r, cc)
    return _with_values(m, "uniform" if values else None, rng)


def block_diagonal(n, b, fill, seed, values=None):
    """n/b dense-pattern diagonal blocks of size b x b, each entry kept with prob ``fill``."""
    if n % b:
        raise ValueError("n must be a multiple of b")
    rng = np.random.default_rng(seed)
    nb = n // b
    keep = rng.random((nb, b, b), dtype=np.float32) < fill
    blk, i, j = np.nonzero(keep)
    m = from_coo(n, n, blk.astype(np.int64) * b + i, blk.astype(np.int64) * b + j)
    return _with_values(m, "uniform" if values else None, rng)


def dense_blocks(n, b):
    """n/b full b x b diagonal blocks."""
    return block_diagonal(n, b, 2.0, 0)


def keep_left_columns(A, k):
    """Sec. VI-A reshape: keep the left k columns of A."""
    rows = np.repeat(np.arange(A.rows, dtype=np.int64), np.diff(A.rpt))
    ok = A.col < k
    return from_coo(A.rows, k, rows[ok], A.col[ok].astype(np.int64), dedup=False)


def keep_top_rows(B, k):
    """Sec. VI-A reshape: keep the top k rows of B."""
    end = int(B.rpt[k])
    return CSR(k, B.cols, B.rpt[: k + 1].copy(), B.col[:end].copy(),
               None if B.val is None else B.val[:end].copy())


def box_3d(n):
    """Box dimensions (nx, ny, nz) with nx*ny*nz == n for the 3D 27-point family."""
    table = {2**12: (16, 16, 16), 2**14: (32, 32, 16), 2**16: (64, 32, 32),
             2**18: (64, 64, 64), 2**20: (128, 128, 64), 2**21: (128, 128, 128)}
    if n in table:
        return table[n]
    e = int(round(np.log2(n)))
    if 2**e != n:
        raise ValueError("n must be a power of two")
    dims = [e // 3 + (1 if k < e % 3 else 0) for k in range(3)]
    return tuple(2**d for d in dims)


STRUCTURES = ("er", "rmat", "lap2d", "st27", "blockdiag")


def family_case(structure, n, variant):
    """One case of the 625-case family: 5 structures x sizes x 25 variants.

    Variant j has density round(2 * 32**(j/24)) (2..64 nnz/row, used by ER and
    R-MAT) and seed j.  Even j: square C = A*A.  Odd j: rectangular
    A(n x n/2) * B(n/2 x n) by the Sec. VI-A reshape rule, with B generated as
    its own n x n instance (next seed).  Returns (A, B, name).
    """
    d = int(round(2 * 32 ** (variant / 24)))
    seed = variant

    def gen(s):
        if structure == "er":
            return erdos_renyi(n, d, 1000 * 4 + 100 * s + int(np.log2(n)))
        if structure == "rmat":
            return rmat(int(round(np.log2(n))), max(d, 1), seed=1000 * 4 + 100 * s + int(np.log2(n)))
        if structure == "lap2d":
            N, Ny = grid_2d(n)
            return laplacian_2d(N, Ny=Ny)
        if structure == "st27":
            return stencil_3d_27(*box_3d(n))
        if structure == "blockdiag":
            return block_diagonal(n, 32, 0.3, 1000 * 4 + 100 * s + int(np.log2(n)))
        raise ValueError(structure)

    A = gen(seed)
    if variant % 2 == 0:
        return A, A, f"{structure}-n{n}-v{variant}-sq"
    B = gen(seed + 1)
    h = n // 2
    return keep_left_columns(A, h), keep_top_rows(B, h), f"{structure}-n{n}-v{variant}-rect"


def tiny_random(M, K, N, density, seed):
    """Small dense-ish random pair for brute-force checks: A (M x K), B (K x N)."""
    rng = np.random.default_rng(seed)
    da = rng.random((M, K)) < density
    db = rng.random((K, N)) < density
    ra, ca = np.nonzero(da)
    rb, cb = np.nonzero(db)
    return from_coo(M, K, ra, ca), from_coo(K, N, rb, cb), da, db
