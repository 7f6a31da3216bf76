"""Host-side reporting of the prediction's real-valued estimates and errors.

The device returns exact integers (F, f*, z*, |S|, per-row predictions); the
quantities the paper reports are ratios of them, formed here as exact rationals
and rounded once to double:
  Z1* = z* / p, p = |S| / M           (reference design, Eq. 2)
  F*  = f* / p                        (Eq. 3)
  Z2* = F z* / f*                     (proposed method, Eq. 4)
  eps1 = (Z1* - Z)/Z, eps_f = (F* - F)/F, eps2 = (Z2* - Z)/Z   (Sec. VI-A)
and Eq. 5 gives eps2 = (eps1 - eps_f) / (1 + eps_f).
"""
from fractions import Fraction

import numpy as np


def estimates(F, Z, f, z, M, S):
    """Dict of the estimates as floats (None where undefined)."""
    q = {}
    q["Z1"] = Fraction(z * M, S) if S else None
    q["F_star"] = Fraction(f * M, S) if S else None
    q["Z2"] = Fraction(F * z, f) if f else None
    q["r_star"] = Fraction(f, z) if z else None
    q["CR"] = Fraction(F, Z) if Z else None
    q["eps1"] = (q["Z1"] - Z) / Z if (S and Z) else None
    q["eps_f"] = (q["F_star"] - F) / F if (S and F) else None
    q["eps2"] = (q["Z2"] - Z) / Z if (f and Z) else None
    return {k: (None if v is None else float(v)) for k, v in q.items()}


def row_errors(pred, nnz):
    """Mean and max of |pred_i - nnz_i| / nnz_i over rows with nnz_i > 0."""
    pred = np.asarray(pred, dtype=np.float64)
    nnz = np.asarray(nnz, dtype=np.float64)
    m = nnz > 0
    if not m.any():
        return {"mean": None, "max": None}
    e = np.abs(pred[m] - nnz[m]) / nnz[m]
    return {"mean": float(e.mean()), "max": float(e.max())}


def accuracy_summary(cases):
    """The statistics of Sec. VI-A over a list of per-case dicts with eps1,
    eps_f, eps2 (cases where an estimate is undefined are left out of it):
    mean and worst |eps| of each, the share of cases where |eps2| < |eps1|
    (ties counted apart), and the correlation of eps1 and eps_f."""
    def col(k):
        return np.array([c[k] for c in cases if c.get(k) is not None], dtype=np.float64)

    out = {"cases": len(cases)}
    for k in ("eps1", "eps_f", "eps2"):
        v = np.abs(col(k))
        out[k] = {"mean_abs": float(v.mean()) if v.size else None, "max_abs": float(v.max()) if v.size else None,
                  "n": int(v.size)}
    both = [c for c in cases if c.get("eps1") is not None and c.get("eps2") is not None]
    if both:
        e1 = np.abs([c["eps1"] for c in both])
        e2 = np.abs([c["eps2"] for c in both])
        out["eps2_better_share"] = float(np.mean(e2 < e1))
        out["tie_share"] = float(np.mean(e2 == e1))
    pair = [c for c in cases if c.get("eps1") is not None and c.get("eps_f") is not None]
    if len(pair) > 1:
        a = np.array([c["eps1"] for c in pair])
        b = np.array([c["eps_f"] for c in pair])
        out["corr_eps1_epsf"] = float(np.corrcoef(a, b)[0, 1]) if a.std() > 0 and b.std() > 0 else None
    return out
