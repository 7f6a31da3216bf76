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
