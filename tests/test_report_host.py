"""Host-side statistics of the accuracy report (Sec. VI-A): mean / worst |eps|,
the share of cases where the proposed estimate beats the reference design, and
the correlation of eps1 with eps_f, on hand-made cases with known answers."""
import numpy as np
import pytest

from paper_2207_13848_gb300.report import accuracy_summary, estimates


def test_summary_on_hand_made_cases():
    cases = [dict(eps1=0.10, eps_f=0.08, eps2=0.02),
             dict(eps1=-0.20, eps_f=-0.25, eps2=0.05),
             dict(eps1=0.01, eps_f=0.0, eps2=0.01),
             dict(eps1=None, eps_f=None, eps2=-0.03)]
    s = accuracy_summary(cases)
    assert s["cases"] == 4
    assert s["eps1"]["n"] == 3 and s["eps1"]["mean_abs"] == pytest.approx((0.10 + 0.20 + 0.01) / 3)
    assert s["eps1"]["max_abs"] == pytest.approx(0.20)
    assert s["eps2"]["n"] == 4 and s["eps2"]["max_abs"] == pytest.approx(0.05)
    assert s["eps2_better_share"] == pytest.approx(2 / 3) and s["tie_share"] == pytest.approx(1 / 3)
    a, b = np.array([0.10, -0.20, 0.01]), np.array([0.08, -0.25, 0.0])
    assert s["corr_eps1_epsf"] == pytest.approx(np.corrcoef(a, b)[0, 1])


def test_summary_matches_eq5_on_estimates():
    # Eq. 5: eps2 = (eps1 - eps_f) / (1 + eps_f) for any integers; the summary
    # only aggregates, so it must see the same per-case values
    rng = np.random.default_rng(3)
    cases = []
    for _ in range(50):
        M = int(rng.integers(100, 10000))
        S = int(rng.integers(1, M))
        F = int(rng.integers(1000, 10 ** 7))
        Z = int(rng.integers(1, F))
        f = int(rng.integers(1, F))
        z = int(rng.integers(1, f + 1))
        e = estimates(F, Z, f, z, M, S)
        assert e["eps2"] == pytest.approx((e["eps1"] - e["eps_f"]) / (1 + e["eps_f"]), rel=1e-9, abs=1e-12)
        cases.append(e)
    s = accuracy_summary(cases)
    assert s["eps2"]["mean_abs"] == pytest.approx(np.mean([abs(c["eps2"]) for c in cases]))
