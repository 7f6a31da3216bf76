"""The accuracy study (bench.py --suite accuracy, Sec. VI-A statistics) is
computed from integers the GPU path returns: F, f*, z*, |S| of the prediction
and Z of the exact symbolic phase.  On a subset of the family, both sampling
rules, each equals the oracle's, so the study's errors are the oracle's errors;
the reals formed from them agree with the oracle's own estimates."""
import pytest

import oracle
import paper_2207_13848_gb300 as sp
from paper_2207_13848_gb300.report import estimates
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

SUBSET = [("er", 1 << 12, 0), ("rmat", 1 << 12, 7), ("lap2d", 1 << 14, 4), ("st27", 1 << 12, 13),
          ("blockdiag", 1 << 14, 21), ("rmat", 1 << 14, 24), ("er", 1 << 16, 11)]


@pytest.mark.parametrize("st,n,v", SUBSET)
def test_study_inputs_equal_the_oracle(st, n, v):
    A, B, name = W.family_case(st, n, v)
    dA = sp.DeviceCSR.from_host(A)
    dB = dA if B is A else sp.DeviceCSR.from_host(B)
    ws = sp.Workspace.for_operands(dA, dB)
    Z = sp.read_result(sp.symbolic_exact(dA, dB, ws=ws).res)["pred_total"]
    _, _, Zo = oracle.symbolic_exact(A, B)
    assert Z == Zo, name
    T = int(0.01 * sp.TWO32)
    for cfg, omode, kw in ((sp.config(threshold=T, seed=v), oracle.BERNOULLI, dict(threshold=T)),
                           (sp.config(mode=sp.SAMPLE_PAPER_DRAW, seed=v), oracle.PAPER_DRAW, {})):
        r = sp.read_result(sp.predict_structure(dA, dB, cfg, ws=ws).res)
        o = oracle.predict(A, B, omode, v, **kw)
        for k in ("flop_total", "flop_s", "nnz_s", "n_sampled"):
            assert r[k] == o[k], (name, omode, k, r[k], o[k])
        e = estimates(r["flop_total"], Z, r["flop_s"], r["nnz_s"], A.rows, r["n_sampled"])
        eo = oracle.estimates(o["flop_total"], Zo, o["flop_s"], o["nnz_s"], A.rows, o["n_sampled"])
        for k in ("eps1", "eps_f", "eps2"):
            if eo[k] is None:
                assert e[k] is None
            else:
                assert e[k] == float(eo[k]), (name, k)
