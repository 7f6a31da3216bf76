"""Shared helpers for the GPU parity tests: run the CUDA path through the C ABI
and the oracle on the same seeded inputs, and compare the integers."""
import numpy as np

import oracle
import paper_2207_13848_gb300 as sp
import workloads as W

TWO32 = 1 << 32


def to_dev(m):
    return sp.DeviceCSR.from_host(m)


def gpu_predict(A, B, mode, seed, threshold=0, sample_num=0, reference=False, ws=None, dA=None, dB=None):
    dA = dA or to_dev(A)
    dB = dB or (dA if B is A else to_dev(B))
    cfg = sp.config(mode=mode, threshold=threshold, sample_num=sample_num, seed=seed)
    p = sp.predict_structure(dA, dB, cfg, ws=ws, want_flop=True, reference=reference)
    return dict(pred=p.pred.cpu().numpy(), offsets=p.offsets.cpu().numpy(), flop=p.flop.cpu().numpy(),
                **sp.read_result(p.res))


def wide_hubs(M, K, N, n_hubs, hub_len, row_len, seed):
    """A (M x K): rows 0..n_hubs-1 with hub_len entries, the others 3; B (K x N)
    with row_len entries per row over all N columns: hub rows of hub_len *
    row_len products."""
    rng = np.random.default_rng(seed)
    ra = [np.full(hub_len, i) for i in range(n_hubs)] + [np.repeat(np.arange(n_hubs, M), 3)]
    ca = [rng.choice(K, size=hub_len, replace=False) for _ in range(n_hubs)] + \
         [rng.integers(0, K, size=3 * (M - n_hubs))]
    A = W.from_coo(M, K, np.concatenate(ra), np.concatenate(ca))
    rb = np.repeat(np.arange(K), row_len)
    cb = rng.integers(0, N, size=K * row_len)
    return A, W.from_coo(K, N, rb, cb)


def oracle_predict(A, B, mode, seed, threshold=0, sample_num=0, reference=False):
    fn = oracle.predict_reference if reference else oracle.predict
    return fn(A, B, mode, seed, threshold, sample_num)


def assert_prediction_equal(g, o, what=""):
    M = o["flop"].shape[0]
    assert g["pred"].shape[0] == M and g["offsets"].shape[0] == M + 1
    np.testing.assert_array_equal(g["flop"].astype(np.int64), o["flop"], err_msg=f"flop {what}")
    for k in ("flop_total", "flop_s", "nnz_s", "n_sampled", "pred_total", "status"):
        assert g[k] == o[k], f"{k} {what}: gpu {g[k]} oracle {o[k]}"
    np.testing.assert_array_equal(g["pred"].astype(np.int64), o["pred"], err_msg=f"pred {what}")
    np.testing.assert_array_equal(g["offsets"], o["offsets"], err_msg=f"offsets {what}")


def gpu_symbolic(A, B, ws=None):
    dA = to_dev(A)
    dB = dA if B is A else to_dev(B)
    p = sp.symbolic_exact(dA, dB, ws=ws)
    return p.pred.cpu().numpy(), p.offsets.cpu().numpy(), sp.read_result(p.res)
