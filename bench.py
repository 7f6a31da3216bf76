#!/usr/bin/env python3
"""Throughput of the sampled-compression-ratio structure prediction on GB300.

One step = one spgemm_predict_structure call: the Bernoulli row sample, the FLOP
and exact nnz of the sampled rows, the compression ratio, the FLOP of every
row, the per-row prediction and its exclusive scan (every step of the hot
path), on C = A*A with A an Erdos-Renyi matrix, n = 2^20, Poisson(16) entries
per row, uniform columns, 1 % of rows sampled.  Inputs are resident in HBM; the
L2 is flushed (512 MiB write) before every timed step, since the operands
(71 MB) fit in the 129 MB L2.

Prints one JSON line.  Other keys: the roofline of the dominant kernel (the
single-launch predictor, k_predict, which is the whole call; timed with CUDA
events on its stream through the library's profiling hook), the end-to-end number through the public API
with host buffers, the GPU exact symbolic phase on the same input, the
prediction errors (Sec. VI-A), the CPU oracle baseline and the SM clocks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs its own replica (weak scaling).
"""
import argparse
import hashlib
import json
import os
import re
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = ("input-nnz/s and HBM GB/s of prediction vs GPU exact symbolic; "
          "predicted-nnz rel. error")
UNIT = "nnz/s"
TWO32 = 1 << 32
L2_FLUSH_BYTES = 512 << 20
WORKLOAD = {
    "workload": "C=A*A, A Erdos-Renyi n=2^20, Poisson(16) nnz/row, uniform columns, "
                "int32 CSR, Bernoulli 1% row sample",
    "n": 1 << 20, "avg_nnz_per_row": 16, "sample_ratio": 0.01, "gen_seed": 2000,
}


def make_input(rank=0):
    return W.erdos_renyi(WORKLOAD["n"], WORKLOAD["avg_nnz_per_row"], WORKLOAD["gen_seed"] + rank)


def threshold():
    return int(WORKLOAD["sample_ratio"] * TWO32)


# ------------------------------------------------------------------ distribution
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(backend):
    import torch.distributed as dist
    ws, rank, _ = dist_env()
    if ws > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend, rank=rank, world_size=ws)
    return ws, rank


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def aggregate(units_local, seconds_local, device=None):
    """Whole-job throughput of replicas: total units / slowest rank's time."""
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
        s = torch.tensor([float(seconds_local)], dtype=torch.float64, device=device)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        dist.all_reduce(s, op=dist.ReduceOp.MAX)
        return float(u.item()), float(s.item())
    return float(units_local), float(seconds_local)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.exe = shutil.which("nvidia-smi")
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        if not self.exe:
            return
        fd, self.path = tempfile.mkstemp(prefix="clocks.", suffix=".csv")
        os.close(fd)
        self.fh = open(self.path, "w")
        self.proc = subprocess.Popen([self.exe, "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits", "-lms", "100"],
                                     stdout=self.fh, stderr=subprocess.DEVNULL)
        t0 = time.time()
        while time.time() - t0 < 5 and os.path.getsize(self.path) == 0:
            time.sleep(0.05)

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ roofline inputs
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    return 6800.0, "fallback (6.8 TB/s)"


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2207_13848_gb300", "csrc")
    for name in ("common.cuh", "k_flop.cuh", "k_dedup.cuh", "k_predict.cuh"):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of k_predict from the committed ncu summary
    (profiles/k_predict_er_n2e20.json), if it was taken on the current kernel
    source (else None)."""
    path = os.path.join(ROOT, "profiles", "k_predict_er_n2e20.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    if d.get("source_hash") != kernel_source_hash():
        return None
    return int(d["traffic_bytes_per_launch"])


def algorithmic_bytes(A, f_s, n_s):
    """Minimum bytes one prediction must move: A.rpt, A.col and B.rpt once each,
    pred (int32) and offsets (int64) written once, and for the sample the B
    column ids of the sampled rows' products and the sampled rows' A offsets.
    The call is one launch, so this is also the kernel's figure."""
    M, nnz, K = A.rows, A.nnz, A.cols
    return 4 * (M + 1) + 4 * nnz + 4 * (K + 1) + 4 * M + 8 * (M + 1) + 4 * f_s + 8 * n_s


# ------------------------------------------------------------------ CPU oracle baseline
def cpu_oracle_baseline(A, seconds=12.0):
    """The oracle on the machine's host cores, all of them and then one (Sec. VI-B
    protocol for the single core: one warm-up run, the mean of ten)."""
    import oracle
    T = threshold()
    n = 0
    t0 = time.perf_counter()
    while True:
        oracle.predict(A, A, oracle.BERNOULLI, n, T)
        n += 1
        dt = time.perf_counter() - t0
        if dt >= seconds or n >= 200:
            break
    out = {"value": A.nnz * n / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
           "sample": f"the full workload, {n} predictions (seeds 0..{n - 1}), {dt:.1f} s"}
    prev = oracle.num_threads()
    oracle.set_num_threads(1)
    try:
        oracle.predict(A, A, oracle.BERNOULLI, 0, T)  # warm-up
        t1 = time.perf_counter()
        for k in range(10):
            oracle.predict(A, A, oracle.BERNOULLI, k, T)
        d1 = time.perf_counter() - t1
    finally:
        oracle.set_num_threads(prev)
    out["single_core"] = {"value": A.nnz * 10 / d1, "unit": UNIT, "cores": 1, "kind": "oracle",
                          "sample": f"the full workload, one warm-up then the mean of 10 predictions, {d1:.1f} s"}
    return out


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, on the machine's host cores,
    one full prediction of the bench workload per step (same config, metric
    and unit as the GPU arm)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    A = make_input(0)
    T = threshold()
    for k in range(args.warmup):
        oracle.predict(A, A, oracle.BERNOULLI, k, T)
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle.predict(A, A, oracle.BERNOULLI, k, T)
    secs = time.perf_counter() - t0
    value = A.nnz * args.steps / secs
    cb = {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
          "sample": f"the full workload, one prediction per step (seeds 0..{args.steps - 1}), {secs:.1f} s"}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": dict(WORKLOAD, nnz=A.nnz), "same_config": True, "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU arm
CONFIG1 = {"workload": "C=A*A, A 2D 5-point Laplacian on a 64x64 grid (n=4096), int32 CSR, Bernoulli 1% row sample",
           "gen": "laplacian_2d(64)", "sample_ratio": 0.01}
CONFIG3 = {"workload": "C=A*A, A R-MAT scale 20, edge factor 16, (a,b,c,d)=(0.57,0.19,0.19,0.05), duplicates "
                       "merged, int32 CSR, Bernoulli 0.5% row sample", "gen_seed": 3000, "sample_ratio": 0.005}


def measure_config(sp, torch, dev, flush, A, ratio, steps, latency=False):
    """One config beside the headline: the prediction call timed with CUDA
    events (L2 flushed before every step), the exact symbolic phase once, the
    prediction errors, and the HBM fraction of the call (its algorithmic bytes
    include the 4 f* bytes of sampled B column ids)."""
    from paper_2207_13848_gb300.report import estimates
    stream = torch.cuda.current_stream()
    dA = sp.DeviceCSR.from_host(A, dev)
    ws = sp.Workspace.for_operands(dA, dA, dev)
    M = A.rows
    pred = torch.empty(M, dtype=torch.int32, device=dev)
    offs = torch.empty(M + 1, dtype=torch.int64, device=dev)
    res = sp.new_result(dev)
    cfg = sp.config(threshold=int(ratio * TWO32), seed=0)

    def call():
        rc = sp.spgemm_predict_structure(dA, dA, cfg, pred, offs, None, res, ws, stream)
        if rc != sp.OK:
            raise RuntimeError(sp.spgemm_status_string(rc))

    for _ in range(3):
        flush.fill_(1)
        call()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k, (a, b) in enumerate(ev):
        flush.fill_(k & 0xff)
        a.record(stream)
        call()
        b.record(stream)
    torch.cuda.synchronize()
    t = sorted(a.elapsed_time(b) for a, b in ev)
    r = sp.read_result(res)
    if r["status"] & (sp.STATUS_ERR_BAD_INPUT | sp.STATUS_ERR_TIMEOUT):
        raise RuntimeError(f"device status {r['status']}")
    nnz_row = torch.empty(M, dtype=torch.int32, device=dev)
    sres = sp.new_result(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.fill_(2)
    e0.record(stream)
    rc = sp.spgemm_symbolic_exact(dA, dA, nnz_row, offs, sres, ws, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    if rc != sp.OK:
        raise RuntimeError(sp.spgemm_status_string(rc))
    Z = sp.read_result(sres)["pred_total"]
    est = estimates(r["flop_total"], Z, r["flop_s"], r["nnz_s"], M, r["n_sampled"])
    p50 = t[len(t) // 2]
    bytes_ = algorithmic_bytes(A, r["flop_s"], r["n_sampled"])
    peak, peak_src = measured_peaks()
    out = {"steps": steps, "nnz": A.nnz, "n": M, "F": r["flop_total"], "f_s": r["flop_s"], "z_s": r["nnz_s"],
           "n_sampled": r["n_sampled"], "Z": Z,
           "call_us": {"p50": 1e3 * p50, "min": 1e3 * t[0], "mean": 1e3 * sum(t) / len(t)},
           "input_nnz_per_s": A.nnz / (p50 * 1e-3), "sampled_products_per_s": r["flop_s"] / (p50 * 1e-3),
           "roofline": {"bound": "hbm", "achieved": bytes_ / (p50 * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                        "frac": bytes_ / (p50 * 1e-3) / 1e9 / peak, "algorithmic_bytes": bytes_,
                        "peak_source": peak_src},
           "exact_symbolic_us": 1e3 * e0.elapsed_time(e1),
           "accuracy": {"eps1": est["eps1"], "eps_f": est["eps_f"], "eps2": est["eps2"]},
           "l2": "flushed before every step (512 MiB write)"}
    if latency:
        out["latency_us_p50_of_%d" % steps] = 1e3 * p50
    return out


def lookup_ceiling(sp, torch, dev, flush, dA, reps=20):
    """The device's rate of scattered one-byte lookups for this A.col stream
    (spgemm_lookup_probe over a table of A.cols bytes), median of `reps` runs
    with the L2 flushed before each."""
    stream = torch.cuda.current_stream()
    tab = torch.randint(0, 32, (dA.cols,), dtype=torch.uint8, device=dev)
    out = torch.zeros(1, dtype=torch.int64, device=dev)
    for _ in range(3):
        flush.fill_(1)
        if sp.spgemm_lookup_probe(dA.col, tab, out, stream) != sp.OK:
            raise RuntimeError("lookup probe failed")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for k, (a, b) in enumerate(ev):
        flush.fill_(k & 0xff)
        a.record(stream)
        sp.spgemm_lookup_probe(dA.col, tab, out, stream)
        b.record(stream)
    torch.cuda.synchronize()
    t = sorted(a.elapsed_time(b) for a, b in ev)
    return dA.nnz / (t[len(t) // 2] * 1e-3), t[len(t) // 2]


def run_ours(args):
    import torch

    import paper_2207_13848_gb300 as sp
    from paper_2207_13848_gb300 import build as spbuild
    from paper_2207_13848_gb300.report import estimates, row_errors

    nranks, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if nranks > 1:
        init_dist("nccl")
    spbuild.build()

    A = make_input(rank)
    dA = sp.DeviceCSR.from_host(A, dev)
    ws = sp.Workspace.for_operands(dA, dA, dev)
    M = A.rows
    pred = torch.empty(M, dtype=torch.int32, device=dev)
    offsets = torch.empty(M + 1, dtype=torch.int64, device=dev)
    res = sp.new_result(dev)
    cfg = sp.config(threshold=threshold(), seed=0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def predict():
        rc = sp.spgemm_predict_structure(dA, dA, cfg, pred, offsets, None, res, ws, stream)
        if rc != sp.OK:
            raise RuntimeError(sp.spgemm_status_string(rc))

    for _ in range(args.warmup):
        flush.fill_(1)
        predict()
    torch.cuda.synchronize()
    r0 = sp.read_result(res)
    if r0["status"] != 0:
        raise RuntimeError(f"device status {r0['status']}: {sp.spgemm_status_string(r0['status'])}")

    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for a, b in kev:  # torch creates the CUDA event on first record; the hook needs the handle
        a.record(stream)
        b.record(stream)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    for k in range(K):
        flush.fill_(k & 0xff)
        sp.spgemm_set_profile_events(kev[k][0], kev[k][1])
        ev[k][0].record(stream)
        predict()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    sp.spgemm_set_profile_events(None, None)
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    kern_ms = [a.elapsed_time(b) for a, b in kev]
    t_step = sum(step_ms) / K
    t_kern = sum(kern_ms) / K
    units, secs = aggregate(A.nnz * K, sum(step_ms) / 1e3, dev)
    value = units / secs
    r = sp.read_result(res)
    if r["status"] & (sp.STATUS_ERR_BAD_INPUT | sp.STATUS_ERR_TIMEOUT):
        raise RuntimeError(f"device status {r['status']} after the timed steps")
    step_sorted = sorted(step_ms)
    step_dist = {"min": step_sorted[0], "p50": step_sorted[K // 2], "p99": step_sorted[min(K - 1, (99 * K) // 100)],
                 "max": step_sorted[-1]}

    # ---- end to end through the public API with host buffers: every step
    # copies its inputs from pinned host memory, predicts, and copies pred,
    # offsets and the result record back.  Steps are double-buffered over two
    # streams (as a caller serving many predictions would run them), so one
    # step's input copy overlaps the previous step's kernel and output copy;
    # the synchronous per-step latency is reported beside it.
    E = max(3, min(K, args.e2e_steps))
    h_rpt = torch.from_numpy(A.rpt).pin_memory()
    h_col = torch.from_numpy(A.col).pin_memory()

    def e2e_set():
        st_ = torch.cuda.Stream(device=dev)
        return {"stream": st_,
                "A": sp.DeviceCSR(A.rows, A.cols, torch.empty_like(dA.rpt), torch.empty_like(dA.col)),
                "ws": sp.Workspace.for_operands(dA, dA, dev),
                "pred": torch.empty(M, dtype=torch.int32, device=dev),
                "off": torch.empty(M + 1, dtype=torch.int64, device=dev),
                "res": sp.new_result(dev),
                "h_pred": torch.empty(M, dtype=torch.int32).pin_memory(),
                "h_off": torch.empty(M + 1, dtype=torch.int64).pin_memory(),
                "h_res": torch.empty(res.numel(), dtype=torch.int64).pin_memory(),
                "done": torch.cuda.Event()}

    sets = [e2e_set(), e2e_set()]

    def e2e_issue(b):
        with torch.cuda.stream(b["stream"]):
            b["A"].rpt.copy_(h_rpt, non_blocking=True)
            b["A"].col.copy_(h_col, non_blocking=True)
            rc = sp.spgemm_predict_structure(b["A"], b["A"], cfg, b["pred"], b["off"], None, b["res"], b["ws"],
                                             b["stream"])
            if rc != sp.OK:
                raise RuntimeError(sp.spgemm_status_string(rc))
            b["h_pred"].copy_(b["pred"], non_blocking=True)
            b["h_off"].copy_(b["off"], non_blocking=True)
            b["h_res"].copy_(b["res"], non_blocking=True)
            b["done"].record(b["stream"])

    for _ in range(3):  # warm-up, and the synchronous latency
        e2e_issue(sets[0])
        sets[0]["done"].synchronize()
    lat = []
    for _ in range(E):
        t0 = time.perf_counter()
        e2e_issue(sets[0])
        sets[0]["done"].synchronize()
        lat.append(time.perf_counter() - t0)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for k in range(E):
        b = sets[k % 2]
        if k >= 2:
            b["done"].synchronize()  # the set's previous step has fully landed on the host
        e2e_issue(b)
    for b in sets:
        b["done"].synchronize()
    e2e_s = time.perf_counter() - t0
    for b in sets:
        rb = [int(x) for x in b["h_res"].tolist()]
        if rb[4] != int(offsets[-1].item()) or (rb[5] & 0xFFFFFFFF) != 0:
            raise RuntimeError("end-to-end result differs from the device-resident run")
    eu, es = aggregate(A.nnz * E, e2e_s, dev)
    h2d = 4 * (M + 1) + 4 * A.nnz
    d2h = 4 * M + 8 * (M + 1) + sp.RESULT_BYTES
    e2e_latency_ms = 1e3 * statistics.median(lat)

    # ---- GPU exact symbolic phase on the same input
    nnz_row = torch.empty(M, dtype=torch.int32, device=dev)
    sres = sp.new_result(dev)
    S = 5
    sev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(S + 1)]
    for k in range(S + 1):
        flush.fill_(3)
        sev[k][0].record(stream)
        rc = sp.spgemm_symbolic_exact(dA, dA, nnz_row, offsets, sres, ws, stream)
        sev[k][1].record(stream)
        if rc != sp.OK:
            raise RuntimeError(sp.spgemm_status_string(rc))
    torch.cuda.synchronize()
    t_sym = sum(a.elapsed_time(b) for a, b in sev[1:]) / S
    sr = sp.read_result(sres)

    # prediction errors against the exact structure (Sec. VI-A)
    predict()
    torch.cuda.synchronize()
    est = estimates(r["flop_total"], sr["pred_total"], r["flop_s"], r["nnz_s"], M, r["n_sampled"])
    rowerr = row_errors(pred.cpu().numpy(), nnz_row.cpu().numpy())

    kern_bytes = call_bytes = algorithmic_bytes(A, r["flop_s"], r["n_sampled"])
    peak, peak_src = measured_peaks()
    achieved = kern_bytes / (t_kern * 1e-3) / 1e9
    traffic = profiled_traffic()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": nranks, "steps": K,
        "warmup": args.warmup, "ms_per_step": t_step, "step_ms": step_dist, "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": dict(WORKLOAD, nnz=A.nnz, l2="flushed before every timed step (512 MiB write)",
                       parallelism=f"replicas x{nranks}"),
        "hbm_gbs_call": call_bytes / (t_step * 1e-3) / 1e9,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "k_predict<predict> (the whole call: B row-length table, sample, "
                               "FLOP per row, heavy sampled rows, prediction, scan)",
                     "algorithmic_bytes": kern_bytes, "kernel_ms": t_kern, "peak_source": peak_src,
                     "l2_lookups_per_s": A.nnz / (t_kern * 1e-3)},
        "e2e": {"value": eu / es, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": E, "pipelined_streams": 2, "latency_ms_per_step": e2e_latency_ms,
                "host_link_gbs": (h2d + d2h) * E / es / 1e9},
        "gpu_launches": K,
        "exact_symbolic": {"ms": t_sym, "input_nnz_per_s": A.nnz / (t_sym * 1e-3),
                           "prediction_speedup": t_sym / t_step, "Z": sr["pred_total"]},
        "accuracy": {"eps1": est["eps1"], "eps_f": est["eps_f"], "eps2": est["eps2"],
                     "row_rel_err_mean": rowerr["mean"], "row_rel_err_max": rowerr["max"],
                     "F": r["flop_total"], "f_s": r["flop_s"], "z_s": r["nnz_s"],
                     "n_sampled": r["n_sampled"]},
        "clocks": clk,
    }
    # the FLOP pass's own ceiling: scattered lookups at the rate the device
    # sustains for this id stream, measured now on the same input
    ceil_rate, ceil_ms = lookup_ceiling(sp, torch, dev, flush, dA)
    rate = A.nnz / (t_kern * 1e-3)
    line["roofline_lookup"] = {"bound": "l2_lookup_rate", "achieved": rate, "peak": ceil_rate, "unit": "lookups/s",
                               "frac": rate / ceil_rate, "lookups_per_launch": A.nnz,
                               "peak_source": "measured in this run: spgemm_lookup_probe (A.col streamed, one "
                                              "scattered byte lookup per id, nothing else), median of 20, "
                                              f"{1e3 * ceil_ms:.1f} us"}
    if not args.skip_configs:
        cf = {}
        cf["config1_lap2d_64"] = dict(CONFIG1, **measure_config(sp, torch, dev, flush, W.laplacian_2d(64), 0.01,
                                                               100, latency=True))
        cf["config3_rmat_20"] = dict(CONFIG3, **measure_config(sp, torch, dev, flush,
                                                              W.rmat(20, 16, seed=CONFIG3["gen_seed"]), 0.005, 20))
        line["configs"] = cf
    if nranks == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_baseline(A, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ other suites
def _family_job(st, n, v):
    A, B, name = W.family_case(st, n, v)
    return st, n, v, A, (None if B is A else B), name


def family_cases(sizes, variants=range(25), structures=None, workers=None):
    """The synthetic family's cases (structure, n, variant, A, B, name), made
    by worker processes (spawn) in parallel; B is A for the square cases."""
    import multiprocessing as mp
    structures = W.STRUCTURES if structures is None else structures
    jobs = [(st, n, v) for st in structures for n in sizes for v in variants]
    workers = workers or max(1, min(16, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(workers) as pool:
        out = pool.starmap(_family_job, jobs, chunksize=1)
    return [(st, n, v, A, A if B is None else B, name) for st, n, v, A, B, name in out]


def _family_pool(sizes, variants, dev):
    import paper_2207_13848_gb300 as sp
    pool, names = [], []
    for st in W.STRUCTURES:
        for k, n in enumerate(sizes):
            v = variants[k % len(variants)]
            A, B, name = W.family_case(st, n, v)
            dA = sp.DeviceCSR.from_host(A, dev)
            dB = dA if B is A else sp.DeviceCSR.from_host(B, dev)
            pool.append((dA, dB))
            names.append(name)
    return pool, names


def run_serve(args):
    """Serving (continuous batching: admission into stream slots by device
    memory, small waiting requests merged into batched launches): saturation
    throughput, then Poisson arrivals at 0.5x and 0.9x of it; requests mix the
    five family structures at n = 2^12 .. 2^21 (log-uniform), operands resident
    on the device, 1 % Bernoulli sample, fresh seed each.  Beside it, on the
    same request stream: one spgemm_predict_structure call per request back to
    back on one stream (the plain predictor, no server), and the server without
    merging; every served result record equals the sequential one."""
    import torch
    import paper_2207_13848_gb300 as sp
    from paper_2207_13848_gb300 import build as spbuild
    from paper_2207_13848_gb300 import serve
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    spbuild.build()
    sizes = [1 << e for e in range(12, 22)]
    pool, names = _family_pool(sizes, (2, 6, 12), dev)
    n = args.serve_requests
    T = threshold()

    # the plain predictor, one call per request in arrival order on one stream
    def sequential(picks):
        stream = torch.cuda.current_stream()
        wss = {}
        outs = []
        for i, k in enumerate(picks):
            A, B = pool[k]
            if k not in wss:
                wss[k] = sp.Workspace.for_operands(A, B, dev)
            pred = torch.empty(A.rows, dtype=torch.int32, device=dev)
            offs = torch.empty(A.rows + 1, dtype=torch.int64, device=dev)
            outs.append((pred, offs, sp.new_result(dev)))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i, k in enumerate(picks):
            A, B = pool[k]
            pred, offs, res = outs[i]
            rc = sp.spgemm_predict_structure(A, B, sp.config(threshold=T, seed=i), pred, offs, None, res, wss[k],
                                             stream)
            if rc != sp.OK:
                raise RuntimeError(sp.spgemm_status_string(rc))
        torch.cuda.synchronize()
        return time.perf_counter() - t0, outs

    if args.serve_sweep:
        for slots, nst in ((8, 1), (8, 8), (16, 1)):
            for br in (0, 1 << 16, 1 << 18, 1 << 22):
                for mb in (128,):
                    sv = serve.Server(slots=slots, memory_budget=16 << 30, device=dev, batch_rows=br, max_batch=mb,
                                      streams=nst)
                    serve.run_poisson(sv, pool, rate=0, n_requests=min(n, 500), seed=99)
                    d, _ = serve.run_poisson(sv, pool, rate=0, n_requests=n, seed=1)
                    sm = serve.latency_summary(d)
                    print(json.dumps({"slots": slots, "streams": nst, "batch_rows": br, "max_batch": mb,
                                      "req_per_s": n / sm["span"],
                                      "batched_launches": sv.stats.batched_launches, "launches": sv.stats.launches}))
        return 0
    srv = serve.Server(slots=args.serve_slots, memory_budget=16 << 30, device=dev, batch_rows=args.serve_batch_rows,
                       max_batch=args.serve_max_batch, streams=args.serve_streams)
    serve.run_poisson(srv, pool, rate=0, n_requests=min(n, 500), seed=99)  # warm-up (pools, caches)
    done, picks = serve.run_poisson(srv, pool, rate=0, n_requests=n, seed=1)
    sat = serve.latency_summary(done)
    sat_rate = n / sat["span"]
    sequential(picks[:200])  # warm-up
    t_seq, seq_out = sequential(picks)
    seq_rate = n / t_seq
    seq_res = torch.stack([o[2] for o in seq_out]).cpu().tolist()
    same = all([int(x) for x in r.res_host.tolist()] == seq_res[r.index] for r in done)
    nomerge = serve.Server(slots=args.serve_slots, memory_budget=16 << 30, device=dev, batch_rows=0,
                           streams=args.serve_streams)
    serve.run_poisson(nomerge, pool, rate=0, n_requests=min(n, 500), seed=99)
    done_nm, _ = serve.run_poisson(nomerge, pool, rate=0, n_requests=n, seed=1)
    nm = serve.latency_summary(done_nm)
    levels = [{"offered": "all at once", **sat, "req_per_s": sat_rate}]
    for f in (0.5, 0.9):
        done_f, _ = serve.run_poisson(srv, pool, rate=f * sat_rate, n_requests=n, seed=int(10 * f))
        summ = serve.latency_summary(done_f)
        levels.append({"offered": f"{f} x saturation", "offered_req_per_s": f * sat_rate, **summ,
                       "req_per_s": n / summ["span"]})
    done_f, _ = serve.run_poisson(srv, pool, rate=5000.0, n_requests=n, seed=50)  # a fixed absolute load
    summ = serve.latency_summary(done_f)
    levels.append({"offered": "5000 req/s", "offered_req_per_s": 5000.0, **summ, "req_per_s": n / summ["span"]})
    bad = [r for r in srv.finished if int(r.res_host[5]) & 0x300]
    line = {"suite": "serve", "metric": "requests/s and p50/p99 latency of served predictions",
            "n_requests": n, "slots": args.serve_slots, "streams": args.serve_streams, "pool": len(pool),
            "pool_sizes": "n = 2^12..2^21, 5 structures", "batch_rows": srv.batch_rows, "max_batch": srv.max_batch,
            "peak_inflight": srv.stats.peak_inflight, "launches": srv.stats.launches,
            "batched_launches": srv.stats.batched_launches, "batched_requests": srv.stats.batched_requests,
            "error_results": len(bad), "failed": srv.stats.failed, "levels": levels,
            "sequential_plain_predictor": {"req_per_s": seq_rate, "s": t_seq,
                                           "how": "one spgemm_predict_structure per request, same operands and "
                                                  "seeds, back to back on one stream"},
            "server_without_merging": {"req_per_s": n / nm["span"], "p50": nm["p50"], "p99": nm["p99"]},
            "speedup_vs_sequential": sat_rate / seq_rate, "identical_to_sequential": same}
    print(json.dumps(line))
    return 0 if same else 1


def run_batch(args):
    """Batched predictor vs one spgemm_predict_structure launch per case on the
    family (5 structures x n = 2^12..2^20 x 25 variants: 625 cases), same
    results."""
    import torch
    import paper_2207_13848_gb300 as sp
    from paper_2207_13848_gb300 import build as spbuild
    T = threshold()
    exps = tuple(args.batch_sizes)
    fam = family_cases([1 << e for e in exps])  # before the first CUDA call (spawned workers)
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    spbuild.build()
    cases = []
    for st, n, v, A, B, _ in fam:
        dA = sp.DeviceCSR.from_host(A, dev)
        dB = dA if B is A else sp.DeviceCSR.from_host(B, dev)
        cases.append((dA, dB, sp.config(threshold=T, seed=v)))
    del fam
    stream = torch.cuda.current_stream()
    # per-case launches: one workspace and output set per case, allocated up front
    per = []
    for dA, dB, cfg in cases:
        ws = sp.Workspace.for_operands(dA, dB, dev)
        pred = torch.empty(dA.rows, dtype=torch.int32, device=dev)
        offs = torch.empty(dA.rows + 1, dtype=torch.int64, device=dev)
        per.append((dA, dB, cfg, ws, pred, offs, sp.new_result(dev)))

    def per_case():
        for dA, dB, cfg, ws, pred, offs, res in per:
            rc = sp.spgemm_predict_structure(dA, dB, cfg, pred, offs, None, res, ws, stream)
            if rc != sp.OK:
                raise RuntimeError(sp.spgemm_status_string(rc))

    def timed(fn, reps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a, b in ev:
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return sorted(a.elapsed_time(b) for a, b in ev)

    steps = max(3, min(args.steps, 20))
    per_case()
    t_per = timed(per_case, steps)
    batch = sp.Batch(cases, device=dev)
    best, best_ms = batch.autotune(reps=3)
    # both forms with the tuned phases: one persistent launch, one launch per phase
    forms = {}
    for launches in (1, 4):
        tu = sp.tuning(**dict(best.as_dict(), launches=launches))
        batch.prepare(tu)
        batch.run()
        t_f = timed(batch.run, steps)
        forms[f"{launches}_launch" + ("es" if launches > 1 else "")] = {"median_ms": t_f[len(t_f) // 2],
                                                                        "tuning": tu.as_dict()}
    batch.prepare(best)
    batch.run()
    t_batch = timed(batch.run, steps)
    # same integers: every case's result record and offsets[M]
    torch.cuda.synchronize()
    rb = batch.results()
    same = all(sp.read_result(per[i][6]) == rb[i] for i in range(len(cases)))
    line = {"suite": "batch", "metric": "ms per pass over all cases: batched vs per-case launches",
            "n_cases": len(cases), "steps": steps,
            "cases": "5 structures x n=" + ",".join(f"2^{e}" for e in exps) + " x 25 variants (2-64 nnz/row, "
                     "odd variants rectangular), 1% Bernoulli",
            "per_case_ms": {"median": t_per[len(t_per) // 2], "min": t_per[0]},
            "batch_ms": {"median": t_batch[len(t_batch) // 2], "min": t_batch[0]},
            "speedup_median": t_per[len(t_per) // 2] / t_batch[len(t_batch) // 2],
            "tuning": best.as_dict(), "autotune_ms": best_ms, "identical_results": same,
            "forms": forms, "gpu_launches_per_pass": {"per_case": len(cases), "batch": best.launches}}
    print(json.dumps(line))
    return 0 if same else 1


def run_accuracy(args):
    """Accuracy of the proposed estimate (Z2*) against the reference design
    (Z1*) over the synthetic family, as in Sec. VI-A: per case the exact Z from
    the GPU symbolic phase, then mean / worst |eps1|, |eps_f|, |eps2|, the share
    of cases where eps2 beats eps1 and corr(eps1, eps_f), for the 1 % Bernoulli
    sample and the paper's min(0.003 M, 300) draws; over all 625 cases (5
    structures x n = 2^12..2^20 x 25 variants) and per size."""
    import torch
    import paper_2207_13848_gb300 as sp
    from paper_2207_13848_gb300 import build as spbuild
    from paper_2207_13848_gb300.report import accuracy_summary, estimates
    exps = tuple(args.batch_sizes)
    fam = family_cases([1 << e for e in exps])  # before the first CUDA call (spawned workers)
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    spbuild.build()
    per_mode = {"bernoulli_1pct": [], "paper_draws": []}
    by_size = {}
    for st, n, v, A, B, name in fam:
        dA = sp.DeviceCSR.from_host(A, dev)
        dB = dA if B is A else sp.DeviceCSR.from_host(B, dev)
        ws = sp.Workspace.for_operands(dA, dB, dev)
        Z = sp.read_result(sp.symbolic_exact(dA, dB, ws=ws).res)["pred_total"]
        for mode, cfg in (("bernoulli_1pct", sp.config(threshold=threshold(), seed=v)),
                          ("paper_draws", sp.config(mode=sp.SAMPLE_PAPER_DRAW, seed=v))):
            r = sp.read_result(sp.predict_structure(dA, dB, cfg, ws=ws).res)
            est = estimates(r["flop_total"], Z, r["flop_s"], r["nnz_s"], A.rows, r["n_sampled"])
            per_mode[mode].append(dict(case=name, **est))
            by_size.setdefault((mode, n), []).append(dict(case=name, **est))
        del dA, dB, ws
    line = {"suite": "accuracy", "metric": "relative error of the predicted NNZ(C), Sec. VI-A statistics",
            "cases": f"5 structures x n={','.join(f'2^{e}' for e in exps)} x 25 variants ({len(fam)}), "
                     "exact Z from the GPU symbolic phase",
            "paper_context": {"mean_abs": {"eps1": 0.0812, "eps_f": 0.0859, "eps2": 0.0156},
                              "max_abs": {"eps1": 1.58, "eps_f": 1.55, "eps2": 0.25},
                              "eps2_better_share": 0.814, "corr_eps1_epsf": 0.9701,
                              "note": "625 SuiteSparse cross-products on CPUs; context only"},
            "results": {m: accuracy_summary(c) for m, c in per_mode.items()},
            "by_size": {f"{m} n=2^{n.bit_length() - 1}": accuracy_summary(c) for (m, n), c in sorted(by_size.items())}}
    print(json.dumps(line))
    return 0


def run_numeric(args):
    """The consumer of the prediction: the numeric product C = A*B with C
    allocated by the predicted offsets (prediction + numeric pass + compaction to
    the exact CSR) against the precise two-phase method (exact symbolic phase +
    numeric pass into the exact offsets), on the ER bench matrix with fp32
    values and on R-MAT scale 16 (rows overflow there).  L2 flushed before every
    step; CUDA events; device-resident inputs."""
    import torch
    import paper_2207_13848_gb300 as sp
    from paper_2207_13848_gb300 import build as spbuild
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    spbuild.build()
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 << 18, dtype=torch.int32, device=dev)
    peak, peak_src = measured_peaks()
    workloads_ = [
        ("ER n=2^20, Poisson(16) nnz/row, C=A*A, fp32 U(0,1) values, 1% Bernoulli",
         W.erdos_renyi(1 << 20, 16, 2000, values=True), threshold()),
        ("R-MAT scale 16, edge factor 16, C=A*A, fp32 U(0,1) values, 0.5% Bernoulli",
         W.rmat(16, 16, seed=3000, values=True), int(0.005 * TWO32)),
    ]
    out = []
    K = max(3, min(args.steps, 20))
    for name, A, T in workloads_:
        dA = sp.DeviceCSR.from_host(A, dev)
        val = torch.from_numpy(np.asarray(A.val, dtype=np.float32)).to(dev)
        ws = sp.Workspace.for_operands(dA, dA, dev)
        cfg = sp.config(threshold=T, seed=0)
        M = A.rows
        # sizes from one untimed run
        ex = sp.symbolic_exact(dA, dA, ws=ws)
        Z = sp.read_result(ex.res)["pred_total"]
        pr = sp.predict_structure(dA, dA, cfg, ws=ws, want_flop=True)
        presult = sp.read_result(pr.res)
        alloc = presult["pred_total"]
        F = presult["flop_total"]
        nnz_row = torch.empty(M, dtype=torch.int32, device=dev)
        row_start = torch.empty(M, dtype=torch.int64, device=dev)
        nres = sp.new_numeric_result(dev)
        c_col = torch.empty(max(alloc, Z, 1), dtype=torch.int32, device=dev)
        c_val = torch.empty(max(alloc, Z, 1), dtype=torch.float32, device=dev)
        o_rpt = torch.empty(M + 1, dtype=torch.int64, device=dev)
        o_col = torch.empty(max(Z, 1), dtype=torch.int32, device=dev)[:Z]
        o_val = torch.empty(max(Z, 1), dtype=torch.float32, device=dev)[:Z]
        pad_col, pad_val = c_col[:alloc], c_val[:alloc]
        exa_col, exa_val = c_col[:Z], c_val[:Z]

        def ok(*rcs):
            if any(rcs):
                raise RuntimeError("numeric call failed: " + ", ".join(sp.spgemm_status_string(r) for r in rcs if r))

        def precise():
            ok(sp.spgemm_symbolic_exact(dA, dA, ex.pred, ex.offsets, ex.res, ws, stream),
               sp.spgemm_numeric_into(dA, val, dA, val, ex.offsets, exa_col, exa_val, row_start, nnz_row, nres,
                                      ws, stream))

        def into(pool):
            ok(sp.spgemm_predict_structure(dA, dA, cfg, pr.pred, pr.offsets, None, pr.res, ws, stream),
               sp.spgemm_numeric_into(dA, val, dA, val, None if pool else pr.offsets, pad_col, pad_val, row_start,
                                      nnz_row, nres, ws, stream))

        def into_compact(pool):
            into(pool)
            ok(sp.spgemm_numeric_compact(dA, val, dA, val, pad_col, pad_val, row_start, nnz_row, o_rpt, o_col,
                                         o_val, nres, ws, stream))

        def numeric_only():
            ok(sp.spgemm_numeric_into(dA, val, dA, val, None, pad_col, pad_val, row_start, nnz_row, nres, ws, stream))

        def timed(fn):
            for _ in range(3):
                flush.fill_(1)
                fn()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
            for k, (a, b) in enumerate(ev):
                flush.fill_(k & 0xff)
                a.record(stream)
                fn()
                b.record(stream)
            torch.cuda.synchronize()
            t = sorted(a.elapsed_time(b) for a, b in ev)
            return {"median_ms": t[K // 2], "min_ms": t[0]}

        clocks = ClockSampler(0)
        clocks.start()
        t_precise = timed(precise)
        modes = {}
        for mode, pool in (("per_row_shares", False), ("pool_of_predicted_total", True)):
            t_c = timed(lambda: into_compact(pool))
            t_i = timed(lambda: into(pool))
            into(pool)
            torch.cuda.synchronize()
            inf = sp.read_numeric_result(nres)
            into_compact(pool)
            torch.cuda.synchronize()
            modes[mode] = {"overflow_rows": inf["overflow_rows"], "overflow_nnz": inf["overflow_nnz"],
                           "exact_csr_ms": t_c, "speedup_exact_csr": t_precise["median_ms"] / t_c["median_ms"],
                           "row_layout_ms": t_i, "row_layout_complete": inf["overflow_rows"] == 0,
                           "speedup_row_layout": t_precise["median_ms"] / t_i["median_ms"],
                           "status": sp.read_numeric_result(nres)["status"]}
        t_num = timed(numeric_only)
        clk = clocks.stop()
        # algorithmic bytes of the numeric pass: A (= B) read once (rpt, col,
        # val), C written once (col, val) plus nnz_row
        bytes_num = 4 * (M + 1) + 8 * A.nnz + 8 * Z + 4 * M
        ach = bytes_num / (t_num["median_ms"] * 1e-3) / 1e9
        out.append({"workload": name, "nnz_A": A.nnz, "F": F, "Z": Z, "alloc_predicted": alloc,
                    "alloc_over_Z": alloc / Z if Z else None, "flop_over_Z": F / Z if Z else None,
                    "precise_symbolic_plus_numeric": t_precise, "predicted": modes,
                    "numeric_pass": {**t_num, "products_per_s": F / (t_num["median_ms"] * 1e-3),
                                     "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                                                  "frac": ach / peak, "algorithmic_bytes": bytes_num,
                                                  "peak_source": peak_src}},
                    "clocks": clk})
        del c_col, c_val, o_col, o_val
        torch.cuda.empty_cache()
    line = {"suite": "numeric", "metric": "ms per numeric SpGEMM: predicted allocation vs exact symbolic phase",
            "l2": "flushed before every step (512 MiB write)", "steps": K, "results": out}
    print(json.dumps(line))
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--e2e-steps", type=int, default=100)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-configs", action="store_true",
                    help="leave out the 2D 5-point (n=4096) and R-MAT scale 20 measurements")
    ap.add_argument("--suite", choices=("predict", "serve", "batch", "accuracy", "numeric"), default="predict",
                    help="predict (default): the headline line; serve / batch: the serving loop "
                         "and the batched predictor")
    ap.add_argument("--batch-sizes", type=int, nargs="+", default=[12, 14, 16, 18, 20],
                    help="log2 of the family's sizes for --suite batch (default: all five, 625 cases)")
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--serve-slots", type=int, default=3)
    ap.add_argument("--serve-batch-rows", type=int, default=1 << 18,
                    help="requests with at most this many rows are merged into batched launches")
    ap.add_argument("--serve-max-batch", type=int, default=128)
    ap.add_argument("--serve-streams", type=int, default=1, help="CUDA streams the slots run on")
    ap.add_argument("--serve-sweep", action="store_true", help="only the saturation rate for a grid of settings")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.suite == "serve":
        return run_serve(args)
    if args.suite == "batch":
        return run_batch(args)
    if args.suite == "accuracy":
        return run_accuracy(args)
    if args.suite == "numeric":
        return run_numeric(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
