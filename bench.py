#!/usr/bin/env python
"""Benchmark: effective TFLOPS (Eq. 4, 2mnk/t) of FP32-accurate two-level Strassen
against the library's own classical tensor-core GEMM at the same accuracy, on GB300.

Default workload: C = A @ B with m = n = k = 16384, A and B uniform[-1, 1] float32
(seeded, synthetic), levels = 2, arithmetic "split3" (FP32 inputs, operand sums split
into BF16 hi/lo, three BF16 tensor-core terms, FP32 accumulation).  A step is one
full library call (beta pass, operand-sum passes, tensor-core kernel) on inputs that
are already resident in HBM; inputs (1 GiB each) are larger than L2, so no flush is
needed between steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle (FP64
classical GEMM in C) on a bounded sample of rows of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "effective TFLOPS (2mnk/t) Strassen vs own classical GEMM on 1 GB300 at stated FP64 error"
UNIT = "TFLOPS"
FALLBACK_PEAK_TFLOPS = 1900.0  # burst bf16, one earlier measurement on a GB300


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=16384, help="m = n")
    ap.add_argument("--k", type=int, default=0, help="inner dimension (default: n)")
    ap.add_argument("--levels", type=int, default=2)
    ap.add_argument("--variant", default="split3")
    ap.add_argument("--algo", default="auto")
    ap.add_argument("--tile-n", type=int, default=0)
    ap.add_argument("--schedule", choices=["auto", "product", "rounds"], default="auto",
                    help="work order of the packed tensor-core kernel (product-major or tile rounds)")
    ap.add_argument("--round-tiles", type=int, default=0,
                    help="tile-rounds schedule: output tiles per round (0 = automatic)")
    ap.add_argument("--err-rows", type=int, default=16)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-seconds", type=float, default=100.0,
                    help="reference arm: CPU seconds for the whole warm-up + timed run")
    ap.add_argument("--no-classical", action="store_true")
    ap.add_argument("--no-fused", action="store_true",
                    help="skip the measurement of the on-chip-sums (fused) algorithm")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the short measurements of the other configurations")
    ap.add_argument("--extra-steps", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true",
                    help="skip the end-to-end measurement through host buffers (sweeps)")
    return ap.parse_args()


DTYPES = {"split3": "bf16x3", "plain_bf16": "bf16", "bf16": "bf16", "f16": "f16"}
TERMS = {"split3": 3, "plain_bf16": 1, "bf16": 1, "f16": 1}


def mma_flops(m, n, k, levels, variant, basis="strassen"):
    """Algorithmic tensor-core work of one product: each level of a basis with R products on
    a g_m x g_k x g_n block grid does R / (g_m g_k g_n) of the classical 2mnk (Strassen 7/8,
    <3,2,3> 15/18), times the tensor-core terms of the arithmetic (split3: 3)."""
    f = 1.0
    if levels >= 1:
        f = 15.0 / 18.0 if basis == "b323" else (7.0 / 8.0) ** levels
    return f * 2.0 * m * n * k * TERMS[variant]


def kernel_name(algo):
    return "fmm_fused_ts_kernel" if algo in ("fused", "hybrid") else "fmm_packed_kernel"


def tensor_peak(peaks):
    """(burst peak, sustained peak, source) in TFLOP/s.  Every timed region of this benchmark
    lasts well under a second, so the burst figure is the denominator; the sustained one
    (seconds of back-to-back GEMMs under the power cap, at a lower clock) is reported beside it."""
    if peaks and "bf16_tflops" in peaks:
        return (float(peaks["bf16_tflops"]), float(peaks.get("bf16_tflops_sustained", 0.0)) or None,
                "measured (burst bf16)")
    return FALLBACK_PEAK_TFLOPS, None, "fallback"


def timed_call(fmm, torch, stream, fn, steps, warmup):
    """Device time per call of fn() (CUDA events on `stream`) and the library's phase
    profile {phase: (ms, launches)} over the timed calls."""
    for _ in range(warmup):
        fn()
    fmm.device_status()
    torch.cuda.synchronize()
    fmm.profile_read()
    fmm.profile_enable(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    fmm.profile_enable(False)
    prof = fmm.profile_read()
    fmm.device_status()
    return e0.elapsed_time(e1) / steps, prof


def workload_name(a, k):
    kind = "square" if k == a.n else "rank-k"
    return f"strassen-L{a.levels}-{a.variant}-{kind}-m{a.n}-n{a.n}-k{k}"


def config_dict(a, k, extra=None):
    d = {
        "workload": workload_name(a, k),
        "m": a.n, "n": a.n, "k": k,
        "levels": a.levels,
        "variant": a.variant,
        "algo": a.algo,
        "schedule": getattr(a, "schedule", "auto"),
        "round_tiles": getattr(a, "round_tiles", 0),
        "inputs": "A, B float32 uniform[-1,1] seeded (synthetic); row-major; alpha=1, beta=0",
        "l2": "inputs larger than L2 (no flush between steps)",
        "comparator": "same library, levels=0, same arithmetic",
    }
    if extra:
        d.update(extra)
    return d


def recorded_traffic(workload):
    """DRAM bytes per launch of the tensor-core kernel from an ncu capture of this workload,
    or None when no capture exists or the kernel's sources changed since it was taken."""
    import glob
    import hashlib
    for path in glob.glob(os.path.join(ROOT, "profiles", "*_traffic_*.json")):
        try:
            with open(path) as f:
                rec = json.load(f)
        except (OSError, ValueError):
            continue
        if rec.get("workload") != workload:
            continue
        h = hashlib.sha256()
        try:
            for src in rec["source_files"]:
                with open(os.path.join(ROOT, src), "rb") as f:
                    h.update(f.read())
        except OSError:
            continue
        if h.hexdigest() == rec.get("source_sha256"):
            return rec["dram_bytes_read"] + rec["dram_bytes_write"]
    return None


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f)
    except OSError:
        return None


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock/throttle samples every 50 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "50"]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self.proc = subprocess.Popen(cmd, stdout=self.tmp, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = [r.strip().split(",") for r in self.tmp.read().splitlines() if r.strip()]
        self.tmp.close()
        os.unlink(self.tmp.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for name, val in zip(names, r[5:9]):
                if val.strip().lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------- multi-rank helpers
def max_over_ranks(x, dist=None, device="cpu"):
    """The largest of every rank's x (the slowest rank's time); x itself with one rank."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, flops_per_rank, ms):
    """Whole-job effective TFLOPS: every rank's product counted, over the slowest rank's
    time (weak scaling: each rank multiplies its own problem of the same shape)."""
    return world * flops_per_rank / (ms * 1e-3) * 1e-12


def rank_problem(n, k, rank):
    """The seeded synthetic problem of one rank (replicas: a different problem per rank)."""
    return synth.uniform((n, k), 1234 + 2 * rank), synth.uniform((k, n), 1235 + 2 * rank)


# ------------------------------------------------------------- other configurations
def sampled_error(oracle, C_d, A, B, rows, a_code=None, b_code=None):
    """Normwise FP64 error of the sampled rows of C_d (A, B: host arrays, FP32 or 16-bit codes)."""
    import torch
    C_s = C_d[torch.from_numpy(rows).to(C_d.device)].cpu().numpy()
    kw = {}
    if a_code is not None:
        kw = {"a_code": a_code, "b_code": b_code}
    C64 = oracle.classical(A, B, rows=rows, **kw)
    Af = A.astype(np.float64) if a_code is None else None
    if a_code is not None:
        import torch as _t
        conv = (lambda X: _t.from_numpy(X.view(np.int16)).view(_t.bfloat16 if a_code == oracle.ORC_BF16
                                                                 else _t.float16).float().numpy())
        Af, Bf = conv(A).astype(np.float64), conv(B).astype(np.float64)
    else:
        Bf = B.astype(np.float64)
    return oracle.normwise_error(C_s, C64, np.linalg.norm(Af[rows]), np.linalg.norm(Bf))


def run_extras(a, fmm, torch, dev, stream, peak, peak_src):
    """Short device-timed runs of the other configurations, each against the classical
    product of the same arithmetic, with its sampled FP64 error and its tensor-core kernel's
    roofline.  Inputs are synthetic and seeded (shapes and distributions of each config)."""
    import oracle
    steps, warm = max(1, a.extra_steps), 1
    out = []

    def entry(workload, cfg, m, n, k, runs, flops, err_of, comparator_levels=0):
        """runs: {label: (levels, variant, basis, fn)}; the first label is the Strassen choice."""
        e = {"config": dict(workload=workload, m=m, n=n, k=k, **cfg)}
        for label, (lv, variant, basis, fn) in runs.items():
            ms, prof = timed_call(fmm, torch, stream, fn, steps, warm)
            ker_ms = prof["tensor"][0] / steps
            mma = mma_flops(m, n, k, lv, variant, basis) * (flops / (2.0 * m * n * k))
            r = {"levels": lv, "variant": variant, "basis": basis,
                 "value": flops / (ms * 1e-3) * 1e-12, "ms_per_step": ms,
                 "roofline": {"bound": "tensor",
                              "kernel": ("fmm_fused_ts_kernel" if label.startswith(("hybrid", "fused"))
                                         else "fmm_packed_kernel"),
                              "kernel_ms_per_step": ker_ms,
                              "launches_per_step": prof["tensor"][1] / steps,
                              "achieved": mma / (ker_ms * 1e-3) * 1e-12 if ker_ms > 0 else None,
                              "peak": peak, "unit": "TFLOP/s", "peak_source": peak_src}}
            if ker_ms > 0:
                r["roofline"]["frac"] = r["roofline"]["achieved"] / peak
            fn()
            torch.cuda.synchronize()
            r["fp64_normwise_err_sampled"] = err_of()
            e[label] = r
        labels = list(runs)
        if "classical" in e and labels[0] != "classical":
            e["speedup_vs_classical"] = e[labels[0]]["value"] / e["classical"]["value"]
        out.append(e)

    def split3_runs(Ad, Bd, Cd, ws, choices, variant="split3"):
        runs = {}
        for label, lv, basis in choices:
            runs[label] = (lv, variant, basis,
                           (lambda lv=lv, basis=basis: fmm.gemm(Ad, Bd, Cd, 1.0, 0.0, levels=lv, variant=variant,
                                                               basis=basis, workspace=ws, stream=stream)))
        return runs

    def ws_for(m, n, k, choices, variant="split3"):
        need = max(fmm.workspace_size(m, n, k, lv, variant, basis=basis) for _, lv, basis in choices)
        return torch.empty(max(need, 256), dtype=torch.uint8, device=dev)

    # rank-k: m = n = 16384, k in {512, 1024, 2048}, uniform[-1, 1], split3
    for k in (512, 1024, 2048):
        m = n = 16384
        A, B = synth.uniform((m, k), 1300 + k), synth.uniform((k, n), 1301 + k)
        Ad, Bd = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
        Cd = torch.empty((m, n), dtype=torch.float32, device=dev)
        ch = [("strassen_L1", 1, "strassen"), ("classical", 0, "strassen")]
        ws = ws_for(m, n, k, ch)
        rows = np.unique(synth.rng(k).integers(0, m, size=8))
        entry(f"strassen-L1-split3-rank-k-m{m}-n{n}-k{k}", {"variant": "split3",
              "inputs": "uniform[-1,1] float32, seeded"}, m, n, k, split3_runs(Ad, Bd, Cd, ws, ch),
              2.0 * m * n * k, lambda: sampled_error(oracle, Cd, A, B, rows))
        del Ad, Bd, Cd, ws

    # <3,2,3> basis at 12288^3 (blocks divide into whole 256-row tiles)
    m = n = k = 12288
    A, B = synth.uniform((m, k), 1400), synth.uniform((k, n), 1401)
    Ad, Bd = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
    Cd = torch.empty((m, n), dtype=torch.float32, device=dev)
    ch = [("b323_L1", 1, "b323"), ("strassen_L1", 1, "strassen"), ("classical", 0, "strassen")]
    ws = ws_for(m, n, k, ch)
    rows = np.unique(synth.rng(12288).integers(0, m, size=8))
    entry("b323-L1-split3-square-m12288-n12288-k12288", {"variant": "split3",
          "inputs": "uniform[-1,1] float32, seeded"}, m, n, k, split3_runs(Ad, Bd, Cd, ws, ch),
          2.0 * m * n * k, lambda: sampled_error(oracle, Cd, A, B, rows))
    del Ad, Bd, Cd, ws, A, B

    # C5: 30001 x 29999 x 4097, N(0, 1), tight (odd) leading dimensions
    m, n, k = 30001, 29999, 4097
    A, B = synth.gaussian((m, k), 1500), synth.gaussian((k, n), 1501)
    Ad, Bd = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
    Cd = torch.empty((m, n), dtype=torch.float32, device=dev)
    rows = np.unique(np.concatenate([[0, m - 1], synth.rng(30001).integers(0, m, size=6)]))
    for variant in ("split3", "plain_bf16"):
        ch = [("strassen_L2", 2, "strassen"), ("strassen_L1", 1, "strassen"), ("classical", 0, "strassen")]
        ws = ws_for(m, n, k, ch, variant)
        wsh = torch.empty(max(fmm.workspace_size(m, n, k, 2, variant, "hybrid"), 256), dtype=torch.uint8,
                          device=dev)
        runs = split3_runs(Ad, Bd, Cd, ws, ch, variant)
        # the same product with the 49 bottom-level operand sums formed on chip (hybrid scheme)
        runs["hybrid_L2"] = (2, variant, "strassen",
                             lambda v=variant, w=wsh: fmm.gemm(Ad, Bd, Cd, 1.0, 0.0, levels=2, variant=v,
                                                               algo="hybrid", workspace=w, stream=stream))
        entry(f"strassen-{variant}-odd-m{m}-n{n}-k{k}", {"variant": variant, "lda": k, "ldb": n, "ldc": n,
              "inputs": "N(0,1) float32, seeded; tight (odd) leading dimensions"}, m, n, k,
              runs, 2.0 * m * n * k, lambda: sampled_error(oracle, Cd, A, B, rows))
        del ws, wsh
    del Ad, Bd, Cd, A, B

    # C3: BF16 linear layer, forward C = A B and backward dA = dC B^T, dB = A^T dC
    m, k, n = 8192, 4096, 4096
    A = synth.gaussian((m, k), 1600)
    B = synth.gaussian((k, n), 1601)
    G = synth.gaussian((m, n), 1602)
    Ad = torch.from_numpy(A).to(dev).to(torch.bfloat16)
    Bd = torch.from_numpy(B).to(dev).to(torch.bfloat16)
    Gd = torch.from_numpy(G).to(dev)
    Cd = torch.empty((m, n), dtype=torch.float32, device=dev)
    runs = {}
    for label, lv in (("strassen_L1", 1), ("strassen_L2", 2), ("classical", 0)):
        wsf = torch.empty(max(fmm.workspace_size(m, n, k, lv, "bf16"), 256), dtype=torch.uint8, device=dev)
        wsb = torch.empty(max(fmm.workspace_size_backward(m, n, k, lv, "bf16"), 256), dtype=torch.uint8,
                          device=dev)

        def layer(lv=lv, wsf=wsf, wsb=wsb):
            fmm.gemm(Ad, Bd, Cd, 1.0, 0.0, levels=lv, variant="bf16", workspace=wsf, stream=stream)
            fmm.gemm_backward(Ad, Bd, Gd, levels=lv, variant="bf16", workspace=wsb, stream=stream)
        runs[label] = (lv, "bf16", "strassen", layer)
    Ab = Ad.cpu().view(torch.int16).numpy().view(np.uint16)
    Bb = Bd.cpu().view(torch.int16).numpy().view(np.uint16)
    rows = np.unique(synth.rng(8192).integers(0, m, size=6))
    entry(f"strassen-bf16-linear-fwd-bwd-m{m}-k{k}-n{n}", {"variant": "bf16",
          "step": "forward C = A B, backward dA = dC B^T and dB = A^T dC (three products)",
          "inputs": "N(0,1) cast to BF16, dC N(0,1) float32, seeded"}, m, n, k, runs,
          3 * 2.0 * m * n * k,
          lambda: sampled_error(oracle, Cd, Ab, Bb, rows, oracle.ORC_BF16, oracle.ORC_BF16))
    del Ad, Bd, Gd, Cd, runs

    # the C3 layer shape in FP32 with every operand sum formed on chip: forward (fused kernel)
    # and backward (the same kernel on the transposed tiles), against the classical layer
    m, k, n = 8192, 4096, 4096
    A = synth.gaussian((m, k), 1610)
    B = synth.gaussian((k, n), 1611)
    G = synth.gaussian((m, n), 1612)
    Ad, Bd, Gd = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev), torch.from_numpy(G).to(dev)
    Cd = torch.empty((m, n), dtype=torch.float32, device=dev)
    runs = {}
    for label, lv, algo in (("fused_L1", 1, "fused"), ("classical", 0, "auto")):
        wsf = torch.empty(max(fmm.workspace_size(m, n, k, lv, "split3", algo), 256), dtype=torch.uint8, device=dev)
        wsb = torch.empty(max(fmm.workspace_size_backward(m, n, k, lv, "split3"), 256), dtype=torch.uint8,
                          device=dev)

        def layer32(lv=lv, algo=algo, wsf=wsf, wsb=wsb):
            fmm.gemm(Ad, Bd, Cd, 1.0, 0.0, levels=lv, algo=algo, workspace=wsf, stream=stream)
            fmm.gemm_backward(Ad, Bd, Gd, levels=lv, algo=algo, workspace=None if algo == "fused" else wsb,
                              stream=stream)
        runs[label] = (lv, "split3", "strassen", layer32)
    rows = np.unique(synth.rng(8193).integers(0, m, size=6))
    entry(f"strassen-split3-linear-fwd-bwd-on-chip-m{m}-k{k}-n{n}", {"variant": "split3",
          "step": "forward C = A B, backward dA = dC B^T and dB = A^T dC; operand sums formed on chip",
          "inputs": "N(0,1) float32, seeded"}, m, n, k, runs, 3 * 2.0 * m * n * k,
          lambda: sampled_error(oracle, Cd, A, B, rows))
    del Ad, Bd, Gd, Cd, runs

    # C4: 256 uneven FP16 products (multiples of 256 in [1024, 8192]) in one persistent
    # launch per tile width, replayed from a CUDA graph; the built-in FP16 table
    shapes = synth.uneven_batch(256, seed=2024)
    g = torch.Generator(device=dev).manual_seed(2025)
    As = [(torch.rand((mm, kk), device=dev, generator=g) * 2 - 1).half() for mm, nn, kk in shapes]
    Bs = [(torch.rand((kk, nn), device=dev, generator=g) * 2 - 1).half() for mm, nn, kk in shapes]
    Cs = [torch.empty((mm, nn), dtype=torch.float32, device=dev) for mm, nn, kk in shapes]
    plan = fmm.BatchedPlan(As, Bs, Cs, variant="f16")
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        plan.execute(side)
    stream.wait_stream(side)
    torch.cuda.synchronize()
    with torch.cuda.graph(graph):
        plan.execute()
    flops = sum(2.0 * mm * nn * kk for mm, nn, kk in shapes)
    ms, prof = timed_call(fmm, torch, stream, graph.replay, steps, warm)
    levels_used = sorted({fmm.tune_select(mm, nn, kk, fmm.tune_table(None, "f16"))[0] for mm, nn, kk in shapes})
    i0 = 0
    mm, nn, kk = shapes[i0]
    rsel = np.unique(synth.rng(2026).integers(0, mm, size=4))
    Ab = As[i0].cpu().view(torch.int16).numpy().view(np.uint16)
    Bb = Bs[i0].cpu().view(torch.int16).numpy().view(np.uint16)
    out.append({"config": {"workload": "batched-f16-256-uneven-1024to8192-graph", "problems": 256,
                           "variant": "f16", "levels_used": levels_used,
                           "inputs": "uniform[-1,1] FP16, m, n, k uniform over multiples of 256 in [1024, 8192]"},
                "batched": {"value": flops / (ms * 1e-3) * 1e-12, "ms_per_step": ms,
                            "fp64_normwise_err_sampled_problem0": sampled_error(
                                oracle, Cs[i0], Ab, Bb, rsel, oracle.ORC_F16, oracle.ORC_F16)}})
    plan.close()
    del As, Bs, Cs, graph
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------- oracle arm
def cpu_oracle_rate(A, B, target_s, rows_hint=None):
    """Time the FP64 classical oracle on a sample of output rows.  Returns
    (TFLOPS, seconds, rows, cores)."""
    import oracle
    oracle.build()
    cores = oracle.num_threads()
    n, k = B.shape[1], A.shape[1]
    if rows_hint is None:
        probe = np.arange(cores) % A.shape[0]
        t0 = time.perf_counter()
        oracle.classical(A, B, rows=probe)
        t1 = time.perf_counter() - t0
        reps = max(1, int(target_s / max(t1, 1e-3)))
        rows_hint = cores * reps
    rows = np.arange(rows_hint) % A.shape[0]
    t0 = time.perf_counter()
    oracle.classical(A, B, rows=rows)
    dt = time.perf_counter() - t0
    return 2.0 * len(rows) * n * k / dt * 1e-12, dt, len(rows), cores


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    k = a.k or a.n
    A = synth.uniform((a.n, k), 1234)
    B = synth.uniform((k, a.n), 1235)
    import oracle
    oracle.build()
    cores = oracle.num_threads()
    # size one step so that warmup + steps end within about two minutes
    budget = a.ref_seconds / max(1, a.steps + a.warmup)
    _, _, rows, _ = cpu_oracle_rate(A, B, budget)
    for _ in range(a.warmup):
        cpu_oracle_rate(A, B, budget, rows_hint=rows)
    times = []
    for _ in range(a.steps):
        _, dt, _, _ = cpu_oracle_rate(A, B, budget, rows_hint=rows)
        times.append(dt)
    t = sum(times) / len(times)
    val = 2.0 * rows * a.n * k / t * 1e-12
    sample = f"{rows} of {a.n} output rows per step (FP64 classical oracle, all columns)"
    line = {
        "impl": "reference",
        "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(a, k),
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
def main():
    a = parse_args()
    if a.impl == "reference":
        return run_reference(a)

    import torch
    import paper_1808_07984_gb300 as fmm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    fmm.build()
    fmm.load()
    k = a.k or a.n
    m = n = a.n
    # replicas: each rank multiplies its own seeded problem of the same shape
    A, B = rank_problem(n, k, rank)
    A_h = torch.from_numpy(A).pin_memory()
    B_h = torch.from_numpy(B).pin_memory()
    C_h = torch.empty((m, n), dtype=torch.float32).pin_memory()
    A_d = A_h.to(dev)
    B_d = B_h.to(dev)
    C_d = torch.empty((m, n), dtype=torch.float32, device=dev)
    ws_bytes = max(fmm.workspace_size(m, n, k, a.levels, a.variant, a.algo, a.tile_n),
                   0 if a.no_classical else fmm.workspace_size(m, n, k, 0, a.variant, a.algo, a.tile_n))
    ws = torch.empty(max(ws_bytes, 256), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step(levels, algo=None, fused_kernel="auto"):
        fmm.gemm(A_d, B_d, C_d, 1.0, 0.0, levels=levels, variant=a.variant, algo=algo or a.algo,
                 tile_n=0 if algo else a.tile_n, workspace=ws, stream=stream, fused_kernel=fused_kernel,
                 schedule="auto" if algo else a.schedule, round_tiles=0 if algo else a.round_tiles)

    def barrier():
        if dist is not None:
            dist.barrier()

    def slowest(x):
        return max_over_ranks(x, dist, dev)

    def timed(levels, steps, warmup, profile=False, algo=None, fused_kernel="auto"):
        for _ in range(warmup):
            step(levels, algo, fused_kernel)
        fmm.device_status()
        barrier()
        torch.cuda.synchronize()
        if profile:
            fmm.profile_read()
            fmm.profile_enable(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step(levels, algo, fused_kernel)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        prof = None
        if profile:
            fmm.profile_enable(False)
            prof = fmm.profile_read()
        fmm.device_status()
        return e0.elapsed_time(e1) / steps, prof

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None

    # ---- Strassen, device-resident (the headline value)
    for _ in range(a.warmup):
        step(a.levels)
    clocks = ClockSampler(uuid)
    clocks.start()
    ms, prof = timed(a.levels, a.steps, 0, profile=True)
    clk = clocks.stop()
    ms = slowest(ms)
    flops = 2.0 * m * n * k
    value = job_value(world, flops, ms)

    # ---- classical comparator at the same arithmetic
    classical = None
    if not a.no_classical:
        ms0, prof0 = timed(0, a.steps, a.warmup, profile=True)
        ms0 = slowest(ms0)
        classical = {"value": job_value(world, flops, ms0), "ms_per_step": ms0,
                     "tensor_kernel_ms": prof0["tensor"][0] / max(prof0["tensor"][1], 1)}

    # ---- the same product with the operand sums formed on chip while the source tiles load
    # (the fused algorithm: no workspace, sums never in HBM), measured beside the default
    fused = None
    do_fused = (not a.no_fused and a.algo == "auto" and a.variant in ("split3", "plain_bf16")
                and a.levels in (1, 2))
    on_chip = [("fused", "tmem", "fused: operand sums formed on chip as the tiles load; A-operand sums in "
                                 "tensor memory, B-operand sums in shared memory; no workspace"),
               ("fused_smem", "smem", "fused: operand sums formed on chip, both operands' sums written to "
                                      "shared memory; no workspace")]
    if a.levels == 2:
        on_chip.append(("hybrid", "tmem", "hybrid: the seven top-level sums materialised in FP32, the 49 "
                                          "bottom-level products' sums formed on chip (A in tensor memory)"))
    if do_fused:
        fused = {}
        fsteps = max(1, min(a.steps, 5))
        for key, fk, desc in on_chip:
            algo = "hybrid" if key == "hybrid" else "fused"
            msf, proff = timed(a.levels, fsteps, 1, profile=True, algo=algo, fused_kernel=fk)
            msf = slowest(msf)
            ker = proff["tensor"][0] / max(proff["tensor"][1], 1)
            mma = mma_flops(m, n, k, a.levels, a.variant)
            fused[key] = {"algo": desc, "value": job_value(world, flops, msf), "ms_per_step": msf,
                          "steps": fsteps, "tensor_kernel_ms": ker,
                          "tensor_kernel_tflops": mma / (ker * 1e-3) * 1e-12,
                          "kernel": "fmm_fused_ts_kernel" if fk == "tmem" else "fmm_fused_kernel"}

    # ---- end to end through host buffers: every step copies its A, B from pinned host memory
    # and its C back to pinned host memory inside the timed region.  Two device buffer sets
    # and three streams (H2D, compute, D2H) let the copies of one step overlap the products
    # of its neighbours, as a serving loop would run.
    e2e = None
    if not a.no_e2e:
        bufs = [(A_d, B_d, C_d)] + [(torch.empty_like(A_d), torch.empty_like(B_d), torch.empty_like(C_d))]
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
        C_hs = [C_h, torch.empty_like(C_h).pin_memory()]

        def e2e_loop(nsteps):
            # buffer set b: step i's inputs may be overwritten once step i-2's product has read
            # them, its C once step i-2's result has been copied out; so the input copies of one
            # step and the output copy of another run at the same time (both directions of the
            # host link) while a third step's product computes
            ev_in = [torch.cuda.Event() for _ in range(2)]
            ev_done = [None, None]
            ev_free = [None, None]
            for i in range(nsteps):
                b = i % 2
                Ab, Bb, Cb = bufs[b]
                with torch.cuda.stream(s_in):
                    if ev_done[b] is not None:
                        s_in.wait_event(ev_done[b])
                    Ab.copy_(A_h, non_blocking=True)
                    Bb.copy_(B_h, non_blocking=True)
                    ev_in[b].record(s_in)
                stream.wait_event(ev_in[b])
                if ev_free[b] is not None:
                    stream.wait_event(ev_free[b])
                fmm.gemm(Ab, Bb, Cb, 1.0, 0.0, levels=a.levels, variant=a.variant, algo=a.algo,
                         tile_n=a.tile_n, workspace=ws, stream=stream, schedule=a.schedule,
                         round_tiles=a.round_tiles)
                ev_done[b] = torch.cuda.Event()
                ev_done[b].record(stream)
                with torch.cuda.stream(s_out):
                    s_out.wait_event(ev_done[b])
                    C_hs[b].copy_(Cb, non_blocking=True)
                    ev_free[b] = torch.cuda.Event()
                    ev_free[b].record(s_out)
            stream.wait_stream(s_in)
            stream.wait_stream(s_out)

        e2e_loop(max(2, a.warmup))
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s_in.wait_stream(stream)
        s_out.wait_stream(stream)
        e2e_loop(a.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        fmm.device_status()
        ms_e2e = slowest(e0.elapsed_time(e1) / a.steps)
        e2e = {"value": job_value(world, flops, ms_e2e), "unit": UNIT,
               "h2d_bytes_per_step": int(A_h.numel() * 4 + B_h.numel() * 4),
               "d2h_bytes_per_step": int(C_h.numel() * 4), "ms_per_step": ms_e2e,
               "overlap": "H2D, compute and D2H on three streams, two device buffer sets; the H2D of "
                          "one step, the D2H of another and the product of a third run concurrently"}
        del bufs

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    # ---- accuracy vs the FP64 oracle on sampled rows (rank 0's problem)
    import oracle
    step(a.levels)
    torch.cuda.synchronize()
    rows = np.unique(synth.rng(7).integers(0, m, size=a.err_rows))
    C_s = C_d[torch.from_numpy(rows).to(dev)].cpu().numpy()
    C64 = oracle.classical(A, B, rows=rows)
    err = oracle.normwise_error(C_s, C64, np.linalg.norm(A[rows].astype(np.float64)),
                                np.linalg.norm(B.astype(np.float64)))
    err0 = None
    if not a.no_classical:
        step(0)
        torch.cuda.synchronize()
        C_s0 = C_d[torch.from_numpy(rows).to(dev)].cpu().numpy()
        err0 = oracle.normwise_error(C_s0, C64, np.linalg.norm(A[rows].astype(np.float64)),
                                     np.linalg.norm(B.astype(np.float64)))
        classical["fp64_normwise_err_sampled"] = err0
    if fused is not None:
        for key, fk, _ in on_chip:
            step(a.levels, "hybrid" if key == "hybrid" else "fused", fk)
            torch.cuda.synchronize()
            C_sf = C_d[torch.from_numpy(rows).to(dev)].cpu().numpy()
            fused[key]["fp64_normwise_err_sampled"] = oracle.normwise_error(
                C_sf, C64, np.linalg.norm(A[rows].astype(np.float64)), np.linalg.norm(B.astype(np.float64)))

    # ---- roofline of the dominant kernel (the tensor-core kernel)
    # per launch of the tensor-core kernel (a pipelined product launches it once per
    # top-level product, each with 1/7 of the work)
    launches_per_step = max(prof["tensor"][1], 1) / a.steps
    ker_ms = prof["tensor"][0] / max(prof["tensor"][1], 1)
    per_launch = mma_flops(m, n, k, a.levels, a.variant) / launches_per_step
    achieved = per_launch / (ker_ms * 1e-3) * 1e-12
    peaks = load_peaks()
    peak, sustained, peak_src = tensor_peak(peaks)
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": (recorded_traffic(workload_name(a, k))
                            if a.schedule == "auto" and a.round_tiles == 0 else None),
                "frac_of_sustained_peak": (achieved / sustained) if sustained else None,
                "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                "peak_source": peak_src + " of measured; timed region " +
                               f"{a.steps * ms / 1e3:.2f} s",
                "kernel": kernel_name(a.algo), "kernel_ms": ker_ms,
                "launches_per_step": launches_per_step,
                "algorithmic_flops_per_launch": per_launch}
    # ---- roofline of the HBM-bound passes: the operand-sum passes (A and B) and the beta pass
    hbm = float(peaks["hbm_gbs"]) if peaks and "hbm_gbs" in peaks else None
    in_b = 2 if a.variant in ("bf16", "f16") else 4
    out_b = 2 * (2 if a.variant == "split3" else 1)  # BF16/FP16 per stored term
    g = 1 << a.levels
    blk = (lambda d: d) if a.levels == 0 else (lambda d: -(-(-(-d // g)) // 8) * 8)
    hm, hn, hk = blk(m), blk(n), blk(k)
    sum_bytes = in_b * (m * k + k * n) + out_b * 7 ** a.levels * (hm * hk + hk * hn)
    pack_ms = prof["pack"][0] / a.steps
    beta_ms = prof["beta"][0] / a.steps
    passes = {
        "operand_sums": {"bound": "hbm", "algorithmic_bytes_per_step": sum_bytes, "ms_per_step": pack_ms,
                         "achieved_gbs": sum_bytes / (pack_ms * 1e-3) * 1e-9 if pack_ms > 0 else None},
        "beta": {"bound": "hbm",
                 "kind": (("none: the classical product stores C (beta = 0)" if a.levels == 0 else
                           "none: the first update of each C block stores it (store-first launch phases)")
                          if prof["beta"][1] == 0 else "C zeroed by cudaMemsetAsync (beta = 0)"),
                 "algorithmic_bytes_per_step": 4 * m * n, "ms_per_step": beta_ms,
                 "achieved_gbs": 4 * m * n / (beta_ms * 1e-3) * 1e-9 if beta_ms > 0 else None},
        "peak_gbs": hbm, "peak_source": "measured (HBM copy)" if hbm else None,
    }
    for v in (passes["operand_sums"], passes["beta"]):
        v["frac"] = (v["achieved_gbs"] / hbm) if (hbm and v["achieved_gbs"]) else None
    phases = {p: {"ms_per_step": v[0] / a.steps, "launches": v[1]} for p, v in prof.items()}
    # kernels of this library only: with beta = 0 and dense rows the beta phase is a
    # cudaMemsetAsync, not a kernel of ours
    gpu_launches = int(prof["pack"][1] + prof["tensor"][1])

    # ---- the other configurations, short runs (one GPU only)
    extra = None
    if not a.no_extra and world == 1:
        del A_d, B_d, C_d, ws
        torch.cuda.empty_cache()
        try:
            extra = run_extras(a, fmm, torch, dev, stream, peak, peak_src + " of measured")
        except Exception as exc:  # noqa: BLE001 - reported in the line, the headline stands
            extra = {"error": f"{type(exc).__name__}: {exc}"}

    cpu = None
    if not a.no_cpu_baseline:
        v, dt, nrows, cores = cpu_oracle_rate(A, B, a.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{nrows} of {m} output rows of the same product (FP64 classical oracle), "
                         f"{dt:.1f} s"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPES[a.variant], "data": "synthetic",
        "config": config_dict(a, k, {"parallelism": f"replicas{world}" if world > 1 else "single"}),
        "fp64_normwise_err_sampled": err,
        "classical": classical,
        "fused": fused,
        "speedup_vs_classical": (value / classical["value"]) if classical else None,
        "phases": phases,
        "roofline": roofline,
        "hbm_passes": passes,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk,
        "gpu_launches": gpu_launches,
        "extra": extra,
    }
    print(json.dumps(line), flush=True)
    print(f"[bench] {workload_name(a, k)}: {value:.1f} eff TFLOPS ({ms:.2f} ms/step), "
          f"classical {classical['value'] if classical else float('nan'):.1f}, "
          f"tensor kernel {ker_ms:.2f} ms = {achieved:.0f} TFLOP/s ({achieved / peak:.1%} of {peak_src}), "
          f"err {err:.2e}", file=sys.stderr)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
