#!/usr/bin/env python
"""Benchmark: effective TFLOP/s (2MNK/t) of the scaled fast multiplication.

Workload (one "step" = the whole hot path on one product): square n = 4096,
FP32 inputs A = D1 X D2, B = D3 Y D4 (X, Y ~ U[0,1), diagonal entries
2^U(-12,12)), outside-then-inside power-of-two scaling (two steps of Alg. 3:
four reduction kernels) followed by the multiply of the Winograd variant,
one recursion level, bf16 hi+lo three-product leaves with FP32
accumulation: under the default (pass) schedule, one combination pass per
operand forms S_r / T_r with the scaling applied, then one tensor-core
launch forms the leaf products and adds them into C.  Inputs stay resident
in HBM; L2 is flushed (256 MiB write, untimed) before every timed step.
Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU float64 oracle on a bounded sample of the
same workload (the reference arm of this method).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

N_DEFAULT = 4096
SEED = 1507 + 1000
METRIC = "effective TFLOP/s (2MNK/t) at stated max error vs FP64; fast vs classical"
UNIT = "TFLOP/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--rule", default="winograd")
    ap.add_argument("--levels", type=int, default=1)
    ap.add_argument("--leaf", default="bf16x3")
    ap.add_argument("--scaling", default="OI")
    ap.add_argument("--schedule", default="auto", choices=["auto", "pass", "load_stage", "pass_accumulate"])
    ap.add_argument("--no-extras", action="store_true", help="skip comparator / variant timings")
    ap.add_argument("--batch", type=int, default=512, help="products in the batched workload extra (0: skip)")
    ap.add_argument("--experiment", default="", choices=["", "scaling_accuracy", "batch", "oracle_timing", "linear", "precision"],
                    help="scaling_accuracy: relative error of Strassen, L = 1..6, under each scaling (Sec. 6.5); "
                         "batch: the batched workload alone (--batch products); oracle_timing: the float64 "
                         "oracle on the host cores, single-threaded and on all cores, n = 256, 4096, 8192; linear: the "
                         "linear layer X[8192,4096] W[4096,4096] forward and backward alone; precision: the precision "
                         "sweep alone")
    ap.add_argument("--samples", type=int, default=100, help="samples per distribution (--experiment)")
    ap.add_argument("--exp-n", type=int, default=2000, help="matrix size (--experiment)")
    return ap.parse_args()


def workload_config(args):
    return {"workload": f"{args.rule} L={args.levels}, n={args.n} square, FP32 data, {args.leaf} leaves, "
                        f"scaling {args.scaling or 'none'}",
            "rule": args.rule, "levels": args.levels, "M": args.n, "K": args.n, "N": args.n,
            "leaf": args.leaf, "scaling_steps": args.scaling, "schedule": args.schedule,
            "inputs": "A=D1 X D2, B=D3 Y D4, X,Y~U[0,1), D=2^U(-12,12), seeded",
            "l2": "flushed before each timed step (256 MiB memset, untimed)"}


# ---------------------------------------------------------------- batched workload

def batched_workload(api, inputs, torch, count: int, rank: int = 0, world: int = 1) -> dict:
    """``count`` independent products, each dimension log-uniform over the
    multiples of 128 in [512, 4096]; BF16 inputs U[-1, 1] (seeded, made on
    the device), BF16 leaves with FP32 accumulation, outside-inside scaling;
    plans chosen per product by the autotuner; the whole batch one launch
    sequence (one persistent tensor-core launch) replayed from a CUDA graph.
    Inputs total several GB, far beyond L2, so no flush is needed.  On
    several GPUs each rank runs its share of the same batch
    (fmm_batch_partition: longest-processing-time by flops, no exchange);
    the batch time is the slowest rank's."""
    all_dims = inputs.log_uniform_dims(count, 512, 4096, 128, seed=1507 + 4000)
    mine = api.partition_batch(all_dims.tolist(), world)[rank] if world > 1 else list(range(count))
    dims = all_dims[mine]
    t0 = time.time()
    tuner = api.Autotuner(leaf="bf16", dtype=torch.bfloat16)
    tune_s = time.time() - t0
    gen = torch.Generator(device="cuda").manual_seed(1507 + 4001)
    probs, choice = [], {}
    for M, K, N in dims.tolist():
        A = (torch.rand((M, K), generator=gen, device="cuda") * 2 - 1).to(torch.bfloat16)
        B = (torch.rand((K, N), generator=gen, device="cuda") * 2 - 1).to(torch.bfloat16)
        plan = tuner.plan(M, K, N)
        key = "-".join(tuner.choose(M, K, N)) or "classical"
        choice[key] = choice.get(key, 0) + 1
        probs.append((plan, A, B, torch.empty((M, N), device="cuda")))
    batch = api.Batch(probs, "OI")
    for _ in range(3):
        batch.run()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        batch.run()
    g.replay()
    torch.cuda.synchronize()
    reps = 10
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    api.sync_status()
    ms = e0.elapsed_time(e1) / reps
    if world > 1:
        ms = max_over_ranks([ms])[0]
    # per-kind breakdown from separate runs with events around every launch
    api.kernel_timing(True)
    for _ in range(3):
        batch.run()
    torch.cuda.synchronize()
    api.kernel_timing(False)
    breakdown = {}
    for kind in ("scale", "combine", "multiply"):
        k_ms, k_n = api.kernel_timing_read(kind)
        breakdown[kind] = {"ms_per_run": k_ms / 3, "launches_per_run": k_n // 3}
    flops = float(sum(2 * M * K * N for M, K, N in all_dims.tolist()))
    # error of a sample of products against an FP64 product of the same inputs
    errs = []
    for i in range(0, count, max(1, count // 16)):
        _, A, B, C = probs[i]
        ref = A.double() @ B.double()
        errs.append(float((C.double() - ref).abs().max() / (A.double().abs().max() * B.double().abs().max() *
                                                             A.shape[1])))
    ws_gb = batch.ws.numel() / 1e9
    del batch, probs, g
    torch.cuda.empty_cache()
    return {"products": count, "tflops": flops / (ms * 1e-3) / 1e12, "ms_per_batch": ms, "total_gflop": flops / 1e9,
            "ranks": world, "products_this_rank": len(mine),
            "plans": choice, "launch": "one CUDA graph replay: 6 scaling + 1 combination + 1 multiply + 1 output launch",
            "workspace_gb": ws_gb, "autotune_s": tune_s,
            "max_err_over_K_normA_normB_sampled": max(errs), "leaf": "bf16", "inputs": "bf16 U[-1,1]",
            "scaling": "OI", "operand_gb": sum(M * K + K * N for M, K, N in dims.tolist()) * 2 / 1e9,
            "breakdown": dict(breakdown, note="separate runs without the graph, events around every launch")}


# ---------------------------------------------------------------- fast-matmul linear layer

def linear_layer_workload(api, torch, reps: int = 10) -> dict:
    """Y = X W with X [8192, 4096] and W [4096, 4096] BF16 (U[-1,1]/sqrt(K),
    seeded, on the device), Strassen two levels, BF16 leaves with FP32
    accumulation: the forward product and the backward pair dX = dY W^T,
    dW = X^T dY through the permuted rules, each timed with CUDA events; the
    tensor-core kernel's share from the library's per-kernel timing."""
    M, K, N = 8192, 4096, 4096
    gen = torch.Generator(device="cuda").manual_seed(1507 + 3000)
    X = ((torch.rand((M, K), generator=gen, device="cuda") * 2 - 1) / K ** 0.5).to(torch.bfloat16)
    W = ((torch.rand((K, N), generator=gen, device="cuda") * 2 - 1) / K ** 0.5).to(torch.bfloat16)
    dY = ((torch.rand((M, N), generator=gen, device="cuda") * 2 - 1)).float()
    plan = api.Plan(["strassen", "strassen"], "bf16")
    Y = api.multiply(plan, X, W)
    api.multiply_backward(plan, dY, X, W)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    api.kernel_timing(True)
    ev[0].record()
    for _ in range(reps):
        api.multiply(plan, X, W, out=Y)
    ev[1].record()
    for _ in range(reps):
        api.multiply_backward(plan, dY, X, W)
    ev[2].record()
    torch.cuda.synchronize()
    api.kernel_timing(False)
    mult_ms, mult_n = api.kernel_timing_read("multiply")
    api.sync_status()
    f_ms = ev[0].elapsed_time(ev[1]) / reps
    b_ms = ev[1].elapsed_time(ev[2]) / reps
    flops = 2.0 * M * K * N
    info = plan.info()
    leaf_flops = 2.0 * info["leaves"] * (M // info["pm"]) * (K // info["pk"]) * (N // info["pn"])
    # forward error against an FP64 product of a row sample
    rows = torch.arange(0, M, 64, device="cuda")
    ref = X[rows].double() @ W.double()
    err = float((Y[rows].double() - ref).abs().max())
    del X, W, dY, Y
    torch.cuda.empty_cache()
    return {"shape": [M, K, N], "plan": "strassen L=2, bf16 leaves", "forward_tflops": flops / (f_ms * 1e-3) / 1e12,
            "backward_tflops": 2 * flops / (b_ms * 1e-3) / 1e12, "forward_ms": f_ms, "backward_ms": b_ms,
            # a product may run as more than one multiply launch: time per product
            # (reps forward products, 2 reps gradient products, equal leaf flops)
            "multiply_kernel_ms_per_product": mult_ms / (3 * reps),
            "multiply_launches_per_product": mult_n / (3 * reps),
            "multiply_kernel_leaf_tflops": leaf_flops / (mult_ms / (3 * reps) * 1e-3) / 1e12,
            "forward_max_abs_err_sampled_rows": err}


# ---------------------------------------------------------------- fast vs classical at n = 8192

def crossover_workload(api, inputs, torch, args, n: int = 8192, reps: int = 10) -> dict:
    """The benchmark's configuration (Winograd one level, bf16 hi+lo leaves,
    FP32 inputs D1 X D2 / D3 Y D4, outside-inside scaling) at n = 8192 beside
    the classical product through the same kernels and scaling: the fast
    step saves 1/8 of the tensor-core work, whose share grows with n, while
    its extra bandwidth passes grow with n^2.  Effective TFLOP/s (2n^3/t)
    and the max-abs error against an FP64 product of a row sample."""
    A64, B64 = inputs.diag_scaled_pair(n, n, n, seed=SEED + 7)
    A = torch.from_numpy(A64).float().cuda()
    B = torch.from_numpy(B64).float().cuda()
    C = torch.empty((n, n), dtype=torch.float32, device="cuda")
    rows = torch.arange(0, n, 128, device="cuda")
    ref = A[rows].double() @ B.double()
    out = {}
    for name, rules in (("fast", [args.rule]), ("classical", [])):
        plan = api.Plan(rules, args.leaf, args.schedule)

        def step():
            eA, d, eB = api.scale(A, B, args.scaling)
            api.multiply(plan, A, B, eA, d, eB, out=C)

        step()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(reps):
            step()
        ev[1].record()
        torch.cuda.synchronize()
        api.sync_status()
        ms = ev[0].elapsed_time(ev[1]) / reps
        out[name] = {"tflops": 2.0 * n**3 / (ms * 1e-3) / 1e12, "ms_per_step": ms,
                     "max_abs_err_sampled_rows": float((C[rows].double() - ref).abs().max())}
        del plan
    del A, B, C, ref
    torch.cuda.empty_cache()
    out["config"] = f"{args.rule} L=1 vs classical, n={n}, FP32 data, {args.leaf} leaves, scaling {args.scaling}"
    return out


# ---------------------------------------------------------------- FP8 dense peak probe

def fp8_peak_probe(torch, n: int = 8192, reps: int = 10) -> dict:
    """The dense E4M3 rate of the library GEMM in torch (a scaled FP8 product
    at n^3, best of `reps`, CUDA events): a measured FP8 reference beside the
    nominal one (the measured bf16 figure x 2) that E4M3 bench lines use; the
    measured-peaks file has no FP8 figure.  Measurement only."""
    try:
        a = torch.randn((n, n), device="cuda").to(torch.float8_e4m3fn)
        b = torch.randn((n, n), device="cuda").to(torch.float8_e4m3fn).t()
        one = torch.ones((), device="cuda")
        best = float("inf")
        for i in range(reps + 2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
            e1.record()
            torch.cuda.synchronize()
            if i >= 2:
                best = min(best, e0.elapsed_time(e1))
        del a, b
        return {"fp8_e4m3_tflops": 2.0 * n**3 / (best * 1e-3) / 1e12, "how": f"torch._scaled_mm {n}^3, best of {reps}"}
    except Exception as e:  # not available in this torch build
        return {"unavailable": str(e)[:200]}


# ---------------------------------------------------------------- precision sweep

def precision_sweep(api, torch, reps: int = 5) -> dict:
    """The precision sweep: n = 8192 square and M = 8192, K = 16384,
    N = 4096; FP32 inputs U[-1, 1] and the scaled-row/column distribution
    A = D1 X D2, B = D3 Y D4 (X, Y ~ U[0, 1), D = 2^U(-12, 12)), seeded, on the
    device; Winograd and Strassen composed with classical <1,2,1> at
    alternating levels, one to four levels, and the classical product through
    the same kernels; BF16, FP16 and E4M3 (128-block power-of-two scales)
    leaves with FP32 accumulation; outside-inside scaling; each configuration
    timed with CUDA events over `reps` calls (inputs far beyond L2), with its
    max-norm error against an FP64 product of the same inputs (measurement
    only), relative to K ||A|| ||B|| and to the plan's Theorem 4.2 bound."""
    out = {}
    gen = torch.Generator(device="cuda").manual_seed(1507 + 5000)
    plans = (["winograd"], ["strassen", "classical121"], ["winograd", "classical121", "winograd"],
             ["strassen", "classical121", "strassen", "classical121"], [])
    eps = {"bf16": 2.0 ** -8, "fp16": 2.0 ** -11, "e4m3b128": 2.0 ** -3 + 2.0 ** -8}
    for M, K, N in ((8192, 8192, 8192), (8192, 16384, 4096)):
        for dist in ("uniform", "scaled"):
            if dist == "uniform":
                A = torch.rand((M, K), generator=gen, device="cuda") * 2 - 1
                B = torch.rand((K, N), generator=gen, device="cuda") * 2 - 1
            else:
                def diag(n):
                    return torch.exp2(torch.rand(n, generator=gen, device="cuda") * 24 - 12)
                A = diag(M)[:, None] * torch.rand((M, K), generator=gen, device="cuda") * diag(K)[None, :]
                B = diag(K)[:, None] * torch.rand((K, N), generator=gen, device="cuda") * diag(N)[None, :]
            ref = A.double() @ B.double()
            normA, normB = float(A.abs().max()), float(B.abs().max())
            scale = K * normA * normB
            flops = 2.0 * M * K * N
            for names in plans:
                for leaf in ("bf16", "fp16", "e4m3b128"):
                    plan = api.Plan(names, leaf)
                    C = torch.empty((M, N), device="cuda")
                    eA, d, eB = api.scale(A, B, "OI")
                    api.multiply(plan, A, B, eA, d, eB, out=C)
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    for _ in range(reps):
                        eA, d, eB = api.scale(A, B, "OI")
                        api.multiply(plan, A, B, eA, d, eB, out=C)
                    e1.record()
                    torch.cuda.synchronize()
                    api.sync_status()
                    ms = e0.elapsed_time(e1) / reps
                    err = float((C.double() - ref).abs().max())
                    key = f"{M}x{K}x{N} {dist} {'-'.join(names) or 'classical'} {leaf}"
                    out[key] = {"tflops": flops / (ms * 1e-3) / 1e12, "ms": ms, "levels": len(names),
                                "max_err_over_K_normA_normB": err / scale,
                                "err_over_theorem_4_2_bound": err / plan.bound(K, normA, normB, eps[leaf])}
                    del C, plan
            del A, B, ref
            torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- clocks

class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"fmm_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- oracle legs

def oracle_inputs(n: int, seed: int):
    from paper_1507_00687_gb300 import inputs
    A, B = inputs.diag_scaled_pair(n, n, n, seed=seed)
    return A.astype(np.float32).astype(np.float64), B.astype(np.float32).astype(np.float64)


def oracle_step(A, B, args):
    """One oracle pass (pow2 scaling + recursive fast product, float64) on a
    sample of the workload; returns seconds."""
    from oracle import fmm as OF
    from oracle import rules as OR
    from oracle import scaling as OS
    rule = {"winograd": OR.winograd, "strassen": OR.strassen}[args.rule]()
    tree = OF.uniform([rule] * args.levels)
    t0 = time.perf_counter()
    if args.scaling:
        st = OS.pow2_repeated(A, B, args.scaling)
        Ap, Bp = OS.pow2_apply(A, B, st.eA, st.d, st.eB)
        OS.pow2_unscale(OF.fmm(Ap, Bp, tree), st.eA, st.eB)
    else:
        OF.fmm(A, B, tree)
    return time.perf_counter() - t0


def host_link(h_src, d_buf, h_dst, reps=5):
    """Copy-engine rates of the host link (GB/s, best of ``reps``): pinned
    host -> device, device -> pinned host, and both at once on two streams
    (each way).  ``h_src``, ``d_buf`` and ``h_dst`` have the same size."""
    import torch
    nbytes = h_src.numel() * h_src.element_size()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    d2 = torch.empty_like(d_buf)

    def best(fn):
        t = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            t = min(t, e0.elapsed_time(e1))
        return nbytes / (t * 1e-3) / 1e9

    def both():
        cur = torch.cuda.current_stream()
        for s in (s1, s2):
            s.wait_stream(cur)
        with torch.cuda.stream(s1):
            d_buf.copy_(h_src, non_blocking=True)
        with torch.cuda.stream(s2):
            h_dst.copy_(d2, non_blocking=True)
        cur.wait_stream(s1)
        cur.wait_stream(s2)

    out = {"h2d_GBps": best(lambda: d_buf.copy_(h_src, non_blocking=True)),
           "d2h_GBps": best(lambda: h_dst.copy_(d_buf, non_blocking=True)),
           "both_ways_GBps_each": best(both)}
    del d2
    return out


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else the kernel's CPU list), or the
    machine type."""
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    return line.split(":", 1)[1].strip()
        with open("/proc/cpuinfo") as f:  # Arm: implementer / part numbers
            parts = {}
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    parts.setdefault(k.strip(), v.strip())
        if "CPU part" in parts:
            return f"Arm implementer {parts.get('CPU implementer')} part {parts.get('CPU part')}"
    except OSError:
        pass
    import platform
    return platform.machine()


def _oracle_timing_child(n: int, which: str, reps: int, q) -> None:
    """Median time of `reps` oracle products (a separate process, so that the
    BLAS thread count set in its environment applies)."""
    from oracle import fmm as OF
    from oracle import rules as OR
    A, B = oracle_inputs(n, SEED)
    tree = None if which == "classical" else OF.uniform([OR.winograd()])
    OF.fmm(A[:256, :256], B[:256, :256], tree)  # warm up
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        OF.fmm(A, B, tree)
        ts.append(time.perf_counter() - t0)
    q.put(statistics.median(ts))


def oracle_timing(args) -> dict:
    """The CPU-baseline leg at more sizes and thread counts: the float64
    oracle as it stands on the host cores at n = 256, 4096 and 8192, the
    classical product and Winograd one level, single-threaded (the paper's
    Sec. 6.5 setting) and on all cores, median of 5 (3 at n = 8192), as
    effective GFLOP/s 2 n^3 / t."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = {"cpu_model": cpu_model(), "nproc": os.cpu_count(), "runs": []}
    for threads in (1, os.cpu_count()):
        for n in (256, 4096, 8192):
            for which in ("classical", "winograd"):
                reps = 3 if n >= 8192 else 5
                env = {k: str(threads) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS",
                                                  "BLIS_NUM_THREADS")}
                old = {k: os.environ.get(k) for k in env}
                os.environ.update(env)
                q = ctx.Queue()
                p = ctx.Process(target=_oracle_timing_child, args=(n, which, reps, q))
                p.start()
                t = q.get()
                p.join()
                for k, v in old.items():
                    if v is None:
                        os.environ.pop(k, None)
                    else:
                        os.environ[k] = v
                out["runs"].append({"threads": threads, "n": n, "algorithm": which, "median_s": t, "reps": reps,
                                    "gflops": 2.0 * n**3 / t / 1e9})
    return out


def cpu_baseline(args) -> dict:
    """The oracle as it stands on the host cores: the workload's own product
    (n capped at 4096), repeated until about 10 s of CPU work (3 to 9 runs),
    median run."""
    n_s = min(args.n, 4096)
    oracle_step(*oracle_inputs(256, SEED), args)  # warm numpy / BLAS
    A, B = oracle_inputs(n_s, SEED)
    ts = []
    while len(ts) < 3 or (sum(ts) < 10.0 and len(ts) < 9):
        ts.append(oracle_step(A, B, args))
    t = statistics.median(ts)
    what = (f"the workload's own n={n_s} product" if n_s == args.n else
            f"one n={n_s} product of the same distribution ({(n_s / args.n) ** 3:.3g} of the workload's flops)")
    return {"value": 2.0 * n_s**3 / t / 1e12, "unit": UNIT, "cores": os.cpu_count(), "cpu_model": cpu_model(),
            "kind": "oracle",
            "sample": f"{what}, float64 numpy oracle with BLAS leaf products, scaling included, median of "
                      f"{len(ts)} runs ({t:.2f} s each, {sum(ts):.1f} s in all)"}


def max_over_ranks(values, device="cuda"):
    """Each value's maximum over the ranks of the initialised process group
    (the values themselves on one rank or without a group): step times are
    taken as the slowest rank's."""
    import torch
    import torch.distributed as dist
    vals = [float(v) for v in values]
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return vals
    t = torch.tensor(vals, device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def whole_job_tflops(flops_per_rank, world, ms_max):
    """Whole-job throughput: the flops all ranks processed (each rank its own
    product, weak scaling) over the slowest rank's time."""
    return world * flops_per_rank / (ms_max * 1e-3) / 1e12


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # size the per-step sample so that warm-up + timed steps take ~2 minutes
    A, B = oracle_inputs(512, SEED)
    oracle_step(A, B, args)
    t512 = min(oracle_step(A, B, args) for _ in range(2))
    per_step = 120.0 / max(1, args.steps + args.warmup)
    n_s = int(512 * (per_step / t512) ** (1.0 / 3.0)) // 64 * 64
    n_s = max(128, min(args.n, 2048, n_s))
    A, B = oracle_inputs(n_s, SEED)
    for _ in range(args.warmup):
        oracle_step(A, B, args)
    tot = 0.0
    for i in range(args.steps):
        tot += oracle_step(A, B, args)
    t = tot / max(args.steps, 1)
    v = 2.0 * n_s**3 / t / 1e12
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": dict(workload_config(args), sample_n=n_s),
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                            "sample": f"each step one n={n_s} product of the workload's distribution "
                                      f"(float64 numpy oracle, BLAS leaf products)"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- accuracy experiment

EXP_SCALINGS = [("none", ""), ("outside", "O"), ("inside", "I"), ("outside-inside", "OI"),
                ("inside-outside", "IO"), ("2x outside-inside", "OIOI"), ("10x outside-inside", "OI" * 10),
                ("adaptive tau=1e-3", None)]


def scaling_accuracy(args):
    """The scaling experiment of Sec. 6.5 on the GPU path: for each of the
    three input distributions, ``samples`` pairs of n x n matrices; for each
    scaling and L = 1..6 levels of Strassen, the largest componentwise
    relative error max_ij |C^_ij - C_ij| / |C_ij| over the samples.  C is
    the float64 classical product of the FP32 inputs (all entries are
    nonnegative, so its own relative error is below n 2^-53)."""
    import torch
    from paper_1507_00687_gb300 import build
    build.build()
    from paper_1507_00687_gb300 import api, inputs
    n, samples, levels = args.exp_n, args.samples, range(1, 7)
    plans = {L: api.Plan(["strassen"] * L, args.leaf, "pass") for L in levels}
    worst = {k: {name: [0.0] * len(levels) for name, _ in EXP_SCALINGS} for k in (1, 2, 3)}
    steps_seen = {k: [] for k in (1, 2, 3)}
    t0 = time.perf_counter()
    for kind in (1, 2, 3):
        for s in range(samples):
            A64, B64 = inputs.paper_distribution(kind, n, seed=100000 * kind + s)
            A = torch.from_numpy(A64).float().cuda()
            B = torch.from_numpy(B64).float().cuda()
            C = A.double() @ B.double()
            Cabs = C.abs()
            for name, steps in EXP_SCALINGS:
                if steps is None:
                    eA, d, eB, t = api.scale_adaptive(A, B, 1e-3, 40)
                    steps_seen[kind].append(int(t.item()))
                elif steps:
                    eA, d, eB = api.scale(A, B, steps)
                else:
                    eA = d = eB = None
                for i, L in enumerate(levels):
                    Ch = api.multiply(plans[L], A, B, eA, d, eB)
                    err = ((Ch.double() - C).abs() / Cabs).max().item()
                    worst[kind][name][i] = max(worst[kind][name][i], err)
        api.sync_status()
    out = {"experiment": "scaling_accuracy", "rule": "strassen", "levels": list(levels), "n": n,
           "samples_per_distribution": samples, "leaf": args.leaf, "inputs": "FP32 (rounded from the samples)",
           "error": "max over samples of max_ij |C^-C|/|C|, C = float64 classical product",
           "adaptive_steps": {str(k): [min(v), max(v)] for k, v in steps_seen.items()},
           "seconds": round(time.perf_counter() - t0, 1),
           "table": {f"distribution {k}": {name: [float(f"{e:.3e}") for e in worst[k][name]]
                                           for name, _ in EXP_SCALINGS} for k in (1, 2, 3)}}
    print(json.dumps(out))


# ---------------------------------------------------------------- GPU leg

def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.experiment == "scaling_accuracy":
        scaling_accuracy(args)
        return
    if args.experiment == "oracle_timing":
        print(json.dumps({"experiment": "oracle_timing", **oracle_timing(args)}))
        return
    if args.experiment == "batch":
        import torch
        from paper_1507_00687_gb300 import build
        build.build()
        from paper_1507_00687_gb300 import api, inputs
        print(json.dumps({"experiment": "batch", **batched_workload(api, inputs, torch, max(1, args.batch))}))
        return
    if args.experiment == "precision":
        import torch
        from paper_1507_00687_gb300 import build
        build.build()
        from paper_1507_00687_gb300 import api
        print(json.dumps({"experiment": "precision", "precision_sweep": precision_sweep(api, torch),
                          "fp8_peak_probe": fp8_peak_probe(torch)}))
        return
    if args.experiment == "linear":
        import torch
        from paper_1507_00687_gb300 import build
        build.build()
        from paper_1507_00687_gb300 import api
        print(json.dumps({"experiment": "linear", **linear_layer_workload(api, torch)}))
        return
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_1507_00687_gb300 import build
    build.build()
    from paper_1507_00687_gb300 import api, inputs

    n = args.n
    A64, B64 = inputs.diag_scaled_pair(n, n, n, seed=SEED + rank)
    hA = torch.from_numpy(A64).float().pin_memory()
    hB = torch.from_numpy(B64).float().pin_memory()
    hC = torch.empty((n, n), dtype=torch.float32).pin_memory()
    A = hA.cuda()
    B = hB.cuda()
    C = torch.empty((n, n), dtype=torch.float32, device="cuda")
    eA = torch.empty(n, dtype=torch.int32, device="cuda")
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    eB = torch.empty(n, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    rules = [args.rule] * args.levels
    plan = api.Plan(rules, args.leaf, args.schedule)
    info = plan.info()

    def step(pl=plan, scaling=args.scaling, kev=None):
        if scaling:
            from paper_1507_00687_gb300 import _native as Nn
            import ctypes
            Nn.check(Nn.lib().fmm_scale(scaling.encode(), ctypes.c_void_p(A.data_ptr()),
                                        ctypes.c_void_p(B.data_ptr()), Nn.DT_F32, n, n, n, n, n,
                                        ctypes.c_void_p(eA.data_ptr()), ctypes.c_void_p(d.data_ptr()),
                                        ctypes.c_void_p(eB.data_ptr()), ctypes.c_void_p(stream.cuda_stream)),
                     "fmm_scale")
        if kev is not None:
            kev[0].record(stream)
        if scaling:
            api.multiply(pl, A, B, eA, d, eB, out=C)
        else:
            api.multiply(pl, A, B, out=C)
        if kev is not None:
            kev[1].record(stream)

    def timed(steps, pl=plan, scaling=args.scaling, clocks=None, kernels=None, kinds=(), call_events=True):
        """Mean step time (ms) over `steps` steps; with `kernels`, the
        library's per-kernel event timing of `kinds` (all when empty) over
        the same steps; with call_events, the mean multiply-call time too.
        Every event between two launches keeps them from overlapping, so the
        headline run records only the multiply kernel's."""
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        kevs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        step(pl, scaling)  # untimed: sizes this plan's cached workspace
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        if kernels is not None:
            api.kernel_timing(True, kinds)
        if clocks:
            clocks.start()
        for i in range(steps):
            flush.zero_()
            evs[i][0].record(stream)
            step(pl, scaling, kevs[i] if call_events else None)
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ck = clocks.stop() if clocks else None
        if kernels is not None:
            api.kernel_timing(False)
            for kind in ("scale", "prepare", "combine", "multiply", ""):
                kernels[kind] = api.kernel_timing_read(kind)
        api.sync_status()
        st = [a.elapsed_time(b) for a, b in evs]
        kt = [a.elapsed_time(b) for a, b in kevs] if call_events else [0.0]
        return statistics.mean(st), statistics.mean(kt), ck

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    api.sync_status()
    clocks = Clocks(local)
    # headline: the whole step, with events around the multiply kernel only
    kern_m = {}
    ms, _, ck = timed(args.steps, clocks=clocks, kernels=kern_m, kinds=("multiply",), call_events=False)
    # breakdown: every kernel timed (events between all launches)
    bd_steps = min(args.steps, 50)
    kern = {}
    _, kms, _ = timed(bd_steps, kernels=kern)
    ms, kms = max_over_ranks([ms, kms])
    flops = 2.0 * n**3
    value = whole_job_tflops(flops, world, ms)

    # ---------------- end to end through the public API with host buffers
    # The public host-memory entry points (fmm_host_*): each step copies A and
    # B in from pinned host memory, scales, multiplies and copies C out; two
    # pipeline slots let one step's copies overlap its neighbours' work.
    pipe = api.HostPipeline(plan, n, n, n, torch.float32, args.scaling, depth=2)
    hCs = [hC, torch.empty((n, n), dtype=torch.float32).pin_memory()]

    def e2e_run(k):
        for i in range(k):
            pipe.submit(hA, hB, hCs[i % 2])
        pipe.wait()

    e2e_run(2)
    torch.cuda.synchronize()
    e_steps = max(3, min(args.steps, 30))
    t0 = time.perf_counter()
    e2e_run(e_steps)
    e_ms = (time.perf_counter() - t0) * 1e3 / e_steps
    del pipe
    link = host_link(hA, A, hCs[1])
    e_ms = max_over_ranks([e_ms])[0]
    api.sync_status()

    # ---------------- accuracy (max-norm vs an FP64 product of the same inputs)
    step()
    torch.cuda.synchronize()
    C_fast = C.double()
    ref = A.double() @ B.double()   # FP64 reference product (measurement only)
    err_fast = float((C_fast - ref).abs().max())
    normA, normB = float(A.abs().max()), float(B.abs().max())
    eps_leaf = {"bf16x3": 3 * 2.0**-16, "bf16": 2.0**-8, "fp16": 2.0**-11, "e4m3b128": 2.0**-3 + 2.0**-8}[args.leaf]
    bound_unscaled = plan.bound(n, normA, normB, eps_leaf)
    extras = {}
    if not args.no_extras:
        plan0 = api.Plan([], args.leaf, args.schedule)
        c_ms, c_kms, _ = timed(max(10, args.steps // 4), plan0, args.scaling)
        step(plan0, args.scaling)
        torch.cuda.synchronize()
        err_cls = float((C.double() - ref).abs().max())
        extras["classical_same_kernel"] = {"tflops": flops / (c_ms * 1e-3) / 1e12, "ms_per_step": c_ms,
                                           "kernel_ms": c_kms, "max_abs_err": err_cls,
                                           "note": "L=0 plan through the same kernels, same scaling"}
        ns_ms, ns_kms, _ = timed(max(10, args.steps // 4), plan, "")
        step(plan, "")
        torch.cuda.synchronize()
        extras["fast_no_scaling"] = {"tflops": flops / (ns_ms * 1e-3) / 1e12, "ms_per_step": ns_ms,
                                     "max_abs_err": float((C.double() - ref).abs().max())}
        if args.schedule != "pass_accumulate":
            plan_acc = api.Plan(rules, args.leaf, "pass_accumulate")
            a_ms, a_kms, _ = timed(max(10, args.steps // 4), plan_acc, args.scaling)
            step(plan_acc, args.scaling)
            torch.cuda.synchronize()
            extras["fast_accumulate"] = {"tflops": flops / (a_ms * 1e-3) / 1e12, "ms_per_step": a_ms,
                                         "kernel_ms": a_kms, "max_abs_err": float((C.double() - ref).abs().max()),
                                         "note": "leaf products added into C by atomic FP32 additions "
                                                 "(no stored products, no output pass)"}
            del plan_acc
        rel = lambda X: float(((X - ref).abs() / ref.abs().clamp_min(1e-300)).max())  # noqa: E731
        step(plan, args.scaling)
        torch.cuda.synchronize()
        extras["componentwise_rel_err"] = {"fast_scaled": rel(C.double())}
        step(plan, "")
        torch.cuda.synchronize()
        extras["componentwise_rel_err"]["fast_unscaled"] = rel(C.double())
        if args.scaling == "OI":
            o_ms, o_kms, _ = timed(max(10, args.steps // 4), plan, "O")
            step(plan, "O")
            torch.cuda.synchronize()
            extras["fast_O_only"] = {"tflops": flops / (o_ms * 1e-3) / 1e12, "ms_per_step": o_ms,
                                     "kernel_ms": o_kms, "max_abs_err": float((C.double() - ref).abs().max()),
                                     "note": "outside scaling only (one O step)"}
        if args.levels == 1:
            for lv in (2, 3):
                try:
                    plan_l = api.Plan([args.rule] * lv, args.leaf, args.schedule)
                    l_ms, l_kms, _ = timed(max(10, args.steps // 4), plan_l, args.scaling)
                    step(plan_l, args.scaling)
                    torch.cuda.synchronize()
                    extras[f"fast_L{lv}"] = {"tflops": flops / (l_ms * 1e-3) / 1e12, "ms_per_step": l_ms,
                                             "kernel_ms": l_kms,
                                             "max_abs_err": float((C.double() - ref).abs().max())}
                    del plan_l
                except Exception as e:  # plan outside the supported range
                    extras[f"fast_L{lv}"] = {"unavailable": str(e)}
        del plan0
    del ref, C_fast
    if not args.no_extras:
        extras["headline_n8192"] = crossover_workload(api, inputs, torch, args)
    if not args.no_extras and args.batch > 0:
        extras["batched"] = batched_workload(api, inputs, torch, args.batch, rank, world)
    if not args.no_extras:
        extras["autograd_linear"] = linear_layer_workload(api, torch)
        extras["precision_sweep"] = precision_sweep(api, torch)
        extras["fp8_peak_probe"] = fp8_peak_probe(torch)

    # ---------------- roofline of the dominant kernel (the tensor-core multiply)
    import json as _json
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = _json.load(open(peaks_path)) if os.path.exists(peaks_path) else {}
    # The multiply kernel is timed alone inside sub-millisecond steps, so its
    # roofline is the burst figure; the sustained one is printed beside it.
    peak = peaks.get("bf16_tflops", 1900.0)
    peak_sus = peaks.get("bf16_tflops_sustained", 1700.0)
    peak_src = "of measured (bf16_tflops, burst)" if peaks else "of fallback"
    lin = extras.get("autograd_linear")
    # E4M3 leaves: the dense FP8 rate, the measured bf16 figure times the
    # nominal FP8 / bf16 ratio of 2
    fp8 = args.leaf == "e4m3b128"
    peak_m = peak * (2 if fp8 else 1)
    peak_sus_m = peak_sus * (2 if fp8 else 1)
    peak_src_m = peak_src + (" x 2 (nominal FP8 / bf16 ratio)" if fp8 else "")
    if lin:
        # forward and backward against the same tensor-core roofline: the
        # leaf kernel's executed flops, and the effective 2MNK/t of each call
        lin["roofline"] = {"bound": "tensor", "peak": peak, "unit": "TFLOP/s", "peak_source": peak_src,
                           "multiply_kernel_frac": lin["multiply_kernel_leaf_tflops"] / peak,
                           "multiply_kernel_frac_of_sustained": lin["multiply_kernel_leaf_tflops"] / peak_sus,
                           "forward_effective_frac": lin["forward_tflops"] / peak,
                           "backward_effective_frac": lin["backward_tflops"] / peak}
    leaf_flops = 2.0 * info["leaves"] * (-(-n // info["pm"])) * (-(-n // info["pk"])) * (-(-n // info["pn"]))
    mma_flops = leaf_flops * (3 if args.leaf == "bf16x3" else 1)
    # the multiply may run as more than one launch per step (tile-row
    # halves): time per step over all of them
    mult_ms, mult_n = kern_m["multiply"]
    mult_launches = max(1, mult_n // max(1, args.steps))
    mult_ms_per = mult_ms / max(1, args.steps)
    achieved = mma_flops / (mult_ms_per * 1e-3) / 1e12
    sched_used = "pass" if kern["combine"][1] > 0 else "load_stage"
    # the pass schedule's leaf blocks of at least 256 x 256 run on CTA pairs
    bt_min = min(-(-n // info["pm"]), -(-n // info["pn"]))
    pairs = os.environ.get("FMM_TILE_PAIRS", "1") != "0" and bt_min >= 256
    kname = ("pair_fmm_kernel" if pairs else "direct_fmm_kernel") if sched_used == "pass" else "fused_fmm_kernel"
    if fp8:
        kname = "fp8_bs_kernel" if os.environ.get("FMM_FP8_FOLD", "0") == "0" else "fp8_fmm_kernel"
    # the bandwidth passes of the pass schedule, per step: the combination
    # of both operands (one launch for small operands, else one per
    # operand; each operand read once, R^L combined leaf blocks written:
    # two bf16 planes for bf16x3, else one 16-bit plane) and, with stored
    # leaf products (every pass-schedule plan with more than one leaf at
    # these sizes), the output pass (reads the R^L fp32 products, writes C)
    comb_ms, comb_n = kern["combine"]
    per_step = comb_n // max(1, bd_steps)
    planes = 2 if args.leaf == "bf16x3" else 1
    R = info["leaves"]
    bt = -(-n // info["pm"])
    tp_a = -(-bt // (256 if bt >= 256 else 128)) * (256 if bt >= 256 else 128)
    tp_b = -(-bt // 256) * 256
    kp = -(-(-(-n // info["pk"])) // 64) * 64
    pass_bytes = 2 * n * n * 4 + planes * R * (tp_a + tp_b) * kp * 2
    if sched_used == "pass" and R > 1 and per_step >= 2:
        # stored leaf products: the output pass reads them and writes C
        pass_bytes += R * tp_a * tp_b * 4 + n * n * 4
    kernel_times = {k or "all": {"ms_total": v[0], "launches": v[1], "ms_per_launch": v[0] / max(1, v[1])}
                    for k, v in kern.items()}
    # DRAM bytes per launch of the multiply kernel and per whole step, from
    # the committed ncu summary (null when no capture of this workload exists)
    traffic, step_traffic = None, None
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(prof):
        tj = _json.load(open(prof))
        key = f"{args.rule}_L{args.levels}_{args.leaf}_n{n}_{args.scaling or 'none'}"
        traffic = tj.get(f"{kname}:{key}")
        st_bytes = tj.get(f"step:{key}")
        if st_bytes:
            # algorithmic minimum per step: read A and B once per scaling
            # step and once for the product, write C
            nsteps = len(args.scaling or "")
            algo = (nsteps + 1) * 2 * n * n * 4 + n * n * 4
            step_traffic = {"dram_bytes": st_bytes, "algorithmic_min_bytes": algo, "ratio": st_bytes / algo}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32-in/bf16x3-leaf/f32-acc" if args.leaf == "bf16x3" else args.leaf,
           "data": "synthetic", "config": workload_config(args),
           "paper_effective_tflops": world * (2.0 * n**3 - n**2) / (ms * 1e-3) / 1e12,
           "multiply_call_ms": kms,
           "schedule": sched_used,
           "kernel_times": dict(kernel_times, steps=bd_steps,
                                note="separate run with events around every kernel (no launch overlap)"),
           "bandwidth_passes": ({"ms_per_step": comb_ms / bd_steps, "launches_per_step": per_step,
                                 "algorithmic_bytes_per_step": pass_bytes,
                                 "achieved_GBps": pass_bytes / (comb_ms / bd_steps * 1e-3) / 1e9,
                                 "peak_GBps": peaks.get("hbm_gbs"),
                                 "frac": (pass_bytes / (comb_ms / bd_steps * 1e-3) / 1e9 / peaks["hbm_gbs"])
                                 if peaks.get("hbm_gbs") else None} if comb_n else None),
           "executed_flop_fraction": achieved / peak_m,
           # a fraction of the measured library GEMM rate, not of a clock-derived tensor-pipe peak
           "executed_flop_fraction_of": peak_src_m,
           "step_dram_traffic": step_traffic,
           "error": {"max_abs_err_vs_fp64": err_fast, "theorem_4_1_bound_unscaled": bound_unscaled,
                     "eps_leaf": eps_leaf, "normA": normA, "normB": normB},
           "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak_m, "unit": "TFLOP/s",
                        "frac": achieved / peak_m, "traffic": traffic, "peak_source": peak_src_m,
                        "peak_sustained": peak_sus_m, "frac_of_sustained": achieved / peak_sus_m,
                        "kernel": kname, "algorithmic_flops_per_step": mma_flops,
                        "launches_per_step": mult_launches, "ms_per_step": mult_ms_per},
           "e2e": {"value": whole_job_tflops(flops, world, e_ms), "unit": UNIT,
                   "h2d_bytes_per_step": 2 * n * n * 4, "d2h_bytes_per_step": n * n * 4,
                   "ms_per_step": e_ms, "path": "fmm_host_submit / fmm_host_wait, two pipeline slots, "
                                                 "pinned host buffers, wall clock over the submissions",
                   # the host link measured in the same run: a step cannot
                   # take less than its input bytes over the host->device rate
                   "host_link": dict(link, bound_ms=2 * n * n * 4 / (link["h2d_GBps"] * 1e9) * 1e3,
                                     frac=2 * n * n * 4 / (link["h2d_GBps"] * 1e9) * 1e3 / e_ms)},
           "gpu_launches": kern[""][1] // max(1, bd_steps) * args.steps,
           "clocks": ck, "plan": info}
    out.update(extras)
    if rank == 0 and world == 1:
        out["cpu_baseline"] = cpu_baseline(args)
    # the comparisons in one short record at the end of the line
    summ = {"fast_scaled": {"tflops": value, "max_abs_err": err_fast}}
    for k in ("classical_same_kernel", "fast_no_scaling", "fast_O_only", "fast_accumulate", "fast_L2", "fast_L3"):
        if k in extras and "tflops" in extras[k]:
            summ[k] = {"tflops": extras[k]["tflops"], "max_abs_err": extras[k].get("max_abs_err")}
    if "headline_n8192" in extras:
        summ["n8192"] = {k: v["tflops"] for k, v in extras["headline_n8192"].items() if isinstance(v, dict)}
    if "batched" in extras and "tflops" in extras["batched"]:
        summ["batched_tflops"] = extras["batched"]["tflops"]
    if "autograd_linear" in extras:
        summ["linear_fwd_bwd_tflops"] = [extras["autograd_linear"]["forward_tflops"],
                                         extras["autograd_linear"]["backward_tflops"]]
    out["summary"] = summ
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
