#!/usr/bin/env python
"""Throughput of msMINRES-CIQ on one B300: K^{1/2}B right-hand-side solves per
second at relative error <= 1e-3.

Workload (the Thompson-sampling-shaped prior draw of Sec. 5.2, synthetic):
N = 50,000 points uniform in [0,1]^6, RBF kernel, lengthscale 0.3,
outputscale 1, sigma^2 = 1e-3, T = 64 right-hand sides ~ N(0, I), Q = 12
quadrature points, K^{1/2}B.  The solve stops per column when the
a-posteriori error bound sum_q w_q t_q |phibar_q| / (t_q + lambda_min) falls
to 1e-3 of ||a_j|| (so every delivered column has relative error <= 1e-3 up
to the O(1e-6) quadrature error at Q = 12); the Lanczos pre-pass (10 MVMs)
and the node computation are inside every step.

One step = one ciq_sqrt call on device-resident inputs.  `e2e` repeats the
same call with host (pageable NumPy) buffers, so the host<->device copies are
inside the timed region.  `--impl reference` times the FP64 CPU oracle on a
bounded sample of the same workload instead.

Multi-GPU: the solves are independent problems, so N ranks run N replicas
(weak scaling), one per GPU, with no data-path collective.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import ciq_inputs as ci  # noqa: E402

WORKLOAD = ci.THOMPSON_50K
TOL = 1e-3
MAX_ITER = 4000
LANCZOS_ITERS = 10
# msMINRES iterations this workload needs to reach the error bound 1e-3 in
# exact-K arithmetic.  A full FP64 oracle solve at N = 50,000 takes hours on
# the host, so the count is the one measured for the library's FP32 path (876),
# whose compensated MVM and FP64 scalars track the FP64 recurrence; the
# FP16-split tiles need 897 because their MVM carries ~4e-6 relative error.
# Only the reference arm uses it, to scale its per-iteration time to a solve.
J_WORKLOAD = 876
# Rows of K per bounded sample of the oracle's kernel MVM: one step of the
# reference arm (about 5 s of host work) and the CPU leg of our arm (8192).
REF_SAMPLE_ROWS = 2048
CPU_SAMPLE_ROWS = 8192
# The headline configuration is checked against the FP64 eigendecomposition
# on the workload's first ORACLE_CHECK_N points (O1 is affordable there), with
# the tensor-core split of three CTAs per row tile that the full-size solve runs.
ORACLE_CHECK_N = 16384
ORACLE_CHECK_TC_SPLIT = 3

# Uneven batch: 512 independent GPs (N log-uniform in [256, 8192], d in 2..12,
# RBF or Matern-5/2, lengthscale log-uniform in [0.05, 1], sigma^2 log-uniform
# in [1e-4, 1e-1]), 8 right-hand sides each, Q = 8, relative residual 1e-4.
BATCH_SEED = 20201108
BATCH_COUNT = 512
BATCH_T = 8
BATCH_Q = 8
BATCH_TOL = 1e-4
BATCH_MAX_ITER = 4000

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
SM_COUNT = 148
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", default="fp16", choices=["fp32", "fp16", "bf16"])
    ap.add_argument("--krylov", default="auto", choices=["auto", "recurrence", "basis"],
                    help="how the solves form their iterates (stored Lanczos basis or Q direction recurrences)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp32-compare", action="store_true")
    ap.add_argument("--workload", default="thompson50k",
                    choices=["thompson50k", "batched512", "precision200k", "learned", "stored", "spectrum", "vjp",
                             "precond", "posterior"],
                    help="batched512: the uneven 512-problem batch through ciq_sqrt_batched; precision200k: "
                         "the 200,000-point Matern precision sweep; learned: train the bound predictor on "
                         "20,000 instances and compare it with the Lanczos pre-pass on 4096 held-out ones; "
                         "spectrum: K^{1/2}b error against Q on matrices with prescribed spectra; "
                         "vjp: forward and backward pass of K^{-1/2}B on the 50,000-point problem; "
                         "precond: pivoted-Cholesky preconditioned roots of ranks 100-400 on the 50,000-point problem; "
                         "posterior: Thompson draws at 50,000 candidates given 256 observations")
    ap.add_argument("--profile-rank", type=int, default=0, metavar="R",
                    help="precond: only run two 40-iteration R' b solves with a rank-R preconditioner "
                         "(a short, fixed launch sequence for profiling)")
    ap.add_argument("--full-fp32", action="store_true",
                    help="precision200k: run the plain FP32 solve to the stop rule too (about 10 minutes)")
    ap.add_argument("--n", type=int, default=0, metavar="N",
                    help="run the headline solve on the first N points only (for profiling captures)")
    ap.add_argument("--mvm-only", type=int, default=0, metavar="N",
                    help="time only the kernel MVM on the first N points of the workload (for profiling)")
    ap.add_argument("--batch-only", action="store_true",
                    help="batched512: only the batched calls, without CUDA graphs (a plain launch sequence "
                         "for profiling captures)")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------- CPU baseline --
def oracle_iteration_seconds(X, B, Q, rows=CPU_SAMPLE_ROWS):
    """FP64 oracle, bounded sample of one full-size msMINRES iteration.

    The O(N^2) part is timed on `rows` of the N rows of K (the oracle's own
    row-block MVM) and scaled by N/rows; the O(QNT) vector/Givens part is one
    full-size oracle msMINRES step with the MVM replaced by the identity.
    """
    from oracle import kernels
    from oracle.msminres import msminres
    from oracle.quadrature import quad_nodes

    W = WORKLOAD
    n = X.shape[0]
    V = np.ascontiguousarray(B.T)
    t0 = time.perf_counter()
    for r0 in range(0, rows, 2048):
        kernels.kernel_matrix(X[r0:min(rows, r0 + 2048)], X, W.kernel, W.lengthscale, W.outputscale) @ V
    t_rows = time.perf_counter() - t0
    w, t = quad_nodes(W.noise, 2100.0, Q)
    t0 = time.perf_counter()
    msminres(lambda Z: Z, V, t, 1)
    t_rec = time.perf_counter() - t0
    return t_rows * n / rows + t_rec, t_rows + t_rec, rows


def cpu_threads():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        if info:
            return max(i.get("num_threads", 1) for i in info)
    except Exception:
        pass
    return os.cpu_count() or 1


def headline_oracle_check(P, torch, dev, opts):
    """CPU leg, second part: the headline configuration's delivered columns
    against the FP64 eigendecomposition (O1, K^{1/2}b = V diag(lambda^{1/2})
    V^T b) on the workload's first ORACLE_CHECK_N points, per right-hand side
    (relative 2-norm).  The solve runs with the bench's options and the
    full-size solve's tensor-core split; only the O(N^3) reference is on the
    host."""
    from oracle import eig, kernels

    W = WORKLOAD
    X, B = W.make(ORACLE_CHECK_N)
    X = X.astype(np.float32)
    B = B.astype(np.float32)
    k = P.Kernel(W.kernel, W.lengthscale, W.outputscale, W.noise)
    out, info = P.ciq_sqrt(torch.from_numpy(X).to(dev), k, torch.from_numpy(B).to(dev), W.q, TOL,
                           **dict(opts, tc_split=ORACLE_CHECK_TC_SPLIT))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    K = kernels.dense_K(X.astype(np.float64), W.kernel, W.lengthscale, W.outputscale, W.noise)
    truth = eig.sqrt_apply(K, B.T.astype(np.float64)).T
    del K
    A = out.cpu().numpy().astype(np.float64)
    err = np.linalg.norm(A - truth, axis=1) / np.linalg.norm(truth, axis=1)
    return {"n": ORACLE_CHECK_N, "columns": int(err.size), "max": float(err.max()),
            "median": float(np.median(err)), "iterations": info["iters"], "errbound_max": info["errbound_max"],
            "tc_split": ORACLE_CHECK_TC_SPLIT, "oracle": "O1: FP64 eigendecomposition (LAPACK dsyevd)",
            "oracle_seconds": time.perf_counter() - t0}


# --------------------------------------------------------------- roofline --
def peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0,
                "sm_max_mhz": 2032.0}, "fallback"


def device_peaks():
    """SFU ex2, FP32 and FP64 FMA rates measured on this device (libciq_peaks)."""
    import ctypes
    path = os.path.join(ROOT, "paper_2006_11267_b300", "libciq_peaks.so")
    L = ctypes.CDLL(path)
    out, ms = ctypes.c_double(), ctypes.c_double()
    L.ciq_peak_sfu_ex2.argtypes = [ctypes.POINTER(ctypes.c_double)] * 2
    L.ciq_peak_fma.argtypes = [ctypes.c_int] + [ctypes.POINTER(ctypes.c_double)] * 2
    L.ciq_peak_sfu_ex2_clock.argtypes = [ctypes.POINTER(ctypes.c_double)] * 4
    res = {}
    per_clk, mhz = ctypes.c_double(), ctypes.c_double()
    if L.ciq_peak_sfu_ex2_clock(ctypes.byref(out), ctypes.byref(ms), ctypes.byref(per_clk), ctypes.byref(mhz)) == 0:
        res["sfu_ex2_per_s"] = out.value
        res["sfu_ex2_per_sm_per_clk"] = per_clk.value
        res["sfu_sm_mhz"] = mhz.value
    if L.ciq_peak_fma(0, ctypes.byref(out), ctypes.byref(ms)) == 0:
        res["fp32_flops"] = out.value
    if L.ciq_peak_fma(1, ctypes.byref(out), ctypes.byref(ms)) == 0:
        res["fp64_flops"] = out.value
    return res


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one in-solve
# launch of mvm_tc_kernel, from one single-pass ncu capture of the default
# command on this workload; kept only while the kernel is unchanged since.
MVM_TC_DRAM_BYTES = {"rbf_n50000_d6_t64_q12": 22.473e6 + 0.147e6}


def headline_config(precision, world=1):
    """The headline workload's configuration, the same object on both arms
    (the GPU path and the oracle); what a run found (iterations, Krylov form,
    bound reached) goes in the line's "run" object."""
    W = WORKLOAD
    return {"workload": W.name, "N": W.n, "d": W.d, "kernel": W.kernel, "lengthscale": W.lengthscale,
            "noise": W.noise, "T": W.t, "Q": W.q, "op": "sqrt", "tol": TOL, "stop_rule": "errbound",
            "precision": precision, "lanczos_iters": LANCZOS_ITERS, "parallelism": f"replicas{world}",
            "l2": "no flush: a step of the GPU arm streams > 40 GB through HBM (48 GiB stored basis, "
                  "> 126 MB L2); the reference arm runs on the host"}


def roofline_tc(W, t_launch_ms, dev, pk, sm_mhz=None):
    # One kernel MVM on tensor cores.  Algorithmic work per kernel entry:
    # 2T flops of the product with V plus 2(d+2) flops of the augmented
    # distance (norm expansion), 1 SFU exp2 (RBF; + sqrt for Matern-5/2).
    # The FP16 hi/lo operand split executes three products for the product
    # with V (3 x 2 TP flops per entry, TP = T rounded to the launch group)
    # and two (d <= 6: 8 augmented features fill half of a K = 16 chunk) or
    # three K = 16 products for the distance.
    # Roofline of an on-the-fly tile (the slower of the two pipes): kernel
    # entries per second the tensor pipe allows at the sustained measured
    # BF16 rate, against entries per second the SFU allows at the measured
    # ex2 rate per SM and clock, scaled to the SM clock sampled during the
    # timed solves.  The line reports the binding one; both are given.
    N, T, d = W.n, W.t, W.d
    entries = float(N) * N
    secs = t_launch_ms * 1e-3
    alg = entries * (2 * T + 2 * (d + 2)) / secs / 1e12
    tp = 32 if T <= 32 else -(-T // 64) * 64
    s_products = 2 if d + 2 <= 8 else 3
    executed = entries * (3 * 2 * tp + s_products * 2 * 16) / secs / 1e12
    # The MVM is timed inside a seconds-long solve: the sustained measured
    # BF16 rate is the denominator (the burst rate is reported beside it).
    peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
    burst = pk.get("bf16_tflops")
    sfu_per_entry = 1 if W.kernel == "rbf" else 2
    sfu_rate = entries * sfu_per_entry / secs
    per_clk = dev.get("sfu_ex2_per_sm_per_clk")
    mhz = sm_mhz or dev.get("sfu_sm_mhz")
    sfu_peak = per_clk * SM_COUNT * mhz * 1e6 if per_clk and mhz else dev.get("sfu_ex2_per_s")
    entry_rate = entries / secs / 1e9                                    # G entries/s
    tensor_roof = peak * 1e12 / (2 * T + 2 * (d + 2)) / 1e9 if peak else None
    sfu_roof = sfu_peak / sfu_per_entry / 1e9 if sfu_peak else None
    roofs = {k: v for k, v in (("tensor", tensor_roof), ("sfu", sfu_roof)) if v}
    bound = min(roofs, key=roofs.get) if roofs else "tensor"
    return {"bound": bound, "achieved": entry_rate, "peak": roofs.get(bound), "unit": "Gentries/s",
            "frac": entry_rate / roofs[bound] if roofs else None,
            "traffic": MVM_TC_DRAM_BYTES.get(W.name), "traffic_unit": "bytes per launch",
            "kernel": "mvm_tc_kernel (tcgen05 on-the-fly kernel MVM, FP16 hi/lo split operands)",
            "peak_source": "min(tensor roof: measured cuBLAS BF16 sustained rate (MEASURED_PEAKS.json) / "
                           "(2T + 2(d+2)) flops per entry; SFU roof: measured ex2 per SM per clock "
                           "(libciq_peaks) x 148 SMs x the SM clock sampled during the timed solves)",
            "tensor": {"achieved_tflops": alg, "peak_tflops": peak, "frac": alg / peak if peak else None,
                       "peak_burst_tflops": burst, "frac_burst": alg / burst if burst else None,
                       "executed_tflops": executed, "frac_executed": executed / peak if peak else None,
                       "roof_gentries_per_s": tensor_roof},
            "sfu": {"achieved_ex2_per_s": sfu_rate, "peak_ex2_per_s": sfu_peak,
                    "frac": sfu_rate / sfu_peak if sfu_peak else None,
                    "ex2_per_sm_per_clk": per_clk, "sm_mhz": mhz,
                    "peak_measured_at_mhz": dev.get("sfu_sm_mhz"),
                    "roof_gentries_per_s": sfu_roof}}


def roofline_fp32(N, T, d, t_launch_ms, pk):
    # Algorithmic work of one kernel MVM on CUDA cores: 2 N^2 T flops for the
    # product with the T-column block plus 3 d N^2 flops for the distances.
    flops = 2.0 * N * N * T + 3.0 * d * N * N
    achieved = flops / (t_launch_ms * 1e-3) / 1e12
    peak = SM_COUNT * FP32_LANES_PER_SM * 2 * pk.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None,
            "kernel": "mvm_wide (FP32 CUDA-core on-the-fly kernel MVM)",
            "peak_note": "148 SMs x 128 FP32 lanes x 2 flop x max SM clock (derived, not measured)"}


# ------------------------------------------------------------------- main --
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def whole_job_rate(elapsed_ms, units_per_rank, dist=None, device="cpu"):
    """The slowest rank's timed region and the whole-job rate over it.

    Every rank passes its own elapsed time (ms) and the units it processed;
    with a process group the times are reduced with MAX, so the rate is the
    units all ranks processed divided by the slowest rank's time.
    """
    world = dist.get_world_size() if dist is not None and dist.is_initialized() else 1
    if world > 1:
        import torch
        t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    return elapsed_ms, units_per_rank * world / (elapsed_ms * 1e-3)


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    W = WORKLOAD
    X, B = W.make()
    X = X.astype(np.float32).astype(np.float64)       # the FP32 inputs our arm solves
    B = B.astype(np.float32).astype(np.float64)
    Q = W.q
    for _ in range(args.warmup):                       # untimed warm-up samples
        oracle_iteration_seconds(X, B, Q, rows=REF_SAMPLE_ROWS)
    steps = []
    for _ in range(args.steps):
        t_iter, t_spent, rows = oracle_iteration_seconds(X, B, Q, rows=REF_SAMPLE_ROWS)
        steps.append(t_iter)
    t_iter = statistics.median(steps)
    t_solve = t_iter * (LANCZOS_ITERS + J_WORKLOAD)
    value = W.t / t_solve
    line = {"impl": "reference", "metric": "K^{1/2}b RHS-solves/s at rel err <=1e-3", "value": value,
            "unit": "RHS-solves/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_solve * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": headline_config(args.precision, world),
            "run": {"arithmetic": "fp64 (the oracle)", "krylov": "recurrence", "iterations": [J_WORKLOAD] * args.steps},
            "cpu_baseline": {"value": value, "unit": "RHS-solves/s", "cores": cpu_threads(), "kind": "oracle",
                             "sample": f"per step: oracle kernel MVM on {rows} of {W.n} rows (scaled x{W.n / rows:.2f}) "
                                       f"+ one full-size oracle msMINRES vector step; x{LANCZOS_ITERS + J_WORKLOAD} iterations"},
            "e2e": {"value": value, "unit": "RHS-solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2006_11267_b300 as P

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    W = WORKLOAD
    if args.n:
        import dataclasses
        W = dataclasses.replace(W, n=args.n, name=f"{W.name}_first{args.n}")
    seed_shift = rank            # independent replica per rank
    X = np.asarray(ci.points(W.seed + seed_shift, W.n, W.d), dtype=np.float32)
    B = np.asarray(ci.rhs(W.seed + seed_shift, W.n, W.t), dtype=np.float32)
    Xd = torch.from_numpy(X).to(dev)
    Bd = torch.from_numpy(B).to(dev)
    out = torch.empty_like(Bd)
    k = P.Kernel(W.kernel, W.lengthscale, W.outputscale, W.noise)
    opts = dict(stop_rule="errbound", max_iter=MAX_ITER, lanczos_iters=LANCZOS_ITERS, precision=args.precision,
                krylov=args.krylov,
                check_every=16)

    def step(profile=0):
        return P.ciq_sqrt(Xd, k, Bd, W.q, TOL, out=out, profile=profile, **opts)[1]

    if args.mvm_only:
        n = args.mvm_only
        Xs, Vs = Xd[:n].contiguous(), Bd[:, :n].contiguous()
        for _ in range(max(1, args.warmup)):
            P.ciq_kernel_mvm(Xs, k, Vs, precision=args.precision)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            P.ciq_kernel_mvm(Xs, k, Vs, precision=args.precision)
        e1.record()
        torch.cuda.synchronize()
        print(json.dumps({"mvm_only": n, "T": W.t, "precision": args.precision,
                          "ms_per_call": e0.elapsed_time(e1) / args.steps}), flush=True)
        return 0

    for _ in range(args.warmup):
        info = step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = []
    for _ in range(args.steps):
        infos.append(step())
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    elapsed_ms, value = whole_job_rate(e0.elapsed_time(e1), W.t * args.steps, dist if world > 1 else None, dev)
    ms_per_step = elapsed_ms / args.steps
    launches = sum(i["launches"] for i in infos)
    # One profiled solve: per-launch CUDA events on the library's stream.
    pinfo = step(profile=1)
    torch.cuda.synchronize()
    t_mvm = pinfo["t_mvm_ms"] / max(1, pinfo["mvm_launches"])
    t_rec = pinfo["t_step_ms"] / max(1, pinfo["step_launches"])
    pk, pk_kind = peaks()
    devpk = device_peaks()
    if args.precision == "fp32":
        roof = roofline_fp32(W.n, W.t, W.d, t_mvm, pk)
        roof["peak_source"] = pk_kind
    else:
        roof = roofline_tc(W, t_mvm, devpk, pk, clocks.get("sm_mhz"))
    fp32 = None
    if not args.no_fp32_compare and args.precision != "fp32":
        o32 = dict(opts, precision="fp32")
        P.ciq_sqrt(Xd, k, Bd, W.q, TOL, out=out, **o32)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record()
        i32 = P.ciq_sqrt(Xd, k, Bd, W.q, TOL, out=out, **o32)[1]
        f1.record()
        torch.cuda.synchronize()
        t32 = f0.elapsed_time(f1)
        fp32 = {"value": W.t / (t32 * 1e-3), "ms_per_step": t32, "iterations": i32["iters"],
                "speedup": (W.t / (t32 * 1e-3)) / (W.t * args.steps / (elapsed_ms * 1e-3) / world)}
        fp32["speedup"] = 1.0 / fp32["speedup"]
    e2e = None
    if not args.no_e2e:
        out_h = np.empty_like(B)
        for _ in range(1):
            P.ciq_sqrt(X, k, B, W.q, TOL, out=out_h, **opts)
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            P.ciq_sqrt(X, k, B, W.q, TOL, out=out_h, **opts)
        _, e2e_rate = whole_job_rate((time.perf_counter() - t0) * 1e3, W.t * args.steps,
                                     dist if world > 1 else None, dev)
        e2e = {"value": e2e_rate, "unit": "RHS-solves/s",
               "h2d_bytes_per_step": int(X.nbytes + B.nbytes), "d2h_bytes_per_step": int(out_h.nbytes)}
    cpu = None
    oracle_err = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.n:
        oracle_err = headline_oracle_check(P, torch, dev, opts)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        J = int(statistics.median(i["iters"] for i in infos))
        t_iter, t_spent, rows = oracle_iteration_seconds(X.astype(np.float64), B.astype(np.float64), W.q)
        cpu = {"value": W.t / (t_iter * (LANCZOS_ITERS + J)), "unit": "RHS-solves/s", "cores": cpu_threads(),
               "kind": "oracle",
               "sample": f"oracle kernel MVM on {rows} of {W.n} rows (scaled x{W.n / rows:.2f}) + one full-size "
                         f"oracle msMINRES vector step = one iteration ({t_spent:.1f} s measured); "
                         f"x{LANCZOS_ITERS + J} iterations (pre-pass + the J={J} this run needed)"}
    if rank == 0:
        it = [i["iters"] for i in infos]
        line = {"metric": "K^{1/2}b RHS-solves/s at rel err <=1e-3", "value": value, "unit": "RHS-solves/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if args.precision == "fp32" else f"{args.precision}x2-split tiles, f32 vectors, f64 scalars",
                "data": "synthetic",
                "config": headline_config(args.precision, world),
                "run": {"krylov": infos[0].get("krylov"), "iterations": it,
                        "errbound_max": max(i["errbound_max"] for i in infos)},
                "roofline": roof,
                "kernels": {"mvm_ms_per_launch": t_mvm, "recurrence_ms_per_launch": t_rec,
                            "mvm_share": pinfo["t_mvm_ms"] / max(pinfo["t_total_ms"], 1e-9),
                            "recurrence_share": pinfo["t_step_ms"] / max(pinfo["t_total_ms"], 1e-9),
                            "prepass_ms": pinfo["t_prepass_ms"], "total_ms": pinfo["t_total_ms"]},
                "oracle_err": oracle_err,
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
                "plain_fp32_gpu_path": fp32, "device_peaks": devpk}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_batched(args):
    """The uneven batch: one ciq_sqrt_batched call per step, against the plain
    FP32 GPU path (one ciq_sqrt call per problem) on the same problems."""
    import torch

    import paper_2006_11267_b300 as P

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    raw = ci.batched_problems(BATCH_SEED + rank, count=BATCH_COUNT, t=BATCH_T)
    host = [dict(X=torch.from_numpy(p["X"].astype(np.float32)).pin_memory(),
                 B=torch.from_numpy(p["B"].astype(np.float32)).pin_memory()) for p in raw]
    probs = [dict(X=h["X"].to(dev), B=h["B"].to(dev),
                  kernel=P.Kernel(p["kernel"], p["lengthscale"], p["outputscale"], p["noise"]))
             for h, p in zip(host, raw)]
    for pr in probs:
        pr["out"] = torch.empty_like(pr["B"])
    opts = dict(max_iter=BATCH_MAX_ITER, lanczos_iters=LANCZOS_ITERS, check_every=8)
    bopts = dict(opts, precision=args.precision)
    if args.batch_only:
        bopts["graph"] = 0
    stream = torch.cuda.current_stream()

    def step():
        return P.ciq_sqrt_batched(probs, BATCH_Q, BATCH_TOL, **bopts)[1]

    for _ in range(args.warmup):
        infos = step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    launches = 0
    for _ in range(args.steps):
        infos = step()
        launches += infos[0]["launches"]
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    elapsed_ms = e0.elapsed_time(e1)
    rhs = BATCH_COUNT * BATCH_T
    value = rhs * args.steps / (elapsed_ms * 1e-3)
    if args.batch_only:
        if rank == 0:
            print(json.dumps({"batch_only": True, "ms_per_batch": elapsed_ms / args.steps,
                              "launches_per_batch": launches // max(args.steps, 1)}), flush=True)
        return 0
    # Plain FP32 GPU path: the same problems, one ciq_sqrt call each.
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    refs = []
    for pr in probs:
        o, _ = P.ciq_sqrt(pr["X"], pr["kernel"], pr["B"], BATCH_Q, BATCH_TOL, **opts)
        refs.append(o)
    f1.record(stream)
    torch.cuda.synchronize()
    t_seq = f0.elapsed_time(f1)
    same = sum(int(torch.equal(o, pr["out"])) for o, pr in zip(refs, probs))
    diffs = [float(torch.linalg.norm((o - pr["out"]).double()) / torch.linalg.norm(o.double())) for o, pr in
             zip(refs, probs)]
    # The batched form with CUDA-core FP32 tiles, for context.
    b32 = None
    if args.precision != "fp32":
        P.ciq_sqrt_batched(probs, BATCH_Q, BATCH_TOL, **opts)
        torch.cuda.synchronize()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        P.ciq_sqrt_batched(probs, BATCH_Q, BATCH_TOL, **opts)
        g1.record(stream)
        torch.cuda.synchronize()
        b32 = {"value": BATCH_COUNT * BATCH_T / (g0.elapsed_time(g1) * 1e-3), "ms_per_step": g0.elapsed_time(g1)}
    # End to end: pinned host inputs in, outputs back to the host, each step.
    outs_h = [torch.empty_like(h["B"]).pin_memory() for h in host]
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for h, pr in zip(host, probs):
            pr["X"].copy_(h["X"], non_blocking=True)
            pr["B"].copy_(h["B"], non_blocking=True)
        step()
        for o, pr in zip(outs_h, probs):
            o.copy_(pr["out"], non_blocking=True)
        torch.cuda.synchronize()
    t_e2e = (time.perf_counter() - t0) / args.steps
    its = [i["iters"] for i in infos]
    # The autotuned launch shape: the first use measures every candidate
    # once (a fresh table), then the tuned shape is timed like the default.
    from paper_2006_11267_b300 import autotune
    tune_path = os.path.join(tempfile.gettempdir(), f"ciq_autotune_bench_{os.getpid()}.json")
    best, cand_ms = autotune.tune(probs, BATCH_Q, BATCH_TOL, path=tune_path, **bopts)
    topts = dict(bopts, **best)
    P.ciq_sqrt_batched(probs, BATCH_Q, BATCH_TOL, **topts)
    torch.cuda.synchronize()
    h0 = torch.cuda.Event(enable_timing=True)
    h1 = torch.cuda.Event(enable_timing=True)
    h0.record(stream)
    for _ in range(args.steps):
        tinfos = P.ciq_sqrt_batched(probs, BATCH_Q, BATCH_TOL, **topts)[1]
    h1.record(stream)
    torch.cuda.synchronize()
    tuned_ms = h0.elapsed_time(h1) / args.steps
    os.unlink(tune_path)
    autotuned = {"autotuned": True, "best": best, "default_ms_per_step": elapsed_ms / args.steps,
                 "tuned_ms_per_step": tuned_ms, "gain": (elapsed_ms / args.steps) / tuned_ms,
                 "tuned_rhs_solves_per_s": BATCH_COUNT * BATCH_T / (tuned_ms * 1e-3),
                 "tuned_unconverged_columns": int(sum(BATCH_T - i["converged"] for i in tinfos)),
                 "candidates_ms": cand_ms,
                 "note": "the line's value is the default launch shape (one CTA per row tile, check_every 8)"}
    # Roofline of the batch: kernel entries evaluated over every live
    # problem (each MVM of problem p, pre-pass included, covers N_p^2
    # entries), against the SFU roof (1 ex2 per RBF entry, sqrt + ex2 per
    # Matern entry; T = 8 leaves the tensor pipe far from binding), at the
    # measured ex2 rate per SM and clock and the clock sampled while timing.
    ent = [float(i["iters"] + i["lanczos_iters"]) * p["n"] ** 2 for i, p in zip(infos, raw)]
    sfu_ops = sum(e * (1 if p["kernel"] == "rbf" else 2) for e, p in zip(ent, raw))
    secs = elapsed_ms / args.steps * 1e-3
    devpk = device_peaks()
    per_clk = devpk.get("sfu_ex2_per_sm_per_clk")
    mhz = clocks.get("sm_mhz") or devpk.get("sfu_sm_mhz")
    sfu_peak = per_clk * SM_COUNT * mhz * 1e6 if per_clk and mhz else None
    roof = {"bound": "sfu", "achieved": sfu_ops / secs / 1e9, "peak": sfu_peak / 1e9 if sfu_peak else None,
            "unit": "G ex2/s", "frac": sfu_ops / secs / sfu_peak if sfu_peak else None, "traffic": None,
            "entries_per_s": sum(ent) / secs,
            "kernel": "the whole batched solve (tensor-core MVM over every live problem, recurrence, pre-pass)",
            "peak_source": "measured ex2 per SM per clock (libciq_peaks) x 148 SMs x the sampled SM clock"}
    line = {"metric": "K^{1/2}b RHS-solves/s, uneven batch (batched vs plain FP32)", "value": value,
            "unit": "RHS-solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else f"{args.precision}x2-split tiles, f32 vectors, f64 scalars",
            "data": "synthetic",
            "config": {"workload": f"batched{BATCH_COUNT}_uneven_t{BATCH_T}_q{BATCH_Q}", "problems": BATCH_COUNT,
                       "T": BATCH_T, "Q": BATCH_Q, "tol": BATCH_TOL, "stop_rule": "residual",
                       "max_iter": BATCH_MAX_ITER, "seed": BATCH_SEED,
                       "sum_n2": int(sum(p["n"] ** 2 for p in raw)),
                       "iterations": {"max": max(its), "median": float(np.median(its)), "mean": float(np.mean(its))},
                       "unconverged_columns": int(sum(BATCH_T - i["converged"] for i in infos)),
                       "l2": "no flush: each step streams every problem's workspace (> 1 GB)"},
            "plain_fp32_gpu_path": {"value": rhs / (t_seq * 1e-3), "ms_per_step": t_seq,
                                    "speedup": t_seq / (elapsed_ms / args.steps),
                                    "outputs_bitwise_equal": f"{same}/{BATCH_COUNT}",
                                    "max_rel_diff": max(diffs), "median_rel_diff": float(np.median(diffs))},
            "batched_fp32": b32,
            "e2e": {"value": rhs / t_e2e, "unit": "RHS-solves/s",
                    "h2d_bytes_per_step": int(sum(h["X"].nbytes + h["B"].nbytes for h in host)),
                    "d2h_bytes_per_step": int(sum(o.nbytes for o in outs_h))},
            "gpu_launches": launches, "clocks": clocks, "cpu_baseline": None, "roofline": roof,
            "autotune": autotuned}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_stored(args):
    """Stored-K MVM (the explicit-matrix case of Sec. 3.3): K = K_XX + sigma^2 I
    of the 50,000-point RBF workload and of its 80,000-point extension formed
    once in HBM (FP32: 10.0 and 25.6 GB), then streamed by every MVM.  One
    column reads K once per MVM with float4 loads and is HBM-bound: 4 Npad^2
    bytes against the measured copy rate (T = 8 reads it once too, four rows
    per warp sharing each V load).  T = 64 runs
    the register-tiled FP32 product (32 flops per byte of K: FP32-FMA-bound,
    reported against the derived FP32 rate).  Beside it the headline solve
    with the stored MVM (FP32) for comparison with the on-the-fly paths."""
    import torch

    import paper_2006_11267_b300 as P

    torch.cuda.set_device(0)
    pk, pk_kind = peaks()
    W = WORKLOAD
    k = P.Kernel(W.kernel, W.lengthscale, W.outputscale, W.noise)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    sizes = {}
    ns = (args.n,) if args.n else (50000, 80000)
    for n in ns:
        npad = -(-n // 128) * 128
        X = torch.from_numpy(ci.points(W.seed, n, W.d).astype(np.float32)).cuda()
        K = torch.empty((npad, npad), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        e0.record()
        P.ciq_kernel_matrix(X, k, K)
        e1.record()
        torch.cuda.synchronize()
        form_ms = e0.elapsed_time(e1)
        res = {"form_ms": form_ms, "K_GB": 4.0 * npad * npad / 1e9}
        for t, prec in ((1, "fp32"), (8, "fp32"), (64, "fp32"), (1, "fp16"), (8, "fp16"), (64, "fp16")):
            V = torch.from_numpy(ci.rhs(W.seed + 3, n, t).astype(np.float32)).cuda()
            out = torch.empty_like(V)
            for _ in range(2):
                P.ciq_stored_mvm(K, V, out, precision=prec)
            torch.cuda.synchronize()
            reps = 5
            e0.record()
            for _ in range(reps):
                P.ciq_stored_mvm(K, V, out, precision=prec)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            nbytes = 4.0 * npad * npad + 4.0 * 2 * t * n
            gbs = nbytes / (ms * 1e-3) / 1e9
            flops = 2.0 * npad * npad * t
            key = f"t{t}" if prec == "fp32" else f"t{t}_fp16"
            res[key] = {"ms": ms, "GB_s": gbs, "frac_hbm": gbs / pk["hbm_gbs"],
                        "TFLOP_s": flops / (ms * 1e-3) / 1e12}
        sizes[str(n)] = res
        del K
        torch.cuda.empty_cache()
    if args.n:                    # a profiling case: the MVMs only
        print(json.dumps({"stored_only": args.n, "sizes": sizes}), flush=True)
        return 0
    # The headline solve with the stored MVM (K of 10 GB formed inside the call).
    n = W.n
    X = torch.from_numpy(ci.points(W.seed, n, W.d).astype(np.float32)).cuda()
    B = torch.from_numpy(ci.rhs(W.seed, n, W.t).astype(np.float32)).cuda()
    P.ciq_sqrt(X, k, B, W.q, 1e-3, stop_rule="errbound", max_iter=4000, mvm="stored")
    torch.cuda.synchronize()
    e0.record()
    _, info = P.ciq_sqrt(X, k, B, W.q, 1e-3, stop_rule="errbound", max_iter=4000, mvm="stored")
    e1.record()
    torch.cuda.synchronize()
    solve_ms = e0.elapsed_time(e1)
    # The same solve with the stored K on tensor cores (FP16 split of K and
    # V), and its MVM time per launch from the library's profile mode.
    P.ciq_sqrt(X, k, B, W.q, 1e-3, stop_rule="errbound", max_iter=4000, mvm="stored", precision="fp16")
    torch.cuda.synchronize()
    e0.record()
    _, info16 = P.ciq_sqrt(X, k, B, W.q, 1e-3, stop_rule="errbound", max_iter=4000, mvm="stored",
                           precision="fp16")
    e1.record()
    torch.cuda.synchronize()
    solve16_ms = e0.elapsed_time(e1)
    _, infop = P.ciq_sqrt(X, k, B, W.q, 0.0, max_iter=40, lanczos_iters=10, mvm="stored", precision="fp16",
                          profile=1)
    mvm16_ms = infop["t_mvm_ms"] / max(1, infop["mvm_launches"])
    fp32_rate = SM_COUNT * FP32_LANES_PER_SM * 2 * pk.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
    head = sizes["50000"]["t64_fp16"]
    npad50 = -(-50000 // 128) * 128
    line = {"metric": "stored-K MVM HBM GB/s (64 columns, N=50,000, tensor cores)", "value": head["GB_s"],
            "unit": "GB/s", "n_gpus": 1, "steps": 5, "warmup": 2, "higher_is_better": True,
            "dtype": "fp16x2 split K and V, f32 accumulation (the fp32 entries: f32 CUDA cores)", "data": "synthetic",
            "config": {"workload": f"stored_{W.name}", "N": [50000, 80000], "T": [1, 8, 64], "d": W.d,
                       "kernel": W.kernel, "l2": "no flush: K (10 / 25.6 GB) is far larger than L2"},
            "roofline": {"bound": "hbm", "achieved": head["GB_s"], "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": head["frac_hbm"], "traffic": None,
                         "kernel": "stored_tc_kernel<64, FP16> (TMA boxes of K, split in TMEM, tcgen05 products); "
                                   "the call also reads K's diagonal and synchronises once. In the solve: "
                                   f"{mvm16_ms:.3f} ms per MVM = "
                                   f"{4.0 * npad50 * npad50 / (mvm16_ms * 1e-3) / 1e9:.0f} GB/s of K",
                         "peak_source": f"{pk_kind} copy rate (MEASURED_PEAKS.json)",
                         "t64_fp32_alu_peak_tflops": fp32_rate},
            "sizes": sizes,
            "stored_solve": {"RHS_solves_per_s": W.t / (solve_ms * 1e-3), "ms": solve_ms, "iterations": info["iters"],
                             "errbound_max": info["errbound_max"], "precision": "fp32"},
            "stored_solve_fp16": {"RHS_solves_per_s": W.t / (solve16_ms * 1e-3), "ms": solve16_ms,
                                  "iterations": info16["iters"], "errbound_max": info16["errbound_max"],
                                  "mvm_ms_in_solve": mvm16_ms}}
    print(json.dumps(line), flush=True)
    return 0


def run_precision(args):
    """Precision sweep, 200,000-point Matern-5/2 workload, K^{-1/2}B, Q = 15:
    per mode (plain FP32, FP16 split, BF16 split, TF32 tiles) the solve error against the
    FP64 eigendecomposition on a 4096-point subsample (T = 256), and at full
    size the MVM time and its difference from the FP32 MVM, and the time per
    msMINRES iteration (a fixed 10-iteration solve)."""
    import torch

    import paper_2006_11267_b300 as P
    from oracle import eig, kernels

    torch.cuda.set_device(0)
    W = ci.PRECISION_200K
    k = P.Kernel(W.kernel, W.lengthscale, W.outputscale, W.noise)
    modes = ("fp32", "fp16", "bf16", "tf32")
    n_sub = 4096
    Xs = ci.points(W.seed, W.n, W.d)[:n_sub].astype(np.float32)
    Bs = ci.rhs(W.seed + 1, n_sub, W.t).astype(np.float32)
    K = kernels.dense_K(Xs.astype(np.float64), W.kernel, W.lengthscale, W.outputscale, W.noise)
    truth = eig.invsqrt_apply(K, Bs.T.astype(np.float64)).T
    Xd, Bd = torch.from_numpy(Xs).cuda(), torch.from_numpy(Bs).cuda()
    sub = {}
    for m in modes:
        out, info = P.ciq_invsqrt(Xd, k, Bd, W.q, 1e-4, max_iter=2000, precision=m)
        torch.cuda.synchronize()
        col = np.linalg.norm(out.cpu().numpy() - truth, axis=1) / np.linalg.norm(truth, axis=1)
        sub[m] = {"rel_err_vs_fp64_eig": float(col.max()), "median_col_err": float(np.median(col)),
                  "iterations": info["iters"], "status": info["status_name"]}
    X = torch.from_numpy(ci.points(W.seed, W.n, W.d).astype(np.float32)).cuda()
    B = torch.from_numpy(ci.rhs(W.seed, W.n, W.t).astype(np.float32)).cuda()
    full = {}
    ref = None
    for m in modes:
        P.ciq_kernel_mvm(X, k, B, precision=m)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        out = P.ciq_kernel_mvm(X, k, B, precision=m)
        e1.record()
        torch.cuda.synchronize()
        if m == "fp32":
            ref = out.clone()
        diff = float(torch.linalg.norm((out - ref).double()) / torch.linalg.norm(ref.double()))
        # msMINRES iterations timed by the library's profile mode (CUDA
        # events between consecutive launches): MVM + recurrence.
        _, info = P.ciq_invsqrt(X, k, B, W.q, 0.0, max_iter=12, lanczos_iters=10, precision=m, profile=1,
                                check_every=4)
        it_ms = (info["t_mvm_ms"] / max(1, info["mvm_launches"]) + info["t_step_ms"] / max(1, info["step_launches"]))
        full[m] = {"mvm_call_ms": e0.elapsed_time(e1), "mvm_rel_diff_vs_fp32": diff, "ms_per_iteration": it_ms,
                   "mvm_ms_in_solve": info["t_mvm_ms"] / max(1, info["mvm_launches"])}
    # Whole solves at the workload's stop rule (relative residual 1e-4):
    # RHS-solves/s and the iterations each mode needs.  The FP32 solve (about
    # 0.75 s per iteration) runs in full only with --full-fp32; otherwise its
    # time is the FP16 solve's iteration count times its measured
    # per-iteration time (labelled as such).
    solves = {}
    for m in modes:
        if m == "fp32" and not args.full_fp32:
            continue
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record()
        _, info = P.ciq_invsqrt(X, k, B, W.q, W.tol, max_iter=3000, lanczos_iters=10, precision=m, check_every=16)
        g1.record()
        torch.cuda.synchronize()
        ms = g0.elapsed_time(g1)
        solves[m] = {"rhs_solves_per_s": W.t / (ms * 1e-3), "ms": ms, "iterations": info["iters"],
                     "status": info["status_name"], "resid_max": info["resid_max"], "measured": "full solve"}
    if "fp32" not in solves and "fp16" in solves:
        J = solves["fp16"]["iterations"] + 10
        ms = J * full["fp32"]["ms_per_iteration"]
        solves["fp32"] = {"rhs_solves_per_s": W.t / (ms * 1e-3), "ms": ms, "iterations": None,
                          "measured": f"extrapolated: the FP16 solve's {J} MVMs x the measured FP32 ms/iteration"}
    line = {"metric": "K^{-1/2}b precision sweep (error vs FP64 oracle per mode)", "value": full["fp16"]["ms_per_iteration"],
            "unit": "ms/iteration (FP16 split, N=200000, T=256)", "n_gpus": 1, "steps": 1, "warmup": 1,
            "higher_is_better": False, "dtype": "f32 / fp16x2 / bf16x2 / tf32 tiles, f64 scalars", "data": "synthetic",
            "config": {"workload": W.name, "N": W.n, "d": W.d, "kernel": W.kernel, "lengthscale": W.lengthscale,
                       "noise": W.noise, "T": W.t, "Q": W.q, "op": "invsqrt", "subsample": n_sub,
                       "subsample_tol": 1e-4},
            "subsample": sub, "full_size": full, "solves": solves}
    print(json.dumps(line), flush=True)
    return 0


def run_learned(args):
    """Learned spectral bounds on the uneven-batch distribution: labels for
    20,000 instances from the library's batched solve with its Lanczos
    pre-pass (FP16 split tiles), GPU training of the predictor, then 4096
    held-out instances solved with predicted bounds (fallback to the
    pre-pass on a spectral check) and with the pre-pass, both timed; the
    oracle judges the 64 smallest held-out problems."""
    import torch

    import paper_2006_11267_b300 as P
    from paper_2006_11267_b300 import learned
    from oracle import eig, kernels

    torch.cuda.set_device(0)
    prec = args.precision
    opts = dict(max_iter=BATCH_MAX_ITER, lanczos_iters=LANCZOS_ITERS, check_every=8, precision=prec)

    def device_batch(raw):
        return [dict(X=torch.from_numpy(p["X"].astype(np.float32)).cuda(),
                     B=torch.from_numpy(p["B"].astype(np.float32)).cuda(),
                     kernel=P.Kernel(p["kernel"], p["lengthscale"], p["outputscale"], p["noise"])) for p in raw]

    t0 = time.perf_counter()
    Fs, Ys = [], []
    n_train = 20000
    label_opts = dict(opts, max_iter=1000)        # iteration labels saturate at 1000
    for b0 in range(0, n_train, BATCH_COUNT):
        raw = ci.batched_problems(BATCH_SEED + 1000 + b0 // BATCH_COUNT, count=min(BATCH_COUNT, n_train - b0),
                                  t=BATCH_T)
        F, Y, _ = learned.label_problems(device_batch(raw), BATCH_Q, BATCH_TOL, **label_opts)
        Fs.append(F)
        Ys.append(Y)
    F = torch.cat(Fs)
    Y = torch.cat(Ys)
    t_label = time.perf_counter() - t0
    n_val = 2000
    t0 = time.perf_counter()
    theta, losses = learned.train_predictor(F[n_val:].contiguous(), Y[n_val:].contiguous(), steps=8000, batch=256,
                                            lr=2e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    Fv, Yv = F[:n_val].contiguous(), Y[:n_val].contiguous()
    margin = learned.lmax_margin_from_validation(theta, Fv, Yv, 0.999)
    pv = P.ciq_mlp_predict(theta, Fv).cpu().numpy()
    yv = Yv.cpu().numpy()
    rmse = np.sqrt(np.mean((pv - yv) ** 2, axis=0)).tolist()
    # Held-out instances, all resident.  The pre-pass pipeline solves them in
    # batches of 512 in index order; the learned pipeline predicts every
    # problem first (its bounds and its iteration count) and sizes its batch
    # schedule ahead of time: the problems predicted to need >= 500
    # iterations in one batch, the rest in batches of 512 in order of
    # predicted iterations, each solved with the predicted bounds.
    raw_test = ci.batched_problems(BATCH_SEED + 999, count=4096, t=BATCH_T)
    test = device_batch(raw_test)
    res = {"prepass": {"ms": 0.0}, "learned": {"ms": 0.0}}
    outs_all = {"prepass": [None] * len(test), "learned": [None] * len(test)}
    fallbacks = 0
    work = {"prepass": 0, "learned": 0}
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    pred = P.ciq_mlp_predict(theta, P.ciq_mlp_features(test))
    schedule = learned.batch_schedule(pred[:, 2].cpu().numpy(), batch=BATCH_COUNT, long_iters=500)
    e1.record()
    torch.cuda.synchronize()
    res["learned"]["ms"] += e0.elapsed_time(e1)
    index_batches = [list(range(b0, min(b0 + BATCH_COUNT, len(test)))) for b0 in range(0, len(test), BATCH_COUNT)]
    for mode, batches in (("prepass", index_batches), ("learned", schedule)):
        for ids in batches:
            probs = [test[i] for i in ids]
            for pr in probs:
                pr["out"] = torch.empty_like(pr["B"])
            torch.cuda.synchronize()
            e0.record()
            if mode == "prepass":
                outs, infos = P.ciq_sqrt_batched(probs, BATCH_Q, BATCH_TOL, **opts)
            else:
                outs, infos = P.ciq_sqrt_batched_learned(probs, BATCH_Q, BATCH_TOL, theta, margin, **opts)
                fallbacks += sum(i["fallback"] for i in infos)
            e1.record()
            torch.cuda.synchronize()
            res[mode]["ms"] += e0.elapsed_time(e1)
            work[mode] += sum(i["iters"] + i["lanczos_iters"] for i in infos)
            for i, o in zip(ids, outs):
                outs_all[mode][i] = o.cpu().numpy()
    # Oracle errors on the 64 smallest held-out problems.
    small = sorted(range(len(raw_test)), key=lambda i: raw_test[i]["n"])[:64]
    errs = {"prepass": [], "learned": []}
    for i in small:
        p = raw_test[i]
        X = p["X"].astype(np.float32).astype(np.float64)
        K = kernels.dense_K(X, p["kernel"], p["lengthscale"], p["outputscale"], p["noise"])
        truth = eig.sqrt_apply(K, p["B"].astype(np.float32).astype(np.float64).T).T
        for mode in errs:
            errs[mode].append(float(np.linalg.norm(outs_all[mode][i] - truth) / np.linalg.norm(truth)))
    rhs = len(raw_test) * BATCH_T
    line = {"metric": "K^{1/2}b RHS-solves/s with learned spectral bounds (vs Lanczos pre-pass)",
            "value": rhs / (res["learned"]["ms"] * 1e-3), "unit": "RHS-solves/s", "n_gpus": 1, "steps": 1,
            "warmup": 0, "higher_is_better": True, "dtype": f"{prec}x2-split tiles, f32 vectors, f64 scalars",
            "data": "synthetic",
            "config": {"workload": "learned_bounds_uneven_t8_q8", "train": n_train, "validation": n_val,
                       "held_out": len(raw_test), "network": "38-64-64-3 tanh, FP32 training, BF16 inference",
                       "label_max_iter": 1000, "tol": BATCH_TOL, "Q": BATCH_Q},
            "prepass_pipeline": {"value": rhs / (res["prepass"]["ms"] * 1e-3), "ms": res["prepass"]["ms"],
                                 "mvm_work": work["prepass"]},
            "learned_pipeline": {"ms": res["learned"]["ms"], "mvm_work": work["learned"], "fallbacks": fallbacks,
                                 "margin_log": margin, "batches": [len(b) for b in schedule]},
            "gain": res["prepass"]["ms"] / res["learned"]["ms"],
            "validation_rmse_log": {"theta_min": rmse[0], "theta_max": rmse[1], "iterations": rmse[2]},
            "oracle_rel_err_64_smallest": {m: {"max": max(v), "median": float(np.median(v))} for m, v in errs.items()},
            "seconds": {"labels": t_label, "training": t_train},
            "final_minibatch_loss": float(losses[-200:].mean())}
    print(json.dumps(line), flush=True)
    return 0


def run_spectrum(args):
    """The Q sweep of Sec. 5 (Fig. quad_error) on explicit matrices through
    ciq_sqrt_dense: spectra lambda_t = 1/sqrt(t) and 1/t^2 (K = U diag(lambda)
    U^T, U Haar-orthogonal) and a one-dimensional Matern-5/2 matrix on random
    points (l = 0.2, sigma^2 = 1e-4, formed by the library), N = 1024 and 4096,
    8 right-hand sides, Lanczos bounds, relative residual 1e-4 or J = 400 as
    in the study.  Error: relative 2-norm against the eigendecomposition of
    the FP32 matrix the solve sees (FP64 eigh on the host)."""
    import torch

    import paper_2006_11267_b300 as P

    torch.cuda.set_device(0)
    T, qs, kinds = 8, (2, 4, 6, 8, 12, 16), ("inv_sqrt", "inv_square", "matern1d")
    table = {}
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    worst8 = 0.0
    for kind in kinds:
        table[kind] = {}
        for n in (1024, 4096):
            if kind == "matern1d":
                npad = -(-n // 128) * 128
                X = torch.from_numpy(ci.points(20201109, n, 1).astype(np.float32)).cuda()
                Kd = torch.empty((npad, npad), dtype=torch.float32, device="cuda")
                P.ciq_kernel_matrix(X, P.Kernel("matern52", 0.2, 1.0, 1e-4), Kd)
                K32 = Kd[:n, :n].cpu().numpy()
                Kd = Kd[:n].contiguous()
            else:
                K32 = ci.spectrum_matrix(20201109, n, kind)[0].astype(np.float32)
                Kd = torch.from_numpy(K32).cuda()
            B = ci.rhs(20201110, n, T).astype(np.float32)
            w, V = np.linalg.eigh(K32.astype(np.float64))
            exact = (V * np.sqrt(np.clip(w, 0.0, None))[None, :]) @ (V.T @ B.T.astype(np.float64))
            Bd = torch.from_numpy(B).cuda()
            row = {"kappa": float(w[-1] / w[0]) if w[0] > 0 else None}
            for q in qs:
                P.ciq_sqrt_dense(Kd, Bd, q, 1e-4, max_iter=400, stop_rule="residual")
                torch.cuda.synchronize()
                e0.record()
                out, info = P.ciq_sqrt_dense(Kd, Bd, q, 1e-4, max_iter=400, stop_rule="residual")
                e1.record()
                torch.cuda.synchronize()
                A = out.cpu().numpy().T.astype(np.float64)
                err = float(np.max(np.linalg.norm(A - exact, axis=0) / np.linalg.norm(exact, axis=0)))
                row[str(q)] = {"rel_err": err, "iters": info["iters"], "ms": e0.elapsed_time(e1)}
                if q == 8:
                    worst8 = max(worst8, err)
            table[kind][str(n)] = row
    line = {"metric": "K^{1/2}b relative error against Q (synthetic spectra, explicit K)", "value": worst8,
            "unit": "max relative error at Q = 8", "n_gpus": 1, "steps": 1, "warmup": 1, "higher_is_better": False,
            "dtype": "f32 stored K, f32 vectors, f64 scalars", "data": "synthetic",
            "config": {"workload": "spectrum_sweep_t8", "T": T, "Q": list(qs), "N": [1024, 4096],
                       "stop_rule": "residual", "tol": 1e-4, "max_iter": 400, "spectra": list(kinds)},
            "table": table}
    print(json.dumps(line), flush=True)
    return 0


def run_vjp(args):
    """Backward pass (Sec. 3.4, Eq. ciq_deriv) on the 50,000-point RBF problem
    with T = 8 right-hand sides (a whitening / SVGP-sized block), Q = 12,
    error bound 1e-3, FP16 split tiles: the forward solve alone against the
    forward-and-backward call (one solve over [B | G], then the gradient
    contractions), and the contractions alone (the VJP call minus a forward
    solve over the same 2T columns).  The contraction pass is CUDA-core FP32:
    algorithmic work N^2 (2 Q T + 30) flops against the derived FP32 rate."""
    import torch

    import paper_2006_11267_b300 as P

    torch.cuda.set_device(0)
    W = WORKLOAD
    T = 8
    X = torch.from_numpy(ci.points(W.seed, W.n, W.d).astype(np.float32)).cuda()
    B = torch.from_numpy(ci.rhs(W.seed, W.n, T).astype(np.float32)).cuda()
    G = torch.from_numpy(ci.rhs(W.seed + 7, W.n, T).astype(np.float32)).cuda()
    BG = torch.cat([B, G], 0).contiguous()
    k = P.Kernel(W.kernel, W.lengthscale, W.outputscale, W.noise)
    opts = dict(stop_rule="errbound", max_iter=MAX_ITER, lanczos_iters=LANCZOS_ITERS, precision=args.precision)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            r = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, r

    reps = max(1, args.steps)
    t_fwd, (_, i_fwd) = timed(lambda: P.ciq_invsqrt(X, k, B, W.q, TOL, **opts), reps)
    t_fwd2, (_, i_fwd2) = timed(lambda: P.ciq_invsqrt(X, k, BG, W.q, TOL, **opts), reps)
    t_vjp, (_, _, gth, i_vjp) = timed(lambda: P.ciq_invsqrt_vjp(X, k, B, G, W.q, TOL, **opts), reps)
    t_con = max(t_vjp - t_fwd2, 1e-6)
    flops = float(W.n) ** 2 * (2 * W.q * T + 30)
    pk, _ = peaks()
    fp32_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * pk.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
    achieved = flops / (t_con * 1e-3) / 1e12
    line = {"metric": "K^{-1/2}B forward + backward (VJP) time", "value": t_vjp, "unit": "ms per call",
            "n_gpus": 1, "steps": reps, "warmup": 1, "higher_is_better": False,
            "dtype": f"{args.precision}x2-split tiles, f32 vectors, f64 scalars; f32 contractions", "data": "synthetic",
            "config": {"workload": "vjp_rbf_n50000_d6_t8_q12", "N": W.n, "d": W.d, "T": T, "Q": W.q, "tol": TOL,
                       "stop_rule": "errbound", "op": "invsqrt", "krylov": i_vjp.get("krylov")},
            "forward_ms": t_fwd, "forward_2T_ms": t_fwd2, "backward_over_forward": t_vjp / t_fwd,
            "iterations": {"forward": i_fwd["iters"], "forward_2T": i_fwd2["iters"], "vjp": i_vjp["iters"]},
            "contractions_ms": t_con, "grad_theta": [float(g) for g in gth],
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": achieved / fp32_peak, "traffic": None,
                         "kernel": "the contraction launches together (basis_solutions, vjp_bilinear on 64 x 64 tiles "
                                   "of K with 4 x 4 register blocks, vjp_dots); work counted is the bilinear pass's",
                         "peak_note": "148 SMs x 128 FP32 lanes x 2 flop x max SM clock (derived, not measured)"}}
    print(json.dumps(line), flush=True)
    return 0


PRECOND_RANKS = (100, 200, 400)
PRECOND_CHECK_N = 8192


def run_precond(args):
    """Preconditioned msMINRES-CIQ (App. "Preconditioning msMINRES-CIQ",
    Eq. precond_sqrt, Eq. precond_sqrt_inverse) on the 50,000-point RBF
    workload, against the unpreconditioned solve: for K^{1/2}-like (R b,
    R R^T = K) and K^{-1/2}-like (R' b, R' R'^T = K^{-1}) roots and pivoted
    Cholesky ranks 100, 200 and 400, the iterations, the time of a whole call
    (factor, eigendecomposition and basis included) and the RHS-solves/s at
    the error bound 1e-3 in the space msMINRES runs in (that of
    A = P^{-1/2} K P^{-1/2}).  CPU leg: the columns' relative error against
    the exact rotated roots (FP64 eigendecompositions of P and of A) on the
    workload's first PRECOND_CHECK_N points with the oracle's own factor, and
    of the unpreconditioned solve against the principal roots."""
    import torch

    import paper_2006_11267_b300 as P

    torch.cuda.set_device(0)
    W = WORKLOAD
    X = torch.from_numpy(ci.points(W.seed, W.n, W.d).astype(np.float32)).cuda()
    B = torch.from_numpy(ci.rhs(W.seed, W.n, W.t).astype(np.float32)).cuda()
    k = P.Kernel(W.kernel, W.lengthscale, W.outputscale, W.noise)
    if args.profile_rank:
        for _ in range(2):
            _, inf = P.ciq_invsqrt_precond(X, k, B, W.q, 0.0, rank=args.profile_rank, max_iter=40,
                                           precision=args.precision, lmin=1.0, lmax=1e5)
        torch.cuda.synchronize()
        print(json.dumps({"profile_rank": args.profile_rank, "iters": inf["iters"], "launches": inf["launches"]}))
        return 0
    opts = dict(stop_rule="errbound", max_iter=MAX_ITER, lanczos_iters=LANCZOS_ITERS, precision=args.precision,
                check_every=16)
    reps = max(1, args.steps)

    def timed(fn):
        for _ in range(max(1, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            r = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, r

    sampler = ClockSampler(0)
    sampler.start()
    table = {}
    # sqrt_mvm: R b = K (R' b), Eq. precond_sqrt as printed (R' b's solve and
    # stop rule, one more MVM); sqrt_identity: P^{1/2} times the estimate of
    # A^{1/2} b (fewer iterations, larger error in the space of K).
    forms = (("sqrt_identity", "sqrt", "identity"), ("sqrt_mvm", "sqrt", "mvm"), ("invsqrt", "invsqrt", "identity"))
    for name, op, form in forms:
        base = P.ciq_sqrt if op == "sqrt" else P.ciq_invsqrt
        pre = P.ciq_sqrt_precond if op == "sqrt" else P.ciq_invsqrt_precond
        ms, (_, inf) = timed(lambda: base(X, k, B, W.q, TOL, **opts))
        rows = {"0": {"iters": inf["iters"], "ms": ms, "rhs_solves_per_s": W.t / (ms * 1e-3)}}
        for r in PRECOND_RANKS:
            ms, (_, inf) = timed(lambda: pre(X, k, B, W.q, TOL, rank=r, sqrt_form=form, **opts))
            _, pinf = pre(X, k, B, W.q, TOL, rank=r, profile=1, sqrt_form=form, **opts)
            mvm = pinf["t_mvm_ms"] / max(1, pinf["mvm_launches"])
            setup = pinf["t_total_ms"] - pinf["t_mvm_ms"] - pinf["t_step_ms"] - pinf["t_prepass_ms"]
            rows[str(r)] = {"iters": inf["iters"], "ms": ms, "rhs_solves_per_s": W.t / (ms * 1e-3),
                            "speedup": rows["0"]["ms"] / ms, "lmax_used": inf["lmax_used"],
                            "precond_rank": inf["precond_rank"], "ms_per_iteration": mvm,
                            "prepass_ms": pinf["t_prepass_ms"], "setup_and_combine_ms": setup}
        table[name] = rows
    clocks = sampler.stop()
    check = None
    if not args.no_cpu_baseline:
        check = precond_oracle_check(P, torch, opts)
    best = max(PRECOND_RANKS, key=lambda r: table["invsqrt"][str(r)]["rhs_solves_per_s"])
    line = {"metric": "rotated K^{-1/2}b (R' b, R' R'^T = K^{-1}) RHS-solves/s at error bound 1e-3 (space of A), "
                      "pivoted-Cholesky preconditioner", "value": table["invsqrt"][str(best)]["rhs_solves_per_s"],
            "unit": "RHS-solves/s",
            "n_gpus": 1, "steps": reps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": f"{args.precision}x2-split tiles, f32 vectors and P^(+-1/2), f64 scalars",
            "data": "synthetic",
            "config": {"workload": "precond_" + W.name, "N": W.n, "d": W.d, "kernel": W.kernel,
                       "lengthscale": W.lengthscale, "noise": W.noise, "T": W.t, "Q": W.q, "tol": TOL,
                       "stop_rule": "errbound (space of A)", "ranks": list(PRECOND_RANKS), "best_rank": best,
                       "precision": args.precision},
            "table": table, "oracle_check": check, "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def precond_oracle_check(P, torch, opts):
    """Per-column relative errors of the preconditioned roots on the first
    PRECOND_CHECK_N points, with the oracle's pivoted Cholesky factor (FP64,
    rounded to FP32) passed to the library, against the exact rotated roots
    R b = K P^{-1/2} A^{-1/2} b and R' b = P^{-1/2} A^{-1/2} b; rank 0 is the
    unpreconditioned solve against the principal roots."""
    from oracle import eig, kernels
    from oracle import precond as PC

    W = WORKLOAD
    n = PRECOND_CHECK_N
    X, B = W.make(n)
    X = X.astype(np.float32)
    B = B.astype(np.float32)
    X64, B64 = X.astype(np.float64), B.astype(np.float64)
    k = P.Kernel(W.kernel, W.lengthscale, W.outputscale, W.noise)
    Kxx = kernels.kernel_matrix(X64, X64, W.kernel, W.lengthscale, W.outputscale)
    K = Kxx + W.noise * np.eye(n)
    Xd, Bd = torch.from_numpy(X).cuda(), torch.from_numpy(B).cuda()

    def errs(A, exact):
        e = np.linalg.norm(A - exact, axis=1) / np.linalg.norm(exact, axis=1)
        return {"max": float(e.max()), "median": float(np.median(e))}

    res = {"n": n}
    t0 = time.perf_counter()
    row = {}
    for op, base, f in (("sqrt", P.ciq_sqrt, eig.sqrt_apply), ("invsqrt", P.ciq_invsqrt, eig.invsqrt_apply)):
        A, inf = base(Xd, k, Bd, W.q, TOL, **opts)
        row[op] = dict(errs(A.cpu().numpy().astype(np.float64), f(K, B64.T).T), iters=inf["iters"])
    res["0"] = row
    for r in PRECOND_RANKS:
        L, _ = PC.pivoted_cholesky(np.diag(Kxx), lambda i: Kxx[:, i], r)
        L32 = L.astype(np.float32)
        Pm = PC.Preconditioner(L32.astype(np.float64), W.noise).dense()
        Rb, Rpb = PC.rotated_roots_exact(K, Pm, B64)
        Ld = torch.from_numpy(np.ascontiguousarray(L32.T)).cuda()
        row = {}
        for name, fn, form, exact in (("sqrt_identity", P.ciq_sqrt_precond, "identity", Rb),
                                      ("sqrt_mvm", P.ciq_sqrt_precond, "mvm", Rb),
                                      ("invsqrt", P.ciq_invsqrt_precond, "identity", Rpb)):
            A, inf = fn(Xd, k, Bd, W.q, TOL, L=Ld, sqrt_form=form, **opts)
            row[name] = dict(errs(A.cpu().numpy().astype(np.float64), exact), iters=inf["iters"])
        res[str(r)] = row
    res["oracle"] = "O1 of the preconditioned problem: FP64 eigendecompositions of P and A (LAPACK dsyevd)"
    res["oracle_seconds"] = time.perf_counter() - t0
    return res


POSTERIOR = dict(n_train=256, n_cand=50_000, d=6, kind="matern52", ls=(0.2, 0.25, 0.3, 0.35, 0.4, 0.45),
                 s=1.0, noise=1e-4, jitter=1e-4, mean=0.0, t=64, q=12, seed=20201112, check_n=4096,
                 pc_check_n=1024)
# Ranks of the posterior's pivoted-Cholesky preconditioner timed beside the
# unpreconditioned draws (the paper's BO runs use a rank-200 preconditioner).
POSTERIOR_PRECOND_RANKS = (100, 200)


def posterior_inputs(n_cand):
    """Synthetic Bayesian-optimisation state: training points and candidates
    uniform in [0,1]^6, observations of a smooth test function (a sum of
    sines; the paper's Hartmann and Lunar Lander runs are not reproduced),
    standard-normal eps."""
    c = POSTERIOR
    Xtr = ci.points(c["seed"], c["n_train"], c["d"]).astype(np.float32)
    Xc = ci.points(c["seed"] + 1, c["n_cand"], c["d"])[:n_cand].astype(np.float32)
    y = np.sin(2.0 * np.pi * Xtr.astype(np.float64) @ np.linspace(0.5, 1.5, c["d"])).astype(np.float32)
    eps = ci.rhs(c["seed"] + 2, c["n_cand"], c["t"])[:, :n_cand].astype(np.float32)
    return Xtr, y, Xc, np.ascontiguousarray(eps)


def run_posterior(args):
    """Posterior Thompson draws (Sec. 5, Eq. thompson_sample): 64 draws at
    50,000 candidates given 256 observations, Matern-5/2 with ARD
    lengthscales, sigma^2 = 1e-4, jitter 1e-4 (the paper's), Q = 12, error
    bound 1e-3 on COV*^{1/2} eps.  One step = one ciq_posterior_sample call
    (setup of the correction, pre-pass, solve, mean).  CPU leg: the draws on
    the first check_n candidates against the FP64 eigendecomposition of the
    dense posterior covariance (O1)."""
    import torch

    import paper_2006_11267_b300 as P

    torch.cuda.set_device(0)
    c = POSTERIOR
    Xtr, y, Xc, eps = posterior_inputs(c["n_cand"])
    dev = lambda a: torch.from_numpy(a).cuda()
    Xtr_d, y_d, Xc_d, eps_d = dev(Xtr), dev(y), dev(Xc), dev(eps)
    opts = dict(stop_rule="errbound", max_iter=MAX_ITER, lanczos_iters=LANCZOS_ITERS, precision=args.precision,
                check_every=16)
    call = lambda: P.ciq_posterior_sample(Xtr_d, y_d, Xc_d, c["kind"], c["ls"], c["s"], c["noise"], c["jitter"],
                                          c["mean"], eps_d, c["q"], TOL, **opts)
    for _ in range(max(1, args.warmup)):
        call()
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = max(1, args.steps)
    e0.record()
    infos = [call()[1] for _ in range(reps)]
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / reps
    _, pinf = P.ciq_posterior_sample(Xtr_d, y_d, Xc_d, c["kind"], c["ls"], c["s"], c["noise"], c["jitter"], c["mean"],
                                     eps_d, c["q"], TOL, profile=1, **opts)
    # The same draws with a pivoted-Cholesky preconditioner of COV* (the
    # rotated root R, R R^T = COV*: draws of the same distribution).
    precond = {}
    for rank in POSTERIOR_PRECOND_RANKS:
        pcall = lambda: P.ciq_posterior_sample(Xtr_d, y_d, Xc_d, c["kind"], c["ls"], c["s"], c["noise"],
                                               c["jitter"], c["mean"], eps_d, c["q"], TOL, precond_rank=rank, **opts)
        pcall()
        torch.cuda.synchronize()
        e0.record()
        pinfos = [pcall()[1] for _ in range(reps)]
        e1.record()
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1) / reps
        precond[str(rank)] = {"draws_per_s": c["t"] / (pms * 1e-3), "ms": pms, "iterations": pinfos[-1]["iters"],
                              "speedup": ms / pms, "precond_rank": pinfos[-1]["precond_rank"]}
    check = None
    if not args.no_cpu_baseline:
        from oracle import posterior as PO
        n = c["check_n"]
        Xtr2, y2, Xc2, eps2 = posterior_inputs(n)
        out, inf = P.ciq_posterior_sample(Xtr2, y2, Xc2, c["kind"], c["ls"], c["s"], c["noise"], c["jitter"],
                                          c["mean"], eps2, c["q"], TOL, **opts)
        t0 = time.perf_counter()
        mu, cov = PO.posterior(Xtr2.astype(np.float64), y2.astype(np.float64), Xc2.astype(np.float64), c["kind"],
                               np.array(c["ls"]), c["s"], c["noise"], c["jitter"], c["mean"])
        exact = PO.thompson_draws(mu, cov, eps2)
        fl = out.astype(np.float64) - mu[None, :]
        ex = exact - mu[None, :]
        e_draw = np.linalg.norm(out - exact, axis=1) / np.linalg.norm(exact, axis=1)
        e_fl = np.linalg.norm(fl - ex, axis=1) / np.linalg.norm(ex, axis=1)
        check = {"n_cand": n, "draw": {"max": float(e_draw.max()), "median": float(np.median(e_draw))},
                 "fluctuation": {"max": float(e_fl.max()), "median": float(np.median(e_fl))},
                 "iterations": inf["iters"], "oracle": "O1: FP64 eigendecomposition of the dense posterior covariance",
                 "oracle_seconds": time.perf_counter() - t0}
        # Preconditioned draws: R R^T against COV* on the first pc_check_n
        # candidates (all columns of the identity), the root's defining property.
        m = c["pc_check_n"]
        Xtr3, y3, Xc3, _ = posterior_inputs(m)
        eye = np.eye(m, dtype=np.float32)
        for rank in POSTERIOR_PRECOND_RANKS:
            o3, i3 = P.ciq_posterior_sample(Xtr3, y3, Xc3, c["kind"], c["ls"], c["s"], c["noise"], c["jitter"],
                                            c["mean"], eye, c["q"], TOL, precond_rank=min(rank, m), **opts)
            mu3, cov3 = PO.posterior(Xtr3.astype(np.float64), y3.astype(np.float64), Xc3.astype(np.float64),
                                     c["kind"], np.array(c["ls"]), c["s"], c["noise"], c["jitter"], c["mean"])
            R = (o3.astype(np.float64) - mu3[None, :]).T
            check[f"precond_{rank}_RRt_rel_err"] = float(np.linalg.norm(R @ R.T - cov3) / np.linalg.norm(cov3))
            check[f"precond_{rank}_iterations"] = i3["iters"]
    line = {"metric": "posterior Thompson draws/s (mu* + COV*^{1/2} eps) at error bound 1e-3",
            "value": c["t"] / (ms * 1e-3), "unit": "draws/s", "n_gpus": 1, "steps": reps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": f"{args.precision}x2-split tiles, f32 vectors and correction, f64 scalars and setup",
            "data": "synthetic",
            "config": {"workload": f"posterior_{c['kind']}_ard_ncand{c['n_cand']}_ntrain{c['n_train']}_d{c['d']}_t{c['t']}",
                       "n_train": c["n_train"], "n_cand": c["n_cand"], "d": c["d"], "kernel": c["kind"] + " ARD",
                       "lengthscales": list(c["ls"]), "noise": c["noise"], "jitter": c["jitter"], "T": c["t"],
                       "Q": c["q"], "tol": TOL, "stop_rule": "errbound", "precision": args.precision},
            "iterations": [i["iters"] for i in infos], "profile": {k: pinf[k] for k in
                                                                   ("t_total_ms", "t_prepass_ms", "t_mvm_ms",
                                                                    "t_step_ms", "mvm_launches")},
            "preconditioned": precond, "oracle_check": check, "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched512":
        return run_batched(args)
    if args.workload == "precision200k":
        return run_precision(args)
    if args.workload == "stored":
        return run_stored(args)
    if args.workload == "learned":
        return run_learned(args)
    if args.workload == "spectrum":
        return run_spectrum(args)
    if args.workload == "vjp":
        return run_vjp(args)
    if args.workload == "precond":
        return run_precond(args)
    if args.workload == "posterior":
        return run_posterior(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
