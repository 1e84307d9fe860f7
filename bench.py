#!/usr/bin/env python3
"""Throughput of the SALS sweep on one GB300, through the library's C ABI.

Metric: nnz*rank updates/s = |Omega| * K * T_in / t_step, where one step is one outer
iteration of Algorithm 1 (ceil(K/C) splits x N modes: R-hat, Gram/rhs, C x C
Cholesky, row writes, residual refresh) followed by the loss / training RMSE of
Eq. (1).  Workload: the 1e5 x 1e5 x 1e3 tensor with 1e8 observed entries, Zipf(1.1)
slice sizes on modes 1-2, rank-50 ground truth + noise, K = 100, C = 10,
lambda = 0.1, T_in = 1, FP32, synthetic (seeded), resident in HBM.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on a
bounded prefix sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import statistics
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "nnz*rank updates/s per SALS sweep"
UNIT = "nnz*rank/s"
WORKLOAD = dict(workload="skewed_3way_1e8", dims=[100_000, 100_000, 1_000], nnz=100_000_000,
                K=100, C=10, T_in=1, lam=0.1, rank_truth=50, zipf=1.1)

# DRAM traffic (read + write) of one mode-pass launch from the ncu capture summarised in
# profiles/k_lean_pass_skewed_3way_1e8.md (2e7-entry case, scaled by entries to a
# 1e8-entry launch), and the hash of the kernel sources it was taken with; the bench
# reports traffic as null once the sources differ or the entry count is not 1e8.
NCU_TRAFFIC = 1.737e9
NCU_TRAFFIC_NNZ = 100_000_000
NCU_SOURCE_HASH = "03862e7fb4cb30ec"


# Utilisation of the L1 data pipe (shared-memory and L1 wavefronts) of the mode pass in the
# same capture, averaged over the three modes' launches; null once the sources differ.
NCU_L1_PIPE_PCT = 70.9


def pass_units(nnz, N, C, avg_launch_ms):
    """The mode pass against the on-chip units that bind it, with this device's measured
    peaks (tf_device_peaks): FP32 FMA throughput, for the algorithmic FLOPs of a pass
    (Eq. 4's Gram lower triangle and right-hand side, the Hadamard products of the other
    modes' rows, and the R-hat refresh over the previous and current columns), and
    shared-memory bandwidth, for the varying-mode slice row every entry reads from on-chip
    copies (C values of each region it needs: two regions where that mode is updated after
    the pass's mode in the split, three where before; averaged over the three modes' passes
    of a three-way tensor)."""
    import paper_1410_5209_gb300 as tf
    dp = tf.device_peaks()
    flops = nnz * (C * (C + 1) + 2 * C + (N - 2) * C + 2 * C * N)
    v_floats = (2 + 3 + 3) * C / 3.0 if N == 3 else 2.0 * C
    sbytes = nnz * 4.0 * v_floats
    s = avg_launch_ms / 1e3
    pct = NCU_L1_PIPE_PCT if NCU_SOURCE_HASH == kernel_source_hash() else None
    return {"fp32": {"peak_tflops": dp["fp32x2_tflops"], "peak_tflops_plain_fma": dp["fp32_tflops"],
                     "algorithmic_flops_per_launch": flops, "achieved_tflops": flops / s / 1e12,
                     "frac": flops / s / 1e12 / dp["fp32x2_tflops"]},
            "shared_memory": {"peak_tbs": dp["smem_tbytes"], "algorithmic_bytes_per_launch": sbytes,
                              "achieved_tbs": sbytes / s / 1e12,
                              "frac": sbytes / s / 1e12 / dp["smem_tbytes"],
                              "ncu_l1_data_pipe_pct": pct},
            "peak_source": "measured on this device (tf_device_peaks, CUDA events)"}


def kernel_source_hash():
    """Hash of the source of the dominant kernel (k_lean_pass), of the plan records it
    reads and of the header that sets its launch shape (the default bin count)."""
    h = hashlib.sha256()
    for f in ("lean_pass.cu", "gather_plan.cuh", "sweep.cuh"):
        with open(os.path.join(ROOT, "paper_1410_5209_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax = float(f[1])
            except ValueError:
                continue
            for name, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(name)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def job_rate(local_ms, local_units, world, device="cuda"):
    """Whole-job figures of N ranks that each timed their own share: the slowest rank's
    time (max over ranks) and the units all ranks processed (sum), as the bench reports
    them; one process group collective each (no-ops at world = 1)."""
    if world <= 1:
        return local_ms, local_units, local_units / (local_ms / 1e3)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    ms, units = float(t.item()), float(u.item())
    return ms, units, units / (ms / 1e3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def oracle_threads():
    """Threads the OpenMP build of the oracle runs with on this host."""
    return int(os.environ.get("OMP_NUM_THREADS", "0") or 0) or (os.cpu_count() or 1)


def run_oracle_sample(m_entries, seed, sweeps=1, parallel=False):
    """The FP64 oracle as it stands on the first m_entries of the workload (a prefix of
    the same seeded draw), K = 100, C = 10: seconds per sweep and the update count.
    parallel: its OpenMP build (rows of a mode in parallel on every host core)."""
    import numpy as np
    import oracle
    import synth
    lib = oracle.load_parallel() if parallel else oracle.load()
    p = synth.skewed_3way(seed=seed, nnz=m_entries, device="cpu")
    c, x = p.numpy()
    t = oracle.Tensor(c, x.astype(np.float64), p.dims)
    A = [a.numpy() for a in p.init_factors()]
    r = oracle.residual(t, A, lib)
    t.groups(lib)
    times = []
    for s in range(sweeps):
        t0 = time.perf_counter()
        oracle.sals_sweep(t, A, r, WORKLOAD["C"], WORKLOAD["lam"], 1,
                          p.column_order(s, WORKLOAD["C"]), lib=lib)
        times.append(time.perf_counter() - t0)
    return times, p.nnz * p.K


def run_oracle_parity_workload(parallel):
    """The parity workload in full (1000 x 1000 x 100, 1e5 entries, K = 10, lambda = 1,
    FP64, five sweeps at C = 5 and at C = 1): seconds per sweep for each C."""
    import oracle
    import synth
    lib = oracle.load_parallel() if parallel else oracle.load()
    p = synth.parity_3way()
    c, x = p.numpy()
    out = {}
    for C in (5, 1):
        t = oracle.Tensor(c, x, p.dims)
        A = [a.numpy() for a in p.init_factors()]
        r = oracle.residual(t, A, lib)
        t.groups(lib)
        t0 = time.perf_counter()
        for s in range(5):
            oracle.sals_sweep(t, A, r, C, 1.0, 1, p.column_order(s, C), lib=lib)
        out[f"C{C}_ms_per_sweep"] = 1e3 * (time.perf_counter() - t0) / 5
        out[f"C{C}_nnz_rank_per_s"] = p.nnz * p.K / ((time.perf_counter() - t0) / 5)
    return out


def reference_arm(args, rank, world):
    if rank != 0:
        return 0
    m = args.ref_sample
    steps = args.warmup + args.steps
    threads = oracle_threads()
    times, units = run_oracle_sample(m, args.seed, steps, parallel=True)
    timed = times[args.warmup:]
    ms = 1e3 * sum(timed) / len(timed)
    value = units / (ms / 1e3)
    sample = (f"first {m} entries (prefix of the seeded 1e8-entry draw) of the workload, "
              f"one full sweep per step (K=100, C=10), FP64 C with OpenMP over rows "
              f"({threads} threads)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {**WORKLOAD, "sample_nnz": m},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def study(args, rank, world):
    """Section 5.5-style studies on the same workload, one JSON line per configuration:
    sweeps at each C (time per sweep, training RMSE and the RMSE on 1% held-out entries
    after each, from the same initial factors; C = K is ALS), then the inner-iteration
    counts T_in at the workload's C, then the row-assignment policies at that C."""
    import numpy as np
    import torch
    import paper_1410_5209_gb300 as tf
    import synth
    from paper_1410_5209_gb300 import build as tfbuild
    if rank != 0:
        return 0
    tfbuild.build()
    tf.load()
    K, lam = WORKLOAD["K"], WORKLOAD["lam"]
    # 1% of the drawn entries are held out (never trained on) for the test RMSE
    p = synth.skewed_3way(seed=args.seed, nnz=args.nnz, device="cuda")
    hold = max(1, p.nnz // 100)
    train_c, train_x = p.coords[:-hold], p.x[:-hold]
    test_c, test_x = p.coords[-hold:].contiguous(), p.x[-hold:].double()
    stream = torch.cuda.current_stream()
    f = tf.Factorization(train_c, train_x, p.dims, K, seed=args.seed, dtype=tf.F32,
                         stream=stream.cuda_stream, device_input=True)
    A0 = [a.numpy().astype(np.float32) for a in p.init_factors(torch.float64, "cpu")]
    p_nnz = int(train_c.shape[0])

    def test_rmse():
        pred = f.predict(test_c).double()
        return float(torch.sqrt(torch.mean((test_x - pred) ** 2)))

    def run(C, sweeps, T_in=1):
        for n in range(3):
            f.set_factors(n, A0[n])
        times, rmses, tests = [], [], []
        for s in range(sweeps):
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ev0.record(stream)
            f.sweep(C, lam, T_in, p.column_order(s, C))
            ev1.record(stream)
            torch.cuda.synchronize()
            times.append(ev0.elapsed_time(ev1))
            rmses.append(f.loss(lam)[1])
            tests.append(test_rmse())
        return times, rmses, tests

    # forms: Gram precision (FP32-level; one TF32 product per term on the tensor cores, wide
    # C only) x row solves (plain FP32 Cholesky; FP64-residual refinement + FP64 re-solve
    # of rows with pivot ratio < 1e-4)
    for C in [int(c) for c in args.study_c.split(",")]:
        for prec in ((0, 1) if C > 16 else (0,)):
            for refine, cond in ((0, 0.0), (1, 1e4)):
                f.set_precision(prec)
                f.set_solve(refine, cond)
                run(C, 1)  # warm-up (kernel selection, buffers)
                f64_0 = f.fp64_rows()
                times, rmses, tests = run(C, args.study_sweeps)
                ms = float(np.median(times))
                print(json.dumps({"study": "C", "C": C, "K": K, "nnz": p_nnz,
                                  "ms_per_sweep": ms,
                                  "precision": ["fp32", "tf32x1"][prec] +
                                               ("+refine+fp64rows" if refine else ""),
                                  "fp64_rows": f.fp64_rows() - f64_0,
                                  "nnz_rank_per_s": p_nnz * K / (ms / 1e3),
                                  "sweep_ms": times, "train_rmse": rmses, "test_rmse": tests,
                                  "pass_path": f.counters()["pass_path"]}), flush=True)
        f.set_precision(0)
        f.set_solve(0, 0.0)
    C = WORKLOAD["C"]
    # inner iterations (Algorithm 1's T_in): the same outer sweeps from the same start, each
    # sweep T_in passes over the modes per column subset; convergence against elapsed time
    for T_in in [int(t) for t in args.study_tin.split(",") if t]:
        run(C, 1, T_in)
        times, rmses, tests = run(C, args.study_sweeps, T_in)
        print(json.dumps({"study": "T_in", "T_in": T_in, "C": C, "K": K,
                          "ms_per_sweep": float(np.median(times)),
                          "elapsed_ms": [float(t) for t in np.cumsum(times)],
                          "train_rmse": rmses, "test_rmse": tests}), flush=True)
    policies = [q for q in args.study_policies.split(",") if q]
    for name, pol in (("lpt", tf.SCHED_LPT), ("greedy_alg3", tf.SCHED_GREEDY),
                      ("seq", tf.SCHED_SEQ), ("ran", tf.SCHED_RAN)):
        if name.split("_")[0] not in policies:
            continue
        f.set_schedule(pol, 0)
        run(C, 1)
        times, rmses, tests = run(C, args.study_sweeps)
        ms = float(np.median(times))
        print(json.dumps({"study": "schedule", "policy": name, "C": C, "ms_per_sweep": ms,
                          "nnz_rank_per_s": p_nnz * K / (ms / 1e3), "train_rmse": rmses,
                          "test_rmse": tests,
                          "split_rows": f.counters()["split_rows"]}), flush=True)
    f.close()
    return 0


def batched(args, rank, world):
    """Many small independent tensors (mode lengths 50..5,000 and 1e3..1e6 entries,
    log-uniform; rank-16 truth; K = 16, C = 4) factorised as one block-diagonal tensor:
    one set of launches per sweep whatever the number of tensors."""
    import numpy as np
    import torch
    import paper_1410_5209_gb300 as tf
    import synth
    from paper_1410_5209_gb300 import build as tfbuild
    if rank != 0:
        return 0
    tfbuild.build()
    tf.load()
    K, C, lam = 16, 4, 0.1
    t0 = time.perf_counter()
    p, row_off, ent_off = synth.batched(args.batched, seed=args.seed, K=K, device="cuda")
    gen_s = time.perf_counter() - t0
    stream = torch.cuda.Stream()   # a capturable stream: sweeps replay as CUDA graphs
    f = tf.Factorization(p.coords, p.x, p.dims, K, seed=args.seed, dtype=tf.F32,
                         stream=stream.cuda_stream, device_input=True)
    f.set_graphs(True)
    tune = None
    if args.autotune:
        Cs, Ps = [2, 4, 8, 16], [0, 152 * 32, 152 * 192]
        bc, bp, tms = f.autotune(Cs, Ps, lam=lam)
        tune = {"C": Cs, "P": [p_ or "default" for p_ in Ps], "ms": tms.round(3).tolist(),
                "best_C": bc, "best_P": bp or "default"}
        f.set_schedule(tf.SCHED_LPT, 0)   # the timed sweeps below keep the default schedule
    for s_ in range(args.warmup):
        f.sweep(C, lam, 1)
    f.loss(lam)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for s_ in range(args.steps):
        f.sweep(C, lam, 1)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    loss, rmse = f.loss(lam)
    cnt = f.counters()
    print(json.dumps({"metric": "nnz*rank updates/s per SALS sweep (batch of tensors)",
                      "value": p.nnz * K / (ms / 1e3), "unit": UNIT, "ms_per_sweep": ms,
                      "tensors": args.batched, "nnz": p.nnz, "dims_total": p.dims, "K": K,
                      "C": C, "kernels_per_sweep": cnt["last_sweep_launches"],
                      "graph_launches_per_sweep": 1 if f.graph_info()["replays"] else None,
                      "autotune": tune,
                      "train_rmse": rmse, "generate_s": gen_s, "dtype": "f32",
                      "data": "synthetic"}), flush=True)
    f.close()
    return 0


def fiveway(args, rank, world):
    """The 5-way workload: mode lengths 1e6, --fiveway uniform-random distinct entries
    (5e8 at full size), rank-20 truth + N(0, 0.1^2), FP32, K = 1000, lambda = 1; one sweep
    per C of --fiveway-c, in sequence (no warm-up sweep: a sweep takes seconds),
    device time by CUDA events, with the layout build time and the memory held."""
    import numpy as np
    import torch
    import paper_1410_5209_gb300 as tf
    import synth
    from paper_1410_5209_gb300 import build as tfbuild
    if rank != 0:
        return 0
    tfbuild.build()
    tf.load()
    K, lam, dims = 1000, 1.0, (1_000_000,) * 5
    t0 = time.perf_counter()
    p = synth.make_problem(dims, args.fiveway, 20, K, args.seed, dtype=torch.float32,
                           device="cuda")
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    s = torch.cuda.Stream()
    used0, _, _ = tf.pool_usage(reset_high=True)
    t0 = time.perf_counter()
    f = tf.Factorization(p.coords, p.x, p.dims, K, seed=args.seed, dtype=tf.F32,
                         stream=s.cuda_stream, device_input=True)
    f.sync()
    create_s = time.perf_counter() - t0
    rows = {}
    Cs = [int(c) for c in args.fiveway_c.split(",") if c]
    for C in Cs:   # one sweep per C, in sequence from the state the previous one left
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        f.sweep(C, lam, 1)
        e1.record(s)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        loss, rmse = f.loss(lam)
        rows[str(C)] = {"ms_per_sweep": ms, "nnz_rank_per_s": p.nnz * K / (ms / 1e3),
                        "train_rmse_after": rmse,
                        "pass_path": f.counters()["pass_path"]}
    _, high, _ = tf.pool_usage()
    est = max(tf.estimate_bytes(p.dims, p.nnz, K, C, tf.F32, device_input=True) for C in Cs)
    print(json.dumps({"metric": "nnz*rank updates/s per SALS sweep (5-way)", "unit": UNIT,
                      "nnz": p.nnz, "dims": list(dims), "K": K, "lam": lam, "dtype": "f32",
                      "per_C": rows, "generate_s": gen_s, "create_s": create_s,
                      "device_bytes_high": high - used0, "device_bytes_estimate": est,
                      "data": "synthetic"}), flush=True)
    f.close()
    return 0


def precision_forms(args, p, K, C, lam, sweeps=3):
    """The precision forms of the mode pass on the same tensor from the same initial factors
    (a fresh context each, the same column orders): device ms per sweep (sweeps after the
    first, which also builds the pass's gather plans) and training RMSE after `sweeps`.
    Forms: FP32 with packed FMAs (the default), bfloat16 slice rows of the varying mode
    (tf_set_precision(2)) or of both other modes (3), TF32 x 1 and x 3 tensor-core Grams,
    and the cp.async pass."""
    import torch
    import paper_1410_5209_gb300 as tf
    forms = {"fp32_packed_fma": (0, 0), "bf16_varying_rows": (0, 2), "bf16_other_rows": (0, 3),
             "tf32x1_tensor_core": (0, 1), "tf32x3_tensor_core": (4, 0), "cp_async_pass": (1, 0)}
    out = {}
    for name, (path, prec) in forms.items():
        s = torch.cuda.Stream()
        g = tf.Factorization(p.coords, p.x, p.dims, K, seed=args.seed, dtype=tf.F32,
                             stream=s.cuda_stream, device_input=True)
        g.set_kernel_path(path)
        g.set_precision(prec)
        ms = []
        for it in range(sweeps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            g.sweep(C, lam, 1)
            e1.record(s)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        _, rmse = g.loss(lam)
        g.close()
        t = sum(ms[1:]) / max(len(ms) - 1, 1)
        out[name] = {"ms_per_sweep": t, "nnz_rank_per_s": p.nnz * K / (t / 1e3),
                     "train_rmse": rmse}
    base = out["fp32_packed_fma"]["train_rmse"]
    for v in out.values():
        v["rmse_rel_to_fp32"] = (v["train_rmse"] - base) / base
    out["what"] = (f"{sweeps} sweeps from the same initial factors, C={C}, lambda={lam}; "
                   "ms per sweep over sweeps 2..; equal RMSE means |rmse_rel_to_fp32| <= 1e-3")
    return out


def batched_config(args, tensors, hbm):
    """The batch of many small tensors (mode lengths 50..5,000 and 1e3..1e6 entries,
    log-uniform, capped at half the cells; rank-16 truth; K = 16, C = 4) as one
    block-diagonal tensor, each sweep one CUDA-graph launch; ms per sweep against the
    sweep's algorithmic HBM bytes, on the default schedule; beside it the autotuner's
    timings of subset sizes and bin counts (tf_autotune: one timed sweep per candidate,
    the state restored after each) and its choice."""
    import torch
    import paper_1410_5209_gb300 as tf
    import synth
    K, C, lam = 16, 4, 0.1
    t0 = time.perf_counter()
    p, _, _ = synth.batched(tensors, seed=args.seed, K=K, device="cuda")
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    s = torch.cuda.Stream()
    t0 = time.perf_counter()
    f = tf.Factorization(p.coords, p.x, p.dims, K, seed=args.seed, dtype=tf.F32,
                         stream=s.cuda_stream, device_input=True)
    f.sync()
    create_s = time.perf_counter() - t0
    del p
    f.set_graphs(True)
    Cs, Ps = [2, 4, 8], [0, 152 * 32]
    bc, bp, tms = f.autotune(Cs, Ps, lam=lam)
    tune = {"C": Cs, "bins": [b or "default" for b in Ps], "ms_per_sweep": tms.round(2).tolist(),
            "best_C": bc, "best_bins": bp or "default", "best_ms_per_sweep": float(tms.min()),
            "best_nnz_rank_per_s": None}
    f.set_schedule(tf.SCHED_LPT, 0)  # the timed sweeps below keep the default schedule
    for _ in range(3):
        f.sweep(C, lam, 1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = 3
    e0.record(s)
    for _ in range(steps):
        f.sweep(C, lam, 1)
    e1.record(s)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    nnz = f.nnz
    _, rmse = f.loss(lam)
    cnt, gi = f.counters(), f.graph_info()
    f.close()
    N = 3
    sweep_bytes = nnz * (N * (4 * (N - 1) + 4) + 4) * math.ceil(K / C)
    achieved = sweep_bytes / (ms / 1e3) / 1e9
    tune["best_nnz_rank_per_s"] = nnz * K / (tune["best_ms_per_sweep"] / 1e3)
    return {"tensors": tensors, "nnz": nnz, "K": K, "C": C, "ms_per_sweep": ms,
            "nnz_rank_per_s": nnz * K / (ms / 1e3), "train_rmse": rmse,
            "kernels_per_sweep": cnt["last_sweep_launches"],
            "graph_launches_per_sweep": 1 if gi["replays"] else None,
            "roofline": {"bound": "hbm", "algorithmic_bytes_per_sweep": sweep_bytes,
                         "floor_ms": sweep_bytes / (hbm * 1e9) * 1e3, "achieved": achieved,
                         "peak": hbm, "unit": "GB/s", "frac": achieved / hbm},
            "autotune": tune, "generate_s": gen_s, "create_s": create_s}


def fiveway_config(args, nnz, hbm):
    """The five-way tensor (mode lengths 1e6, uniform-random distinct entries, rank-20
    truth + N(0, 0.1^2), FP32; K = 1000, C = 10, lambda = 1): one sweep, against its
    algorithmic bytes -- the streams and the factor-row gathers, which go to HBM here
    (each 1e6-row slice is larger than a share of L2)."""
    import torch
    import paper_1410_5209_gb300 as tf
    import synth
    K, C, lam, dims = 1000, 10, 1.0, (1_000_000,) * 5
    t0 = time.perf_counter()
    p = synth.make_problem(dims, nnz, 20, K, args.seed, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    s = torch.cuda.Stream()
    t0 = time.perf_counter()
    f = tf.Factorization(p.coords, p.x, p.dims, K, seed=args.seed, dtype=tf.F32,
                         stream=s.cuda_stream, device_input=True)
    f.sync()
    create_s = time.perf_counter() - t0
    nnz = p.nnz
    del p
    torch.cuda.empty_cache()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    f.sweep(C, lam, 1)
    e1.record(s)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    _, rmse = f.loss(lam)
    f.close()
    N = 5
    splits = math.ceil(K / C)
    stream = nnz * (N * (4 * (N - 1) + 4) + 4) * splits
    gathers = nnz * N * (N - 1) * 4 * C * splits
    achieved = (stream + gathers) / (ms / 1e3) / 1e9
    # the gathers with the R-hat refresh regions every pass reads: each other mode's row
    # brings its current and previous columns, and for modes updated earlier in the split
    # its old ones too: (N - 1) * 2.5 * C values per entry and pass on average over the modes
    gathers_r = nnz * N * (N - 1) * 2.5 * 4 * C * splits
    achieved_r = (stream + gathers_r) / (ms / 1e3) / 1e9
    return {"nnz": nnz, "dims": list(dims), "K": K, "C": C, "ms_per_sweep": ms,
            "nnz_rank_per_s": nnz * K / (ms / 1e3), "train_rmse_after": rmse,
            "roofline": {"bound": "hbm", "algorithmic_bytes_per_sweep": stream + gathers,
                         "stream_bytes": stream, "gather_bytes": gathers,
                         "floor_ms": (stream + gathers) / (hbm * 1e9) * 1e3,
                         "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm,
                         "with_refresh_regions": {
                             "gather_bytes": gathers_r,
                             "floor_ms": (stream + gathers_r) / (hbm * 1e9) * 1e3,
                             "achieved": achieved_r, "frac": achieved_r / hbm}},
            "generate_s": gen_s, "create_s": create_s}


def small_sweeps(args):
    """The 1e5-entry FP64 parity workload (1000 x 1000 x 100, K = 10), C = 1 (CDTF) and
    C = 5: device time per sweep with eager launches and with the sweep replayed as a
    CUDA graph (tf_set_graphs).  At this size a sweep is launch-bound."""
    import torch
    import paper_1410_5209_gb300 as tf
    import synth
    p = synth.parity_3way(seed=1, device="cuda")
    s = torch.cuda.Stream()
    out = {}
    for C in (1, 5):
        row = {}
        for graphs in (False, True):
            f = tf.Factorization(p.coords, p.x, p.dims, p.K, seed=1, dtype=tf.F64,
                                 stream=s.cuda_stream, device_input=True)
            f.set_graphs(graphs)
            for _ in range(3):
                f.sweep(C, 1.0, 1)
            f.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 20
            e0.record(s)
            for _ in range(reps):
                f.sweep(C, 1.0, 1)
            e1.record(s)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / reps
            row["graph_ms" if graphs else "eager_ms"] = ms
            row["launches_per_sweep"] = f.counters()["last_sweep_launches"]
            f.close()
        row["nnz_rank_per_s_graph"] = p.nnz * p.K / (row["graph_ms"] / 1e3)
        out[f"C={C}"] = row
    out["what"] = ("1e5-entry FP64 parity workload, K=10: ms per sweep, eager launches vs "
                   "one CUDA-graph launch per sweep")
    return out


def serve_with_jobs(args, f, p, lam):
    """Fold-in requests and factorisation jobs through the serving loop (tf_server.h), in
    real time: Poisson arrivals of both kinds submitted from this thread; the server
    admits jobs against free device memory (each on its own stream and host thread) and
    batches the fold-ins continuously on a high-priority stream against the frozen model
    `f`.  Fold-in latency is the server's own submission-to-result time."""
    import numpy as np
    import torch
    import paper_1410_5209_gb300 as tf
    import synth
    rng = np.random.default_rng(args.seed + 53)
    reqs = synth.foldin_requests(p, args.serve_server_requests, args.seed + 59)
    # jobs shaped like the batched workload's tensors: mode lengths log-uniform in
    # [50, 5000], entries log-uniform in [1e3, 1e6], rank-16 truth, K = 16, C = 4
    u = rng.random((args.serve_jobs, 4))
    jobs = []
    for b in range(args.serve_jobs):
        dims = [int(math.exp(math.log(50) + u[b, n] * (math.log(5000) - math.log(50))))
                for n in range(3)]
        nnz = int(math.exp(math.log(1e3) + u[b, 3] * (math.log(1e6) - math.log(1e3))))
        q = synth.make_problem(dims, nnz, 16, 16, args.seed * 7919 + b, dtype=torch.float32,
                               device="cuda")
        c, x = q.numpy()
        jobs.append((c, x.astype(np.float32), q.dims))
    job_sweeps, job_C = 5, 4
    srv = tf.Server(f, max_running=8, max_batch=args.serve_batch)
    # warm-up: one job and a few fold-ins
    wj = srv.submit_job(*jobs[0], 16, job_C, lam, 1, seed=1)
    for o, v in reqs[:8]:
        srv.wait_foldin(srv.submit_foldin(0, o, v, lam))
    srv.wait_job(wj)
    srv.release_job(wj)
    tf_ = np.cumsum(rng.exponential(1.0 / args.serve_server_rate, len(reqs)))
    tj = np.cumsum(rng.exponential(1.0 / args.serve_job_rate, len(jobs)))
    fids, jids, lag = [], [], []
    t0 = time.perf_counter()

    def submit_jobs():   # jobs from a second host thread (the input copy releases the GIL)
        for i, t in enumerate(tj):
            while time.perf_counter() - t0 < t:
                time.sleep(0)
            c, x, dims = jobs[i]
            jids.append(srv.submit_job(c, x, dims, 16, job_C, lam, job_sweeps, seed=i))

    th = threading.Thread(target=submit_jobs)
    th.start()
    for i, t in enumerate(tf_):
        while time.perf_counter() - t0 < t:
            pass
        lag.append(time.perf_counter() - t0 - t)
        fids.append(srv.submit_foldin(0, reqs[i][0], reqs[i][1], lam))
    t_sub = time.perf_counter() - t0
    lat = np.array([srv.wait_foldin(r)[2] for r in fids])
    t_f = time.perf_counter() - t0
    th.join()
    infos = [srv.wait_job(j) for j in jids]
    t_all = time.perf_counter() - t0
    assert all(i["state"] == tf.JOB_DONE for i in infos), infos
    for j in jids:
        srv.release_job(j)
    st = srv.stats()
    srv.close()
    jlat = np.array([i["finished_s"] - i["queued_s"] for i in infos])
    jwait = np.array([i["started_s"] - i["queued_s"] for i in infos])
    return {"foldin_p50_ms": float(np.percentile(lat, 50) * 1e3),
            "foldin_p99_ms": float(np.percentile(lat, 99) * 1e3),
            "foldin_req_per_s": len(fids) / t_f, "foldin_offered_req_per_s": args.serve_server_rate,
            "foldin_requests": len(fids), "foldin_batches": st["foldin_batches"],
            "foldin_submitted_per_s": len(fids) / t_sub,
            "submit_lag_p99_ms": float(np.percentile(lag, 99) * 1e3),
            "jobs": len(jids), "job_p50_ms": float(np.percentile(jlat, 50) * 1e3),
            "job_p99_ms": float(np.percentile(jlat, 99) * 1e3),
            "job_admission_wait_p99_ms": float(np.percentile(jwait, 99) * 1e3),
            "jobs_per_s": len(jids) / t_all, "job_offered_per_s": args.serve_job_rate,
            "job_entries": [int(j[1].shape[0]) for j in jobs],
            "running_peak": st["running_peak"], "bytes_admitted_peak": st["bytes_admitted_peak"],
            "what": "tf_server: Poisson fold-ins (new mode-1 slices, K=100) and Poisson "
                    f"factorisation jobs ({job_sweeps} sweeps, K=16, C={job_C}) admitted "
                    "against free device memory, in real time"}


def serve_beside_large_job(args, f, p, K, C, lam, sm_limits=(0, 144)):
    """Fold-ins against the frozen model `f` (through the serving loop, continuous batching
    on a high-priority stream) while a second context of the same size (the 1e8-entry
    tensor, K = 100, C = 10) sweeps back to back on its own low-priority stream from another
    host thread: fold-in p50 / p99 and the concurrent sweep's rate, for each SM limit of
    the sweeping context (0: every SM)."""
    import numpy as np
    import torch
    import paper_1410_5209_gb300 as tf
    import synth
    reqs = synth.foldin_requests(p, args.serve_large_requests, args.seed + 61)
    js = torch.cuda.Stream(priority=0)   # the least urgent priority
    g = tf.Factorization(p.coords, p.x, p.dims, K, seed=args.seed + 1, dtype=tf.F32,
                         stream=js.cuda_stream, device_input=True)
    g.sweep(C, lam, 1)
    g.sync()
    out = {}
    for lim in sm_limits:
        g.set_sm_limit(max(lim, 0))
        g.sweep(C, lam, 1)
        g.sync()
        srv = tf.Server(f, max_batch=args.serve_batch, reserve_sms=-1)
        for o, v in reqs[:8]:
            srv.wait_foldin(srv.submit_foldin(0, o, v, lam))
        stop = threading.Event()
        sweeps = []

        def sweeper():
            while not stop.is_set():
                t0 = time.perf_counter()
                g.sweep(C, lam, 1)
                g.sync()
                sweeps.append(time.perf_counter() - t0)

        th = threading.Thread(target=sweeper)
        if lim >= 0:
            th.start()
            time.sleep(0.05)
        rng = np.random.default_rng(args.seed + 67)
        ta = np.cumsum(rng.exponential(1.0 / args.serve_large_rate, len(reqs)))
        t0 = time.perf_counter()
        ids = []
        for i, t in enumerate(ta):
            while time.perf_counter() - t0 < t:
                pass
            ids.append(srv.submit_foldin(0, reqs[i][0], reqs[i][1], lam))
        lat = np.array([srv.wait_foldin(r)[2] for r in ids])
        t_f = time.perf_counter() - t0
        stop.set()
        if lim >= 0:
            th.join()
        srv.close()
        ms = float(np.median(sweeps) * 1e3) if sweeps else None
        key = "no_concurrent_sweep" if lim < 0 else f"sm_limit_{lim or 'all'}"
        out[key] = {
            "foldin_p50_ms": float(np.percentile(lat, 50) * 1e3),
            "foldin_p99_ms": float(np.percentile(lat, 99) * 1e3),
            "foldin_req_per_s": len(ids) / t_f, "offered_req_per_s": args.serve_large_rate,
            "concurrent_sweeps": len(sweeps), "concurrent_sweep_ms_p50": ms,
            "concurrent_nnz_rank_per_s": (p.nnz * K / (ms / 1e3)) if ms else None}
    g.close()
    out["what"] = ("Poisson fold-ins (new mode-1 slices of 10-10,000 entries, K=100) through "
                   "tf_server against the frozen model while a second 1e8-entry context "
                   "(K=100, C=10) sweeps back to back on another stream; sm_limit = blocks of "
                   "its persistent mode passes (tf_set_sm_limit)")
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--ref-sample", type=int, default=400_000)
    ap.add_argument("--cpu-sample", type=int, default=1_000_000)
    ap.add_argument("--cpu-sample-parallel", type=int, default=8_000_000)
    ap.add_argument("--configs", type=int, default=1,
                    help="also run the precision forms, the batched and the five-way configs")
    ap.add_argument("--batched-tensors", type=int, default=4096)
    ap.add_argument("--serve-large-requests", type=int, default=1500)
    ap.add_argument("--serve-large-rate", type=float, default=5000.0)
    ap.add_argument("--serve-large-sm-limits", default="-1,0,144,112,96,80,64",
                    help="SM limits of the concurrently sweeping context (-1: no sweep)")
    ap.add_argument("--fiveway-nnz", type=int, default=500_000_000)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nnz", type=int, default=WORKLOAD["nnz"])
    ap.add_argument("--C", type=int, default=0,
                    help="subset size of the timed sweeps (0: the workload's C = 10)")
    ap.add_argument("--foldin-requests", type=int, default=200)
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-rate", type=float, default=20000.0)
    ap.add_argument("--serve-batch", type=int, default=256)
    ap.add_argument("--autotune", type=int, default=1,
                    help="with --batched: time (C, P) candidates with tf_autotune first")
    ap.add_argument("--small-sweeps", type=int, default=1,
                    help="1: time the 1e5-entry parity workload eager vs CUDA graphs")
    ap.add_argument("--serve-jobs", type=int, default=24,
                    help="factorisation jobs mixed into the server-driven fold-in stream")
    ap.add_argument("--serve-job-rate", type=float, default=40.0)
    ap.add_argument("--serve-server-rate", type=float, default=10000.0)
    ap.add_argument("--serve-server-requests", type=int, default=4000)
    ap.add_argument("--study", action="store_true",
                    help="C-sweep and row-assignment policy study instead of the benchmark")
    ap.add_argument("--study-c", default="1,2,4,10,20,50,100")
    ap.add_argument("--study-sweeps", type=int, default=3)
    ap.add_argument("--study-policies", default="lpt,greedy,seq,ran")
    ap.add_argument("--study-tin", default="1,2,3,5",
                    help="inner-iteration counts of the T_in study (empty: skip it)")
    ap.add_argument("--fiveway", type=int, default=0,
                    help="entries of the 5-way workload to time instead (5e8 at full size)")
    ap.add_argument("--fiveway-c", default="10,50,1")
    ap.add_argument("--batched", type=int, default=0,
                    help="factorise this many small independent tensors as one batch instead")
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.study:
        return study(args, rank, world)
    if args.batched > 0:
        return batched(args, rank, world)
    if args.fiveway > 0:
        return fiveway(args, rank, world)
    if args.impl == "reference":
        return reference_arm(args, rank, world)

    import numpy as np
    import torch
    import paper_1410_5209_gb300 as tf
    import synth
    from paper_1410_5209_gb300 import build as tfbuild

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0:
        tfbuild.build()
    if world > 1:
        dist.barrier()
    tf.load()

    if args.C:
        WORKLOAD["C"] = args.C
    K, C, lam, T_in = WORKLOAD["K"], WORKLOAD["C"], WORKLOAD["lam"], WORKLOAD["T_in"]
    # each rank factorises its own replica (independent problems: no data-path collective)
    p = synth.skewed_3way(seed=args.seed + rank, nnz=args.nnz, device="cuda")
    nnz, N = p.nnz, p.N
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()  # the generator's kernels are not part of the build
    t0 = time.perf_counter()
    f = tf.Factorization(p.coords, p.x, p.dims, K, seed=args.seed + rank, dtype=tf.F32,
                         stream=stream.cuda_stream, device_input=True)
    torch.cuda.synchronize()
    create_s = time.perf_counter() - t0

    def step():
        f.sweep(C, lam, T_in)
        return f.loss(lam)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    f.profile(True)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        loss, rmse = step()
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    prof = f.get_profile()
    cnt = f.counters()
    f.profile(False)
    # each rank factorises its own replica: whole-job units over the slowest rank's time
    ms, units, value = job_rate(ms, nnz * K * T_in, world)

    # roofline of the dominant kernel: the fused mode pass
    hbm, peak_kind = peaks()
    mp_n, mp_ms = prof["mode_pass"]
    mp_avg_ms = mp_ms / max(mp_n, 1)
    bytes_per_launch = nnz * (4 * (N - 1) + 4 + 4.0 / (N * T_in))
    achieved = bytes_per_launch / (mp_avg_ms / 1e3) / 1e9
    traffic = NCU_TRAFFIC if (NCU_SOURCE_HASH == kernel_source_hash()
                              and nnz == NCU_TRAFFIC_NNZ and C == 10) else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": traffic,
                "kernel": " + ".join(n for b, n in ((1, "k_pass_wide" if C > 16 else "k_mode_pass"),
                                                   (2, "k_mode_pass_tma"), (4, "k_pass_wide_tc"),
                                                   (8, "k_lean_pass"))
                                     if cnt["pass_path"] & b) or "?",
                "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": bytes_per_launch,
                "avg_launch_ms": mp_avg_ms}
    # the same launch with the factor-row gathers counted as bytes: C values of each other
    # mode's row per entry (the slices fit L2, so these are L2/L1 bytes, not HBM bytes)
    gather_bytes = nnz * (N - 1) * 4.0 * C
    with_g = (bytes_per_launch + gather_bytes) / (mp_avg_ms / 1e3) / 1e9
    roofline["with_gathers"] = {"achieved": with_g, "frac": with_g / hbm,
                                "gather_bytes_per_launch": gather_bytes}
    roofline["units"] = pass_units(nnz, N, C, mp_avg_ms)
    nsplit = math.ceil(K / C)
    sweep_bytes = nnz * (T_in * N * (4 * (N - 1) + 4) + 4) * nsplit
    sweep_ms = sum(v[1] for k, v in prof.items()
                   if k in ("pack", "mode_pass", "combine", "solve")) / args.steps
    kernel_breakdown = {k: {"launches": v[0], "ms": v[1]} for k, v in prof.items()}
    launches_per_step = cnt["last_sweep_launches"] + cnt["loss_launches"]

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {**WORKLOAD, "nnz": nnz, "l2": "inputs larger than L2 (>= 2.4 GB per sweep)",
                      "parallelism": f"replicas{world}", "create_s": create_s},
           "roofline": roofline,
           "sweep_roofline": {"bound": "hbm", "algorithmic_bytes": sweep_bytes,
                              "device_ms": sweep_ms,
                              "achieved": sweep_bytes / (sweep_ms / 1e3) / 1e9 if sweep_ms else None,
                              "peak": hbm, "frac": (sweep_bytes / (sweep_ms / 1e3) / 1e9 / hbm)
                              if sweep_ms else None},
           "kernels": kernel_breakdown, "gpu_launches": launches_per_step * args.steps,
           "clocks": clocks, "loss": loss, "train_rmse": rmse}
    # fold-in latency (Eq. 2 row solve for a new mode-1 slice) against the factors the
    # timed sweeps left: one synchronous tf_foldin per request, submit to result on host
    if args.foldin_requests > 0:
        reqs = synth.foldin_requests(p, args.foldin_requests + 10, args.seed + 17 + rank)
        lat = []
        for q, (other, xv) in enumerate(reqs):
            t0 = time.perf_counter()
            f.foldin(0, other, xv, lam)
            if q >= 10:   # the first ten are a warm-up
                lat.append(time.perf_counter() - t0)
        lat_ms = np.sort(np.array(lat)) * 1e3
        ms_sizes = [r[0].shape[0] for r in reqs[10:]]
        out["foldin"] = {"p50_ms": float(np.percentile(lat_ms, 50)),
                         "p99_ms": float(np.percentile(lat_ms, 99)),
                         "requests": len(lat), "req_per_s": len(lat) / float(lat_ms.sum() / 1e3),
                         "entries_min": int(min(ms_sizes)), "entries_max": int(max(ms_sizes)),
                         "K": K, "what": "sequential tf_foldin calls: host request -> device "
                                         "Gram + Cholesky -> host row"}
    # serving: Poisson arrivals of fold-in requests, continuous batching (every batch
    # takes all requests that arrived while the previous one ran, up to --serve-batch);
    # a virtual clock advances by the measured wall time of each tf_foldin_batch call
    if args.serve_requests > 0:
        reqs = synth.foldin_requests(p, args.serve_requests, args.seed + 29 + rank)
        f.foldin_batch(0, reqs[:8], lam)   # warm-up
        rng = np.random.default_rng(args.seed + 31)
        arrive = np.cumsum(rng.exponential(1.0 / args.serve_rate, len(reqs)))

        def serve():
            clock, nxt, lat, batches = 0.0, 0, np.zeros(len(reqs)), []
            while nxt < len(reqs):
                clock = max(clock, arrive[nxt])
                end = nxt
                while end < len(reqs) and arrive[end] <= clock and end - nxt < args.serve_batch:
                    end += 1
                t0 = time.perf_counter()
                _, status = f.foldin_batch(0, reqs[nxt:end], lam)
                clock += time.perf_counter() - t0
                assert not status.any()
                lat[nxt:end] = clock - arrive[nxt:end]
                batches.append(end - nxt)
                nxt = end
            return {"p50_ms": float(np.percentile(lat, 50) * 1e3),
                    "p99_ms": float(np.percentile(lat, 99) * 1e3),
                    "req_per_s": len(reqs) / clock, "offered_req_per_s": args.serve_rate,
                    "requests": len(reqs), "mean_batch": float(np.mean(batches)),
                    "max_batch": args.serve_batch}

        out["serving"] = {**serve(), "what": "Poisson fold-in arrivals, continuous batching "
                          "through tf_foldin_batch (latency = arrival -> rows on host)"}
        if args.serve_jobs > 0:
            out["serving_server"] = serve_with_jobs(args, f, p, lam)
    if args.serve_large_requests > 0 and world == 1:
        out["serving_beside_large_job"] = serve_beside_large_job(
            args, f, p, K, C, lam, [int(v) for v in args.serve_large_sm_limits.split(",")])
    f.close()
    del f
    if args.configs and rank == 0 and world == 1:
        out["precision"] = precision_forms(args, p, K, C, lam)
    if args.small_sweeps:
        out["small_sweeps"] = small_sweeps(args)

    # end to end through the C ABI from pinned host buffers: upload + layout + one sweep
    # + loss + factors back, per step
    c_pin = torch.empty((nnz, N), dtype=torch.int32, pin_memory=True)
    x_pin = torch.empty(nnz, dtype=torch.float32, pin_memory=True)
    c_pin.copy_(p.coords)
    x_pin.copy_(p.x)
    del p
    torch.cuda.empty_cache()
    cn, xn = c_pin.numpy(), x_pin.numpy()
    # the results land in page-locked host buffers, as the inputs come from them
    outs = [torch.empty((d, K), dtype=torch.float32, pin_memory=True).numpy()
            for d in WORKLOAD["dims"]]
    e2e_times, e2e_phases = [], []
    for s in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = tf.Factorization(cn, xn, WORKLOAD["dims"], K, seed=args.seed + rank, dtype=tf.F32,
                             stream=stream.cuda_stream)
        t1 = time.perf_counter()
        g.sweep(C, lam, T_in)
        g.loss(lam)
        t2 = time.perf_counter()
        for n in range(N):
            g._check(g._lib.tf_get_factors(g.handle, n, outs[n].ctypes.data_as(
                __import__("ctypes").c_void_p)))
        g.close()
        t3 = time.perf_counter()
        if s > 0:   # the first one is a warm-up
            e2e_times.append(t3 - t0)
            e2e_phases.append({"create_ms": (t1 - t0) * 1e3, "sweep_and_loss_ms": (t2 - t1) * 1e3,
                               "factors_and_destroy_ms": (t3 - t2) * 1e3})
    # the median step: a shared host occasionally stalls one upload or copy for tens of
    # milliseconds; every step's time and phases are reported beside it, and the mean
    e2e_s = statistics.median(e2e_times) if e2e_times else float("nan")
    e2e_mean_s = sum(e2e_times) / len(e2e_times) if e2e_times else float("nan")
    e2e_value = None
    if e2e_times:
        _, _, e2e_value = job_rate(e2e_s * 1e3, nnz * K * T_in, world)
    out["e2e"] = None if not e2e_times else {"value": e2e_value, "unit": UNIT,
                  "h2d_bytes_per_step": nnz * (4 * N + 4),
                  "d2h_bytes_per_step": sum(WORKLOAD["dims"]) * K * 4 + 16,
                  "what": "tf_create from pinned host COO + 1 sweep + tf_loss + factors to "
                          "pinned host memory + tf_destroy, median over the timed steps",
                  "mean_value": job_rate(e2e_mean_s * 1e3, nnz * K * T_in, world)[2],
                  "steps_ms": [t * 1e3 for t in e2e_times], "phases": e2e_phases}

    if args.configs and rank == 0 and world == 1:
        torch.cuda.empty_cache()
        if args.batched_tensors > 0:
            out["batched"] = batched_config(args, args.batched_tensors, hbm)
            torch.cuda.empty_cache()
        if args.fiveway_nnz > 0:
            out["fiveway"] = fiveway_config(args, args.fiveway_nnz, hbm)
            torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle as it stands, after the timed region: its OpenMP build on every host
        # core over a larger prefix, the serial build over a smaller one, and the parity
        # workload in full with both
        threads = oracle_threads()
        tp, up = run_oracle_sample(args.cpu_sample_parallel, args.seed, 1, parallel=True)
        ts, us = run_oracle_sample(args.cpu_sample, args.seed, 1)
        out["cpu_baseline"] = {
            "value": up / tp[0], "unit": UNIT, "cores": threads, "kind": "oracle",
            "host_cpus": os.cpu_count(),
            "sample": f"first {args.cpu_sample_parallel} entries (prefix of the seeded draw) "
                      f"of the same workload, one full sweep, K=100, C=10, FP64 C with "
                      f"OpenMP over rows ({threads} threads)",
            "single_thread": {"value": us / ts[0], "unit": UNIT, "cores": 1,
                              "sample": f"first {args.cpu_sample} entries, one full sweep"},
            "parity_workload": {"single_thread": run_oracle_parity_workload(False),
                                "openmp": run_oracle_parity_workload(True),
                                "what": "1000x1000x100, 1e5 entries, K=10, lambda=1, FP64, "
                                        "5 sweeps at C=5 and at C=1, in full"}}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
