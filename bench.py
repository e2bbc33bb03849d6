#!/usr/bin/env python
"""Benchmark of the GPU interior-point solver: time to the 1e-7 stopping tolerance
(paper §3: ε_abs = ε_rel = 1e-7) on the minimum-fuel trajectory SOCP with N = 20000
stages (N_K = 540018, ~2e6 KKT nonzeros; seeded synthetic data).

One step = one complete solve from a fresh initial point to the stopping tolerance
(every iteration: residuals, NT scaling, −W² update, LDLᵀ refactorisation, predictor
and corrector solves with refinement, steps).  `value` is seconds per solve with the
problem already resident in HBM (setup excluded, as in the paper's split of setup
and solve time, §3.2); `e2e` is the same metric through the C ABI with host buffers:
setup (host analysis + host→device copies), solve, copy of the solution back.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank solves its own replica; the reported time is the
max over ranks ("replicas only": a single solve is not sharded).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time_to_1e-7_gap"
WORKLOAD = "trajectory_socp_N20000"
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
HBM_FALLBACK_GBS = 6800.0
BF16_FALLBACK_TFLOPS = 1900.0
# TF32 : BF16 dense tensor-core rate of this part (1.1 : 2.25 PFLOP/s nominal, ~1/2)
TF32_OVER_BF16 = 0.5


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true",
                    help="mpc_batch: skip timing the plain solver on a sample of the instances")
    ap.add_argument("--stages", type=int, default=20000, help="trajectory stages (default: the benchmark size)")
    ap.add_argument("--workload", default="trajectory", choices=["trajectory", "lasso", "mpc_batch", "portfolio"],
                    help="trajectory (default, the headline line); lasso: the lasso QP scaled by 1/10 "
                         "(F 5000x10000, FP64 or --mixed); mpc_batch: 4096 MPC instances, solves/s; "
                         "portfolio: n = 20000 assets, solve plus the adjoint of ||x - 1/n||^2")
    ap.add_argument("--mixed", action="store_true", help="FP32 large fronts with FP64 refinement")
    ap.add_argument("--full", action="store_true",
                    help="lasso: the full size, F 50000x100000 with density 1e-3 (one 50440-row dense front)")
    ap.add_argument("--batch-schedule", type=int, default=0,
                    help="mpc_batch: 0 = the persistent batched kernel (default), 1-5 = the host-driven loop schedules")
    ap.add_argument("--factor-only", action="store_true",
                    help="lasso: time K factorisations at the initial scaling (W = I) instead of K solves")
    ap.add_argument("--ordering", default="auto", choices=["auto", "amd", "nd"],
                    help="fill-reducing ordering of the lasso / portfolio / mpc_batch workloads "
                         "(auto: the analysis' cost model, which counts a batch's independent trees)")
    ap.add_argument("--cpu-baseline-child", action="store_true", help=argparse.SUPPRESS)
    return ap.parse_args()


def workload(stages):
    from workloads import trajectory_socp
    return trajectory_socp(N=stages, seed=0)


def golden_iters(stages):
    path = os.path.join(ROOT, "tests", "golden", f"trajectory_socp_N{stages}.json")
    if os.path.exists(path):
        with open(path) as f:
            return int(json.load(f)["iters"])
    return None


def config(prob, extra=None):
    cfg = {"workload": f"trajectory_socp_N{prob.meta['N']}: min-fuel 3-D double integrator, "
                       f"{prob.meta['N']} stages, one Q^4 per stage + 7 orthant rows per stage",
           "n": prob.n, "m": prob.m, "p": prob.p, "kkt_dim": prob.kkt_dim(),
           "size_nnzA_nnzG_nnzPupper": prob.size(), "tolerance": 1e-7,
           "l2": "flushed between timed steps (256 MiB write); working set > L2"}
    if extra:
        cfg.update(extra)
    return cfg


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_uuid=None):
        self.uuid = dev_uuid
        self.proc = None
        self.lines = []

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- CPU baseline
def cpu_baseline_child(stages):
    """Runs in a subprocess with one BLAS/OpenMP thread: the oracle on a bounded sample
    of the workload (its initial point, then two iterations), scaled to one solve."""
    from oracle import ipm
    prob = workload(stages)
    t0 = time.perf_counter()
    ipm.solve(prob, ipm.Settings(max_iter=0))
    t_init = time.perf_counter() - t0
    t0 = time.perf_counter()
    ipm.solve(prob, ipm.Settings(max_iter=2))
    t2 = time.perf_counter() - t0
    per_iter = max(0.0, (t2 - t_init) / 2.0)
    iters = golden_iters(stages) or 30
    est = t_init + per_iter * iters
    print(json.dumps({"value": est, "t_init": t_init, "per_iter": per_iter, "iters": iters,
                      "sample_seconds": t_init + t2}))


def run_cpu_baseline(stages):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-baseline-child",
                        "--stages", str(stages)], capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        return {"value": None, "unit": "s", "cores": 1, "kind": "oracle",
                "sample": "failed: " + r.stderr.strip().splitlines()[-1] if r.stderr else "failed"}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": d["value"], "unit": "s", "cores": 1, "kind": "oracle",
            "sample": (f"oracle IPM on the same instance: initial point ({d['t_init']:.2f} s) plus 2 "
                       f"iterations timed ({d['sample_seconds']:.1f} s of CPU work); "
                       f"{d['per_iter']:.2f} s/iteration × {d['iters']} iterations (oracle's count) "
                       f"+ initial point"),
            "nproc": os.cpu_count()}


# --------------------------------------------------------------------------- helpers
def peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def tf32_peak():
    """TF32 dense tensor rate (GFLOP/s): the measured bf16 burst rate × the nominal
    TF32:BF16 ratio of this part."""
    try:
        with open(MEASURED_PEAKS) as f:
            return float(json.load(f)["bf16_tflops"]) * 1e3 * TF32_OVER_BF16, "measured bf16 burst x 1/2 (nominal TF32:BF16)"
    except Exception:
        return BF16_FALLBACK_TFLOPS * 1e3 * TF32_OVER_BF16, "fallback bf16 x 1/2 (nominal TF32:BF16)"


_FP64 = None


def fp64_peaks(q):
    """(DFMA, DMMA) GFLOP/s of this GPU, measured once by the library's own kernels."""
    global _FP64
    if _FP64 is None:
        _FP64 = q.fp64_peaks()
    return _FP64


# The sources each profiled kernel is built from (its own file and the headers it
# includes); the DRAM traffic ncu measured stays valid while these are unchanged.
# the kernel's own CUDA sources and the host sources that shape the supernodal tree it
# walks (ordering, amalgamation, plan): a change to either changes its DRAM traffic
KERNEL_SOURCES = {
    "k_factor_dataflow": ["factor.cu", "fronts.cuh", "factor.h", "common.cuh", "plan.h", "plan.cpp",
                          "ordering.cpp", "symbolic.cpp"],
    "k_solve_dataflow": ["factor.cu", "fronts.cuh", "factor.h", "common.cuh", "plan.h", "plan.cpp",
                         "ordering.cpp", "symbolic.cpp"],
}


def kernel_source_digest(kernel=None):
    """Digest of the sources of `kernel` (KERNEL_SOURCES; every CUDA source when it has
    no entry there): DRAM traffic measured by ncu is only reported while the kernel and
    the tree it walks are the ones it was measured on."""
    import hashlib
    h = hashlib.sha256()
    src = os.path.join(ROOT, "paper_2603_29197_gb300", "csrc")
    names = KERNEL_SOURCES.get(kernel) or [n for n in os.listdir(src) if n.endswith((".cu", ".cuh", ".h"))]
    for name in sorted(names):
        with open(os.path.join(src, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, stages):
    """dram__bytes_read.sum + dram__bytes_write.sum per launch of `kernel`, from the ncu
    summary in profiles/ (a line `traffic <kernel> <stages> <bytes> <source digest>`),
    or None when no capture matches this workload and this kernel's sources."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    digest = kernel_source_digest(kernel)
    with open(path) as f:
        for line in f:
            t = line.split()
            if len(t) == 5 and t[0] == "traffic" and t[1] == kernel and t[2] == str(stages) and t[4] == digest:
                return float(t[3])
    return None


def roofline(profile, info, stages, fp64):
    """Roofline of the phase with the largest device time (CUDA events on the solver's
    stream over the timed steps); fp64 = measured (DFMA, DMMA) GFLOP/s."""
    hbm, hbm_src = peaks()
    N = info["kkt_dim"]
    nnz = info["kkt_nnz"]
    ph = max(profile, key=lambda k: profile[k]["ms"])
    rec = profile[ph]
    per_call_ms = rec["ms"] / max(1, rec["calls"])
    if ph == "factor":
        flops = info["factor_flops"]
        ach = flops / (per_call_ms * 1e-3) / 1e9
        peak = max(fp64)
        return {"kernel": "k_factor_dataflow (one launch per LDLᵀ factorisation, the predictor's forward "
                          "sweep fused into it; achieved counts the factorisation's flops only)",
                "bound": "alu", "achieved": ach, "peak": peak, "unit": "GFLOP/s",
                "frac": ach / peak, "traffic": ncu_traffic("k_factor_dataflow", stages),
                "per_launch_unit": f"{flops:.4g} algorithmic flops per factorisation",
                "peak_source": (f"measured in this run by the library's FP64 kernels: DFMA {fp64[0]:.0f}, "
                                f"DMMA m8n8k4 {fp64[1]:.0f} GFLOP/s (the larger)"),
                "avg_ms": per_call_ms, "launches_per_call": rec["launches"] / max(1, rec["calls"])}
    if ph == "solve":
        by = 2.0 * info["l_nnz"] * 12.0 + N * 8.0 * 4.0
        name = "k_solve_dataflow (forward, diagonal and backward solve in one launch)"
    elif ph == "row":
        by = nnz * 12.0 + N * 8.0 * 3.0
        name = "k_residual / k_spmv_res / k_norm_inf (one pass)"
    else:
        by = info.get("m_cone", 0) * 8.0 * 12.0
        name = "cone kernels (one pass)"
    ach = by / (per_call_ms * 1e-3) / 1e9
    return {"kernel": name, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
            "frac": ach / hbm, "traffic": ncu_traffic(name.split()[0], stages), "per_launch_unit": f"{by:.4g} algorithmic bytes per call",
            "peak_source": f"{hbm_src} copy bandwidth", "avg_ms": per_call_ms,
            "launches_per_call": rec["launches"] / max(1, rec["calls"])}


def reduce_max(value, device=None):
    """Max of a float over the ranks (identity without a process group); the tensor lives
    on `device` (CUDA for NCCL, CPU for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "ours":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
    return ws, rank, local


# --------------------------------------------------------------------------- arms
def run_reference(args, ws, rank):
    if rank != 0:
        return
    from oracle import ipm
    prob = workload(args.stages)
    iters = golden_iters(args.stages) or 30
    t_init = []
    for _ in range(max(1, args.warmup)):
        t0 = time.perf_counter()
        ipm.solve(prob, ipm.Settings(max_iter=0))
        t_init.append(time.perf_counter() - t0)
    ti = statistics.median(t_init)
    vals, step_s = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        ipm.solve(prob, ipm.Settings(max_iter=1))
        dt = time.perf_counter() - t0
        step_s.append(dt)
        vals.append(ti + max(0.0, dt - ti) * iters)
    v = statistics.mean(vals)
    sample = (f"each step: oracle initial point + 1 iteration of the full instance "
              f"({statistics.mean(step_s):.1f} s), scaled to {iters} iterations")
    out = {"metric": METRIC, "value": v, "unit": "s", "impl": "reference", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(step_s) * 1e3,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded generator)", "config": config(prob),
           "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_ours(args, ws, rank, local):
    import torch
    import paper_2603_29197_gb300 as q
    from paper_2603_29197_gb300 import build as qbuild
    if not os.path.exists(qbuild.LIB):
        qbuild.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    prob = workload(args.stages)
    stream = torch.cuda.current_stream(dev)
    S = q.Solver(prob)
    setup_info = S.info()
    for _ in range(args.warmup):
        st = S.solve(stream.cuda_stream)
        if st != 0:
            raise RuntimeError(f"warm-up solve returned {q.STATUS_NAMES.get(st, st)}")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        if not uuid.startswith("GPU-"):
            uuid = "GPU-" + uuid
    except Exception:
        uuid = None
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(uuid)
    clocks.start()
    # inside the timed region only the factorisation (the dominant phase) is timed by
    # events: two per factorisation; the phase split comes from one more solve below
    S.set_profiling(2)
    times, launches, iters = [], 0, []
    t_wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = S.solve(stream.cuda_stream)
        e1.record(stream)
        e1.synchronize()
        if st != 0:
            raise RuntimeError(f"solve returned {q.STATUS_NAMES.get(st, st)}")
        times.append(e0.elapsed_time(e1))
        inf = S.info()
        launches += int(inf["kernel_launches"])
        iters.append(int(inf["iters"]))
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t_wall0
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    prof = S.profile()
    # the phase split: one more solve, every phase timed (outside the timed region)
    S.set_profiling(True)
    if S.solve(stream.cuda_stream) != 0:
        raise RuntimeError("profiled solve failed")
    split = S.profile()
    S.set_profiling(False)
    info = S.info()
    info["m_cone"] = prob.m
    ms = statistics.mean(times)
    ms_max = reduce_max(ms, dev)
    dominant = max(split, key=lambda k: split[k]["ms"])
    rl = roofline(prof if dominant == "factor" else split, info, args.stages, fp64_peaks(q))

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(q, prob, args, stream, dev)
        e2e["value"] = reduce_max(e2e["value"], dev)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = run_cpu_baseline(args.stages)
    if rank == 0:
        out = {"metric": METRIC, "value": ms_max / 1e3, "unit": "s", "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": False,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic (seeded generator, no dataset)",
               "config": config(prob, {"parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                                       "ordering": info["ordering_used"], "iterations": iters[-1],
                                       "n_supernodes": info["n_supernodes"], "tree_levels": info["n_levels"],
                                       "factor_flops": info["factor_flops"], "l_nnz": info["l_nnz"],
                                       "kkt_nnz": info["kkt_nnz"], "setup_s": setup_info["setup_time_s"],
                                       "analysis_s": setup_info["analysis_time_s"]}),
               "gpu_launches": launches,
               "refactor_gflops": info["factor_flops"] / (prof["factor"]["ms"] / max(1, prof["factor"]["calls"]) * 1e-3) / 1e9
               if prof["factor"]["calls"] else None,
               "phase_ms_per_solve": {k: v["ms"] for k, v in split.items()},
               "phase_note": "phase split of one solve after the timed region; inside it only the "
                             "factorisation phase carries events",
               "roofline": rl, "clocks": clk, "e2e": e2e, "cpu_baseline": cpu,
               "wall_s_timed": wall}
        print(json.dumps(out), flush=True)
    S.close()


def run_e2e(q, prob, args, stream, dev):
    """Same metric through the C ABI with host buffers: setup (analysis + host→device
    copies from pinned memory), solve, device→host copy of the solution, cleanup."""
    import numpy as np
    import torch

    def pinned(a, dtype):
        t = torch.empty(len(a), dtype=dtype, pin_memory=True)
        t.numpy()[:] = a
        return t.numpy()

    class Pinned:
        pass

    pp = Pinned()
    for k in ("n", "m", "p", "l", "q", "meta"):
        setattr(pp, k, getattr(prob, k))
    for k in ("c", "b", "h"):
        setattr(pp, k, pinned(getattr(prob, k), torch.float64))
    for k in ("P", "A", "G"):
        M = getattr(prob, k).tocsc()
        M2 = M.copy()
        M2.data = pinned(M.data, torch.float64)
        M2.indices = pinned(M.indices.astype(np.int32), torch.int32)
        M2.indptr = pinned(M.indptr.astype(np.int32), torch.int32)
        setattr(pp, k, M2)
    times = []
    h2d = d2h = 0
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        S = q.Solver(pp)
        st = S.solve(stream.cuda_stream)
        sol = S.solution()
        S.close()
        t1 = time.perf_counter()
        if st != 0:
            raise RuntimeError(f"e2e solve returned {st}")
        if i >= args.warmup:
            times.append(t1 - t0)
        inf = sol["info"]
        h2d = int(inf["h2d_bytes"])
        d2h = int(inf["d2h_bytes"]) + 8 * (prob.n + 2 * prob.m + prob.p)
    return {"value": statistics.mean(times), "unit": "s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h,
            "note": "setup incl. host ordering + symbolic analysis, solve, solution copy-back"}


# --------------------------------------------------------------------------- other workloads
def other_workload(args, rank=0, ws=1):
    """The instances of one rank: the lasso and portfolio problems are replicated; the
    MPC batch is one job of ws × 4096 instances (seed 0; the first 4096 are the 1-GPU
    batch) split into contiguous ranges balanced by N_K³ (paper_2603_29197_gb300.shard),
    and rank r solves its own range; nothing crosses ranks until the final gather."""
    from workloads import lasso_qp, mpc_batch, portfolio_socp
    if args.workload == "lasso":
        if args.full:
            return [lasso_qp(rows=50000, cols=100000, density=1e-3, seed=0)]
        return [lasso_qp(rows=5000, cols=10000, density=5e-3, seed=0)]
    if args.workload == "portfolio":
        return [portfolio_socp(n=20000, k=200, seed=0)]
    from paper_2603_29197_gb300.shard import instance_cost, partition
    job = mpc_batch(count=4096 * ws, seed=0)
    starts = partition([instance_cost(p) for p in job], ws)
    args.batch_job, args.batch_starts = len(job), starts
    return job[starts[rank]:starts[rank + 1]]


def lasso_certificate(prob, x_all, pobj):
    """Optimality of the lasso part of a solution, from the data alone: with
    g = Fᵀ(Fx − y), the subgradient condition is |g_j| ≤ λ everywhere and g_j = −λ·sign(x_j)
    on the support.  Returned relative to λ (the 1e-7 stopping tolerance leaves ~1e-6)."""
    import numpy as np
    F, y, lam = prob.meta["F"], prob.meta["y"], prob.meta["lam"]
    x = np.asarray(x_all[:F.shape[1]], float)
    res = F @ x - y
    g = F.T @ res
    supp = np.abs(x) > 1e-3 * float(np.max(np.abs(x)))  # the clear support
    obj = 0.5 * float(res @ res) + lam * float(np.abs(x).sum())
    return {"max_abs_g_over_lambda_minus_1": float(np.max(np.abs(g)) / lam - 1.0),
            "support": int(supp.sum()),
            "support_sign_residual": float(np.max(np.abs(g[supp] + lam * np.sign(x[supp]))) / lam)
            if supp.any() else 0.0,
            "lasso_objective": obj, "objective_vs_pobj_rel": abs(obj - pobj) / max(1.0, abs(obj))}


def batch_check(S, args, ws, rank, dev):
    """After the timed region: every rank's per-instance status and primal objective are
    gathered to rank 0 (the one collective of the sharded batch), which reports how many
    instances solved and compares a seeded sample of objectives with the oracle's values
    stored in tests/golden/mpc_batch_4096_sample.json (the first 4096 instances of the
    job are the 1-GPU batch)."""
    import numpy as np
    bi = S.batch_info()
    mine = (rank, [int(v) for v in bi["status"]], [float(v) for v in bi["pobj"]])
    if ws > 1:
        import torch.distributed as dist
        got = [None] * ws if rank == 0 else None
        dist.gather_object(mine, got, dst=0)
    else:
        got = [mine]
    if rank != 0:
        return None
    status, pobj = [0] * args.batch_job, [0.0] * args.batch_job
    for r, st, po in got:
        a = args.batch_starts[r]
        status[a:a + len(st)] = st
        pobj[a:a + len(po)] = po
    out = {"instances": args.batch_job, "solved": int(sum(1 for v in status if v == 0))}
    path = os.path.join(ROOT, "tests", "golden", "mpc_batch_4096_sample.json")
    if os.path.exists(path):
        with open(path) as f:
            g = json.load(f)
        errs = [abs(pobj[i] - v) / max(1.0, abs(v)) for i, v in zip(g["idx"], g["pobj"])]
        out["pobj_rel_vs_oracle_max"] = float(np.max(errs))
        out["sample"] = f"{len(errs)} seeded instances, oracle values in tests/golden/mpc_batch_4096_sample.json"
    return out


def golden_error(name, sol, pobj):
    """Deviation of the solution from the stored oracle values (tests/golden), if any."""
    path = os.path.join(ROOT, "tests", "golden", name + ".json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        g = json.load(f)
    out = {"pobj_rel": abs(pobj - g["pobj"]) / max(1.0, abs(g["pobj"]))}
    for key in ("x", "y", "z"):
        if f"{key}_idx" in g:
            got = [float(sol[key][i]) for i in g[f"{key}_idx"]]
            d = max(abs(a - b) for a, b in zip(got, g[f"{key}_val"]))
            out[f"{key}_rel_sampled"] = d / max(1.0, g[f"{key}_inf"])
    out["reference"] = f"oracle values stored in tests/golden/{name}.json"
    return out


def run_other(args, ws, rank, local):
    """The lasso QP (time to the 1e-7 gap, FP64 or mixed) or the MPC batch (solves/s),
    timed like the headline workload: W warm-up solves, K timed solves with CUDA events,
    L2 flushed between them; e2e includes set-up from host data and the copy-back."""
    import numpy as np
    import torch
    import paper_2603_29197_gb300 as q
    from paper_2603_29197_gb300 import build as qbuild
    if not os.path.exists(qbuild.LIB):
        qbuild.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    probs = other_workload(args, rank, ws)
    batch = args.workload == "mpc_batch"
    kw = dict(mixed_precision=1 if args.mixed else 0, ordering={"auto": 0, "amd": 1, "nd": 2}[args.ordering])
    if batch:
        kw["batch_schedule"] = args.batch_schedule
    make = (lambda: q.BatchSolver(probs, **kw)) if batch else (lambda: q.Solver(probs[0], **kw))
    S = make()
    stream = torch.cuda.current_stream(dev)
    fp64 = fp64_peaks(q)
    if args.factor_only:
        return run_factor_only(args, S, probs[0], stream, dev, fp64)
    failed = None  # a rank whose solve fails stops every rank together (below)
    for _ in range(args.warmup):
        st = S.solve(stream.cuda_stream)
        if st != 0:
            failed = failed or f"warm-up solve returned {st}"
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    clocks = ClockSampler(None)
    clocks.start()
    S.set_profiling(True)
    times, launches = [], 0
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.synchronize(dev)
        dist.barrier()
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = S.solve(stream.cuda_stream)
        e1.record(stream)
        e1.synchronize()
        if st != 0:
            failed = failed or f"solve returned {st}"
        times.append(e0.elapsed_time(e1))
        launches += int(S.info()["kernel_launches"])
    if ws > 1:
        torch.cuda.synchronize(dev)
        dist.barrier()
    clk = clocks.stop()
    if reduce_max(1.0 if failed else 0.0, dev) > 0.0:
        raise RuntimeError(failed or "a solve failed on another rank")
    prof = S.profile()
    info = S.info()
    S.set_profiling(False)
    ms = reduce_max(statistics.mean(times), dev)  # the slowest rank
    adj = None
    if args.workload == "portfolio":
        # the adjoint of L = ||x - 1/n||^2 after the last timed solve (reuses its factor)
        x = S.solution_tensors()[0]
        gx = 2.0 * (x - 1.0 / x.numel())
        bts = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            S.backward(dx=gx)
            e1.record(stream)
            e1.synchronize()
            bts.append(e0.elapsed_time(e1))
        bi = S.backward_info()
        adj = {"backward_ms": statistics.mean(bts), "refine_steps": bi["refine_steps"],
               "backward_error": bi["backward_error"], "refactored": bi["refactored"],
               "solve_plus_backward_ms": ms + statistics.mean(bts)}
    plain = None
    if batch and not args.no_plain and ws == 1:
        # the plain FP64 form on the same instances, one solver per instance, one at a
        # time: a seeded sample of 16 instances (device-timed solves, set-up excluded)
        idx = sorted(np.random.default_rng(0).choice(len(probs), size=16, replace=False).tolist())
        pts = []
        for i in idx:
            one = q.Solver(probs[i])
            if one.solve(stream.cuda_stream) != 0:
                raise RuntimeError(f"plain solve of instance {i} failed")
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st1 = one.solve(stream.cuda_stream)
            e1.record(stream)
            e1.synchronize()
            if st1 != 0:
                raise RuntimeError(f"plain solve of instance {i} failed")
            pts.append(e0.elapsed_time(e1))
            one.close()
        per_s = 1e3 / statistics.mean(pts)
        plain = {"value": per_s, "unit": "solves/s", "ms_per_solve": statistics.mean(pts),
                 "sample": "16 seeded instances, each on its own solver, one after the other",
                 "batched_over_plain": (len(probs) / (ms * 1e-3)) / per_s}
    fcalls = prof["factor"]["calls"]
    if fcalls:
        f_ms = prof["factor"]["ms"] / fcalls
        gflops = info["factor_flops"] / (f_ms * 1e-3) / 1e9
        rl = factor_roofline(args.mixed and info["fp32_factors"] > 0, gflops, f_ms, info, fp64)
    else:
        # the persistent batched kernel: one launch per batched solve runs every step; its
        # algorithmic work counted here is the factorisations alone, Σ over instances of
        # (iterations + 1) × that instance's factor flops (≈ the stack's flops × (mean
        # iterations + 1)), a lower bound on the FP64 work of the launch
        bi = S.batch_info()
        mean_it = float(np.mean(bi["iters"]))
        flops = info["factor_flops"] * (mean_it + 1.0)
        gflops = flops / (ms * 1e-3) / 1e9
        peak = max(fp64)
        rl = {"kernel": "k_batch_ipm (one persistent launch per batched solve)", "bound": "alu",
              "achieved": gflops, "peak": peak, "unit": "GFLOP/s", "frac": gflops / peak, "traffic": None,
              "per_launch_unit": f"{flops:.4g} algorithmic factorisation flops per launch "
                                 f"(stack {info['factor_flops']:.4g} x (mean iterations {mean_it:.2f} + 1))",
              "peak_source": f"measured in this run: DFMA {fp64[0]:.0f}, DMMA {fp64[1]:.0f} GFLOP/s (the larger)",
              "avg_ms": ms, "note": "latency-bound: per-instance level chains of small fronts"}
        f_ms = None
    # e2e: set-up from host data, solve, copy-back
    e2e_s, sol, e2e_split = None, None, None
    if not args.no_e2e:
        t0 = time.perf_counter()
        E = make()
        t1 = time.perf_counter()
        st = E.solve(stream.cuda_stream)
        t2 = time.perf_counter()
        sol = E.solution()
        e2e_s = reduce_max(time.perf_counter() - t0, dev)
        ei = E.info()
        e2e_split = {"setup_s": t1 - t0, "library_setup_s": ei["setup_time_s"],
                     "analysis_s": ei["analysis_time_s"], "first_solve_s": t2 - t1,
                     "copy_back_s": t0 + e2e_s - t2}
        E.close()
    # CPU oracle on a bounded sample
    from oracle import ipm
    t0 = time.perf_counter()
    if args.no_cpu_baseline or ws > 1:
        cpu = None
    elif batch:
        sample = probs[:16]
        for pr in sample:
            ipm.solve(pr)
        cpu_s = (time.perf_counter() - t0) / len(sample) * len(probs)
        cpu = {"value": len(probs) / cpu_s, "unit": "solves/s", "cores": 1, "kind": "oracle",
               "sample": f"oracle IPM on 16 of the {len(probs)} instances, scaled"}
    elif args.full:
        cpu = {"value": None, "unit": "s", "cores": 1, "kind": "oracle",
               "sample": "not run: one sparse LU of this KKT (a dense 50440-row Schur complement) takes hours "
                         "on one core"}
    else:
        ipm.solve(probs[0], ipm.Settings(max_iter=0))
        t_init = time.perf_counter() - t0
        cpu = {"value": t_init * (info["iters"] + 1), "unit": "s", "cores": 1, "kind": "oracle",
               "sample": f"oracle initial point (one sparse LU of the KKT, {t_init:.1f} s) × "
                         f"{info['iters'] + 1} factorisations"}
    if batch:
        # whole job: every rank's instances over the slowest rank's time
        metric, value, unit, hib = "batched_solves_per_s", args.batch_job / (ms * 1e-3), "solves/s", True
        e2e = {"value": args.batch_job / e2e_s, "unit": unit} if e2e_s else None
    else:
        metric, value, unit, hib = "time_to_1e-7_gap", ms * 1e-3, "s", False
        e2e = {"value": e2e_s, "unit": unit} if e2e_s else None
    if e2e:
        e2e["split"] = e2e_split
        e2e.update({"h2d_bytes_per_step": int(sol["info"]["h2d_bytes"]),
                    "d2h_bytes_per_step": int(sol["info"]["d2h_bytes"]) + 8 * (S.n + 2 * S.m + S.p)})
    wl = {"mpc_batch": "mpc_batch_4096: horizons U{10..60}, state 4, control 2, Q^3 input cone, box bounds",
          "lasso": ("lasso_qp_r50000_c100000: F 50000x100000, density 1e-3 (100 nnz/row)" if args.full else
                    "lasso_qp_r5000_c10000: F 5000x10000, 50 nnz/row"),
          "portfolio": "portfolio_socp_n20000: 20000 assets, factor model k=200, Q^201 risk cone"}
    cfg = {"workload": wl[args.workload],
           "kkt_dim": info["kkt_dim"], "kkt_nnz": info["kkt_nnz"], "factor_flops": info["factor_flops"],
           "iterations": info["iters"], "max_front": info["max_front"], "large_fronts": info["large_fronts"],
           "precision": "mixed (FP32 large fronts, FP64 refinement)" if args.mixed else "fp64",
           "ordering": {0: "auto", 1: "amd", 2: "nd", 3: "natural"}.get(info["ordering_used"], "?") +
                       (" (requested)" if args.ordering != "auto" else " (cost model)"),
           "fp32_factors": info["fp32_factors"], "fp64_escalations": info["fp64_escalations"],
           "fp32_floor_raises": info["fp32_floor_raises"],
           "krylov_steps": info["krylov_steps"], "refine_steps": info["refine_steps"],
           "batch_schedule": info["batch_schedule_used"] if batch else None,
           "batch_tile": ({"warps_per_cta": info["batch_warps"], "thread_fronts": info["batch_thread_fronts"],
                           "warps_per_sm": info["batch_warps_per_sm"]} if batch else None),
           "l2": "flushed between timed steps (256 MiB write)",
           "parallelism": ("single GPU" if ws == 1 else
                           f"one job of {ws} x 4096 instances in {ws} contiguous ranges balanced by N_K^3, "
                           f"one gather of the results to rank 0 after the timed region" if batch else
                           f"replicas x{ws}")}
    out = {"metric": metric, "value": value, "unit": unit, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": hib, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32+f64" if args.mixed else "f64", "data": "synthetic (seeded generator)",
           "config": cfg, "gpu_launches": launches, "refactor_gflops": gflops,
           "phase_ms_per_solve": {k: v["ms"] / args.steps for k, v in prof.items()},
           "roofline": rl, "clocks": clk, "e2e": e2e, "cpu_baseline": cpu}
    if batch:
        out["batch_check"] = batch_check(S, args, ws, rank, dev)
    if not batch:
        final = S.solution()
        if args.workload == "lasso" and args.full:
            # no oracle run at this size: the solution is certified from the data alone
            out["certificate"] = lasso_certificate(probs[0], final["x"], info["pobj"])
        else:
            gname = {"lasso": "lasso_qp_r5000_c10000", "portfolio": "portfolio_socp_n20000"}[args.workload]
            out["error_vs_oracle"] = golden_error(gname, final, info["pobj"])
    if adj:
        out["adjoint"] = adj
    if plain:
        out["plain_fp64_one_at_a_time"] = plain
    if rank == 0:
        print(json.dumps(out), flush=True)
    S.close()


def factor_roofline(mixed, gflops, f_ms, info, fp64):
    """Roofline of one factorisation: FP64 against the measured FP64 rate; mixed
    precision (FP32 large fronts, their trailing updates as three TF32 tensor-core
    products) against the TF32 tensor peak, with the products issued (3× the useful
    flops of those updates) stated beside the useful rate."""
    if mixed:
        peak, src = tf32_peak()
        return {"kernel": "factorisation (large fronts: FP32 panels + 3xTF32 tcgen05 trailing updates)",
                "bound": "tensor", "achieved": gflops, "peak": peak, "unit": "GFLOP/s", "frac": gflops / peak,
                "traffic": None, "issued_tf32_gflops_upper_bound": 3.0 * gflops,
                "per_launch_unit": f"{info['factor_flops']:.4g} algorithmic flops per factorisation",
                "peak_source": src, "avg_ms": f_ms}
    peak = max(fp64)
    return {"kernel": "factorisation (large-front panel kernels + supernodal kernels)", "bound": "alu",
            "achieved": gflops, "peak": peak, "unit": "GFLOP/s", "frac": gflops / peak, "traffic": None,
            "per_launch_unit": f"{info['factor_flops']:.4g} algorithmic flops per factorisation",
            "peak_source": f"measured in this run: DFMA {fp64[0]:.0f}, DMMA m8n8k4 {fp64[1]:.0f} GFLOP/s (the larger)",
            "avg_ms": f_ms}


def run_factor_only(args, S, prob, stream, dev, fp64):
    """K factorisations of the KKT matrix at the initial scaling s = z = e (W = I), each
    timed with CUDA events on the solver's stream after W warm-up ones: the refactor
    GFLOP/s of a size whose full solve is too long to repeat (FP64)."""
    import numpy as np
    import torch
    e = torch.zeros(prob.m, dtype=torch.float64, device=dev)
    o = 0
    if prob.l:
        e[:prob.l] = 1.0
        o = prob.l
    for qk in prob.q:
        e[o] = 1.0
        o += qk
    for _ in range(args.warmup):
        S.kkt_factor_at(e, e, stream.cuda_stream)
    times = []
    clocks = ClockSampler(None)
    clocks.start()
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        S.kkt_factor_at(e, e, stream.cuda_stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    info = S.info()
    f_ms = statistics.mean(times)
    gflops = info["factor_flops"] / (f_ms * 1e-3) / 1e9
    out = {"metric": "kkt_refactor_gflops", "value": gflops, "unit": "GFLOP/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": f_ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if args.mixed else "f64",
           "data": "synthetic (seeded generator)",
           "config": {"workload": ("lasso_qp_r50000_c100000" if args.full else "lasso_qp_r5000_c10000") +
                                  ": one factorisation at W = I (includes the NT-scaling kernel and the norm pass)",
                      "kkt_dim": info["kkt_dim"], "factor_flops": info["factor_flops"],
                      "max_front": info["max_front"], "front_entries": info["front_entries"],
                      "setup_s": info["setup_time_s"], "analysis_s": info["analysis_time_s"],
                      "precision": "mixed (FP32 large fronts)" if args.mixed else "fp64"},
           "roofline": factor_roofline(args.mixed, gflops, f_ms, info, fp64), "clocks": clk,
           "fp64_peaks_gflops": {"dfma": fp64[0], "dmma": fp64[1]}}
    print(json.dumps(out), flush=True)
    S.close()


def main():
    args = parse()
    if args.cpu_baseline_child:
        cpu_baseline_child(args.stages)
        return
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
    elif args.workload != "trajectory":
        run_other(args, ws, rank, local)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
