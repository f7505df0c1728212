#!/usr/bin/env python
"""Benchmark: CP solves per second to ||grad f|| / #params < 1e-7 on the dense
256 x 256 x 256 FP32 tensor (planted rank 16, collinearity 0.9, 10 %
homoscedastic + 10 % heteroscedastic noise), solved at R = 16 by N-GMRES
(w = 20) accelerated ALS with the More-Thuente line search.

One step = one complete solve from the same seeded N(0,1) initial guess with
the tensor already resident in HBM; L2 is flushed (512 MiB write, 256 MiB read) before
every timed step, outside the timed interval.  Prints ONE JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec mixed|fp64]
  python bench.py --impl reference ...   (the FP64 CPU oracle on host cores)

With more than one process (torchrun), every rank solves its own replica
(no collective on the data path); value = all ranks' solves / max time.
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

METRIC = "CP solves/s & p99 latency to rel-grad 1e-7; MTTKRP %roofline, mixed vs FP64"
UNIT = "solves/s"
WORKLOAD = ("dense 256x256x256 fp32, planted R=16, collinearity 0.9, 10% homoscedastic + "
            "10% heteroscedastic noise; N-GMRES w=20 + More-Thuente, R=16, stop ||g||/P < 1e-7")
DIMS = (256, 256, 256)
R = 16
TOL = 1e-7
# FP64 FMA issue rate of the part: 2 FP64 FMA per clock per SM (152 SMs at
# 2070 MHz max) -> 2 * 2 * 152 * 2.07e9 flop/s.  cuBLAS DGEMM measured 1.10.
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.070e9 / 1e12


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--mttkrp-only", default=None,
                   choices=["dense_256", "dense_4way", "sparse", "sparse_scaled", "dimtree_256"],
                   help="time only cp_mttkrp on that workload (profiling driver)")
    p.add_argument("--many-only", action="store_true",
                   help="cp_solve_many calls on one fixed case (default: 16 requests of 48^3, R=8, mixed, 20 "
                        "iterations each, clusters of 2 CTAs; profiling driver for the cluster engine's kernel)")
    p.add_argument("--many-shape", type=int, default=48, help="--many-only: side of the cubic tensors")
    p.add_argument("--many-rank", type=int, default=8, help="--many-only: planted and fitted rank")
    p.add_argument("--many-count", type=int, default=16, help="--many-only: requests per call")
    p.add_argument("--many-iters", type=int, default=20, help="--many-only: iterations per request")
    p.add_argument("--many-cluster", type=int, default=2, help="--many-only: CTAs per cluster")
    p.add_argument("--many-prec", default="mixed", choices=["mixed", "fp64"], help="--many-only: precision")
    p.add_argument("--reps", type=int, default=3)
    p.add_argument("--accuracy-report", default=None, choices=["dense_256", "dense_4way"],
                   help="mixed (with FP64 polish) against FP64 solves of one workload; one JSON line")
    p.add_argument("--solve-only", action="store_true",
                   help="time only the headline solves (profiling driver; no side reports)")
    p.add_argument("--small-kernels", action="store_true",
                   help="run the solve's small kernels eagerly on the 256^3 workload (f/g, ALS sweep with "
                        "normalisation, N-GMRES step, line search) so that ncu can profile them")
    p.add_argument("--kernel-breakdown", action="store_true",
                   help="one headline solve under the CUDA profiler (CUPTI): per-kernel launches, device "
                        "time and critical-path share (ncu does not see kernels inside conditional graph bodies)")
    p.add_argument("--serve-requests", type=int, default=1024,
                   help="requests of the 200/s Poisson serving stream replayed (0: skip)")
    p.add_argument("--serve-fp64-requests", type=int, default=32,
                   help="requests solved by the FP64 path in saturation for the mixed-vs-FP64 figure")
    p.add_argument("--serve-slots", type=int, default=48)
    p.add_argument("--dimtree", type=int, default=-1, choices=[-1, 0, 1],
                   help="dimension-tree MTTKRP pairs in the mixed solve: -1 library default, 0 off, 1 on")
    p.add_argument("--fixed-iters", type=int, default=0,
                   help="solve-only timing at exactly this many iterations (tolerance out of reach): ms per iteration")
    p.add_argument("--precision-table", type=int, default=0,
                   help="solve the first N serving-stream requests alone in FP64 and in mixed precision; "
                        "one JSON line per request (time, iterations, entries)")
    p.add_argument("--table-mixed-only", action="store_true", help=argparse.SUPPRESS)
    p.add_argument("--mixed-stall", type=int, default=0, help=argparse.SUPPRESS)
    p.add_argument("--serve-only", action="store_true", help="only the serving stream block (profiling driver)")
    p.add_argument("--no-workloads", action="store_true",
                   help="skip the 20^3, 96^4 and sparse workload blocks of the bench line")
    p.add_argument("--cpu-sample", action="store_true", help=argparse.SUPPRESS)
    p.add_argument("--cpu-c1", action="store_true", help=argparse.SUPPRESS)
    p.add_argument("--cpu-iters", type=int, default=1, help=argparse.SUPPRESS)
    p.add_argument("--cpu-workload", default="dense_256", choices=["dense_256", "sparse_20000"],
                   help=argparse.SUPPRESS)
    return p.parse_args()


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class L2Flush:
    """Between timed launches: write a 512 MiB buffer (larger than the 129 MB
    L2), then read a second 256 MiB buffer, so that the next kernel starts
    with a cold L2 that holds no dirty lines of the flush (whose write-back
    would otherwise be charged to it)."""

    def __init__(self, dev):
        import torch
        self.w = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        self.r = torch.ones(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        self.sink = torch.empty(1, dtype=torch.float32, device=dev)

    def __call__(self, stream, k):
        import torch
        with torch.cuda.stream(stream):
            self.w.fill_(float(k))
            torch.sum(self.r, dim=0, keepdim=True, out=self.sink)


# ---------------------------------------------------------------- CPU oracle
def oracle_solve(name="dense_256"):
    """The oracle's own solve of a workload (iterations, f/g evaluations, ...)
    as stored by oracle/workload_iters.py, or None."""
    path = os.path.join(ROOT, "oracle", "workload_iters.json")
    try:
        return json.load(open(path))[name]
    except Exception:
        return None


def oracle_iters(name="dense_256"):
    s = oracle_solve(name)
    return s["iters"] if s else None


def cpu_sample(n_iters: int, name: str = "dense_256") -> dict:
    """Time the oracle on a workload (dense_256: 256^3 R=16; sparse_20000:
    20000^3 with 2e6 nonzeros, R=10): its start-up (normalise + f/g) and
    then n_iters N-GMRES iterations of one solve, each timed on its own (an
    iteration starts at its Step I, the ALS sweep), with the time of every
    ALS sweep and every f/g evaluation inside it."""
    import synth
    from oracle import cp_oracle as O
    if name == "sparse_20000":
        prob, u0 = synth.workload_sparse()
        X = O.SparseTensor(prob.coords, prob.vals, prob.dims)
        Rw = prob.R
    else:
        prob, u0 = synth.workload_dense_256()
        X = O.DenseTensor(prob.T)
        Rw = R
    marks, sweeps, fgs = [], [], []
    real_sweep, real_fg = O.als_sweep, O.fg

    def timed_sweep(*a, **k):
        marks.append(time.perf_counter())
        r = real_sweep(*a, **k)
        sweeps.append(time.perf_counter() - marks[-1])
        return r

    def timed_fg(*a, **k):
        t = time.perf_counter()
        r = real_fg(*a, **k)
        fgs.append((len(marks), time.perf_counter() - t))
        return r
    O.als_sweep, O.fg = timed_sweep, timed_fg
    try:
        t0 = time.perf_counter()
        _, _, rep = O.cp_solve(X, u0, O.SolveOpts(R=Rw, tol=TOL), max_iters=n_iters)
        t_end = time.perf_counter()
    finally:
        O.als_sweep, O.fg = real_sweep, real_fg
    bounds = marks + [t_end]
    per_iter = [bounds[i + 1] - bounds[i] for i in range(len(marks))]
    # f/g evaluations of iteration i (1-based: made after its sweep began)
    fg_n = [sum(1 for k, _ in fgs if k == i + 1) for i in range(len(marks))]
    fg_t = [sum(d for k, d in fgs if k == i + 1) for i in range(len(marks))]
    t_init = (marks[0] if marks else t_end) - t0
    res = dict(workload=name, t_init_s=t_init, per_iter_s=per_iter, sweep_s=sweeps, fg_count=fg_n, fg_s=fg_t,
               iters_sampled=rep.iters)
    res.update(extrapolate(res, 0))
    return res


def extrapolate(s: dict, skip: int) -> dict:
    """Seconds of a whole oracle solve from a sample: the start-up, plus the
    oracle's own iteration count times the mean ALS sweep and the rest of an
    iteration (Step II, normalisations), plus its own count of f/g
    evaluations after the start-up times the mean evaluation; means over the
    sampled iterations after the first `skip`.  (Per-iteration times are
    skewed by the line search: a search may take 1 or 20 evaluations.)"""
    full = oracle_solve(s["workload"])
    it = range(skip, len(s["per_iter_s"]))
    if not full or not it:
        return dict(oracle_iters=None, oracle_fg_evals=None, est_solve_s=None)
    sweep = sum(s["sweep_s"][i] for i in it) / len(it)
    nfg = sum(s["fg_count"][i] for i in it)
    fg = sum(s["fg_s"][i] for i in it) / max(nfg, 1)
    rest = sum(s["per_iter_s"][i] - s["sweep_s"][i] - s["fg_s"][i] for i in it) / len(it)
    est = s["t_init_s"] + full["iters"] * (sweep + rest) + (full["fg_evals"] - 1) * fg
    return dict(oracle_iters=full["iters"], oracle_fg_evals=full["fg_evals"], mean_sweep_s=sweep,
                mean_fg_s=fg, mean_rest_s=rest, est_solve_s=est)


def cpu_solves_c1(n_solves: int) -> dict:
    """Whole oracle solves of the 20x20x20 R=3 workload to ||g||/P < 1e-7,
    each timed from the initial guess to convergence."""
    import synth
    from oracle import cp_oracle as O
    prob, u0 = synth.workload_dense_small()
    X = O.DenseTensor(prob.T)
    times, iters = [], None
    for _ in range(n_solves):
        t0 = time.perf_counter()
        _, _, rep = O.cp_solve(X, u0, O.SolveOpts(R=3, tol=TOL))
        times.append(time.perf_counter() - t0)
        iters = rep.iters
    return dict(solves=n_solves, mean_s=sum(times) / len(times), iters=iters)


def host_cpu() -> dict:
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:  # noqa: BLE001
        pass
    return {"nproc": os.cpu_count(), "model": model}


def run_cpu_child(flag: str, n: int, threads: int = 1, extra=()) -> dict:
    """Run one CPU timing in a child process with `threads` BLAS threads and
    no GPU visible; returns its JSON result (or {"error": ...})."""
    t = str(threads)
    env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t,
               CUDA_VISIBLE_DEVICES="")
    try:
        out = subprocess.run([sys.executable, os.path.abspath(__file__), flag, "--cpu-iters", str(n), *extra],
                             capture_output=True, text=True, env=env, timeout=1800)
        return json.loads(out.stdout.strip().splitlines()[-1])
    except Exception as exc:  # noqa: BLE001
        return {"error": str(exc)[:200]}


def run_cpu_baseline_subprocess(n_iters: int, threads: int = 1, name: str = "dense_256") -> dict | None:
    return run_cpu_child("--cpu-sample", n_iters, threads, ("--cpu-workload", name))


def sample_text(s: dict, how: str) -> str:
    per = s.get("per_iter_s") or [0.0]
    if not s.get("est_solve_s"):
        return (f"oracle start-up + {len(per)} N-GMRES iteration(s) of this workload timed ({how}); no stored "
                f"oracle solve to scale to")
    return (f"oracle start-up + {len(per)} N-GMRES iteration(s) of this workload timed (numpy {how}; "
            f"start-up {s['t_init_s']:.2f} s, ALS sweep {s['mean_sweep_s']:.2f} s, f/g evaluation "
            f"{s['mean_fg_s']:.2f} s, rest {s['mean_rest_s']:.3f} s per iteration), scaled to the oracle's own "
            f"solve of it: {s['oracle_iters']} iterations and {s['oracle_fg_evals']} f/g evaluations "
            f"(oracle/workload_iters.json)")


def cpu_baseline_obj(s: dict, threads: int = 1) -> dict:
    est = s.get("est_solve_s")
    how = "single thread" if threads == 1 else f"{threads} BLAS threads"
    return {"value": 1.0 / est if est else None, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": sample_text(s, how), "host": host_cpu()}


def cpu_samples_obj(one: dict, allc: dict | None, nproc: int) -> dict:
    """cpu_baseline from a one-thread sample, with the all-cores sample of
    the same workload beside it (the oracle as it stands: its loops do not
    use more threads, so the two agree)."""
    if "error" in one:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": one["error"]}
    res = cpu_baseline_obj(one)
    if allc is not None:
        if "error" in allc:
            res["all_cores"] = {"error": allc["error"]}
        else:
            a = cpu_baseline_obj(allc, nproc)
            res["all_cores"] = {"value": a["value"], "unit": UNIT, "blas_threads": nproc, "sample": a["sample"],
                                "note": "the oracle's MTTKRP (numpy einsum) runs on one thread whatever "
                                        "the BLAS thread count; only its small matrix products can use more"}
    return res


def cpu_c1_block() -> dict:
    """The oracle's whole solves of the 20x20x20 workload on the host, one
    BLAS thread and all cores (no extrapolation)."""
    h = host_cpu()
    one = run_cpu_child("--cpu-c1", 20, 1)
    allc = run_cpu_child("--cpu-c1", 20, h["nproc"] or 1)
    res = {"host": h, "kind": "oracle", "workload": "dense 20x20x20 fp64, R=3, c=0.5, 10% noise, tol 1e-7"}
    for name, r in (("one_thread", one), ("all_cores", allc)):
        if "error" in r:
            res[name] = r
        else:
            res[name] = {"solves_per_s": 1.0 / r["mean_s"], "ms_per_solve": 1e3 * r["mean_s"],
                         "solves_timed": r["solves"], "iters": r["iters"],
                         "threads": 1 if name == "one_thread" else h["nproc"]}
    return res


# ------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[4:8]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- our arm
def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    import synth
    import paper_1105_5331_gb300 as cp

    cpu = cpu_c1 = cpu_c4 = None
    if rank == 0 and not args.no_cpu_baseline and not args.solve_only:
        nproc = host_cpu()["nproc"] or 1
        # before any GPU work: the headline workload on one thread and on all
        # cores, the 20^3 workload as whole solves, the sparse workload
        cpu = cpu_samples_obj(run_cpu_baseline_subprocess(args.cpu_iters),
                              run_cpu_baseline_subprocess(args.cpu_iters, nproc), nproc)
        cpu_c1 = cpu_c1_block()
        if not args.no_workloads and oracle_iters("sparse_20000"):
            cpu_c4 = cpu_samples_obj(run_cpu_baseline_subprocess(args.cpu_iters, 1, "sparse_20000"), None, 1)

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(dev)
    prob, u0 = synth.workload_dense_256()
    T_host = torch.from_numpy(prob.T).pin_memory()
    u0_host = torch.from_numpy(u0).pin_memory()
    P = u0.size
    ctx = cp.cp_ctx_create(local_rank, stream)
    prec = cp.CP_MIXED_BF16X3 if args.prec == "mixed" else cp.CP_FP64
    with torch.cuda.stream(stream):
        T_dev = T_host.to(dev, non_blocking=True)
        u0_dev = u0_host.to(dev, non_blocking=True)
        u = torch.empty_like(u0_dev)
    flush = L2Flush(dev)
    stream.synchronize()
    t = cp.cp_tensor_dense(ctx, T_dev)

    def opts_for(p):
        o = cp.cp_solve_opts_default(R)
        o.tol = TOL
        o.prec = p
        o.dimtree = args.dimtree
        if args.fixed_iters > 0:
            o.tol = 1e-30
            o.maxit = args.fixed_iters
            o.polish = 0
        return o

    def timed_solves(p, n_warm, n_timed, launch_count=None):
        o = opts_for(p)
        times, reps = [], []
        for k in range(n_warm + n_timed):
            if k == n_warm and launch_count is not None:
                launch_count.append(cp.cp_kernel_launches())
            flush(stream, k)
            with torch.cuda.stream(stream):
                u.copy_(u0_dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rep = cp.cp_solve(ctx, t, o, u)
            e1.record(stream)
            e1.synchronize()
            if k >= n_warm:
                times.append(e0.elapsed_time(e1) / 1e3)
                reps.append(rep)
        return times, reps

    # headline precision
    lc = []
    barrier(world)
    with ClockSampler(local_rank) as clk:
        times, reps = timed_solves(prec, args.warmup, args.steps, lc)
    launches = cp.cp_kernel_launches() - lc[0]   # the K timed solves only
    value, total_max = aggregate_replicas(times, world)
    # the other precision at the same tolerance, for the mixed-vs-FP64 figure
    other = cp.CP_FP64 if prec != cp.CP_FP64 and not args.solve_only else None
    other_obj = None
    if other is not None:
        ot, orp = timed_solves(other, 1, 1)
        other_obj = {"precision": "fp64", "solves_per_s": 1.0 / ot[0], "ms_per_solve": ot[0] * 1e3,
                     "iters": orp[0]["iters"], "gnorm_over_P": orp[0]["gnorm_over_P"], "f": orp[0]["f"]}

    # roofline of the dominant kernel (the MTTKRP), timed live on the ctx stream
    roof = None if args.solve_only else mttkrp_roofline(cp, ctx, t, u0_dev, stream, flush, prec)

    # end to end through the public API with host buffers
    e2e = None if args.solve_only else e2e_run(cp, ctx, prob, u0, prec, min(args.steps, 3), T_host)

    serving = serving_run(cp, ctx, args) if rank == 0 and not args.solve_only else None

    # the other workloads: the 20^3 plain method, the 96^4 mixed solve with
    # its errors, the sparse solve with its one-off sort (not in `value`)
    workloads = None
    if rank == 0 and not args.solve_only and not args.no_workloads:
        t.close()
        workloads = {"dense_20_fp64": c1_block(cp, ctx, stream), "dense_4way_96": c3_block(cp, ctx, stream),
                     "sparse_20000": c4_block(cp, ctx, stream)}
        workloads["dense_20_fp64"]["many_small"] = many_block(cp, ctx, stream)
        workloads["sparse_20000"]["scaled_2e8"] = sparse_scaled_block(cp, ctx, stream)
        if cpu_c1 is not None:
            workloads["dense_20_fp64"]["cpu_oracle"] = cpu_c1
        if cpu_c4 is not None:
            workloads["sparse_20000"]["cpu_oracle"] = cpu_c4
        t = None

    clocks = clk.summary()
    lat = sorted(times)
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16x3(fp32 acc)+f64" if prec != cp.CP_FP64 else "f64",
        "data": "synthetic (seeded generator; no dataset)",
        "config": {"workload": WORKLOAD, "dims": list(DIMS), "R": R, "tol": TOL, "w": 20,
                   "precision": args.prec, "l2": "flushed before every timed step: 512 MiB write, then 256 MiB read (cold, clean L2)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "latency_ms": {"p50": 1e3 * lat[len(lat) // 2], "p99": 1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))]},
        "us_per_iteration": 1e6 * sum(times) / max(1, sum(r["iters"] for r in reps)),
        "solve": {"iters": reps[-1]["iters"], "fg_evals": reps[-1]["fg_evals"],
                  "restarts": reps[-1]["restarts"], "ls_failures": reps[-1]["ls_failures"],
                  "mixed_iters": reps[-1]["mixed_iters"], "fp64_iters": reps[-1]["fp64_iters"],
                  "gnorm_over_P": reps[-1]["gnorm_over_P"], "f": reps[-1]["f"]},
        "vs_fp64_path": other_obj,
        "serving": serving,
        "workloads": workloads,
        "roofline": roof,
        "e2e": e2e,
        "clocks": clocks,
        "gpu_launches": launches,
    }
    if cpu is not None:
        res["cpu_baseline"] = cpu
    if t is not None:
        t.close()
    ctx.close()
    return res


# DRAM bytes (read + write) per launch of mttkrp_tc_kernel, mode 0 of the
# 256^3 R=16 workload, from one ncu --set full capture of the current kernel
# (dram__bytes_read.sum 67.180800 MB + dram__bytes_write.sum 0.438528 MB).
TC_NCU_TRAFFIC = 67619328


def mttkrp_roofline(cp, ctx, t, u, stream, flush, prec):
    """Dominant kernel: the MTTKRP kernel itself, timed live with CUDA events
    around each of its launches on the context stream (library kernel
    timers), L2 flushed before every call; the whole cp_mttkrp call (FP32
    factor copy, kernel, split-K reduction) is reported beside it."""
    import torch
    out = torch.empty(DIMS[0] * R, dtype=torch.float64, device=u.device)
    K = DIMS[0] * DIMS[1] * DIMS[2]
    fam = cp.TIMER_F64 if prec == cp.CP_FP64 else cp.TIMER_TC
    call = []
    for warm in (True, False):
        cp.cp_ctx_timer_enable(ctx, True)
        for n in range(3):
            for k in range(2 if warm else 5):
                flush(stream, k)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                cp.cp_mttkrp(ctx, t, R, u, n, out, prec)
                e1.record(stream)
                e1.synchronize()
                if not warm:
                    call.append(e0.elapsed_time(e1) / 1e3)
    total_ms, launches = cp.cp_ctx_timer_read(ctx, fam)
    cp.cp_ctx_timer_enable(ctx, False)
    d = total_ms / 1e3 / max(launches, 1)
    dc = sum(call) / len(call)
    peaks = measured_peaks()
    if prec == cp.CP_FP64:
        flops = 2.0 * K * R
        ach = flops / d / 1e12
        return {"kernel": "mttkrp_f64_kernel", "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS, "traffic": None,
                "per_launch": {"flops": flops, "avg_kernel_ms": d * 1e3, "launches_timed": launches,
                               "avg_cp_mttkrp_call_ms": dc * 1e3},
                "peak_source": "derived: 2 FP64 FMA/clk/SM x 152 SMs x 2070 MHz"}
    # compulsory traffic of one launch: the bf16 hi/lo planes of T_(n) (4 B
    # per element), the FP32 factor tables of the other modes and one FP32
    # I x R result (the split-K partials beyond it stay in L2)
    bytes_ = 4.0 * K + 4.0 * R * (DIMS[1] + DIMS[2]) + 4.0 * DIMS[0] * R
    ach = bytes_ / d / 1e9
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    return {"kernel": "mttkrp_tc_kernel (tcgen05 bf16x3)", "bound": "hbm", "achieved": ach, "peak": peak,
            "unit": "GB/s", "frac": ach / peak, "traffic": TC_NCU_TRAFFIC,
            "per_launch": {"bytes": bytes_, "avg_kernel_ms": d * 1e3, "launches_timed": launches,
                           "avg_cp_mttkrp_call_ms": dc * 1e3,
                           "call_achieved_GBps": bytes_ / dc / 1e9},
            "peak_source": ("MEASURED_PEAKS.json hbm_gbs (burst copy) - of measured" if peaks
                            else "fallback 6.8 TB/s - of fallback")}


def _gen_request(r):
    """One request's tensor and initial guess (worker of the generation pool)."""
    import synth
    prob, u0 = synth.request_problem(r, config=5)
    return prob.T, u0


def generate_requests(reqs, workers=16):
    """The requests' tensors, drawn by a pool of spawned processes (about
    56 ms of host work each), in request order."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(min(workers, os.cpu_count() or 1)) as pool:
        return pool.map(_gen_request, reqs, chunksize=8)


def serving_run(cp, ctx, args):
    """The serving stream (dense 3-way requests, sides U{16..192}, R U{2..32},
    collinearity {0.5, 0.9}, 1-10 % noise, tol {1e-5, 1e-7}, Poisson arrivals
    at 200/s): the first `serve_requests` requests (default: all 1024)
    replayed open-loop through the request server (p50/p99 time to
    tolerance), then the same requests all submitted at t=0 (saturation
    solves/s), with the server's default routing (requests up to
    ENGINE_MAX_WORK entries x R on the cluster engine, the rest on graph
    slots) and with graph slots only; then the first `serve_fp64_requests`
    in FP64 and in mixed precision, at saturation and one by one (the
    per-request table, cp_solve)."""
    import numpy as np
    import synth
    n = args.serve_requests
    if n <= 0:
        return None
    reqs = synth.request_stream(n, rate_per_s=200.0, config=5)
    t0 = time.perf_counter()
    probs = generate_requests(reqs)                           # generated before timing
    t_gen = time.perf_counter() - t0

    def opts(r, prec):
        o = cp.cp_solve_opts_default(r.R)
        o.tol = r.tol
        o.prec = prec
        o.dimtree = args.dimtree
        return o

    def run(prec, count, open_loop, engine=True):
        srv = cp.cp_server_create(ctx, 64 << 30, args.serve_slots)
        cp.cp_server_set_engine(srv, engine, ENGINE_MAX_WORK)
        outs = [np.zeros_like(u0) for _, u0 in probs[:count]]
        t0 = time.perf_counter()
        ids = []
        for r, (T, u0), out in zip(reqs[:count], probs[:count], outs):
            if open_loop:
                delay = r.arrival_s - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
            ids.append(cp.cp_server_submit(srv, T, opts(r, prec), u0, out))
        cp.cp_server_drain(srv, 1800.0)
        wall = time.perf_counter() - t0
        st = cp.cp_server_stats(srv)
        conv = sum(1 for i in ids if cp.cp_server_poll(srv, i)[1]["converged"])
        srv.close()
        return {"requests": count, "converged": conv, "wall_s": wall, "p50_ms": st["p50_s"] * 1e3,
                "p99_ms": st["p99_s"] * 1e3, "solves_per_s": count / wall,
                "peak_admitted_bytes": st["peak_bytes"]}

    def one_by_one(count):
        """Each request solved alone, FP64 then mixed, wall time of cp_solve
        (synchronous) after its tensor is made: [id, entries, R, fp64 ms,
        mixed ms, fp64 iterations, mixed iterations]."""
        rows = []
        for r, (T, u0) in zip(reqs[:count], probs[:count]):
            t = cp.cp_tensor_dense(ctx, T)
            row = [r.request_id, int(T.size), r.R]
            ms, its = [], []
            for prec in (cp.CP_FP64, cp.CP_MIXED_BF16X3):
                u = np.array(u0, copy=True)
                cp.cp_solve(ctx, t, opts(r, prec), u)          # warm-up (graph capture, planes)
                u = np.array(u0, copy=True)
                t1 = time.perf_counter()
                rep = cp.cp_solve(ctx, t, opts(r, prec), u)
                ms.append(1e3 * (time.perf_counter() - t1))
                its.append(rep["iters"])
            t.close()
            rows.append(row + [round(ms[0], 2), round(ms[1], 2)] + its)
        return rows

    routed = sum(1 for r in reqs if r.R * int(np.prod(r.dims)) <= ENGINE_MAX_WORK and max(r.dims) <= 256
                 and max(r.dims) * r.R <= 8192)   # (mixed requests; FP64 ones up to a 64th of it)
    res = {"stream": "Poisson 200/s, sides U{16..192}, R U{2..32}, c {0.5,0.9}, noise U(1%,10%), tol {1e-5,1e-7}",
           "slots": args.serve_slots, "generation_s": t_gen,
           "routing": {"cluster_engine_max_entries_x_R": ENGINE_MAX_WORK, "to_cluster_engine": routed,
                       "to_graph_slots": n - routed}}
    res["open_loop_mixed"] = run(cp.CP_MIXED_BF16X3, n, True)
    res["saturation_mixed"] = run(cp.CP_MIXED_BF16X3, n, False)
    res["saturation_mixed_graph_slots_only"] = run(cp.CP_MIXED_BF16X3, n, False, engine=False)
    if args.serve_fp64_requests > 0:
        m = min(n, args.serve_fp64_requests)
        res["saturation_fp64"] = run(cp.CP_FP64, m, False)
        res["saturation_mixed_same_requests"] = run(cp.CP_MIXED_BF16X3, m, False)
        rows = one_by_one(m)
        res["one_by_one"] = {"columns": ["id", "entries", "R", "fp64_ms", "mixed_ms", "fp64_iters", "mixed_iters"],
                             "rows": rows,
                             "mixed_not_slower": sum(1 for x in rows if x[4] <= x[3]),
                             "fp64_total_ms": sum(x[3] for x in rows), "mixed_total_ms": sum(x[4] for x in rows)}
    return res


# Requests up to this many entries x R go to the cluster engine (the server's
# default routing; larger ones to graph slots with tensor-core MTTKRPs).
ENGINE_MAX_WORK = 1 << 26


def e2e_run(cp, ctx, prob, u0, prec, n, T_host):
    """Solves through the public C-ABI with HOST buffers: tensor upload,
    solve with a host iterate (uploaded and read back inside the call)."""
    import numpy as np
    o = cp.cp_solve_opts_default(R)
    o.tol = TOL
    o.prec = prec
    times = []
    for k in range(n + 1):
        u = np.array(u0, copy=True)
        t0 = time.perf_counter()
        tt = cp.cp_tensor_dense(ctx, T_host.numpy())
        cp.cp_solve(ctx, tt, o, u)
        tt.close()
        dt = time.perf_counter() - t0
        if k > 0:
            times.append(dt)
    return {"value": len(times) / sum(times), "unit": UNIT,
            "h2d_bytes_per_step": int(prob.T.nbytes + u0.nbytes), "d2h_bytes_per_step": int(u0.nbytes),
            "note": "host-clock wall time per solve incl. tensor upload, per-mode copies and iterate H2D/D2H"}


# ------------------------------------------------------------ reference arm
def run_reference(args):
    """The FP64 CPU oracle on the host cores (one BLAS thread, in a child
    process), on the 256^3 workload: one solve's start-up, then warmup +
    steps N-GMRES iterations of that solve; a step is one iteration, timed
    on its own.  solves/s = 1 / the whole solve's seconds scaled from the
    timed iterations (extrapolate(): the oracle's own counts of iterations
    and f/g evaluations times the mean sweep, evaluation and rest)."""
    s = run_cpu_baseline_subprocess(args.warmup + args.steps)
    if "error" in s:
        return {"impl": "reference", "unavailable": f"oracle sample failed: {s['error']}"}
    timed = s["per_iter_s"][args.warmup:]
    mean = sum(timed) / len(timed)
    est = extrapolate(s, args.warmup)
    value = 1.0 / est["est_solve_s"] if est.get("est_solve_s") else None
    cb = cpu_baseline_obj(dict(s, **est))
    cb["sample"] = (f"one oracle solve of this workload: {args.warmup} untimed + {args.steps} timed N-GMRES "
                    f"iterations after the start-up (mean {mean:.2f} s each); " + cb["sample"])
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * mean,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded generator; no dataset)",
            "config": {"workload": WORKLOAD, "dims": list(DIMS), "R": R, "tol": TOL, "w": 20,
                       "precision": "fp64 (CPU oracle)", "step": "one N-GMRES iteration of the oracle"},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# -------------------------------------------------------------- distributed
def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x, world):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    v = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(v, op=dist.ReduceOp.MAX)
    return float(v.item())


def aggregate_replicas(times, world):
    """Whole-job solves/s over `world` independent replicas, each of which
    timed len(times) solves: every replica's total, the MAX over ranks (the
    job ends when the slowest replica does), value = world x steps / max."""
    total_max = allreduce_max(float(sum(times)), world)
    return world * len(times) / total_max, total_max


def dimtree_timing(cp, reps=5):
    """The 256^3 R=16 workload: cp_mttkrp_dimtree (W = T x_c A^(c) on the
    tensor cores, both other modes' MTTKRPs from W) against two mixed
    cp_mttkrp calls for the same modes; CUDA events around each call, the
    tensor-core kernel timed alone by the library timers, L2 flushed before."""
    import torch
    import synth
    prob, u0 = synth.workload_dense_256()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    ctx = cp.cp_ctx_create(0, stream)
    with torch.cuda.stream(stream):
        T = torch.from_numpy(prob.T).to(dev)
        u = torch.from_numpy(u0).to(dev)
    flush = L2Flush(dev)
    stream.synchronize()
    t = cp.cp_tensor_dense(ctx, T)
    out = torch.empty(2 * 256 * 16, dtype=torch.float64, device=dev)
    res = {}
    for c in (0, 2):
        modes = [m for m in range(3) if m != c]
        for name, fn in (("dimtree", lambda: cp.cp_mttkrp_dimtree(ctx, t, 16, u, c, out)),
                         ("two_mttkrps", lambda: [cp.cp_mttkrp(ctx, t, 16, u, m, out[k * 4096:(k + 1) * 4096],
                                                                cp.CP_MIXED_BF16X3) for k, m in enumerate(modes)])):
            call = []
            for k in range(reps + 1):
                if k == 1:
                    cp.cp_ctx_timer_enable(ctx, True)
                flush(stream, k)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                e1.synchronize()
                if k > 0:
                    call.append(e0.elapsed_time(e1) * 1e3)
            tc_ms, launches = cp.cp_ctx_timer_read(ctx, cp.TIMER_TC)
            cp.cp_ctx_timer_enable(ctx, False)
            res[f"c{c}_{name}"] = {"call_us": sum(call) / len(call), "tc_kernel_us_total": 1e3 * tc_ms / reps,
                                   "tc_launches_per_call": launches / reps}
    return res


def run_precision_table(args):
    """Each of the first N requests of the serving stream solved alone, FP64
    and mixed (FP64-polished), from the same start, CUDA-event timed after one
    warm-up solve of each: the size at which mixed precision starts to pay."""
    import torch
    import synth
    import paper_1105_5331_gb300 as cp
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    ctx = cp.cp_ctx_create(0, stream)
    reqs = synth.request_stream(args.precision_table, rate_per_s=200.0, config=5)
    rows = []
    for r in reqs:
        prob, u0 = synth.request_problem(r, config=5)
        with torch.cuda.stream(stream):
            T = torch.from_numpy(prob.T).to(dev)
            u0d = torch.from_numpy(u0).to(dev)
        stream.synchronize()
        t = cp.cp_tensor_dense(ctx, T)
        row = {"id": r.request_id, "dims": list(r.dims), "R": r.R, "tol": r.tol, "entries": int(T.numel())}
        for name, prec in (("fp64", cp.CP_FP64), ("mixed", cp.CP_MIXED_BF16X3)):
            if args.table_mixed_only and prec == cp.CP_FP64:
                continue
            o = cp.cp_solve_opts_default(r.R)
            o.tol = r.tol
            o.prec = prec
            o.mixed_stall = args.mixed_stall
            o.dimtree = args.dimtree
            for k in range(2):
                with torch.cuda.stream(stream):
                    u = u0d.clone()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                rep = cp.cp_solve(ctx, t, o, u)
                e1.record(stream)
                e1.synchronize()
            row[name] = {"ms": e0.elapsed_time(e1), "iters": rep["iters"], "converged": rep["converged"]}
        t.close()
        rows.append(row)
        print(json.dumps(row), flush=True)
    ctx.close()


def run_many_only(args):
    """The cluster engine on one fixed case (profiling driver): `many-count`
    requests of a cubic tensor of side `many-shape`, planted rank
    `many-rank`, c=0.5, 5 % noise, exactly `many-iters` iterations each in
    `many-prec`, clusters of `many-cluster` CTAs; `reps` cp_solve_many calls
    from the same start; prints the wall time of each and the best call's
    time per iteration."""
    import numpy as np
    import torch
    import synth
    import paper_1105_5331_gb300 as cp
    S, R, n = args.many_shape, args.many_rank, args.many_count
    ctx = cp.cp_ctx_create(0, torch.cuda.current_stream())
    ts, u0s, opts = [], [], []
    for k in range(n):
        rng = synth.rng_for(33, k)
        prob = synth.dense_problem(rng, (S, S, S), R, 0.5, eta=0.05, dtype=np.float32)
        ts.append(cp.cp_tensor_dense(ctx, prob.T))
        u0s.append(synth.initial_guess(rng, prob.dims, R))
        o = cp.cp_solve_opts_default(R)
        o.prec = cp.CP_MIXED_BF16X3 if args.many_prec == "mixed" else cp.CP_FP64
        o.tol = 1e-300
        o.maxit = args.many_iters
        opts.append(o)
    walls, iters = [], 0
    for _ in range(max(1, args.reps)):
        us = [u.copy() for u in u0s]
        t0 = time.perf_counter()
        reps = cp.cp_solve_many(ctx, ts, opts, us, cluster=args.many_cluster)
        walls.append(time.perf_counter() - t0)
        iters = max(r["iters"] for r in reps)
    print(json.dumps({"many_only": f"{n} x {S}^3 R={R} {args.many_prec}, {args.many_iters} iterations, "
                                   f"clusters of {args.many_cluster}",
                      "wall_s": walls, "iters": iters, "us_per_iter_best": min(walls) / max(iters, 1) * 1e6}))
    for t in ts:
        t.close()
    ctx.close()


def run_mttkrp_only(args):
    """cp_mttkrp on every mode of a workload, `reps` launches per mode with an
    L2 flush before each; prints per-mode average times (profiling driver)."""
    import torch

    import synth
    import paper_1105_5331_gb300 as cp
    if args.mttkrp_only == "dimtree_256":
        print(json.dumps({"mttkrp_only": "dimtree_256", **dimtree_timing(cp)}))
        return
    if args.mttkrp_only == "sparse_scaled":
        dev = torch.device("cuda", 0)
        stream = torch.cuda.Stream(dev)
        ctx = cp.cp_ctx_create(0, stream)
        print(json.dumps({"mttkrp_only": "sparse_scaled", **sparse_scaled_block(cp, ctx, stream)}))
        return
    sparse = args.mttkrp_only == "sparse"
    if args.mttkrp_only == "dense_256":
        prob, u0 = synth.workload_dense_256()
    elif args.mttkrp_only == "dense_4way":
        prob, u0 = synth.workload_dense_4way()
    else:
        prob, u0 = synth.workload_sparse()
    Rk = prob.R
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    ctx = cp.cp_ctx_create(0, stream)
    prec = cp.CP_MIXED_BF16X3 if args.prec == "mixed" else cp.CP_FP64
    with torch.cuda.stream(stream):
        u = torch.from_numpy(u0).to(dev)
        if sparse:
            coords = torch.from_numpy(prob.coords).to(dev)
            vals = torch.from_numpy(prob.vals).to(dev)
        else:
            T = torch.from_numpy(prob.T).to(dev)
    flush = L2Flush(dev)
    stream.synchronize()
    t = cp.cp_tensor_coo(ctx, prob.dims, coords, vals) if sparse else cp.cp_tensor_dense(ctx, T)
    res = {}
    fam = cp.TIMER_COO if sparse else (cp.TIMER_TC if prec == cp.CP_MIXED_BF16X3 else cp.TIMER_F64)
    for n in range(len(prob.dims)):
        out = torch.empty(prob.dims[n] * Rk, dtype=torch.float64, device=dev)
        ms = []
        for k in range(args.reps + 1):
            if k == 1:
                cp.cp_ctx_timer_enable(ctx, True)
            flush(stream, k)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            cp.cp_mttkrp(ctx, t, Rk, u, n, out, prec)
            e1.record(stream)
            e1.synchronize()
            if k > 0:
                ms.append(e0.elapsed_time(e1))
        kms, kl = cp.cp_ctx_timer_read(ctx, fam)
        cp.cp_ctx_timer_enable(ctx, False)
        res[f"mode{n}_ms"] = sum(ms) / len(ms)
        res[f"mode{n}_kernel_ms"] = kms / max(kl, 1)
        if not sparse and prec == cp.CP_MIXED_BF16X3:
            K = 1
            for d in prob.dims:
                K *= d
            res[f"mode{n}_kernel_GBps"] = 4.0 * K / (res[f"mode{n}_kernel_ms"] / 1e3) / 1e9
        if sparse:
            nnz = prob.coords.shape[0]
            sf = 4 if args.prec == "mixed" else 8
            comp = nnz * (4 + 4 * (len(prob.dims) - 1))          # values + other coordinates
            access = comp + nnz * (len(prob.dims) - 1) * Rk * sf   # + gathered factor rows
            res[f"mode{n}_compulsory_GBps"] = comp / (res[f"mode{n}_ms"] / 1e3) / 1e9
            res[f"mode{n}_access_GBps"] = access / (res[f"mode{n}_ms"] / 1e3) / 1e9
    cp.cp_ctx_sync(ctx)
    print(json.dumps({"mttkrp_only": args.mttkrp_only, "prec": args.prec, **res}))


def match_factors(prob, um, uf):
    """Rank-one terms of two solutions matched greedily by congruence (the
    product over modes of |cos| of the columns); per mode the relative error
    of the first against the second, column signs matched."""
    import numpy as np
    Rk = prob.R
    As, Bs, off = [], [], 0
    for n in prob.dims:
        As.append(um[off:off + n * Rk].reshape(n, Rk))
        Bs.append(uf[off:off + n * Rk].reshape(n, Rk))
        off += n * Rk
    C = np.ones((Rk, Rk))
    for A, Bf in zip(As, Bs):
        C *= np.abs((A / np.linalg.norm(A, axis=0)).T @ (Bf / np.linalg.norm(Bf, axis=0)))
    perm, used = [-1] * Rk, set()
    for idx in np.argsort(-C, axis=None):
        r, q = divmod(int(idx), Rk)
        if perm[r] < 0 and q not in used:
            perm[r] = q
            used.add(q)
    errs = []
    for A, Bf in zip(As, Bs):
        Bp = Bf[:, perm]
        sg = np.sign(np.sum(A * Bp, axis=0))
        sg[sg == 0] = 1.0
        errs.append(float(np.linalg.norm(A - Bp * sg) / np.linalg.norm(Bf)))
    return errs, perm


def mixed_vs_fp64(cp, ctx, t, prob, u0, stream, timed=1):
    """The mixed-precision solve (bf16x3 MTTKRP, FP64 polish) and the FP64
    solve of one dense workload from the same start, CUDA-event timed; at the
    mixed solution, f and grad f of the mixed evaluation against the FP64
    one; the mixed solution's factors against the FP64 solution's."""
    import numpy as np
    import torch
    Rk = prob.R
    dev = torch.device("cuda", torch.cuda.current_device())
    out = {"dims": list(prob.dims), "R": Rk, "tol": TOL}
    sols = {}
    with torch.cuda.stream(stream):
        u0d = torch.from_numpy(u0).to(dev)
    for name, prec in (("mixed", cp.CP_MIXED_BF16X3), ("fp64", cp.CP_FP64)):
        o = cp.cp_solve_opts_default(Rk)
        o.tol = TOL
        o.prec = prec
        times = []
        for k in range(1 + timed):
            with torch.cuda.stream(stream):
                u = u0d.clone()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = cp.cp_solve(ctx, t, o, u)
            e1.record(stream)
            e1.synchronize()
            if k > 0 or timed == 0:
                times.append(e0.elapsed_time(e1) / 1e3)
        sols[name] = u
        out[name] = {"solves_per_s": len(times) / sum(times), "ms_per_solve": 1e3 * sum(times) / len(times),
                     "iters": r["iters"], "mixed_iters": r["mixed_iters"], "fp64_iters": r["fp64_iters"],
                     "converged": r["converged"], "f": r["f"], "gnorm_over_P": r["gnorm_over_P"]}
    um = sols["mixed"]
    P = um.numel()
    ev = {}
    for name, prec in (("mixed", cp.CP_MIXED_BF16X3), ("fp64", cp.CP_FP64)):
        f = torch.zeros(1, dtype=torch.float64, device=dev)
        g = torch.empty(P, dtype=torch.float64, device=dev)
        cp.cp_fg(ctx, t, Rk, um, f, g, prec)
        cp.cp_ctx_sync(ctx)
        ev[name] = (f.item(), g.cpu().numpy())
    f64, g64 = ev["fp64"]
    fm, gm = ev["mixed"]
    out["at_mixed_solution"] = {"f_fp64": f64, "f_mixed_rel_err": abs(fm - f64) / abs(f64),
                                "g_fp64_over_P": float(np.linalg.norm(g64)) / P,
                                "g_mixed_err_over_P": float(np.linalg.norm(gm - g64)) / P}
    errs, perm = match_factors(prob, um.cpu().numpy(), sols["fp64"].cpu().numpy())
    out["factors_rel_err_vs_fp64_solve"] = errs
    out["f_rel_diff_vs_fp64_solve"] = abs(out["mixed"]["f"] - out["fp64"]["f"]) / abs(out["fp64"]["f"])
    out["note"] = ("errors against the FP64 GPU path, which matches the FP64 oracle within 1e-10 per call "
                   "(tests/test_gpu_dense.py, tests/test_gpu_trajectories.py)")
    return out, sols


def run_accuracy_report(args):
    """mixed_vs_fp64 on one workload, one JSON line."""
    import torch

    import synth
    import paper_1105_5331_gb300 as cp
    prob, u0 = synth.workload_dense_4way() if args.accuracy_report == "dense_4way" else synth.workload_dense_256()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    ctx = cp.cp_ctx_create(0, stream)
    with torch.cuda.stream(stream):
        T = torch.from_numpy(prob.T).to(dev)
    stream.synchronize()
    t = cp.cp_tensor_dense(ctx, T)
    out, _ = mixed_vs_fp64(cp, ctx, t, prob, u0, stream, timed=0)
    out["accuracy_report"] = args.accuracy_report
    print(json.dumps(out))


def c1_block(cp, ctx, stream, n_solves=30):
    """The 20x20x20 R=3 workload (the paper's plain method, FP64): whole GPU
    solves to ||g||/P < 1e-7, CUDA-event timed, and the oracle's whole solves
    on the host cores."""
    import torch
    import synth
    prob, u0 = synth.workload_dense_small()
    dev = torch.device("cuda", torch.cuda.current_device())
    with torch.cuda.stream(stream):
        T = torch.from_numpy(prob.T).to(dev)
        u0d = torch.from_numpy(u0).to(dev)
    stream.synchronize()
    t = cp.cp_tensor_dense(ctx, T)
    o = cp.cp_solve_opts_default(3)
    o.tol = TOL
    times = []
    for k in range(3 + n_solves):
        with torch.cuda.stream(stream):
            u = u0d.clone()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = cp.cp_solve(ctx, t, o, u)
        e1.record(stream)
        e1.synchronize()
        if k >= 3:
            times.append(e0.elapsed_time(e1) / 1e3)
    t.close()
    lat = sorted(times)
    return {"workload": "dense 20x20x20 fp64, planted R=3, c=0.5, 10% noise; N-GMRES w=20, R=3, fp64, "
                        "stop ||g||/P < 1e-7",
            "solves_per_s": len(times) / sum(times), "p50_ms": 1e3 * lat[len(lat) // 2],
            "p99_ms": 1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))], "solves_timed": len(times),
            "iters": r["iters"], "converged": r["converged"]}


def many_block(cp, ctx, stream, n=1024, n_single=30):
    """Many small decompositions in one persistent launch: n independent
    problems shaped like the 20x20x20 workload (FP64, R=3, c=0.5, 10 % noise,
    seeds 1000..1000+n-1), each solved to ||g||/P < 1e-7, by cp_solve_many
    (every thread-block cluster runs one problem's whole solve at a time) and
    by cp_solve_batch (one CUDA graph per problem, each on its own stream);
    wall clock of the call, tensors resident, initial guesses and solutions
    on the device.  Also the 20^3 workload itself solved alone through
    cp_solve_many (CUDA-event timed)."""
    import numpy as np
    import torch
    import synth
    dev = torch.device("cuda", torch.cuda.current_device())
    ts, u0s, opts = [], [], []
    for k in range(n):
        rng = synth.rng_for(1, 1000 + k)
        prob = synth.dense_problem(rng, (20, 20, 20), 3, 0.5, eta=0.10, dtype=np.float64)
        with torch.cuda.stream(stream):
            ts.append(cp.cp_tensor_dense(ctx, torch.from_numpy(prob.T).to(dev)))
            u0s.append(torch.from_numpy(synth.initial_guess(rng, prob.dims, 3)).to(dev))
        o = cp.cp_solve_opts_default(3)
        o.tol = TOL
        o.prec = cp.CP_FP64
        opts.append(o)
    stream.synchronize()
    out = {"workload": f"{n} independent dense 20x20x20 fp64 problems (planted R=3, c=0.5, 10% noise), "
                       "N-GMRES w=20, R=3, stop ||g||/P < 1e-7"}
    for name, fn in (("cp_solve_many", lambda us: cp.cp_solve_many(ctx, ts, opts, us)),
                     ("cp_solve_batch", lambda us: cp.cp_solve_batch(ctx, ts, opts, us))):
        for rep in range(2):   # the first call tunes / captures
            us = [u.clone() for u in u0s]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            reps = fn(us)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
        out[name] = {"solves_per_s": n / dt, "wall_s": dt, "converged": sum(r["converged"] for r in reps),
                     "iters_total": sum(r["iters"] for r in reps)}
    out["speedup_many_vs_batch"] = out["cp_solve_many"]["solves_per_s"] / out["cp_solve_batch"]["solves_per_s"]
    # the 20^3 workload alone through the engine
    prob, u0 = synth.workload_dense_small()
    with torch.cuda.stream(stream):
        T = torch.from_numpy(prob.T).to(dev)
        u0d = torch.from_numpy(u0).to(dev)
    stream.synchronize()
    t = cp.cp_tensor_dense(ctx, T)
    o = cp.cp_solve_opts_default(3)
    o.tol = TOL
    o.prec = cp.CP_FP64
    times = []
    for k in range(3 + n_single):
        u = u0d.clone()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        (r,) = cp.cp_solve_many(ctx, [t], [o], [u])
        e1.record(stream)
        e1.synchronize()
        if k >= 3:
            times.append(e0.elapsed_time(e1) / 1e3)
    t.close()
    for x in ts:
        x.close()
    lat = sorted(times)
    out["dense_20_alone"] = {"solves_per_s": len(times) / sum(times), "p50_ms": 1e3 * lat[len(lat) // 2],
                             "iters": r["iters"], "converged": r["converged"]}
    return out


def c3_block(cp, ctx, stream):
    """The 96^4 R=32 workload: mixed (FP64-polished) and FP64 solves, and the
    errors of f, grad f and the factors of the mixed solution."""
    import synth
    import torch
    prob, u0 = synth.workload_dense_4way()
    dev = torch.device("cuda", torch.cuda.current_device())
    with torch.cuda.stream(stream):
        T = torch.from_numpy(prob.T).to(dev)
    stream.synchronize()
    t = cp.cp_tensor_dense(ctx, T)
    del T
    out, _ = mixed_vs_fp64(cp, ctx, t, prob, u0, stream, timed=1)
    out["workload"] = "dense 96x96x96x96 fp32, planted R=32, c=0.5, 5% noise; N-GMRES w=20, R=32, stop ||g||/P < 1e-7"
    t.close()
    return out


def sparse_scaled_on_device(I, nnz, R=10, seed=11055731):
    """A scaled version of the sparse workload, drawn on the GPU (a host draw
    of 2e8 distinct coordinates takes minutes): I x I x I, uniform int64
    coordinates made distinct through their linear index (sorted by it), a
    planted rank-R model with U(0,1) factors evaluated there plus 1 % noise,
    FP32 values.  Returns device coords (nnz' x 3), values, nnz' (nnz' may
    fall a few short of nnz when draws collide)."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    key = torch.randint(0, I * I * I, (nnz,), generator=g, device="cuda", dtype=torch.int64)
    key = torch.unique(key)
    coords = torch.stack([key // (I * I), (key // I) % I, key % I], dim=1).contiguous()
    del key
    m = torch.ones(coords.shape[0], R, dtype=torch.float64, device="cuda")
    for n in range(3):
        A = torch.rand(I, R, generator=g, dtype=torch.float64, device="cuda")
        m *= A[coords[:, n]]
    m = m.sum(dim=1)
    noise = torch.randn(coords.shape[0], generator=g, dtype=torch.float64, device="cuda")
    vals = (m + 0.01 * torch.linalg.vector_norm(m) * noise / torch.linalg.vector_norm(noise)).to(torch.float32)
    return coords, vals.contiguous(), int(coords.shape[0])


def sparse_scaled_block(cp, ctx, stream, variants=((2_000_000, 200_000_000), (500_000, 200_000_000))):
    """The sparse MTTKRP at 2e8 nonzeros (kernel timers, every mode, FP32
    products and FP64): I = 2e6 as planned (the two gathered FP32 factor
    tables, 2 x 128 MB, exceed the 129 MB L2), and I = 5e5 (2 x 32 MB, L2
    resident), with the one-off sort and segmentation."""
    import torch
    res = {}
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    Rk = 10
    for I, want in variants:
        coords, vals, nnz = sparse_scaled_on_device(I, want, Rk)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t = cp.cp_tensor_coo(ctx, (I, I, I), coords, vals)
        cp.cp_ctx_sync(ctx)
        build_s = time.perf_counter() - t0
        del coords, vals
        u = torch.rand(3 * I * Rk, dtype=torch.float64, device="cuda")
        out = torch.empty(I * Rk, dtype=torch.float64, device="cuda")
        blk = {"I": I, "nnz": nnz, "sort_and_segment_s": build_s}
        for pname, prec, sf in (("fp32_products", cp.CP_MIXED_BF16X3, 4), ("fp64", cp.CP_FP64, 8)):
            cp.cp_mttkrp(ctx, t, Rk, u, 0, out, prec)
            cp.cp_ctx_timer_enable(ctx, True)
            for n in range(3):
                for _ in range(2):
                    cp.cp_mttkrp(ctx, t, Rk, u, n, out, prec)
            ms, launches = cp.cp_ctx_timer_read(ctx, cp.TIMER_COO)
            cp.cp_ctx_timer_enable(ctx, False)
            d = ms / 1e3 / max(launches, 1)
            comp = nnz * 12
            access = comp + nnz * 2 * Rk * sf
            blk[pname] = {"avg_kernel_ms": 1e3 * d, "compulsory_GBps": comp / d / 1e9,
                          "compulsory_frac_of_hbm": comp / d / 1e9 / peak, "access_GBps": access / d / 1e9,
                          "access_frac_of_hbm": access / d / 1e9 / peak, "launches_timed": launches}
        t.close()
        del u, out
        torch.cuda.empty_cache()
        res[f"I{I}"] = blk
    res["bytes"] = ("compulsory = 12 B per nonzero (FP32 value + two int32 coordinates); access = compulsory + "
                    "the two gathered factor rows (R x 4 B FP32 / R x 8 B FP64 each)")
    return res


def c4_block(cp, ctx, stream, maxit=3000):
    """The sparse 20000^3 workload (2e6 nonzeros, planted rank 10 + 1 %
    noise, R=10, w=20): the one-off sort and segmentation, the sparse MTTKRP
    of every mode (kernel timers; compulsory and access bytes), and FP64 and
    FP32-product solves."""
    import torch
    import synth
    prob, u0 = synth.workload_sparse()
    Rk = prob.R
    dev = torch.device("cuda", torch.cuda.current_device())
    with torch.cuda.stream(stream):
        coords = torch.from_numpy(prob.coords).to(dev)
        vals = torch.from_numpy(prob.vals).to(dev)
        u0d = torch.from_numpy(u0).to(dev)
    stream.synchronize()
    build = []
    for k in range(2):
        t0 = time.perf_counter()
        t = cp.cp_tensor_coo(ctx, prob.dims, coords, vals)
        cp.cp_ctx_sync(ctx)
        build.append(time.perf_counter() - t0)
        if k == 0:
            t.close()
    nnz = prob.coords.shape[0]
    N = len(prob.dims)
    res = {"workload": "sparse 20000^3 COO, 2e6 distinct uniform nonzeros, planted rank-10 U(0,1) + 1% noise, "
                       "fp32 values; N-GMRES w=20, R=10, stop ||g||/P < 1e-7",
           "nnz": nnz, "sort_and_segment_s": build[-1],
           "sort_note": "cp_tensor_coo on device arrays, synchronised: validation, per-mode stable sort, "
                        "segmentation, work units (second call; the first is warm-up)"}
    out = torch.empty(max(prob.dims) * Rk, dtype=torch.float64, device=dev)
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    for pname, prec, sf in (("fp64", cp.CP_FP64, 8), ("fp32_products", cp.CP_MIXED_BF16X3, 4)):
        cp.cp_ctx_timer_enable(ctx, True)
        for n in range(N):
            for _ in range(5):
                cp.cp_mttkrp(ctx, t, Rk, u0d, n, out, prec)
        ms, launches = cp.cp_ctx_timer_read(ctx, cp.TIMER_COO)
        cp.cp_ctx_timer_enable(ctx, False)
        d = ms / 1e3 / max(launches, 1)
        comp = nnz * (4 + 4 * (N - 1))
        access = comp + nnz * (N - 1) * Rk * sf
        res[f"mttkrp_{pname}"] = {"avg_kernel_us": 1e6 * d, "compulsory_GBps": comp / d / 1e9,
                                  "access_GBps": access / d / 1e9, "compulsory_frac_of_hbm": comp / d / 1e9 / peak,
                                  "launches_timed": launches}
    for pname, prec in (("fp64", cp.CP_FP64), ("fp32_products", cp.CP_MIXED_BF16X3)):
        o = cp.cp_solve_opts_default(Rk)
        o.tol = TOL
        o.prec = prec
        o.maxit = maxit
        with torch.cuda.stream(stream):
            u = u0d.clone()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = cp.cp_solve(ctx, t, o, u)
        e1.record(stream)
        e1.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        res[f"solve_{pname}"] = {"solves_per_s": 1.0 / sec, "ms_per_solve": 1e3 * sec, "iters": r["iters"],
                                 "converged": r["converged"], "f": r["f"], "gnorm_over_P": r["gnorm_over_P"],
                                 "maxit": maxit}
    t.close()
    return res


def run_small_kernels(args):
    """Three rounds of cp_fg, cp_als_sweep (normalising), ngmres_step (window
    of 20) and linesearch on the 256^3 R=16 workload, outside any graph."""
    import numpy as np
    import torch

    import synth
    import paper_1105_5331_gb300 as cp
    prec = cp.CP_MIXED_BF16X3 if args.prec == "mixed" else cp.CP_FP64
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    prob, u0 = synth.workload_dense_256()
    ctx = cp.cp_ctx_create(0, stream)
    rng = np.random.default_rng(5)
    P = u0.size
    with torch.cuda.stream(stream):
        T = torch.from_numpy(prob.T).to(dev)
        u = torch.from_numpy(u0).to(dev)
        U = torch.from_numpy(rng.standard_normal((20, P))).to(dev)
        G = torch.from_numpy(rng.standard_normal((20, P))).to(dev)
        ub = torch.from_numpy(rng.standard_normal(P)).to(dev)
        gb = torch.from_numpy(rng.standard_normal(P)).to(dev)
        uh = torch.empty(P, dtype=torch.float64, device=dev)
        f = torch.zeros(1, dtype=torch.float64, device=dev)
        g = torch.empty(P, dtype=torch.float64, device=dev)
        x = torch.empty_like(g)
        gx = torch.empty_like(g)
    stream.synchronize()
    t = cp.cp_tensor_dense(ctx, T)
    for _ in range(3):
        cp.cp_fg(ctx, t, R, u, f, g, prec)
        w = u.clone()
        cp.cp_als_sweep(ctx, t, R, w, True, prec)
        cp.ngmres_step(ctx, U, G, ub, gb, 1e-12, uh)
        cp.cp_fg(ctx, t, R, w, f, g, prec)
        cp.cp_ctx_sync(ctx)
        d = w - u
        fu = torch.zeros(1, dtype=torch.float64, device=dev)
        gu = torch.empty_like(g)
        cp.cp_fg(ctx, t, R, u, fu, gu, prec)
        cp.cp_ctx_sync(ctx)
        if float((gu * d).sum()) < 0:
            cp.linesearch(ctx, t, R, u, float(fu.item()), gu, d, x, gx, prec=prec)
    cp.cp_ctx_sync(ctx)
    print(json.dumps({"small_kernels": "done"}))


def run_kernel_breakdown(args):
    """One warm headline solve, then one under torch.profiler (CUPTI activity
    records, which include kernels launched by CUDA graphs and their
    conditional bodies).  Prints per-kernel launches, total device time and
    the time during which each kernel ran alone or shared the GPU."""
    import collections

    import torch
    from torch.profiler import ProfilerActivity, profile

    import synth
    import paper_1105_5331_gb300 as cp
    prec = cp.CP_MIXED_BF16X3 if args.prec == "mixed" else cp.CP_FP64
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    prob, u0 = synth.workload_dense_256()
    ctx = cp.cp_ctx_create(0, stream)
    with torch.cuda.stream(stream):
        T = torch.from_numpy(prob.T).to(dev)
        u0d = torch.from_numpy(u0).to(dev)
        u = torch.empty_like(u0d)
    stream.synchronize()
    t = cp.cp_tensor_dense(ctx, T)
    o = cp.cp_solve_opts_default(R)
    o.tol = TOL
    o.prec = prec

    def solve():
        with torch.cuda.stream(stream):
            u.copy_(u0d)
        stream.synchronize()
        return cp.cp_solve(ctx, t, o, u)

    solve()
    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        rep = solve()
        stream.synchronize()
    kern = [e for e in prof.events() if e.device_type == torch.autograd.DeviceType.CUDA
            and "memcpy" not in e.name.lower() and "memset" not in e.name.lower()]

    def short(name):
        return name.replace("(anonymous namespace)::", "").split("(")[0].replace("cpg::", "").replace("void ", "")

    agg = collections.defaultdict(lambda: [0, 0.0])
    for e in kern:
        a = agg[short(e.name)]
        a[0] += 1
        a[1] += e.time_range.end - e.time_range.start
    ev = sorted([(e.time_range.start, 1, short(e.name)) for e in kern] + [(e.time_range.end, -1, short(e.name)) for e in kern])
    active = collections.Counter()
    alone = collections.defaultdict(float)
    shared = collections.defaultdict(float)
    last = ev[0][0]
    for ts, kind, nm in ev:
        dt = ts - last
        names = [k for k, v in active.items() if v]
        if len(names) == 1:
            alone[names[0]] += dt
        elif len(names) > 1:
            for k in names:
                shared[k] += dt / len(names)
        active[nm] += kind
        last = ts
    tot = sum(v[1] for v in agg.values())
    print(json.dumps({"kernel_breakdown": "mixed" if prec != cp.CP_FP64 else "fp64", "iters": rep["iters"],
                      "fg_evals": rep["fg_evals"], "launches": len(kern), "device_time_ms": tot / 1e3}))
    print(f"{'kernel':34s} {'launches':>9s} {'total ms':>9s} {'share':>6s} {'avg us':>8s} {'alone ms':>9s} {'shared ms':>9s}")
    for k, (c, tt) in sorted(agg.items(), key=lambda x: -x[1][1]):
        print(f"{k:34s} {c:9d} {tt / 1e3:9.3f} {100 * tt / tot:5.1f}% {tt / c:8.2f} {alone[k] / 1e3:9.3f} {shared[k] / 1e3:9.3f}")


def main():
    args = parse()
    if args.cpu_sample:
        print(json.dumps(cpu_sample(args.cpu_iters, args.cpu_workload)))
        return
    if args.cpu_c1:
        print(json.dumps(cpu_solves_c1(args.cpu_iters)))
        return
    if args.kernel_breakdown:
        run_kernel_breakdown(args)
        return
    if args.accuracy_report:
        run_accuracy_report(args)
        return
    if args.small_kernels:
        run_small_kernels(args)
        return
    if args.mttkrp_only:
        run_mttkrp_only(args)
        return
    if args.many_only:
        run_many_only(args)
        return
    if args.precision_table:
        run_precision_table(args)
        return
    if args.serve_only:
        import torch
        import paper_1105_5331_gb300 as cp
        stream = torch.cuda.Stream(torch.device("cuda", 0))
        ctx = cp.cp_ctx_create(0, stream)
        print(json.dumps({"serve_only": True, "dimtree": args.dimtree, **serving_run(cp, ctx, args)}))
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)))
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    res = run_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
