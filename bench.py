#!/usr/bin/env python
"""Benchmark of the LocalPower hot path on GB300.

One "step" is one complete LocalPower solve of the FP32 workload (n = 1,000,000
rows, d = 1,024, k = 16, m = 64 row partitions, p decaying 8 -> 4 -> 2 -> 1 over
10 rounds each and then 10 more rounds at p = 1, sign-fixing, then a
Rayleigh-Ritz pass): 50 aggregations, 160 local power steps and one Ritz pass,
each pass streaming all of A (4.1 GB) from HBM, ending below distance 1e-4 to
the top-16 subspace.  The headline runs the FP32 data as hi/lo BF16 planes on
the tensor cores (FP32-level results); the plain FP32 (SIMT) path and a BF16
copy are timed beside it.  The metric is algorithmic GB/s of A streamed;
solves/s, per-solve latency percentiles and the accuracy ride along.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank solves its own replica of the workload (the
solves are independent problems: weak scaling, no data-path collective); the
elapsed time is the maximum over ranks.  ``--impl reference`` times the FP64
CPU oracle on a bounded sample of the same workload.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LocalPower GB/s & solves/s at dist≤1e-4 vs plain FP32 path; p50/p99 latency"
WORKLOAD = "fp32"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--agg", choices=["sign", "opt"], default="sign")
    ap.add_argument("--e2e-steps", type=int, default=4)
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-bf16", action="store_true", help="skip the BF16-storage (tensor-core) run of the workload")
    ap.add_argument("--requests", type=int, default=2000, help="serving: number of requests")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: Poisson arrival rate (requests/s)")
    ap.add_argument("--shape", default="1024x16", help="kernels: d x k of the step-kernel comparison")
    ap.add_argument("--autotune", action="store_true",
                    help="kernels workload: let the autotuner pick the tensor-core step's tuning first")
    ap.add_argument("--instances", type=int, default=256, help="batching: number of instances")
    ap.add_argument("--workload", choices=["fp32", "lowprec", "plain", "serving", "kernels", "batching", "rounds"],
                    default="fp32",
                    help="fp32: the FP32 workload (default, with its BF16-storage and split-plane runs alongside); "
                         "lowprec: the reduced-precision workload n=4e6, d=2048, k=32 (BF16, then FP8-E4M3); "
                         "plain: the small plain configuration n=4000, d=100, k=5 (latency-bound); "
                         "serving: a Poisson stream of BF16 truncated-SVD requests through the request server; "
                         "kernels: every step kernel on one shape (--shape, --rows), one-step solves, for profiling; "
                         "batching: independent BF16 instances of mixed shapes solved by one graph launch; "
                         "rounds: rounds-to-accuracy and the residual error rho_t for constant p in {1, 2, 4, 8}")
    ap.add_argument("--profile-solve", action="store_true",
                    help="batching: after the timed solves, one more batch solve between cudaProfilerStart and "
                         "cudaProfilerStop (for ncu --profile-from-start off); not timed")
    ap.add_argument("--rows", type=int, default=None,
                    help="override n (same spectrum and partition count): a smaller case for profiler captures")
    return ap.parse_args()


def _dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


class Clocks:
    """nvidia-smi samples (200 ms) while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# host seconds spent generating synthetic inputs (outside every timed region),
# reported beside the results as data_generation_s
_DATA_GEN_S = [0.0]


def _emit(line: dict) -> None:
    print(json.dumps(dict(line, data_generation_s=_DATA_GEN_S[0])))


def _workload(rank: int, rows: int | None = None, name: str = WORKLOAD):
    import synth
    t = time.perf_counter()
    c = dict(synth.CONFIGS[name])
    if rows:
        c["n"] = int(rows)
    A, sizes, Y0 = synth.make_config_data(name, n=c["n"])
    _DATA_GEN_S[0] += time.perf_counter() - t
    return c, A, sizes, Y0, synth.config_schedule(name)


def _oracle_sample_gbps(parts, Y0, passes: int):
    """The FP64 oracle's local power step (eq. (2)) over every partition, `passes` times."""
    import oracle
    Z = oracle.orth(Y0)
    nbytes = sum(p.nbytes for p in parts)
    t = time.perf_counter()
    for _ in range(passes):
        for P in parts:
            oracle.local_step(P, Z)
    dt = time.perf_counter() - t
    return passes * nbytes / dt / 1e9, dt


def run_reference(args):
    rank, world, _ = _dist_env()
    if rank != 0:
        return
    import synth
    c, A, sizes, Y0, sched = _workload(0, args.rows)
    parts = synth.split_rows(A, sizes)
    sample = parts[:16]
    for _ in range(args.warmup):
        _oracle_sample_gbps(sample, Y0, 1)
    t = time.perf_counter()
    vals = [_oracle_sample_gbps(sample, Y0, 1)[0] for _ in range(args.steps)]
    dt = time.perf_counter() - t
    bytes_step = sum(p.nbytes for p in sample)
    value = args.steps * bytes_step / dt / 1e9
    cores = os.cpu_count()
    sample_txt = (f"each step: one FP64 oracle local power step (eq. (2)) over 16 of the 64 partitions "
                  f"({bytes_step / 1e9:.2f} GB of FP32 A)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(c, sched),
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": sample_txt},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    _emit(line)


# DRAM bytes per launch over algorithmic bytes, from ncu captures (dram__bytes_read.sum +
# dram__bytes_write.sum) of each step kernel at n = 262,144, d = 1,024, k = 16; the traffic
# grows with the rows, so a full launch's traffic is this ratio times its algorithmic bytes.
# Keys: (path, planes, cache hints).  Configurations without a capture report null.
# DRAM bytes per launch / algorithmic bytes at d = 1024, k = 16, from ncu
# captures of the current kernels, keyed by (path, planes, cache hints, slice
# columns, lag); other configurations report traffic as unknown.
DRAM_RATIO = {(0, 0, 0, 0, 0): 1081.1 / 1073.7,    # SIMT FP32, Z_i in TMEM (n = 262,144)
              (3, 2, 0, 0, 0): 2118.4 / 2048.0}    # pass-split pair tcgen05, hi/lo planes (n = 500,000)
# the precision workload's shape (d = 2,048, k = 32), from captures at n = 131,072 scaled by rows
DRAM_RATIO_PRECISION = {"bf16": 552.866 / 536.871,   # streaming tcgen05 (profiles/step_tcs_bf16_d2048_k32.md)
                        "e4m3": 275.163 / 268.960}   # FP8 tcgen05, codes + scales (profiles/step_tcs8_e4m3_d2048_k32.md)


def _traffic(path, planes, tuning, launch_bytes, d=1024, k=16):
    t = tuning or {}
    key = (path, planes, t.get("cache_hints", 0), t.get("slice_cols", 0), t.get("lag_units", 0))
    r = DRAM_RATIO.get(key) if (d, k) == (1024, 16) else None
    return None if r is None else r * launch_bytes


KERNELS = {0: "step_simt2_kernel (SIMT FP32 fused A_i^T (A_i Z_i))",
           1: "step_tc_kernel (tcgen05, tile resident in shared memory, cluster-split d)",
           2: "step_tcs_kernel (tcgen05 streaming, second pass re-read from L2)",
           3: "step_pair_kernel (tcgen05, the two passes on the two CTAs of a cluster: HBM pass forms W, "
              "L2 pass accumulates A^T W)"}


def _kernel(path, dtype="f32", d=1024, k=16):
    """Name of the step kernel a solve ran (lp_stats.path plus the shape for the SIMT path)."""
    if path == 2 and dtype == "e4m3":
        return "step_tcs8_kernel (tcgen05 streaming, E4M3 codes widened to FP16 in shared memory, row scales factored out)"
    if path != 0:
        return KERNELS[path]
    if dtype != "f32":
        return "step_simt_kernel (SIMT, rows widened to FP32 in shared memory)"
    if 8 < k <= 16 and d == 1024:
        return ("step_simt_tmem_d1024_kernel (SIMT FP32 fused A_i^T (A_i Z_i), Z_i resident in TMEM, "
                "tiles software-pipelined)")
    if 8 < k <= 16 and d <= 1024:
        return "step_simt_tmem_kernel (SIMT FP32 fused A_i^T (A_i Z_i), Z_i resident in TMEM)"
    return KERNELS[0]


def _config(c, sched, name: str = WORKLOAD):
    if name == "plain":
        text = (f"LocalPower plain: n={c['n']:,} d={c['d']} k={c['k']} m={c['m']}, p=4 x20 rounds, sign-fixing "
                f"(FP32 A)")
        return {"workload": text, "n": c["n"], "d": c["d"], "k": c["k"], "m": c["m"], "rounds": len(sched),
                "local_steps": sum(sched), "l2": "inputs fit in L2 (1.6 MB); latency-bound configuration"}
    if name == "lowprec":
        text = (f"LocalPower BF16 storage: n={c['n']:,} d={c['d']} k={c['k']} m={c['m']}, p=4 x30 rounds + 3 "
                f"FP32-accumulated p=1 refinement rounds ({sum(sched)} local steps) + Rayleigh-Ritz pass")
        size = f"A is {c['n'] * c['d'] * 2 / 1e9:.1f} GB BF16"
    else:
        text = (f"LocalPower FP32: n={c['n']:,} d={c['d']} k={c['k']} m={c['m']}, p=8,4,2,1 x10 rounds then "
                f"p=1 x{len(sched) - 40} (T={len(sched)}, {sum(sched)} local steps) + Rayleigh-Ritz pass")
        size = f"A is {c['n'] * c['d'] * 4 / 1e9:.1f} GB FP32"
    return {"workload": text, "n": c["n"], "d": c["d"], "k": c["k"], "m": c["m"], "rounds": len(sched),
            "local_steps": sum(sched), "l2": f"inputs larger than L2 ({size}; L2 is 129 MB)"}


def run_lowprec(args):
    """The reduced-precision workload: BF16 storage on the tensor cores (kernel
    chosen by the autotuner), then the same matrix in FP8-E4M3 with row scales."""
    import torch
    import torch.distributed as dist

    import oracle
    import synth
    from paper_2002_08014_gb300 import binding as B

    rank, world, local = _dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    c, A, sizes, Y0, sched = _workload(rank, args.rows, "lowprec")
    _timed.y0 = Y0
    k, d = c["k"], c["d"]
    parts = synth.split_rows(A, sizes)
    bits = [synth.f32_to_bf16_bits(p) for p in parts]
    stream = torch.cuda.Stream(device=dev)
    hbm_peak, _, peak_src = _peaks()
    lpb = B.LocalPower(bits, dtype="bf16", device=local, stream=stream)
    choice = B.lp_autotune(lpb.ctx, k)
    # the workload's arithmetic: FP32 accumulation, the k x k work in FP64 (LP_FLAG_KXK_FP64)
    for _ in range(args.warmup):
        lpb.submit(k, sched, args.agg, Y0, ritz=True, timing=True, kxk_fp64=True)
        lpb.result(k)
    ms, stats, Z, sig, clk = _timed(torch, dist, world, dev, stream, lpb, k, sched, args.agg, args.steps,
                                    Clocks(local), kxk_fp64=True)
    s = _summary(world, args.steps, ms, stats, 2, c)
    # the same solves with the k x k work in FP32, for the cost of the FP64 k x k work
    for _ in range(max(1, args.warmup // 2)):
        lpb.submit(k, sched, args.agg, Y0, ritz=True, timing=True)
        lpb.result(k)
    ms32, stats32, Z32, _, _ = _timed(torch, dist, world, dev, stream, lpb, k, sched, args.agg, args.steps)
    s32 = _summary(world, args.steps, ms32, stats32, 2, c)
    lpb.close()
    gbs_k = s["launch_bytes"] / (s["step_ms"] / 1e3) / 1e9
    line = {"metric": METRIC, "value": s["gbs"], "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": s["ms_per_solve"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic", "config": _config(c, sched, "lowprec"),
            "solves_per_s": s["solves_per_s"], "latency_ms": s["latency_ms"], "clocks": clk,
            "gpu_launches": s["launches"], "e2e": None, "autotune": choice,
            "roofline": {"kernel": _kernel(s["path"], "bf16", c["d"], c["k"]), "bound": "hbm",
                         "achieved": gbs_k, "peak": hbm_peak, "unit": "GB/s", "frac": gbs_k / hbm_peak,
                         "traffic": (DRAM_RATIO_PRECISION["bf16"] * s["launch_bytes"] if s["path"] == 2 else None),
                         "traffic_unit": "bytes per launch", "launch_ms": s["step_ms"],
                         "peak_source": f"{peak_src} HBM copy bandwidth"}}
    line["orthonormality"] = float(np.abs(Z.T @ Z - np.eye(k)).max())
    line["sigma_top3"] = [float(x) for x in sig[:3]]
    line["kxk"] = {"precision": "fp64 (Gram/Cholesky of CholQR2, Procrustes SVD, Ritz eigen-solve)",
                   "fp32_kxk_solves_per_s": s32["solves_per_s"], "fp32_kxk_ms_per_solve": s32["ms_per_solve"],
                   "fp64_cost_frac": (s["ms_per_solve"] - s32["ms_per_solve"]) / s["ms_per_solve"]}

    # the same matrix as FP8-E4M3 codes with one FP32 scale per row (tensor cores: codes widened to FP16)
    fp8 = None
    try:
        codes, scales = zip(*[synth.f32_to_e4m3_rowscaled(p) for p in parts])
        lp8 = B.LocalPower(list(codes), dtype="e4m3", row_scales=list(scales), device=local, stream=stream)
        choice8 = B.lp_autotune(lp8.ctx, k)
        for _ in range(args.warmup):
            lp8.submit(k, sched, args.agg, Y0, ritz=True, timing=True, kxk_fp64=True)
            lp8.result(k)
        ms8, st8, Z8, sig8, clk8 = _timed(torch, dist, world, dev, stream, lp8, k, sched, args.agg, args.steps,
                                          Clocks(local), kxk_fp64=True)
        s8 = _summary(world, args.steps, ms8, st8, 1, c)
        lp8.close()
        gbs8 = (s8["launch_bytes"] + 4.0 * c["n"]) / (s8["step_ms"] / 1e3) / 1e9
        fp8 = {"dtype": "e4m3 codes x FP32 row scales, FP32 accumulation", "step_kernel": _kernel(s8["path"], "e4m3", c["d"], c["k"]),
               "gbs": s8["gbs"], "solves_per_s": s8["solves_per_s"], "ms_per_solve": s8["ms_per_solve"],
               "step_launch_ms": s8["step_ms"], "clocks": clk8, "latency_ms": s8["latency_ms"],
               "speedup_solves_vs_bf16": s8["solves_per_s"] / s["solves_per_s"],
               "roofline": {"bound": "hbm", "achieved": gbs8, "peak": hbm_peak, "unit": "GB/s",
                            "frac": gbs8 / hbm_peak, "launch_ms": s8["step_ms"],
                            "traffic": (DRAM_RATIO_PRECISION["e4m3"] * (s8["launch_bytes"] + 4.0 * c["n"])
                                        if s8["path"] == 2 else None),
                            "traffic_unit": "bytes per launch",
                            "algorithmic_bytes_per_launch": s8["launch_bytes"] + 4.0 * c["n"],
                            "peak_source": f"{peak_src} HBM copy bandwidth"},
               "autotune": choice8,
               "note": "E4M3 codes widened to FP16 in shared memory, row scales factored out (Q^T diag(s^2) Q Z)"}
    except Exception as e:  # reported, not hidden
        fp8 = {"error": str(e)[:300]}
    line["fp8_path"] = fp8

    if rank == 0 and not args.no_accuracy:
        # FP64 truth of the decoded BF16 problem (the matrix the solver is given) and of the FP32 original
        t0 = time.perf_counter()
        Vb, _ = _truth(bits, c, oracle.decode_bf16)
        Vf, _ = _truth(parts, c)
        line["accuracy"] = {"dist_to_eigh_topk_bf16_problem": oracle.subspace_dist(oracle.orth(Z), Vb),
                            "dist_to_eigh_topk_fp32_problem": oracle.subspace_dist(oracle.orth(Z), Vf),
                            "dist_to_eigh_topk_bf16_problem_fp32_kxk": oracle.subspace_dist(oracle.orth(Z32), Vb),
                            "quantisation_shift": oracle.subspace_dist(Vb, Vf),
                            "host_fp64_seconds": time.perf_counter() - t0}
        if fp8 and "error" not in fp8:
            line["fp8_path"]["dist_to_eigh_topk_fp32_problem"] = oracle.subspace_dist(oracle.orth(Z8), Vf)
    if rank == 0:
        _emit(line)
    if world > 1:
        dist.destroy_process_group()


def run_plain(args):
    """The small plain configuration (FP32, n=4000, d=100, k=5, m=4): latency-bound,
    reported as solves/s and per-solve latency over many solves."""
    import torch
    import torch.distributed as dist

    import oracle
    import synth
    from paper_2002_08014_gb300 import binding as B

    rank, world, local = _dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    c, A, sizes, Y0, sched = _workload(rank, None, "plain")
    _timed.y0 = Y0
    k = c["k"]
    parts = synth.split_rows(A, sizes)
    stream = torch.cuda.Stream(device=dev)
    lp = B.LocalPower(parts, device=local, stream=stream)
    solves = max(args.steps, 50)
    for _ in range(max(args.warmup, 3)):
        lp.submit(k, sched, "sign", Y0, ritz=True, timing=True)
        lp.result(k)
    ms, stats, Z, sig, clk = _timed(torch, dist, world, dev, stream, lp, k, sched, "sign", solves, Clocks(local))
    s = _summary(world, solves, ms, stats, 4, c)
    # the other two aligners of eq. (3) on the same solves (latency and launches)
    others = {}
    for agg in ("opt", "identity"):
        for _ in range(max(args.warmup, 3)):
            lp.submit(k, sched, agg, Y0, ritz=True, timing=True)
            lp.result(k)
        ms_a, st_a, Za, _, clk_a = _timed(torch, dist, world, dev, stream, lp, k, sched, agg, solves, Clocks(local))
        sa = _summary(world, solves, ms_a, st_a, 4, c)
        ref_a = oracle.localpower(parts, k, sched, agg, Y0)
        others[agg] = {"solves_per_s": sa["solves_per_s"], "latency_ms": sa["latency_ms"],
                       "launches_per_solve": sa["launches"] / solves, "clocks": clk_a,
                       "dist_to_oracle": oracle.subspace_dist(oracle.orth(Za), ref_a["Z"])}
    lp.close()
    ref = oracle.localpower(parts, k, sched, "sign", Y0)
    line = {"metric": METRIC, "value": s["gbs"], "unit": "GB/s", "n_gpus": world, "steps": solves,
            "warmup": max(args.warmup, 3), "ms_per_step": s["ms_per_solve"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": _config(c, sched, "plain"), "solves_per_s": s["solves_per_s"], "latency_ms": s["latency_ms"],
            "clocks": clk, "gpu_launches": s["launches"], "e2e": None,
            "launches_per_solve": s["launches"] / solves, "step_kernel": _kernel(s["path"], "f32", c["d"], c["k"]),
            "dist_to_oracle": oracle.subspace_dist(oracle.orth(Z), ref["Z"]), "other_aggregators": others}
    if rank == 0 and not args.no_cpu_baseline:
        rate, runs = _oracle_solves(parts, k, sched, "sign", Y0, 10.0)
        rate1, runs1 = _oracle_solves(parts, k, sched, "sign", Y0, 10.0, one_thread=True)
        solve_bytes = s["bytes_solve"] / 1e9     # algorithmic GB per solve (all step passes)
        line["cpu_baseline"] = {"value": rate * solve_bytes, "unit": "GB/s", "cores": os.cpu_count(),
                                "kind": "oracle", "solves_per_s": rate,
                                "sample": f"{runs} whole FP64 oracle solves (Alg. 1, sign-fixing, Ritz output) "
                                          f"in about 10 s, NumPy's BLAS on all cores",
                                "one_thread_solves_per_s": rate1,
                                "one_thread_gbs": None if rate1 is None else rate1 * solve_bytes,
                                "one_thread_sample": f"{runs1} whole oracle solves in about 10 s, BLAS limited "
                                                     f"to one thread", **_cpu_info()}
    if rank == 0:
        _emit(line)
    if world > 1:
        dist.destroy_process_group()


SERVING_WIDTHS = [64, 90, 128, 181, 256, 362, 512, 724, 1024]   # log-spaced pool widths
# Sec. 3's decaying p for each request, ending with enough p = 1 rounds that the
# small, heterogeneous partitions of the request mix leave no error floor (an
# offline oracle study of the request shapes: every shape below 1e-4, worst 4e-6)
SERVING_SCHEDULE = [4] * 10 + [2] * 10 + [1] * 60


def _serving_requests(n_req: int, rate: float, seed: int):
    """Request shapes (log-uniform n, m; d log-uniform rounded to the nearest
    pool width; k uniform in {4, 8, 16, 32}) and Poisson arrival times."""
    rng = np.random.default_rng(seed)
    lu = lambda lo, hi, size: np.exp(rng.uniform(np.log(lo), np.log(hi), size))
    n = np.round(lu(2_000, 200_000, n_req)).astype(int)
    w = np.log(np.array(SERVING_WIDTHS, dtype=float))
    d = np.array([SERVING_WIDTHS[int(np.argmin(np.abs(w - np.log(x))))] for x in lu(64, 1024, n_req)])
    m = np.round(lu(4, 32, n_req)).astype(int)
    k = rng.choice([4, 8, 16, 32], n_req)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
    offs = rng.integers(0, 1, n_req)  # filled by the caller once the pool size is known
    return [dict(n=int(n[i]), d=int(d[i]), m=int(m[i]), k=int(k[i]), t=float(arrivals[i]), off=int(offs[i]),
                 seed=seed * 100_000 + i) for i in range(n_req)]


def _width_pools(torch, local, seed, pool_rows, fp32=False):
    """Device pools of spiked BF16 rows, one per width in SERVING_WIDTHS, each with
    its own Haar rotation and lambda_j = 0.85^j (j <= width); host copies too.
    fp32: also device pools of the FP32 rows the BF16 ones are rounded from."""
    import synth
    t = time.perf_counter()
    bits, dev, dev32 = {}, {}, {}
    for wi, w in enumerate(SERVING_WIDTHS):
        lam = 0.85 ** np.arange(1, w + 1)
        rows = synth.spiked_rows(pool_rows, w, lam, 0.0, seed + 10 + wi, out_dtype=np.float32,
                                 threads=os.cpu_count())
        bits[w] = synth.f32_to_bf16_bits(rows)
        dev[w] = torch.from_numpy(bits[w].view(np.int16)).cuda(local)
        if fp32:
            dev32[w] = torch.from_numpy(rows).cuda(local)
        del rows
    _DATA_GEN_S[0] += time.perf_counter() - t
    return (bits, dev, dev32) if fp32 else (bits, dev)


def run_batching(args):
    """Batching: independent instances (n log-uniform [2e3, 2e5], d log-uniform
    [64, 1024] rounded to the pool widths, m [4, 32], k in {4, 8, 16, 32}; BF16;
    p = 4, T = 30) loaded once into a batch; instances of one (d, k) form a group
    whose every step kind is one launch over all of them, with the group's step
    kernel chosen by the autotuner; every solve of the whole batch is one CUDA
    graph launch.  Beside it: the same instances solved one after another (each
    its own replayed graph)."""
    import torch

    import oracle
    import synth
    from paper_2002_08014_gb300 import binding as B

    rank, world, local = _dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    seed = synth.configs.SEED_BASE + 4
    inst = _serving_requests(args.instances, 1.0, seed)
    pool_rows = 400_000
    bits, dev = _width_pools(torch, local, seed, pool_rows)
    orng = np.random.default_rng(seed + 1)
    sched = [4] * 30
    a_bytes = 0.0
    with B.Batch(device=local) as bt:
        for r in inst:
            r["off"] = int(orng.integers(0, pool_rows - r["n"]))
            sizes = synth.partition_sizes(r["n"], r["m"])
            offs = r["off"] + np.cumsum([0] + sizes[:-1])
            parts = [dev[r["d"]][o:o + s_] for o, s_ in zip(offs, sizes)]
            bt.add(parts, r["k"], sched, "sign", synth.gaussian_start(r["d"], r["k"], r["seed"]), dtype="bf16")
        t_tune = time.perf_counter()
        bt.autotune()
        t_tune = time.perf_counter() - t_tune
        t_cap = time.perf_counter()
        bt.solve()                      # captures and instantiates the graph, then runs it
        for i in range(len(inst)):
            bt.result(i)
        t_cap = time.perf_counter() - t_cap
        for _ in range(max(args.warmup - 1, 1)):
            bt.solve()
            bt.result(0)
        clocks = Clocks(local)
        torch.cuda.synchronize()
        clocks.start()
        ms = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            bt.solve()
            bt.result(0)               # waits for the whole batch
            ms.append((time.perf_counter() - t0) * 1e3)
        clk = clocks.stop()
        if args.profile_solve:
            torch.cuda.synchronize()
            torch.cuda.profiler.start()
            bt.solve()
            bt.result(0)
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
        outs = [bt.result(i) for i in range(len(inst))]
        n_groups = bt.groups()
        a_bytes = sum(o[2]["a_bytes"] for o in outs)
        # instances of one group (here: one (d, k), every other parameter is shared)
        # report their group's launches; count each group once
        group_of = {}
        for r, o in zip(inst, outs):
            group_of[(r["d"], r["k"])] = (o[2]["kernel_launches"], KERNELS[o[2]["path"]])
        launches = sum(v[0] for v in group_of.values())
        paths = {}
        for _, pth in group_of.values():
            paths[pth] = paths.get(pth, 0) + 1
    # the same instances one after another, each with its own context and replayed graph
    seq_ms = None
    try:
        t0 = time.perf_counter()
        for r in inst:
            sizes = synth.partition_sizes(r["n"], r["m"])
            offs = r["off"] + np.cumsum([0] + sizes[:-1])
            parts = [dev[r["d"]][o:o + s_] for o, s_ in zip(offs, sizes)]
            with B.LocalPower(parts, dtype="bf16") as lp:
                lp.solve(r["k"], sched, "sign", synth.gaussian_start(r["d"], r["k"], r["seed"]))
        seq_ms = (time.perf_counter() - t0) * 1e3
    except Exception as e:
        seq_ms = f"error: {str(e)[:200]}"
    acc, acc_o = [], []
    cheap = [i for i, r in enumerate(inst) if r["n"] * r["d"] * r["k"] <= 3e8]
    for i in [cheap[j] for j in np.linspace(0, len(cheap) - 1, min(6, len(cheap))).astype(int)]:
        r = inst[i]
        rows = oracle.decode_bf16(bits[r["d"]][r["off"]:r["off"] + r["n"]])
        w, V = np.linalg.eigh(rows.T @ rows / r["n"])
        acc.append(oracle.subspace_dist(oracle.orth(outs[i][0]), V[:, ::-1][:, :r["k"]]))
        ref = oracle.localpower(synth.split_rows(rows, synth.partition_sizes(r["n"], r["m"])), r["k"], sched, "sign",
                                synth.gaussian_start(r["d"], r["k"], r["seed"]))
        acc_o.append(oracle.subspace_dist(oracle.orth(outs[i][0]), ref["Z"]))
    best = min(ms)
    line = {"metric": METRIC, "value": a_bytes / (best / 1e3) / 1e9, "unit": "GB/s", "n_gpus": 1, "steps": args.steps,
            "warmup": max(args.warmup - 1, 1) + 1, "ms_per_step": float(np.mean(ms)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": f"LocalPower batching: {len(inst)} independent BF16 instances, n log-uniform "
                                   f"[2e3, 2e5], d log-uniform [64, 1024] rounded to 9 widths, m [4, 32], k in "
                                   f"{{4, 8, 16, 32}}, p=4 x30 rounds, one graph launch per step (instances "
                                   f"of one (d, k) merged into a group: each step kind one launch per group)",
                       "instances": len(inst), "groups": n_groups, "a_bytes_per_step": a_bytes,
                       "l2": "instances' A from 2.7 GB of device pools (larger than L2)"},
            "solves_per_s": len(inst) / (best / 1e3), "latency_ms": {"p50": float(np.percentile(ms, 50)),
                                                                    "p99": float(np.percentile(ms, 99)),
                                                                    "samples": len(ms)},
            "kernel_launches_per_step": launches, "step_kernels_chosen_per_group": paths,
            "autotune_s": t_tune, "first_solve_with_capture_s": t_cap,
            "sequential_ms": seq_ms,
            "speedup_vs_sequential": (seq_ms / best) if isinstance(seq_ms, float) else None,
            "clocks": clk, "e2e": None,
            "accuracy_sample": {"dist_to_oracle": [float(x) for x in acc_o], "max_dist_to_oracle": float(max(acc_o)),
                                "dist_to_eigh_topk": [float(x) for x in acc]}}
    _emit(line)


def run_rounds(args):
    """Rounds to accuracy for constant p in {1, 2, 4, 8} (sign-fixing and OPT) on
    the FP32 workload's matrix (n rows from --rows, default 250,000): the traced
    solve gives Z_t after every aggregation and the residual error rho_t of
    Def. 3; the distance of Z_t to the FP64 eigendecomposition's top-k gives the
    first round at 1e-4 and 1e-6 (the analogue of the paper's communication vs
    accuracy experiments, on synthetic data)."""
    import oracle
    import synth
    from paper_2002_08014_gb300 import binding as B

    rank, world, local = _dist_env()
    if rank != 0:
        return
    c, A, sizes, Y0, _ = _workload(0, args.rows or 250_000)
    parts = synth.split_rows(A, sizes)
    k, d = c["k"], c["d"]
    V, _ = _truth(parts, c)
    T = 120
    out = {}
    with B.LocalPower(parts, device=local) as lp:
        for agg in ("sign", "opt"):
            for p in (1, 2, 4, 8):
                B.lp_solve(lp.ctx, k, [p] * T, agg, Y0, 0, B.LP_FLAG_TRACE)
                lp.result(k)
                Zt, rho = B.lp_trace(lp.ctx, T, d, k)
                dist = [oracle.subspace_dist(oracle.orth(Zt[t]), V) for t in range(T)]
                first = lambda tol: next((t + 1 for t, x in enumerate(dist) if x <= tol), None)
                out[f"{agg}_p{p}"] = {"rounds_to_1e-4": first(1e-4), "rounds_to_1e-6": first(1e-6),
                                      "final_dist": dist[-1], "dist_every_10": dist[9::10],
                                      "rho_mean": float(np.mean(rho)), "rho_last": float(rho[-1])}
        # iteration rank r > k (Alg. 1): dist(Z_t, U_k) = ||(I - Z_t Z_t^T) U_k||_2 with Z_t of r columns
        ranks = {}
        rng = np.random.default_rng(synth.configs.SEED_BASE + 7)
        for r in (k, k + 8, 2 * k):
            Yr = np.concatenate([Y0, rng.standard_normal((d, r - k))], axis=1) if r > k else Y0
            B.lp_solve(lp.ctx, r, [4] * T, "sign", Yr, 0, B.LP_FLAG_TRACE)
            lp.result(r)
            Zt, _ = B.lp_trace(lp.ctx, T, d, r)
            dist = [oracle.subspace_dist(oracle.orth(Zt[t]), V) for t in range(T)]
            first = lambda tol: next((t + 1 for t, x in enumerate(dist) if x <= tol), None)
            ranks[f"r{r}"] = {"rounds_to_1e-4": first(1e-4), "rounds_to_1e-6": first(1e-6), "final_dist": dist[-1]}
        # eta of Def. 2 on the device, beside the oracle's value on the same matrix
        t0 = time.perf_counter()
        eta, norms = lp.eta()
        eta_ms = (time.perf_counter() - t0) * 1e3
    eta_ref = oracle.eta(parts)[0]
    print(json.dumps({"workload": "rounds", "n": c["n"], "d": d, "k": k, "m": c["m"], "T": T,
                      "note": "rounds = aggregations = the paper's communications; rho_t is max_i ||Z_i G_i - Z_b||_2",
                      "results": out,
                      "iteration_rank": {"note": "sign-fixing, p = 4; the first k columns of Y_0 are shared",
                                         "results": ranks},
                      "eta": {"value": eta, "oracle": eta_ref, "rel_err": abs(eta - eta_ref) / eta_ref,
                              "norm_M": float(norms[-1]), "ms": eta_ms,
                              "note": "Def. 2: max_i ||M_i - M||_2 / ||M||_2; lp_eta forms the M_i with "
                                      "ceil(d/K) fused steps and measures norms by Lanczos"}}))


def run_serving(args):
    """Continuous batching: a Poisson stream of truncated-SVD requests of mixed
    shapes through the request server, admitted against an HBM budget.  Each
    request is BF16 and solved to dist <= 1e-4 with the decaying schedule
    p = 4 x 10, 2 x 10, 1 x 60 rounds, then 3 refinement rounds (p = 1) and
    Rayleigh-Ritz: 123 local steps, like a constant p = 4 x 30 + 3, but without
    the constant-p error floor that small, heterogeneous partitions leave.  Rows
    come from device-resident pools of spiked BF16 rows, one per width d, each
    with its own Haar rotation and lambda_j = 0.85^j (j <= d); a request names a
    row range of the pool of its width.  Beside it: the same stream on the plain
    FP32 path (the FP32 rows the BF16 pools are rounded from), and both paths with
    every request submitted at once (the largest throughput each sustains)."""
    import torch

    import oracle
    import synth
    from paper_2002_08014_gb300 import binding as B

    rank, world, local = _dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    seed = synth.configs.SEED_BASE + 5
    reqs = _serving_requests(args.requests, args.rate, seed)
    pool_rows = 400_000
    pool_bits, dev_pool, dev_pool32 = _width_pools(torch, local, seed, pool_rows, fp32=True)
    orng = np.random.default_rng(seed + 1)
    for r in reqs:
        r["off"] = int(orng.integers(0, pool_rows - r["n"]))
    sched = SERVING_SCHEDULE
    budget = 120 << 30

    def serve(dtype, pools, saturated=False, clocks=None):
        """The request stream through a server: arrivals at their Poisson times, or
        all at once (saturated).  Returns per-request completion times (from the
        arrival, or from the start when saturated), the A bytes, the wall time, the
        peaks and the results."""
        done_t, a_bytes, Zs = {}, 0.0, {}
        with B.Server(device=local, hbm_budget_bytes=budget, max_active=64) as srv:
            def submit(r):
                sizes = synth.partition_sizes(r["n"], r["m"])
                offs = r["off"] + np.cumsum([0] + sizes[:-1])
                parts = [pools[r["d"]][o:o + s_] for o, s_ in zip(offs, sizes)]
                return srv.submit(parts, r["k"], sched, "sign", synth.gaussian_start(r["d"], r["k"], r["seed"]),
                                  dtype=dtype, refine_rounds=3)
            for r in reqs[:4]:  # warm-up: a few requests of the same kind, not timed
                rid = submit(r)
                while rid not in srv.progress():
                    time.sleep(0.0005)
                srv.result(rid)
            torch.cuda.synchronize()
            if clocks:
                clocks.start()
            t0 = time.perf_counter()
            nxt, ids = 0, {}
            peak = {"active": 0, "queued": 0}
            while len(done_t) < len(reqs):
                now = time.perf_counter() - t0
                while nxt < len(reqs) and (saturated or reqs[nxt]["t"] <= now):
                    ids[submit(reqs[nxt])] = nxt
                    nxt += 1
                fin = srv.progress()
                tnow = time.perf_counter() - t0
                for rid in fin:
                    i = ids[rid]
                    done_t[i] = tnow
                    Z, sig, st = srv.result(rid)
                    a_bytes += st["a_bytes"]
                    Zs[i] = Z
                info = srv.query()
                peak["active"] = max(peak["active"], info["active"])
                peak["queued"] = max(peak["queued"], info["queued"])
                if not fin:
                    time.sleep(0.0002)
            wall = time.perf_counter() - t0
            hbm_peak = srv.query()["hbm_peak"]
        clk = clocks.stop() if clocks else None
        return done_t, a_bytes, wall, peak, hbm_peak, Zs, clk

    clocks = Clocks(local)
    done_t, a_bytes, wall, peak, hbm_peak, Zs, clk = serve("bf16", dev_pool, clocks=clocks)
    for i, Z in Zs.items():
        reqs[i]["Z"] = Z
    lats = np.array([(done_t[i] - reqs[i]["t"]) * 1e3 for i in range(len(reqs))])
    span = max(done_t.values()) - reqs[0]["t"]
    # a sample of requests against the FP64 oracle run on the same decoded data and schedule
    # (parity) and against the eigendecomposition of the request's matrix (convergence of the
    # schedule on that matrix's sample spectrum)
    acc, acc_o = [], []
    cheap = [i for i, r in enumerate(reqs) if r["n"] * r["d"] * r["k"] <= 3e8]
    for i in [cheap[j] for j in np.linspace(0, len(cheap) - 1, min(8, len(cheap))).astype(int)]:
        r = reqs[i]
        rows = oracle.decode_bf16(pool_bits[r["d"]][r["off"]:r["off"] + r["n"]])
        w, V = np.linalg.eigh(rows.T @ rows / r["n"])
        acc.append(oracle.subspace_dist(oracle.orth(r["Z"]), V[:, ::-1][:, :r["k"]]))
        ref = oracle.localpower(synth.split_rows(rows, synth.partition_sizes(r["n"], r["m"])), r["k"],
                                sched + [1, 1, 1], "sign", synth.gaussian_start(r["d"], r["k"], r["seed"]))
        acc_o.append(oracle.subspace_dist(oracle.orth(r["Z"]), ref["Z"]))
    # the plain FP32 path on the same request stream (the FP32 rows the BF16 pools
    # are rounded from), then both with every request submitted at once: the
    # largest throughput each path sustains
    d32, b32, wall32, peak32, _, Zs32, clk32 = serve("f32", dev_pool32, clocks=Clocks(local))
    lats32 = np.array([(d32[i] - reqs[i]["t"]) * 1e3 for i in range(len(reqs))])
    span32 = max(d32.values()) - reqs[0]["t"]
    acc32 = []
    for i in [cheap[j] for j in np.linspace(0, len(cheap) - 1, min(4, len(cheap))).astype(int)]:
        r = reqs[i]
        rows = dev_pool32[r["d"]][r["off"]:r["off"] + r["n"]].cpu().numpy().astype(np.float64)
        w, V = np.linalg.eigh(rows.T @ rows / r["n"])
        acc32.append(oracle.subspace_dist(oracle.orth(Zs32[i]), V[:, ::-1][:, :r["k"]]))
    sat = {}
    for dtype, pools in (("bf16", dev_pool), ("f32", dev_pool32)):
        dsat, bsat, wsat, psat, _, _, _ = serve(dtype, pools, saturated=True)
        lsat = np.array(list(dsat.values())) * 1e3
        sat[dtype] = {"solves_per_s": len(reqs) / max(dsat.values()), "gbs": bsat / max(dsat.values()) / 1e9,
                      "completion_ms": {"p50": float(np.percentile(lsat, 50)), "p99": float(np.percentile(lsat, 99))},
                      "peak_active": psat["active"]}
    sat["speedup_solves_bf16_vs_plain_fp32"] = sat["bf16"]["solves_per_s"] / sat["f32"]["solves_per_s"]
    line = {"metric": METRIC, "value": a_bytes / span / 1e9, "unit": "GB/s", "n_gpus": 1, "steps": len(reqs),
            "warmup": 4, "ms_per_step": span * 1e3 / len(reqs), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": f"LocalPower serving: {len(reqs)} truncated-SVD requests, Poisson arrivals at "
                                   f"{args.rate:g} req/s, n log-uniform [2e3, 2e5], d log-uniform [64, 1024] "
                                   f"rounded to 9 pool widths, m [4, 32], "
                                   f"k in {{4, 8, 16, 32}}, BF16, p=4 x10, 2 x10, 1 x60 rounds + 3 refinement "
                                   f"rounds + Ritz (123 local steps), "
                                   f"admission budget 120 GB",
                       "requests": len(reqs), "rate_per_s": args.rate, "budget_bytes": budget, "max_active": 64,
                       "l2": "requests' A from 2.7 GB of device pools (larger than L2)"},
            "solves_per_s": len(reqs) / span, "latency_ms": {"p50": float(np.percentile(lats, 50)),
                                                             "p99": float(np.percentile(lats, 99)),
                                                             "max": float(lats.max()), "samples": len(lats)},
            "offered_solves_per_s": args.rate, "wall_s": wall, "peak_active": peak["active"],
            "peak_queued": peak["queued"], "hbm_peak_bytes": int(hbm_peak), "clocks": clk, "e2e": None,
            "accuracy_sample": {"dist_to_oracle": [float(x) for x in acc_o], "max_dist_to_oracle": float(max(acc_o)),
                                "dist_to_eigh_topk": [float(x) for x in acc],
                                "max_dist_to_eigh_topk": float(max(acc)), "target": 1e-4,
                                "met": bool(max(acc) <= 1e-4),
                                "truth": "FP64 eigendecomposition of each sampled request's decoded BF16 matrix"},
            "plain_fp32_serving": {"dtype": "f32 (SIMT FP32 step kernels)", "solves_per_s": len(reqs) / span32,
                                   "gbs": b32 / span32 / 1e9,
                                   "latency_ms": {"p50": float(np.percentile(lats32, 50)),
                                                  "p99": float(np.percentile(lats32, 99)),
                                                  "max": float(lats32.max()), "samples": len(lats32)},
                                   "peak_active": peak32["active"], "clocks": clk32,
                                   "accuracy_sample": {"dist_to_eigh_topk": [float(x) for x in acc32],
                                                       "max_dist_to_eigh_topk": float(max(acc32)),
                                                       "met": bool(max(acc32) <= 1e-4),
                                                       "truth": "FP64 eigendecomposition of the FP32 rows"}},
            "saturated": sat}
    _emit(line)


def run_kernels(args):
    """Each step kernel on one shape: one-step solves (a single fused-step launch
    each) per kernel, in a fixed order, for profiler captures and quick scans:
    SIMT FP32, streaming tcgen05 BF16, resident tcgen05 BF16, streaming tcgen05
    on hi/lo planes of the FP32 data, the pass-split pair kernel on BF16 and on
    the hi/lo planes, then the FP8-E4M3 tensor-core kernel on the codes and row
    scales of the same rows."""
    import synth
    from paper_2002_08014_gb300 import binding as B

    d, k = (int(x) for x in args.shape.lower().split("x"))
    n = int(args.rows or (1 << 31) // (d * 4))
    m = 64
    lam = 10.0 * 0.9 ** np.arange(1, min(32, d) + 1)
    A = synth.spiked_rows(n, d, lam, np.sqrt(0.1), synth.configs.SEED_BASE + 9, threads=os.cpu_count())
    parts = synth.split_rows(A, synth.partition_sizes(n, m))
    Y0 = synth.gaussian_start(d, k, 1)
    runs = [("f32", parts, 0, None), ("bf16", None, 0, "stream"), ("bf16", None, B.LP_FLAG_TC_RESIDENT, None),
            ("f32_bf16x2", parts, 0, "stream"), ("bf16", None, 0, "pair"), ("f32_bf16x2", parts, 0, "pair"),
            ("e4m3", None, 0, None)]
    bits = [synth.f32_to_bf16_bits(p) for p in parts]
    codes, scales = map(list, zip(*[synth.f32_to_e4m3_rowscaled(p) for p in parts]))
    out = {}
    for dtype, data, flags, kern in runs:
        eb = {"bf16": 2, "e4m3": 1 + 4.0 / d}.get(dtype, 4)
        name = f"{dtype}{'_resident' if flags else ''}{'_' + kern if kern else ''}"
        if data is None:
            data = codes if dtype == "e4m3" else bits
        try:
            with B.LocalPower(data, dtype=dtype, row_scales=scales if dtype == "e4m3" else None) as lp:
                if kern:
                    B.lp_set_tuning(lp.ctx, kernel=kern)
                tuned = (B.lp_autotune(lp.ctx, k) if args.autotune and dtype != "f32" and not flags and kern != "pair"
                         else None)
                ms = []
                for _ in range(max(args.steps, 2)):
                    B.lp_solve(lp.ctx, k, [1], "sign", Y0, 0, B.LP_FLAG_TIMING | B.LP_FLAG_NO_GRAPH | flags)
                    _, _, st = lp.result(k)
                    ms.append(st["ms_step_kernels"])
            best = min(ms[1:])
            out[name] = {
                "kernel": _kernel(st["path"], dtype if dtype in ("f32", "e4m3") else "bf16", d, k), "tuning": tuned,
                "launch_ms": best, "gbs": n * d * eb / (best / 1e3) / 1e9}
        except Exception as e:
            out[name] = {"error": str(e)[:200]}
    print(json.dumps({"workload": "kernels", "n": n, "d": d, "k": k, "m": m, "results": out}))


def _timed(torch, dist, world, dev, stream, lp, k, sched, agg, steps, clocks=None, kxk_fp64=False):
    """K back-to-back solves on the library's stream, bracketed by a barrier and a
    device synchronize; CUDA events on that stream.  Returns (ms, stats, Z, sigma, clocks)."""
    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
    barrier()
    if clocks:
        clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    stats, Z, sig = [], None, None
    for _ in range(steps):
        lp.submit(k, sched, agg, _timed.y0, ritz=True, timing=True, kxk_fp64=kxk_fp64)
        Z, sig, st = lp.result(k)
        stats.append(st)
    ev1.record(stream)
    barrier()
    clk = clocks.stop() if clocks else None
    ms = max_over_ranks(torch, dist, world, dev, ev0.elapsed_time(ev1))
    return ms, stats, Z, sig, clk


def max_over_ranks(torch, dist, world, dev, ms: float) -> float:
    """The slowest rank's time (every rank gets it); the identity at world == 1."""
    if world <= 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, steps: int, bytes_per_solve: float, ms: float) -> tuple[float, float]:
    """Whole-job (GB/s, solves/s): every rank solves `steps` problems of
    `bytes_per_solve` algorithmic bytes; `ms` is the slowest rank's time."""
    return world * steps * bytes_per_solve / (ms / 1e3) / 1e9, world * steps / (ms / 1e3)


def _summary(world, steps, ms, stats, elem_bytes, c):
    """Throughput, latency percentiles and the step kernel's live launch time."""
    bytes_solve = stats[-1]["a_bytes"]
    lat = sorted(s["ms_solve"] for s in stats)
    step_ms = sum(s["ms_step_kernels"] for s in stats) / sum(s["step_launches"] for s in stats)
    gbs, sps = job_throughput(world, steps, bytes_solve, ms)
    return {"gbs": gbs,
            "solves_per_s": sps,
            "ms_per_solve": ms / steps,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "samples": len(lat)},
            "step_ms": step_ms,
            "launch_bytes": float(c["n"]) * c["d"] * elem_bytes,
            "launch_flops": 4.0 * c["n"] * c["d"] * c["k"],
            "launches": int(sum(s["kernel_launches"] for s in stats)),
            "path": stats[-1]["path"],
            "bytes_solve": bytes_solve}


def _truth(parts, c, decode=None):
    """Top-k eigenvectors / eigenvalues of M = A^T A / n (FP64, on the host);
    `decode` maps a stored partition to its FP64 values, a few at a time."""
    M = np.zeros((c["d"], c["d"]))
    for i in range(0, len(parts), 8):
        blk = np.concatenate([decode(p) if decode else p for p in parts[i:i + 8]]).astype(np.float64)
        M += blk.T @ blk
    lam, V = np.linalg.eigh(M / c["n"])
    return V[:, ::-1][:, :c["k"]], lam[::-1][:c["k"]]


def _cpu_info() -> dict:
    """Host CPU model and the BLAS library NumPy calls (for the CPU baseline)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    blas = None
    try:
        cfg = np.show_config(mode="dicts")
        b = cfg.get("Build Dependencies", {}).get("blas", {})
        blas = f"{b.get('name')} {b.get('version', '')}".strip()
    except Exception:
        pass
    return {"cpu_model": model, "blas": blas}


def _oracle_one_thread_gbps(parts, Y0) -> float | None:
    """The oracle's local step on the given partitions in a child process pinned to
    one BLAS thread (GB/s of FP32 A)."""
    fd, path = tempfile.mkstemp(suffix=".npz")
    os.close(fd)
    try:
        np.savez(path, Y0=Y0, **{f"p{i}": p for i, p in enumerate(parts)})
        code = ("import sys, time, numpy as np; sys.path.insert(0, %r); import oracle; "
                "f = np.load(%r); Z = oracle.orth(f['Y0']); P = [f[k] for k in f.files if k != 'Y0']; "
                "t = time.perf_counter(); [oracle.local_step(x, Z) for x in P]; "
                "print(sum(x.nbytes for x in P) / (time.perf_counter() - t) / 1e9)") % (ROOT, path)
        env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
        out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=300)
        return float(out.stdout.strip().splitlines()[-1])
    except Exception:
        return None
    finally:
        os.unlink(path)


def _oracle_solves(parts, k, sched, agg, Y0, seconds: float, one_thread: bool = False):
    """Whole oracle solves (Alg. 1 with Ritz output) repeated for about `seconds`;
    returns (solves/s, solves run).  With one_thread, in a child process whose BLAS
    is limited to one thread."""
    if not one_thread:
        import oracle
        t = time.perf_counter()
        runs = 0
        while True:
            r = oracle.localpower(parts, k, sched, agg, Y0)
            oracle.ritz(parts, r["Z"])
            runs += 1
            if time.perf_counter() - t >= seconds:
                return runs / (time.perf_counter() - t), runs
    fd, path = tempfile.mkstemp(suffix=".npz")
    os.close(fd)
    try:
        np.savez(path, Y0=Y0, sched=np.asarray(sched), **{f"p{i}": p for i, p in enumerate(parts)})
        code = ("import sys, time, numpy as np; sys.path.insert(0, %r); import oracle; f = np.load(%r); "
                "P = [f['p%%d' %% i] for i in range(%d)]; s = [int(x) for x in f['sched']]; "
                "t = time.perf_counter(); n = 0\n"
                "while True:\n"
                "    r = oracle.localpower(P, %d, s, %r, f['Y0']); oracle.ritz(P, r['Z']); n += 1\n"
                "    if time.perf_counter() - t >= %r: break\n"
                "print(n / (time.perf_counter() - t), n)") % (ROOT, path, len(parts), k, agg, seconds)
        env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
        out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=300)
        rate, runs = out.stdout.strip().splitlines()[-1].split()
        return float(rate), int(runs)
    except Exception:
        return None, 0
    finally:
        os.unlink(path)


def run_ours(args):
    """The FP32 workload (the default).  Three runs of the same matrix, one after
    another on the device, each timed over K solves after W warm-up solves:
      headline  the FP32 data held as hi + lo BF16 planes (4 bytes per element, within
                2^-17 of the FP32 values), pass-split tcgen05 step: FP32-level results;
      plain     the FP32 data on the SIMT FP32 step (the plain FP32 path the metric
                compares with);
      bf16      the data rounded to BF16 (reduced precision), same tcgen05 step;
    and the headline again with the other aligner (sign-fixing and OPT both run).
    Each run's result is compared with the FP64 eigendecomposition of A^T A / n
    (the metric's accuracy bar is 1e-4), and a traced solve gives rounds to 1e-4."""
    import torch
    import torch.distributed as dist

    import oracle
    import synth
    from paper_2002_08014_gb300 import binding as B

    rank, world, local = _dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    c, A, sizes, Y0, sched = _workload(rank, args.rows)
    _timed.y0 = Y0
    parts = synth.split_rows(A, sizes)
    k, d = c["k"], c["d"]
    stream = torch.cuda.Stream(device=dev)
    hbm_peak, sm_max_mhz, peak_src = _peaks()
    alu_peak = 152 * 128 * 2 * sm_max_mhz * 1e6 / 1e12      # FP32 FMA lanes x 2 flop x max SM clock
    want_acc = rank == 0 and not args.no_accuracy

    def run_path(data, dtype, elem_bytes, agg=None):
        agg = agg or args.agg
        lpx = B.LocalPower(data, dtype=dtype, device=local, stream=stream)
        for _ in range(args.warmup):
            lpx.submit(k, sched, agg, Y0, ritz=True, timing=True)
            lpx.result(k)
        ms, stats, Z, sig, clk = _timed(torch, dist, world, dev, stream, lpx, k, sched, agg, args.steps,
                                        Clocks(local))
        summ = _summary(world, args.steps, ms, stats, elem_bytes, c)
        ztrace = None
        if want_acc:  # one traced solve outside the timed region: Z_t after every round
            B.lp_solve(lpx.ctx, k, sched, agg, Y0, 0, B.LP_FLAG_TRACE)
            lpx.result(k)
            ztrace, _ = B.lp_trace(lpx.ctx, len(sched), d, k)
        lpx.close()
        return summ, Z, sig, clk, ztrace

    # ---------------- headline: FP32 data as hi/lo planes on the tensor cores
    hl, Z, sig, clk, tr_hl = run_path(parts, "f32_bf16x2", 4)
    gbs_hl = hl["launch_bytes"] / (hl["step_ms"] / 1e3) / 1e9

    # ---------------- end to end through the public API, host buffers (pinned)
    # Every step loads the FP32 matrix from pinned host memory (lp_load_partitions
    # splits it into planes on the device), solves and reads the result back.  Two
    # contexts alternate, so step i+1's host-to-device copy overlaps step i's solve.
    e2e = None
    if args.e2e_steps > 0:
        pinned = torch.from_numpy(A).pin_memory()
        host_parts = [t.numpy() for t in torch.split(pinned, sizes)]
        streams = [stream, torch.cuda.Stream(device=dev)]
        ctxs = [B.LocalPower(host_parts, dtype="f32_bf16x2", device=local, stream=st_) for st_ in streams]
        for c2 in ctxs:   # warm-up: every context has loaded and solved (graphs captured) once
            B.lp_load_partitions(c2.ctx, host_parts, "f32_bf16x2")
            c2.submit(k, sched, args.agg, Y0, ritz=True)
            c2.result(k)
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        B.lp_load_partitions(ctxs[0].ctx, host_parts, "f32_bf16x2")
        ctxs[0].submit(k, sched, args.agg, Y0, ritz=True)
        for it in range(1, args.e2e_steps):
            c2 = ctxs[it % 2]
            B.lp_load_partitions(c2.ctx, host_parts, "f32_bf16x2")  # overlaps the previous step's solve
            ctxs[(it - 1) % 2].result(k)                              # previous step's result back to the host
            c2.submit(k, sched, args.agg, Y0, ritz=True)              # solves run one after another
        ctxs[(args.e2e_steps - 1) % 2].result(k)
        torch.cuda.synchronize(dev)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        e2e_t = max_over_ranks(torch, dist, world, dev, e0.elapsed_time(e1))
        for c2 in ctxs:
            c2.close()
        del pinned, host_parts
        e2e = {"value": job_throughput(world, args.e2e_steps, hl["bytes_solve"], e2e_t)[0], "unit": "GB/s",
               "h2d_bytes_per_step": int(A.nbytes + Y0.nbytes), "d2h_bytes_per_step": int(d * k * 8 + 8 * k),
               "ms_per_step": e2e_t / args.e2e_steps, "steps": args.e2e_steps,
               "pipelining": "two contexts: step i+1's host-to-device copy (FP32, split into planes on the "
                             "device) overlaps step i's solve; solves in sequence"}

    # ---------------- the headline path with the other aligner (the workload runs both)
    other = "opt" if args.agg == "sign" else "sign"
    ho, Zo, sigo, clko, tr_o = run_path(parts, "f32_bf16x2", 4, agg=other)

    # ---------------- the plain FP32 path (SIMT FP32 step) and the BF16 copy
    f32, Zf, sigf, clkf, tr_f = run_path(parts, "f32", 4)
    Zb = None
    if not args.no_bf16:
        bits = [synth.f32_to_bf16_bits(p) for p in parts]
        b16, Zb, sigb, clkb, tr_b = run_path(bits, "bf16", 2)
        del bits
    achieved_tf = f32["launch_flops"] / (f32["step_ms"] / 1e3) / 1e12
    gbs_f = f32["launch_bytes"] / (f32["step_ms"] / 1e3) / 1e9

    line = {"metric": METRIC, "value": hl["gbs"], "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": hl["ms_per_solve"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 data as bf16 hi/lo planes, bf16 x bf16 products, f32 accumulation",
            "data": "synthetic", "config": _config(c, sched),
            "solves_per_s": hl["solves_per_s"], "latency_ms": hl["latency_ms"], "clocks": clk,
            "gpu_launches": hl["launches"], "e2e": e2e,
            "roofline": {"kernel": _kernel(hl["path"], "bf16", c["d"], c["k"]), "bound": "hbm",
                         "achieved": gbs_hl, "peak": hbm_peak, "unit": "GB/s", "frac": gbs_hl / hbm_peak,
                         "traffic": _traffic(hl["path"], 2, None, hl["launch_bytes"]),
                         "traffic_unit": "bytes per launch", "launch_ms": hl["step_ms"],
                         "algorithmic_bytes_per_launch": hl["launch_bytes"],
                         "peak_source": f"{peak_src} HBM copy bandwidth", "frac_of_nominal_8000": gbs_hl / 8000.0},
            "speedup_solves_vs_plain_fp32": hl["solves_per_s"] / f32["solves_per_s"],
            "other_aggregator": {"aggregator": other, "solves_per_s": ho["solves_per_s"],
                                 "ms_per_solve": ho["ms_per_solve"], "latency_ms": ho["latency_ms"],
                                 "step_launch_ms": ho["step_ms"], "clocks": clko, "gpu_launches": ho["launches"]},
            "plain_fp32_path": {
                "dtype": "f32", "step_kernel": _kernel(f32["path"], "f32", c["d"], c["k"]), "gbs": f32["gbs"],
                "solves_per_s": f32["solves_per_s"], "ms_per_solve": f32["ms_per_solve"],
                "latency_ms": f32["latency_ms"], "clocks": clkf, "gpu_launches": f32["launches"],
                "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": alu_peak, "unit": "TFLOP/s",
                             "frac": achieved_tf / alu_peak, "launch_ms": f32["step_ms"],
                             "peak_source": f"derived: 152 SMs x 128 FP32 lanes x 2 flop x {sm_max_mhz:.0f} MHz",
                             "hbm_frac": gbs_f / hbm_peak,
                             "traffic": _traffic(0, 0, None, f32["launch_bytes"])}}}
    if Zb is not None:
        gbs_b = b16["launch_bytes"] / (b16["step_ms"] / 1e3) / 1e9
        line["precision_path"] = {
            "dtype": "bf16 storage, bf16 x bf16 products (Z and W as hi/lo pairs), f32 accumulation",
            "step_kernel": KERNELS[b16["path"]], "gbs": b16["gbs"],
            "solves_per_s": b16["solves_per_s"], "ms_per_solve": b16["ms_per_solve"],
            "latency_ms": b16["latency_ms"], "clocks": clkb, "gpu_launches": b16["launches"],
            "speedup_solves_vs_plain_fp32": b16["solves_per_s"] / f32["solves_per_s"],
            "roofline": {"bound": "hbm", "achieved": gbs_b, "peak": hbm_peak, "unit": "GB/s",
                         "frac": gbs_b / hbm_peak, "traffic": _traffic(b16["path"], 1, None, b16["launch_bytes"]),
                         "traffic_unit": "bytes per launch", "launch_ms": b16["step_ms"],
                         "peak_source": f"{peak_src} HBM copy bandwidth"}}

    if want_acc:
        V, lam = _truth(parts, c)

        def acc_of(Zx, sigx, trace):
            dists = [oracle.subspace_dist(oracle.orth(z), V) for z in trace] if trace is not None else []
            first = next((t + 1 for t, x in enumerate(dists) if x <= 1e-4), None)
            dist_ = oracle.subspace_dist(oracle.orth(Zx), V)
            return {"dist_to_eigh_topk": dist_, "target": 1e-4, "met": bool(dist_ <= 1e-4),
                    "rounds_to_1e-4": first, "local_steps_to_1e-4": (sum(sched[:first]) if first else None),
                    "dist_every_10_rounds": [dists[t] for t in range(9, len(dists), 10)],
                    "sigma_rel_err": float(np.max(np.abs(sigx - np.sqrt(c["n"] * lam)) / np.sqrt(c["n"] * lam)))}
        line["accuracy"] = acc_of(Z, sig, tr_hl)
        line["accuracy"]["dist_to_plain_fp32_output"] = oracle.subspace_dist(oracle.orth(Z), oracle.orth(Zf))
        line["plain_fp32_path"]["accuracy"] = acc_of(Zf, sigf, tr_f)
        line["other_aggregator"]["accuracy"] = acc_of(Zo, sigo, tr_o)
        if Zb is not None:
            line["precision_path"]["accuracy"] = acc_of(Zb, sigb, tr_b)
            line["precision_path"]["accuracy"]["dist_to_plain_fp32_output"] = oracle.subspace_dist(
                oracle.orth(Zb), oracle.orth(Zf))
    if rank == 0 and not args.no_cpu_baseline:
        gbs, dt = _oracle_sample_gbps(parts, Y0, 3)
        one = _oracle_one_thread_gbps(parts[:4], Y0)
        line["cpu_baseline"] = {"value": gbs, "unit": "GB/s", "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"3 FP64 oracle local power steps (eq. (2)) over all 64 partitions "
                                          f"({dt:.1f} s)",
                                "one_thread_gbs": one,
                                "one_thread_sample": "one FP64 oracle local power step over 4 partitions, "
                                                     "BLAS limited to one thread",
                                **_cpu_info()}
    if rank == 0:
        _emit(line)
    if world > 1:
        dist.destroy_process_group()

if __name__ == "__main__":
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "lowprec":
        run_lowprec(a)
    elif a.workload == "plain":
        run_plain(a)
    elif a.workload == "serving":
        run_serving(a)
    elif a.workload == "kernels":
        run_kernels(a)
    elif a.workload == "batching":
        run_batching(a)
    elif a.workload == "rounds":
        run_rounds(a)
    else:
        run_ours(a)
