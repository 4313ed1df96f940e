#!/usr/bin/env python
"""Benchmark of the LocalPower hot path on GB300.

One "step" is one complete LocalPower solve of the FP32 workload (n = 1,000,000
rows, d = 1,024, k = 16, m = 64 row partitions, p decaying 8 -> 4 -> 2 -> 1 over
10 rounds each, sign-fixing, then a Rayleigh-Ritz pass): 40 aggregations, 150
local power steps and one Ritz pass, each pass streaming all of A (4.1 GB) from
HBM.  The metric is algorithmic GB/s of A streamed; solves/s and per-solve
latency percentiles ride along.

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
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-bf16", action="store_true", help="skip the BF16-storage (tensor-core) run of the workload")
    ap.add_argument("--workload", choices=["fp32", "lowprec"], default="fp32",
                    help="fp32: the FP32 workload (default, with its BF16-storage run alongside); "
                         "lowprec: the BF16-storage workload n=4e6, d=2048, k=32")
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


def _workload(rank: int, rows: int | None = None, name: str = WORKLOAD):
    import synth
    c = dict(synth.CONFIGS[name])
    if rows:
        c["n"] = int(rows)
    A, sizes, Y0 = synth.make_config_data(name, n=c["n"])
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
    print(json.dumps(line))


def _config(c, sched, name: str = WORKLOAD):
    if name == "lowprec":
        text = (f"LocalPower BF16 storage: n={c['n']:,} d={c['d']} k={c['k']} m={c['m']}, p=4 x30 rounds + 3 "
                f"FP32-accumulated p=1 refinement rounds ({sum(sched)} local steps) + Rayleigh-Ritz pass")
        size = f"A is {c['n'] * c['d'] * 2 / 1e9:.1f} GB BF16"
    else:
        text = (f"LocalPower FP32: n={c['n']:,} d={c['d']} k={c['k']} m={c['m']}, p=8,4,2,1 x10 rounds "
                f"(T={len(sched)}, {sum(sched)} local steps) + Rayleigh-Ritz pass")
        size = f"A is {c['n'] * c['d'] * 4 / 1e9:.1f} GB FP32"
    return {"workload": text, "n": c["n"], "d": c["d"], "k": c["k"], "m": c["m"], "rounds": len(sched),
            "local_steps": sum(sched), "l2": f"inputs larger than L2 ({size}; L2 is 129 MB)"}


def run_lowprec(args):
    """The low-precision workload (BF16 storage) on the tensor-core path alone."""
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
    for _ in range(args.warmup):
        lpb.submit(k, sched, args.agg, Y0, ritz=True, timing=True)
        lpb.result(k)
    ms, stats, Z, sig, clk = _timed(torch, dist, world, dev, stream, lpb, k, sched, args.agg, args.steps,
                                    Clocks(local))
    s = _summary(world, args.steps, ms, stats, 2, c)
    lpb.close()
    gbs_k = s["launch_bytes"] / (s["step_ms"] / 1e3) / 1e9
    line = {"metric": METRIC, "value": s["gbs"], "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": s["ms_per_solve"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic", "config": _config(c, sched, "lowprec"),
            "solves_per_s": s["solves_per_s"], "latency_ms": s["latency_ms"], "clocks": clk,
            "gpu_launches": s["launches"], "e2e": None,
            "roofline": {"kernel": "step_tc_kernel (tcgen05, BF16 A, hi/lo BF16 Z and W)", "bound": "hbm",
                         "achieved": gbs_k, "peak": hbm_peak, "unit": "GB/s", "frac": gbs_k / hbm_peak,
                         "traffic": None, "launch_ms": s["step_ms"], "peak_source": f"{peak_src} HBM copy bandwidth"}}
    line["orthonormality"] = float(np.abs(Z.T @ Z - np.eye(k)).max())
    line["sigma_top3"] = [float(x) for x in sig[:3]]
    if rank == 0 and not args.no_accuracy and c["n"] * d <= 2_200_000_000:
        # truth of the decoded BF16 problem (the matrix the solver is given) and of the FP32 original;
        # forming M in FP64 on the host is skipped above about the FP32 workload's size
        dec = [oracle.decode_bf16(b) for b in bits]
        Vb, _ = _truth(dec, c)
        Vf, _ = _truth(parts, c)
        line["accuracy"] = {"dist_to_eigh_topk_bf16_problem": oracle.subspace_dist(oracle.orth(Z), Vb),
                            "dist_to_eigh_topk_fp32_problem": oracle.subspace_dist(oracle.orth(Z), Vf),
                            "quantisation_shift": oracle.subspace_dist(Vb, Vf)}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def _timed(torch, dist, world, dev, stream, lp, k, sched, agg, steps, clocks=None):
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
        lp.submit(k, sched, agg, _timed.y0, ritz=True, timing=True)
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


def _truth(parts, c):
    """Top-k eigenvectors / eigenvalues of M = A^T A / n (FP64, on the host)."""
    M = np.zeros((c["d"], c["d"]))
    for i in range(0, len(parts), 8):
        blk = np.concatenate(parts[i:i + 8]).astype(np.float64)
        M += blk.T @ blk
    lam, V = np.linalg.eigh(M / c["n"])
    return V[:, ::-1][:, :c["k"]], lam[::-1][:c["k"]]


def run_ours(args):
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

    # ---------------- plain FP32 path: device-resident timed region
    lp = B.LocalPower(parts, device=local, stream=stream)
    for _ in range(args.warmup):
        lp.submit(k, sched, args.agg, Y0, ritz=True, timing=True)
        lp.result(k)
    ms, stats, Z, sig, clk = _timed(torch, dist, world, dev, stream, lp, k, sched, args.agg, args.steps,
                                    Clocks(local))
    f32 = _summary(world, args.steps, ms, stats, 4, c)
    achieved_tf = f32["launch_flops"] / (f32["step_ms"] / 1e3) / 1e12
    achieved_gbs = f32["launch_bytes"] / (f32["step_ms"] / 1e3) / 1e9

    # ---------------- end to end through the public API, host buffers (pinned)
    e2e_ms = []
    if args.e2e_steps > 0:
        pinned = torch.from_numpy(A).pin_memory()
        host_parts = [t.numpy() for t in torch.split(pinned, sizes)]
        for it in range(args.e2e_steps + 1):
            torch.cuda.synchronize(dev)
            if world > 1:
                dist.barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.lp_load_partitions(lp.ctx, host_parts, "f32")
            lp.submit(k, sched, args.agg, Y0, ritz=True)
            lp.result(k)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            if it > 0:   # the first is a warm-up
                e2e_ms.append(e0.elapsed_time(e1))
        del pinned, host_parts
    e2e = None
    if e2e_ms:
        e2e_t = max_over_ranks(torch, dist, world, dev, max(e2e_ms))
        e2e = {"value": job_throughput(world, 1, f32["bytes_solve"], e2e_t)[0], "unit": "GB/s",
               "h2d_bytes_per_step": int(A.nbytes + Y0.nbytes), "d2h_bytes_per_step": int(d * k * 8 + 8 * k),
               "ms_per_step": e2e_t}
    lp.close()

    line = {"metric": METRIC, "value": f32["gbs"], "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": f32["ms_per_solve"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": _config(c, sched),
            "solves_per_s": f32["solves_per_s"], "latency_ms": f32["latency_ms"], "clocks": clk,
            "gpu_launches": f32["launches"], "e2e": e2e,
            "roofline": {"kernel": "step_simt_kernel (fused A_i^T (A_i Z_i), FP32)", "bound": "alu",
                         "achieved": achieved_tf, "peak": alu_peak, "unit": "TFLOP/s", "frac": achieved_tf / alu_peak,
                         "traffic": None, "launch_ms": f32["step_ms"],
                         "peak_source": f"derived: 152 SMs x 128 FP32 lanes x 2 flop x {sm_max_mhz:.0f} MHz"},
            "roofline_hbm": {"achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                             "frac": achieved_gbs / hbm_peak, "peak_source": f"{peak_src} HBM copy bandwidth",
                             "frac_of_nominal_8000": achieved_gbs / 8000.0}}

    # ---------------- the same workload stored in BF16 (tensor-core step kernel)
    Zb = None
    if not args.no_bf16:
        bits = [synth.f32_to_bf16_bits(p) for p in parts]
        lpb = B.LocalPower(bits, dtype="bf16", device=local, stream=stream)
        for _ in range(args.warmup):
            lpb.submit(k, sched, args.agg, Y0, ritz=True, timing=True)
            lpb.result(k)
        msb, statsb, Zb, sigb, clkb = _timed(torch, dist, world, dev, stream, lpb, k, sched, args.agg, args.steps,
                                             Clocks(local))
        b16 = _summary(world, args.steps, msb, statsb, 2, c)
        lpb.close()
        gbs_b = b16["launch_bytes"] / (b16["step_ms"] / 1e3) / 1e9
        line["precision_path"] = {
            "dtype": "bf16 storage, FP32 accumulation (hi/lo BF16 operands)", "step_kernel":
            "step_tc_kernel (tcgen05)" if b16["path"] == 1 else "step_simt_kernel", "gbs": b16["gbs"],
            "solves_per_s": b16["solves_per_s"], "ms_per_solve": b16["ms_per_solve"],
            "latency_ms": b16["latency_ms"], "clocks": clkb, "gpu_launches": b16["launches"],
            "speedup_solves_vs_fp32": b16["solves_per_s"] / f32["solves_per_s"],
            "roofline": {"bound": "hbm", "achieved": gbs_b, "peak": hbm_peak, "unit": "GB/s",
                         "frac": gbs_b / hbm_peak, "traffic": None, "launch_ms": b16["step_ms"],
                         "peak_source": f"{peak_src} HBM copy bandwidth"}}

    if rank == 0 and not args.no_accuracy:
        V, lam = _truth(parts, c)
        acc = {"dist_to_eigh_topk": oracle.subspace_dist(oracle.orth(Z), V),
               "orthonormality": float(np.abs(Z.T @ Z - np.eye(k)).max()),
               "sigma_rel_err": float(np.max(np.abs(sig - np.sqrt(c["n"] * lam)) / np.sqrt(c["n"] * lam)))}
        line["accuracy"] = acc
        if Zb is not None:
            line["precision_path"]["accuracy"] = {
                "dist_to_eigh_topk_of_fp32_problem": oracle.subspace_dist(oracle.orth(Zb), V),
                "dist_to_fp32_path_output": oracle.subspace_dist(oracle.orth(Zb), oracle.orth(Z))}
    if rank == 0 and not args.no_cpu_baseline:
        gbs, dt = _oracle_sample_gbps(parts, Y0, 3)
        line["cpu_baseline"] = {"value": gbs, "unit": "GB/s", "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"3 FP64 oracle local power steps (eq. (2)) over all 64 partitions "
                                          f"({dt:.1f} s)"}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "lowprec":
        run_lowprec(a)
    else:
        run_ours(a)
