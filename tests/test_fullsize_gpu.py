"""The benchmark's workloads at full size against the FP64 oracle, through the
C ABI, in the launch configurations the benchmark times.

  * FP32 workload (n = 1,000,000, d = 1,024, k = 16, m = 64, 4.1 GB): one power
    step element-wise on sampled partitions and as the aggregate sum_i p_i Y_i
    over all of them, for the plain FP32 path (SIMT) and the headline path (the
    FP32 data as hi/lo BF16 planes on the tensor cores); then the whole 50-round
    solve (160 local steps) against the oracle's own whole solve, both
    aggregators, both paths, at the FP32 bar of 1e-6 in subspace distance.
  * Precision workload (d = 2,048, k = 32, BF16 or FP8-E4M3, p = 4 x 30 + 3
    refinement rounds): the whole solve on 8 of its 128 partitions (31,250 rows
    each, the workload's partition size; the oracle would need 65 GB for all
    128) against the oracle on the decoded values, at the reduced-precision bar
    of 1e-4, with the k x k work in FP64 (as the workload states) and in FP32.

These tests take minutes (the oracle's whole FP32-workload solve is ~160 FP64
passes over 8 GB)."""
import numpy as np
import pytest

import oracle as O
import synth
from paper_2002_08014_gb300 import binding as B

pytestmark = pytest.mark.gpu

FP32_SOLVE_TOL = 1e-6
TC_SOLVE_TOL = 1e-4


@pytest.fixture(scope="module")
def fp32_workload():
    A, sizes, Y0 = synth.make_config_data("fp32", threads=16)
    parts = synth.split_rows(A, sizes)
    return parts, sizes, Y0, synth.config_schedule("fp32")


def _elementwise_ok(Y, ref, P, Z, c):
    a = O.as_f64(P)
    bound = c * (np.abs(a).T @ (np.abs(a) @ np.abs(Z))) / a.shape[0]
    return bool((np.abs(Y - ref) <= bound).all())


def test_fp32_workload_step_elementwise_and_aggregate(gpu_lib, fp32_workload):
    parts, sizes, Y0, _ = fp32_workload
    Z = O.orth(Y0)
    w = O.weights(sizes)
    MZ = sum(w[i] * O.local_step(P, Z) for i, P in enumerate(parts))   # (1/n) sum_i A_i^T A_i Z
    for dtype in ("f32", "f32_bf16x2"):
        with B.LocalPower(parts, dtype=dtype) as lp:
            Y = lp.power_step(16, Z, shared=True)
        for i in (0, 31, 63):
            if dtype == "f32":
                P = parts[i]
            else:  # the oracle runs on the stored planes, hi + lo
                hi, lo = synth.f32_to_bf16x2_planes(parts[i])
                P = O.decode_bf16(hi) + O.decode_bf16(lo)
            ref = O.local_step(P, Z)
            if dtype == "f32":
                # FP32 FMAs over d then s_i terms: well inside 1e-5 of each entry's absolute sum
                assert _elementwise_ok(Y[i], ref, P, Z, 1e-5), i
            else:
                # tensor cores: a common round-toward-zero scale first (<= one ulp per MMA of the
                # longest chain), then the hi/lo split bound of Z and W on each entry
                alpha = float(np.vdot(Y[i], ref) / np.vdot(Y[i], Y[i]))
                assert 0.0 <= alpha - 1.0 <= 600 * 2.0 ** -23, (i, alpha)
                assert _elementwise_ok(alpha * Y[i], ref, P, Z, 2e-5), i
        agg = sum(w[i] * Y[i] for i in range(len(sizes)))
        rel = np.linalg.norm(agg - MZ) / np.linalg.norm(MZ)
        # the planes differ from the FP32 data by up to 2^-17 per element
        assert rel < (2e-6 if dtype == "f32" else 2e-5), (dtype, rel)


@pytest.mark.parametrize("agg", ["sign", "opt"])
def test_fp32_workload_whole_solve_matches_oracle(gpu_lib, fp32_workload, agg):
    parts, sizes, Y0, sched = fp32_workload
    ref = O.localpower(parts, 16, sched, agg, Y0)["Z"]
    got = {}
    for dtype in ("f32", "f32_bf16x2"):
        with B.LocalPower(parts, dtype=dtype) as lp:
            Z, _, st = lp.solve(16, sched, agg, Y0)
        got[dtype] = (O.subspace_dist(Z, ref), st["path"])
    print(f"full-size FP32 workload, {agg}: dist to the oracle's solve {got}")
    for dtype, (dist, _) in got.items():
        assert dist < FP32_SOLVE_TOL, (dtype, dist)


@pytest.mark.parametrize("dtype,agg", [("bf16", "sign"), ("bf16", "opt"), ("e4m3", "sign")])
def test_precision_workload_subset_whole_solve(gpu_lib, dtype, agg):
    A, _, Y0 = synth.make_config_data("lowprec", n=8 * 31_250, m=8, threads=16)
    sizes = [31_250] * 8
    parts = synth.split_rows(A, sizes)
    del A
    if dtype == "bf16":
        stored = [synth.f32_to_bf16_bits(p) for p in parts]
        exact, scales = [("bf16", b) for b in stored], None
    else:
        stored, scales = map(list, zip(*[synth.f32_to_e4m3_rowscaled(p) for p in parts]))
        exact = [("e4m3", c, s) for c, s in zip(stored, scales)]
    del parts
    sched = synth.config_schedule("lowprec")        # p = 4 x 30, then 3 rounds at p = 1
    ref = O.localpower(exact, 32, sched, agg, Y0)["Z"]
    with B.LocalPower(stored, dtype=dtype, row_scales=scales) as lp:
        B.lp_autotune(lp.ctx, 32)
        # the workload's k x k arithmetic (FP64 Gram/Cholesky and Procrustes SVD), then the default
        Z64, _, st = lp.solve(32, sched[:30], agg, Y0, refine_rounds=3, kxk_fp64=True)
        Z32, _, _ = lp.solve(32, sched[:30], agg, Y0, refine_rounds=3)
    d64, d32 = O.subspace_dist(Z64, ref), O.subspace_dist(Z32, ref)
    print(f"precision workload ({dtype}, {agg}), 8 of 128 partitions: dist to the oracle's solve "
          f"{d64:.3e} with FP64 k x k, {d32:.3e} with FP32 k x k (path {st['path']})")
    assert d64 < TC_SOLVE_TOL and d32 < TC_SOLVE_TOL, (d64, d32)
