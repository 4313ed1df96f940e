"""Parity of the CUDA path with the FP64 oracle, one kernel at a time and end to
end, through the C ABI.  Inputs are seeded synthetic data; the oracle runs on
the exact values of the stored bytes.

Tolerances (the arithmetic is FP32 with FP64 k x k factorisations):
  * one power step: ||Y_gpu - Y_ref||_F <= 2e-6 ||Y_ref||_F (FP32 accumulation
    over s_i + d terms, u = 6e-8);
  * orth: ||Z^T Z - I|| <= 1e-5, columns equal to the oracle's (same diag(R) > 0
    convention) within 2e-5;
  * whole solves: subspace distance to the oracle's output <= 1e-6 (FP32 path).
"""
import numpy as np
import pytest

import oracle as O
import synth
from paper_2002_08014_gb300 import binding as B

pytestmark = pytest.mark.gpu

# BF16-stored A runs on the tensor cores with Z and W split into BF16 hi + lo
# parts (each split leaves at most 2^-18 relative error), FP32 accumulation.
# One step is checked at 1e-5; whole solves at the reduced-precision bar of
# 1e-4 in subspace distance.
TC_STEP_TOL = 1e-5
TC_SOLVE_TOL = 1e-4
# Path codes of lp_stats.path.
SIMT, TC_RESIDENT, TC_STREAM, TC_PAIR = 0, 1, 2, 3


def _decode_planes(hi, lo):
    return O.decode_bf16(hi) + O.decode_bf16(lo)


def _parts(sizes, d, seed, dtype="f32", spikes=40):
    # lam_j = 10 * 0.9^j: a relative eigengap of about 10% at every k <= 32, so
    # the top-k subspace is well defined (a noise-level gap would make any
    # rounding difference look like a parity failure).
    n = sum(sizes)
    lam = 10.0 * 0.9 ** np.arange(1, min(spikes, d) + 1)
    A = synth.spiked_rows(n, d, lam, 0.3, seed, threads=4)
    A32 = synth.split_rows(A, sizes)
    if dtype == "f32":
        return A32, A32, None
    if dtype == "bf16":
        bits = [synth.f32_to_bf16_bits(a) for a in A32]
        return bits, [("bf16", b) for b in bits], None
    if dtype == "f32_bf16x2":
        # the caller hands FP32; the oracle runs on the stored hi + lo planes
        planes = [synth.f32_to_bf16x2_planes(a) for a in A32]
        return A32, [_decode_planes(h, l) for h, l in planes], None
    codes, scales = [], []
    for a in A32:
        c, s = synth.f32_to_e4m3_rowscaled(a)
        codes.append(c)
        scales.append(s)
    return codes, [("e4m3", c, s) for c, s in zip(codes, scales)], scales


def _relF(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "e4m3", "f32_bf16x2"])
@pytest.mark.parametrize("sizes,d,k", [
    ([37, 64, 21], 100, 5),            # ragged tiles, d not a multiple of 16
    ([500, 333, 129, 700], 257, 16),   # d just over a 256-column block
    ([96, 96], 1024, 16),              # widest SIMT column count
    ([40, 41, 42], 64, 32),            # k = 32
    ([20], 7, 1),                      # tiny d, k = 1
    ([300, 29], 512, 24),              # k padded to 32, partition of 29 rows
    ([13] * 40 + [600], 200, 12),      # many tiny partitions: CTAs restage Z_i often (k padded to 16)
    ([12, 15, 16, 17, 33, 500], 1024, 12),  # d = 1024 pipelined kernel: ragged last tiles, short segments
    ([37] * 30 + [2000], 1024, 16),    # d = 1024: many partitions per CTA, Z_i restaged in TMEM
])
def test_power_step_matches_oracle(gpu_lib, dtype, sizes, d, k):
    stored, exact, scales = _parts(sizes, d, 100 + d + k, dtype)
    rng = np.random.default_rng(1)
    Z = O.orth(rng.standard_normal((d, k)))
    tol = TC_STEP_TOL if dtype in ("bf16", "f32_bf16x2", "e4m3") else 2e-6
    with B.LocalPower(stored, dtype=dtype, row_scales=scales) as lp:
        Y = lp.power_step(k, Z, shared=True)
        for i, P in enumerate(exact):
            ref = O.local_step(P, Z)
            assert _relF(Y[i], ref) < tol, (i, _relF(Y[i], ref))
        # per-partition bases
        Zs = np.stack([O.orth(rng.standard_normal((d, k))) for _ in sizes])
        Y2 = B.lp_power_step(lp.ctx, k, Zs, False, len(sizes), d)
        for i, P in enumerate(exact):
            assert _relF(Y2[i], O.local_step(P, Zs[i])) < tol


@pytest.mark.parametrize("d,k,batch", [(100, 5, 3), (1024, 16, 4), (257, 32, 2), (9, 1, 5), (2048, 32, 1)])
def test_orth_matches_oracle(gpu_lib, d, k, batch):
    rng = np.random.default_rng(d + k)
    Y = rng.standard_normal((batch, d, k)) @ np.diag(np.linspace(1.0, 30.0, k))
    ctx = B.lp_create(0)
    try:
        Z = B.lp_orth(ctx, Y)
    finally:
        B.lp_destroy(ctx)
    for b in range(batch):
        assert np.abs(Z[b].T @ Z[b] - np.eye(k)).max() < 1e-5
        ref = O.orth(Y[b])
        assert np.abs(Z[b] - ref).max() < 2e-5
        assert O.subspace_dist(Z[b], ref) < 1e-6


def test_orth_reports_rank_deficiency(gpu_lib):
    Y = np.zeros((1, 50, 4))
    Y[0, :, :3] = np.random.default_rng(0).standard_normal((50, 3))
    ctx = B.lp_create(0)
    try:
        with pytest.raises(B.LPError) as e:
            B.lp_orth(ctx, Y)
        assert e.value.status == B.LP_ERR_NUMERIC
    finally:
        B.lp_destroy(ctx)


@pytest.mark.parametrize("agg", ["identity", "sign", "opt"])
@pytest.mark.parametrize("d,k,m,base", [(100, 5, 4, 0), (513, 16, 7, 3), (64, 32, 3, 2), (30, 1, 5, 4),
                                        # odd k next to the column padding (a dummy column in the
                                        # Jacobi's round-robin pairing), 16 partition slices with a
                                        # ragged last pass, a single partition, the FP32 workload's shape
                                        (257, 13, 20, 19), (40, 31, 17, 0), (16, 3, 1, 0), (1024, 16, 64, 5)])
def test_align_aggregate_matches_oracle(gpu_lib, agg, d, k, m, base):
    rng = np.random.default_rng(7 * d + k)
    Zb = O.orth(rng.standard_normal((d, k)))
    Zs, Ys = [], []
    for i in range(m):
        Q = O.orth(rng.standard_normal((k, k)))
        S = np.diag(rng.choice([-1.0, 1.0], size=k))
        Zi = O.orth(Zb @ (Q if agg == "opt" else S) + 0.05 * rng.standard_normal((d, k)))
        Zs.append(Zi)
        Ys.append(Zi @ np.diag(np.linspace(3, 1, k)) + 0.01 * rng.standard_normal((d, k)))
    Zs[base] = Zb
    sizes = [100] * m
    sizes[base] = 150
    w = np.array(sizes, float) / sum(sizes)
    ctx = B.lp_create(0)
    try:
        Y, D = B.lp_align_aggregate(ctx, agg, base, w, np.stack(Ys), np.stack(Zs))
    finally:
        B.lp_destroy(ctx)
    ref = O.aggregate(Ys, Zs, sizes, agg)
    assert _relF(Y, ref) < 5e-6
    for i in range(m):
        Dref = np.eye(k) if i == base else O.align(agg, Zs[i], Zb)
        if agg == "sign":
            assert np.array_equal(D[i], Dref)          # the +-1 decisions are exact
        else:
            assert np.abs(D[i] - Dref).max() < 1e-5
            assert np.abs(D[i].T @ D[i] - np.eye(k)).max() < 1e-5


@pytest.mark.parametrize("agg", ["sign", "opt", "identity"])
def test_plain_config_end_to_end(gpu_lib, agg):
    """The plain workload: n=4,000, d=100, k=5, m=4, p=4, T=20."""
    c = synth.CONFIGS["plain"]
    A, sizes, Y0 = synth.make_config_data("plain")
    parts = synth.split_rows(A, sizes)
    ref = O.localpower(parts, c["k"], c["schedule"], agg, Y0)
    with B.LocalPower(parts) as lp:
        Z, sig, st = lp.solve(c["k"], c["schedule"], agg, Y0, ritz=True)
    assert O.subspace_dist(Z, ref["Z"]) < 1e-6
    assert st["rounds"] == 20 and st["local_steps"] == 80 and st["step_launches"] == 81
    Zr, sr = O.ritz(parts, ref["Z"])
    assert np.allclose(sig, sr, rtol=1e-6)
    for j in range(c["k"]):
        assert abs(abs(Z[:, j] @ Zr[:, j]) - 1.0) < 1e-5
    assert np.abs(Z.T @ Z - np.eye(c["k"])).max() < 1e-5


@pytest.mark.parametrize("agg", ["sign", "opt"])
def test_fp32_workload_shape_decay_schedule(gpu_lib, agg):
    """The FP32 workload's shape (d=1024, k=16, m=64, spectrum 10*0.9^j) on
    64,000 rows with the 8-4-2-1 decay cut to 2 rounds per level."""
    A, sizes, Y0 = synth.make_config_data("fp32", n=64_000, m=64)
    parts = synth.split_rows(A, sizes)
    sched = [8, 8, 4, 4, 2, 2, 1, 1]
    ref = O.localpower(parts, 16, sched, agg, Y0)
    with B.LocalPower(parts) as lp:
        Z, _, st = lp.solve(16, sched, agg, Y0)
    assert O.subspace_dist(Z, ref["Z"]) < 1e-6
    assert st["rounds"] == len(sched) and st["local_steps"] == sum(sched)


@pytest.mark.parametrize("dtype,flags,path", [
    ("bf16", 0, TC_PAIR), ("bf16", B.LP_FLAG_TC_RESIDENT, TC_RESIDENT), ("bf16", B.LP_FLAG_SIMT, SIMT),
    ("e4m3", 0, TC_STREAM), ("e4m3", B.LP_FLAG_SIMT, SIMT), ("f32_bf16x2", 0, TC_PAIR)])
def test_reduced_precision_storage_end_to_end(gpu_lib, dtype, flags, path):
    """BF16 / FP8-E4M3 / split-plane stored A: the oracle runs on the decoded
    stored values.  BF16 and split planes run on the tensor cores (the pass-split
    pair kernel by default, the resident one or the SIMT kernel on request)."""
    sizes = [900, 1100, 1000, 1000]
    stored, exact, scales = _parts(sizes, 200, 55, dtype, spikes=10)
    Y0 = synth.gaussian_start(200, 8, 56)
    sched = [4] * 6 + [1] * 3
    ref = O.localpower(exact, 8, sched, "sign", Y0)
    with B.LocalPower(stored, dtype=dtype, row_scales=scales) as lp:
        B.lp_solve(lp.ctx, 8, sched, "sign", Y0, 0, flags)
        Z, _, st = lp.result(8)
    assert st["path"] == path
    assert O.subspace_dist(Z, ref["Z"]) < (TC_SOLVE_TOL if path != SIMT else 1e-6)


@pytest.mark.parametrize("d,k,sizes", [
    (1024, 16, [2500, 3100, 2601, 2399]),  # streaming: whole rows per CTA; resident: 4-CTA clusters
    (2048, 32, [640, 385]),                # streaming: 4-CTA clusters; resident: 8-CTA clusters, k = 32
    (2048, 16, [700, 1301]),               # streaming: 2-CTA clusters
    (3000, 32, [500, 260]),                # streaming: 8-CTA clusters, ragged last slice (no resident plan)
    (300, 5, [129, 2000, 77]),             # resident: 2-CTA clusters, last slice mostly past d
    (100, 8, [260, 140]),                  # one CTA, two 64-column chunks
    (513, 13, [3000]),                     # one partition, ragged everything
])
def test_tensor_core_step_shapes(gpu_lib, d, k, sizes):
    stored, exact, _ = _parts(sizes, d, 7 * d + k, "bf16")
    rng = np.random.default_rng(d)
    Zs = np.stack([O.orth(rng.standard_normal((d, k))) for _ in sizes])
    Y0 = synth.gaussian_start(d, k, 3)
    sched = [4, 4, 2, 1]
    got = {}
    with B.LocalPower(stored, dtype="bf16") as lp:
        Y = B.lp_power_step(lp.ctx, k, Zs, False, len(sizes), d)
        for i, P in enumerate(exact):
            assert _relF(Y[i], O.local_step(P, Zs[i])) < TC_STEP_TOL, (i, _relF(Y[i], O.local_step(P, Zs[i])))
        # whether the pair kernel has a plan here decides what the default runs
        B.lp_set_tuning(lp.ctx, kernel="pair")
        try:
            B.lp_power_step(lp.ctx, k, Zs, False, len(sizes), d)
            default_path = TC_PAIR
        except B.LPError as e:
            assert e.status == B.LP_ERR_UNSUPPORTED
            default_path = TC_STREAM
        # the whole solve on every tensor-core kernel (and the SIMT kernel where it exists)
        runs = [("default", 0, default_path), ("stream", 0, TC_STREAM)]
        if default_path == TC_PAIR:
            runs.append(("pair", 0, TC_PAIR))
        if d <= 2048:
            runs.append(("default", B.LP_FLAG_TC_RESIDENT, TC_RESIDENT))
        if d <= 1024:
            runs.append(("default", B.LP_FLAG_SIMT, SIMT))
        for kern, flags, path in runs:
            B.lp_set_tuning(lp.ctx, kernel=kern)
            B.lp_solve(lp.ctx, k, sched, "opt", Y0, 0, flags)
            Z, _, st = lp.result(k)
            assert st["path"] == path
            got[path] = Z
    ref = O.localpower(exact, k, sched, "opt", Y0)
    for path, Z in got.items():
        assert O.subspace_dist(Z, ref["Z"]) < (TC_SOLVE_TOL if path != SIMT else 1e-6), path


@pytest.mark.parametrize("d,k,sizes", [
    (1024, 16, [2500, 3100, 2601, 2399]),  # whole rows per CTA, 16 ring units per tile
    (2048, 32, [6000, 4001]),              # 4-CTA clusters
    (300, 5, [129, 2000, 77]),
    (40, 3, [50, 60]),                     # one 128-column block, mostly padding
])
def test_split_plane_storage(gpu_lib, d, k, sizes):
    """FP32 data stored as hi + lo BF16 planes on the tensor cores: one step and a
    whole solve against the oracle on the stored planes, and the stored planes
    against the FP32 data within the 2^-17 representation bound."""
    A32, exact, _ = _parts(sizes, d, 11 * d + k, "f32_bf16x2")
    for a, e in zip(A32, exact):
        a64 = a.astype(np.float64)
        assert np.all(np.abs(e - a64) <= 2.0 ** -17 * np.abs(a64))
    rng = np.random.default_rng(d + 1)
    Zs = np.stack([O.orth(rng.standard_normal((d, k))) for _ in sizes])
    Y0 = synth.gaussian_start(d, k, 5)
    sched = [4, 2, 1, 1]
    with B.LocalPower(A32, dtype="f32_bf16x2") as lp:
        Y = B.lp_power_step(lp.ctx, k, Zs, False, len(sizes), d)
        for i, P in enumerate(exact):
            assert _relF(Y[i], O.local_step(P, Zs[i])) < TC_STEP_TOL, (i, _relF(Y[i], O.local_step(P, Zs[i])))
        Z, _, st = lp.solve(k, sched, "sign", Y0)
        assert st["path"] in (TC_PAIR, TC_STREAM)
        with pytest.raises(B.LPError) as e:  # no SIMT kernel reads split planes
            B.lp_solve(lp.ctx, k, sched, "sign", Y0, 0, B.LP_FLAG_SIMT)
        assert e.value.status == B.LP_ERR_UNSUPPORTED
    ref = O.localpower(exact, k, sched, "sign", Y0)
    # Z and W enter the MMAs as hi + lo BF16 pairs (<= 2^-18 relative per
    # element): the reduced-precision bar applies.  Measured 1.7e-6 at d = 1024,
    # k = 16 and 1.4e-5 at d = 2048, k = 32 (gap/||M|| five times smaller).
    assert O.subspace_dist(Z, ref["Z"]) < TC_SOLVE_TOL


def test_split_plane_device_input(gpu_lib):
    """Split-plane load from device FP32 partitions gives the same solve as from host."""
    torch = pytest.importorskip("torch")
    sizes = [700, 650]
    A32, _, _ = _parts(sizes, 96, 21, "f32_bf16x2")
    Y0 = synth.gaussian_start(96, 6, 22)
    with B.LocalPower(A32, dtype="f32_bf16x2") as lp:
        Zh, _, _ = lp.solve(6, [2, 1], "sign", Y0)
    dev = [torch.from_numpy(a).cuda() for a in A32]
    with B.LocalPower(dev, dtype="f32_bf16x2") as lp:
        Zd, _, _ = lp.solve(6, [2, 1], "sign", Y0)
    assert np.array_equal(Zh, Zd)


def test_uneven_partitions_base_not_first(gpu_lib):
    sizes = [50, 13, 400, 77, 399]
    A, _, _ = _parts(sizes, 60, 9)
    Y0 = synth.gaussian_start(60, 6, 10)
    sched = [5, 3, 2, 1]
    for agg in ("sign", "opt", "identity"):
        ref = O.localpower(A, 6, sched, agg, Y0)
        with B.LocalPower(A) as lp:
            Z, _, _ = lp.solve(6, sched, agg, Y0)
        assert O.subspace_dist(Z, ref["Z"]) < 1e-6, agg


def test_single_partition_and_refine_rounds(gpu_lib):
    A, _, _ = _parts([800], 48, 11)
    Y0 = synth.gaussian_start(48, 4, 12)
    ref = O.localpower(A, 4, [3, 3, 1, 1], "sign", Y0)
    with B.LocalPower(A) as lp:
        lp_ = lp
        B.lp_solve(lp_.ctx, 4, [3, 3], "sign", Y0, refine_rounds=2)
        Z, _, st = lp_.result(4)
    assert O.subspace_dist(Z, ref["Z"]) < 1e-6
    assert st["rounds"] == 4


def test_invalid_arguments_and_state(gpu_lib):
    A, _, _ = _parts([30, 40], 20, 13)
    ctx = B.lp_create(0)
    try:
        with pytest.raises(B.LPError) as e:
            B.lp_solve(ctx, 4, [2], "sign", np.zeros((20, 4)))
        assert e.value.status == B.LP_ERR_STATE
        B.lp_load_partitions(ctx, A)
        for k in (0, 31, 33):       # k > min s_i = 30, k > 32
            with pytest.raises(B.LPError) as e:
                B.lp_solve(ctx, k, [2], "sign", np.zeros((20, max(k, 1))))
            assert e.value.status == B.LP_ERR_INVALID
        with pytest.raises(B.LPError) as e:
            B.lp_solve(ctx, 4, [2, 0], "sign", np.ones((20, 4)))
        assert e.value.status == B.LP_ERR_INVALID
        with pytest.raises(B.LPError) as e:
            B.lp_result(ctx, 20, 4)
        assert e.value.status == B.LP_ERR_STATE
    finally:
        B.lp_destroy(ctx)


def test_budget_is_enforced(gpu_lib):
    A, _, _ = _parts([1000, 1000], 256, 14)
    ctx = B.lp_create(0, hbm_budget_bytes=1 << 20)
    try:
        with pytest.raises(B.LPError) as e:
            B.lp_load_partitions(ctx, A)
        assert e.value.status == B.LP_ERR_OOM
    finally:
        B.lp_destroy(ctx)


def test_nonfinite_input_is_reported(gpu_lib):
    A, _, _ = _parts([60, 60], 16, 15)
    A[1][5, 3] = np.nan
    with B.LocalPower(A) as lp:
        with pytest.raises(B.LPError) as e:
            lp.solve(4, [2, 1], "sign", synth.gaussian_start(16, 4, 1))
        assert e.value.status == B.LP_ERR_NUMERIC


def test_full_size_bf16_step_sampled(gpu_lib):
    """The precision workload at full size (n=4e6, d=2048, k=32, m=128, BF16,
    16.4 GB on the device), in the benchmark's launch configuration (the
    autotuner's choice): one power step, checked on sampled partitions against
    the oracle on the decoded BF16 values."""
    A, sizes, Y0 = synth.make_config_data("lowprec", threads=16)
    bits = [synth.f32_to_bf16_bits(p) for p in synth.split_rows(A, sizes)]
    del A
    Z = O.orth(Y0)
    with B.LocalPower(bits, dtype="bf16") as lp:
        B.lp_autotune(lp.ctx, 32)
        Y = lp.power_step(32, Z, shared=True)
    # The tensor cores round the FP32 accumulator toward zero on every MMA, so an
    # accumulation chain shrinks Y_i by a nearly uniform factor: at most one unit
    # in the last place (2^-23) per MMA that adds into an entry.  The library cuts
    # the tensor-core segments into pieces of at most 4,096 rows, so a chain is at
    # most 32 tiles x 8 MMAs in the second contraction plus d / 16 in the first.
    # A common scale does not move span(Y_i); Y_i is checked at the step bar both
    # as it is and after removing the best scale.
    for i in (0, 77, 127):
        ref = O.local_step(("bf16", bits[i]), Z)
        alpha = float(np.vdot(Y[i], ref) / np.vdot(Y[i], Y[i]))
        chain = (4096 // 128 + 1) * 8 + 2048 // 16
        assert 0.0 <= alpha - 1.0 <= chain * 2.0 ** -23, (i, alpha)
        assert _relF(alpha * Y[i], ref) < TC_STEP_TOL, (i, _relF(alpha * Y[i], ref), alpha)
        assert _relF(Y[i], ref) < TC_STEP_TOL, (i, _relF(Y[i], ref))
        # element-wise, after the common scale: within the hi/lo split bound of Z and W
        # on each entry's own dot products (|A|^T |A| |Z| / s_i)
        a = O.decode_bf16(bits[i])
        bound = 2e-5 * (np.abs(a).T @ (np.abs(a) @ np.abs(Z))) / a.shape[0]
        assert (np.abs(alpha * Y[i] - ref) <= bound).all(), i


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f32_bf16x2"])
def test_reload_same_shape_reuses_the_context(gpu_lib, dtype):
    """New data of the same shapes go into the existing buffers (tables, plans and
    the captured graph stay): the result equals a fresh context's on that data,
    and the old result is gone until the next solve."""
    sizes, d, k = [700, 500, 900], 96, 6
    A1, _, _ = _parts(sizes, d, 71, dtype)
    A2, _, _ = _parts(sizes, d, 72, dtype)
    Y0 = synth.gaussian_start(d, k, 73)
    with B.LocalPower(A1, dtype=dtype) as lp:
        lp.solve(k, [4, 2, 1], "sign", Y0)
        B.lp_load_partitions(lp.ctx, A2, dtype)
        with pytest.raises(B.LPError) as e:
            lp.result(k)
        assert e.value.status == B.LP_ERR_STATE
        Z2, _, _ = lp.solve(k, [4, 2, 1], "sign", Y0)
    with B.LocalPower(A2, dtype=dtype) as fresh:
        Zf, _, _ = fresh.solve(k, [4, 2, 1], "sign", Y0)
    assert np.array_equal(Z2, Zf)


def test_tuning_changes_speed_not_results(gpu_lib):
    """Ring depth, lag, L2 prefetch and cache hints reorder loads only: the
    streaming kernel's products and their summation order are unchanged."""
    sizes = [3000, 2500, 1777]
    stored, exact, _ = _parts(sizes, 512, 31, "bf16")
    Y0 = synth.gaussian_start(512, 16, 32)
    sched = [2, 1]
    outs = []
    with B.LocalPower(stored, dtype="bf16") as lp:
        for ring, lag, pf, hint in [(0, 0, 0, 0), (2, 1, 0, 0), (3, 4, 0, 1), (0, 2, 4, 1), (5, 3, 8, 0)]:
            B.lp_set_tuning(lp.ctx, ring, lag, pf, hint, kernel="stream")
            Z, _, st = lp.solve(16, sched, "sign", Y0)
            assert st["path"] == TC_STREAM
            outs.append(Z)
        with pytest.raises(B.LPError) as e:
            B.lp_set_tuning(lp.ctx, -1, 0, 0, 0)
        assert e.value.status == B.LP_ERR_INVALID
        B.lp_set_tuning(lp.ctx, reset=True)
    for Z in outs[1:]:
        assert np.array_equal(Z, outs[0])
    ref = O.localpower(exact, 16, sched, "sign", Y0)
    assert O.subspace_dist(outs[0], ref["Z"]) < TC_SOLVE_TOL
    # narrower column slices (a cluster splits d): another summation order, same result to the bar
    with B.LocalPower(stored, dtype="bf16") as lp:
        B.lp_set_tuning(lp.ctx, slice_cols=128, kernel="stream")
        Zs, _, st = lp.solve(16, sched, "sign", Y0)
        assert st["path"] == TC_STREAM
        with pytest.raises(B.LPError) as e:
            B.lp_set_tuning(lp.ctx, slice_cols=100)
        assert e.value.status == B.LP_ERR_INVALID
    assert O.subspace_dist(Zs, ref["Z"]) < TC_SOLVE_TOL


@pytest.mark.parametrize("dtype", ["bf16", "f32_bf16x2", "f32"])
def test_autotune_picks_a_working_kernel(gpu_lib, dtype):
    sizes = [2000, 2100]
    stored, exact, scales = _parts(sizes, 384, 41, dtype)
    Y0 = synth.gaussian_start(384, 12, 42)
    with B.LocalPower(stored, dtype=dtype, row_scales=scales) as lp:
        choice = B.lp_autotune(lp.ctx, 12)
        Z, _, st = lp.solve(12, [3, 1], "opt", Y0)
    assert st["path"] == choice["path_code"]
    if dtype == "f32":
        assert choice["path_code"] == SIMT
    else:
        assert choice["path_code"] in (TC_RESIDENT, TC_STREAM, TC_PAIR) and choice["ms_per_step"] > 0
    ref = O.localpower(exact, 12, [3, 1], "opt", Y0)
    assert O.subspace_dist(Z, ref["Z"]) < (1e-6 if dtype == "f32" else TC_SOLVE_TOL)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_graph_replay_matches_eager_launches(gpu_lib, dtype):
    """The solve's captured CUDA graph replays exactly the eager launch sequence;
    a changed schedule or aggregator is captured anew."""
    sizes = [700, 900, 650]
    stored, exact, _ = _parts(sizes, 160, 51, dtype)
    Y0 = synth.gaussian_start(160, 8, 52)
    with B.LocalPower(stored, dtype=dtype) as lp:
        runs = []
        for sched, agg in [([3, 2, 1], "sign"), ([3, 2, 1], "sign"), ([2, 2], "opt"), ([3, 2, 1], "sign")]:
            for flags in (B.LP_FLAG_RITZ | B.LP_FLAG_NO_GRAPH | B.LP_FLAG_TIMING, B.LP_FLAG_RITZ,
                          B.LP_FLAG_RITZ | B.LP_FLAG_TIMING):
                B.lp_solve(lp.ctx, 8, sched, agg, Y0, 1, flags)
                Z, sig, st = lp.result(8)
                if flags & B.LP_FLAG_TIMING:   # step events recorded eagerly and inside the graph
                    assert st["ms_step_kernels"] > 0
                runs.append((sched, agg, Z, sig, st))
    for i in range(0, len(runs), 3):
        eager, first, replay = runs[i:i + 3]
        for other in (first, replay):
            assert np.array_equal(eager[2], other[2]) and np.array_equal(eager[3], other[3])
            assert other[4]["kernel_launches"] == eager[4]["kernel_launches"]
            assert other[4]["local_steps"] == eager[4]["local_steps"]
    for sched, agg, Z, _, _ in runs[:3] + runs[6:9]:
        ref = O.localpower(exact, 8, list(sched) + [1], agg, Y0)
        assert O.subspace_dist(Z, ref["Z"]) < (1e-6 if dtype == "f32" else TC_SOLVE_TOL)


@pytest.mark.parametrize("agg", ["identity", "sign", "opt"])
def test_trace_and_residual_error_match_oracle(gpu_lib, agg):
    """LP_FLAG_TRACE: Z_t after every aggregation and rho_t (Def. 3) against the
    oracle's per-round trace, a decaying schedule with p = 1 rounds at the end."""
    sizes = [1500, 1400, 1650, 1450]
    A, _, _ = _parts(sizes, 96, 61)
    Y0 = synth.gaussian_start(96, 6, 62)
    sched = [4, 4, 2, 1, 1]
    ref = O.localpower(A, 6, sched, agg, Y0, keep_trace=True)
    with B.LocalPower(A) as lp:
        B.lp_solve(lp.ctx, 6, sched, agg, Y0, 0, B.LP_FLAG_TRACE)
        lp.result(6)
        Zt, rho = B.lp_trace(lp.ctx, len(sched), 96, 6)
        B.lp_solve(lp.ctx, 6, sched, agg, Y0, 0, 0)
        lp.result(6)
        with pytest.raises(B.LPError) as e:       # the last solve was not traced
            B.lp_trace(lp.ctx, len(sched), 96, 6)
        assert e.value.status == B.LP_ERR_STATE
    for t, entry in enumerate(ref["trace"]):
        assert O.subspace_dist(Zt[t], entry["Z"]) < 1e-6, t
        if entry["p"] == 1:
            assert rho[t] == 0.0
        else:
            assert entry["rho"] > 1e-4          # the local bases really differ
            assert abs(rho[t] - entry["rho"]) <= 1e-4 * entry["rho"] + 1e-7, (t, rho[t], entry["rho"])


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_seeded_solve_matches_oracle_from_the_same_start(gpu_lib, dtype):
    """lp_solve_seeded draws Y_0 itself (SplitMix64 + Box-Muller); the oracle runs
    from the start block the test side generates from the same definition, and
    lp_solve given that block gives the same result as the seeded call."""
    from tests.seeded_start import seeded_start
    sizes = [700, 900, 650]
    stored, exact, _ = _parts(sizes, 160, 81, dtype)
    seed, k, sched = 2002_08014, 8, [4, 2, 1, 1]
    Y0 = seeded_start(seed, 160, k)
    ref = O.localpower(exact, k, sched, "sign", Y0)["Z"]
    with B.LocalPower(stored, dtype=dtype) as lp:
        B.lp_solve_seeded(lp.ctx, k, sched, "sign", seed)
        Zs, _, _ = lp.result(k)
        Zg, _, _ = lp.solve(k, sched, "sign", Y0)
    assert O.subspace_dist(Zs, ref) < (1e-6 if dtype == "f32" else TC_SOLVE_TOL)
    assert O.subspace_dist(Zs, Zg) < 1e-9
