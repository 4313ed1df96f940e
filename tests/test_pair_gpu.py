"""The pass-split pair step kernel (LP_KERNEL_PAIR: rank 0 of a CTA pair forms
W = A_t Z from HBM, rank 1 accumulates A_t^T W from L2) against the FP64 oracle,
through the C ABI: one power step element-wise on ragged shapes, and whole
solves.  Same tolerances as the other tensor-core paths (Z and W split into
BF16 hi + lo, FP32 accumulation)."""
import numpy as np
import pytest

import oracle as O
from paper_2002_08014_gb300 import binding as B
from tests.test_parity_gpu import TC_SOLVE_TOL, TC_STEP_TOL, _parts, _relF

pytestmark = pytest.mark.gpu

TC_PAIR = 3  # lp_stats::path of the pair kernel


def _path_of(lp, k):
    """Path code a solve on this context runs with its current tuning."""
    d = lp.d
    y0 = np.random.default_rng(0).standard_normal((d, k))
    _, _, st = lp.solve(k, [1], "sign", y0)
    return st["path"]


@pytest.mark.parametrize("dtype", ["bf16", "f32_bf16x2"])
@pytest.mark.parametrize("sizes,d,k", [
    ([37, 64, 21], 100, 5),            # ragged tiles, d not a multiple of 16, K = 8
    ([500, 333, 129, 700], 257, 16),   # d just over a 256-column block
    ([96, 96], 1024, 16),              # the FP32 workload's width
    ([40, 41, 42], 64, 32),            # K = 32, one 128-column block
    ([300, 29], 512, 24),              # k padded to 32 at d = 512 (rank 1 Y slice fills TMEM)
    ([13] * 40 + [600], 200, 12),      # many tiny partitions: rank 0 restages Z_i often
    ([12, 15, 16, 17, 33, 500], 1024, 12),
    ([37] * 30 + [2000], 1024, 16),
])
def test_pair_power_step_matches_oracle(gpu_lib, dtype, sizes, d, k):
    stored, exact, _ = _parts(sizes, d, 300 + d + k, dtype)
    rng = np.random.default_rng(2)
    Z = O.orth(rng.standard_normal((d, k)))
    with B.LocalPower(stored, dtype=dtype) as lp:
        B.lp_set_tuning(lp.ctx, kernel="pair")
        Y = lp.power_step(k, Z, shared=True)
        for i, P in enumerate(exact):
            ref = O.local_step(P, Z)
            assert _relF(Y[i], ref) < TC_STEP_TOL, (i, _relF(Y[i], ref))
            # element-wise: every entry within the bound of the hi/lo splits of Z and W
            # (each within 2^-17 relative) on its own dot products, with slack for the
            # FP32 accumulation: |dY| <= 1.6e-5 (|A|^T |A| |Z|) / s_i
            bound = 1.6e-5 * (np.abs(O.as_f64(P)).T @ (np.abs(O.as_f64(P)) @ np.abs(Z))) / O.as_f64(P).shape[0]
            assert (np.abs(Y[i] - ref) <= bound + 1e-30).all()
        Zs = np.stack([O.orth(rng.standard_normal((d, k))) for _ in sizes])
        Y2 = B.lp_power_step(lp.ctx, k, Zs, False, len(sizes), d)
        for i, P in enumerate(exact):
            assert _relF(Y2[i], O.local_step(P, Zs[i])) < TC_STEP_TOL
        assert _path_of(lp, k) == TC_PAIR


def test_pair_many_pieces_per_pair(gpu_lib):
    """Enough rows that each CTA pair owns several 4,096-row pieces (rank 1
    alternates its two TMEM Y slices) and partitions change inside a pair."""
    sizes = [200_000, 150_001, 4_096, 70_000]
    d, k = 256, 8
    stored, exact, _ = _parts(sizes, d, 77, "bf16")
    Z = O.orth(np.random.default_rng(3).standard_normal((d, k)))
    with B.LocalPower(stored, dtype="bf16") as lp:
        B.lp_set_tuning(lp.ctx, kernel="pair")
        Y = lp.power_step(k, Z, shared=True)
        for i, P in enumerate(exact):
            assert _relF(Y[i], O.local_step(P, Z)) < TC_STEP_TOL, i
        assert _path_of(lp, k) == TC_PAIR


@pytest.mark.parametrize("agg", ["sign", "opt"])
def test_pair_solve_matches_oracle_and_streaming_kernel(gpu_lib, agg):
    """A whole solve on hi/lo planes of FP32 data at the FP32 workload's width:
    within the reduced-precision bar of the oracle on the stored planes, and no
    further from the oracle than the same solve on the single-CTA streaming
    kernel (the two sum each W in a different order, so they differ by rounding)."""
    sizes = [5000, 9000, 4097, 700]
    d, k = 1024, 16
    stored, exact, _ = _parts(sizes, d, 91, "f32_bf16x2")
    y0 = np.random.default_rng(4).standard_normal((d, k))
    sched = [2, 2, 1]
    ref = O.localpower(exact, k, sched, agg, y0)["Z"]
    with B.LocalPower(stored, dtype="f32_bf16x2") as lp:
        B.lp_set_tuning(lp.ctx, kernel="pair")
        Zp, _, st = lp.solve(k, sched, agg, y0)
        assert st["path"] == TC_PAIR
        B.lp_set_tuning(lp.ctx, kernel="stream")
        Zs, _, st2 = lp.solve(k, sched, agg, y0)
        assert st2["path"] == 2
    dp, ds = O.subspace_dist(Zp, ref), O.subspace_dist(Zs, ref)
    assert dp < TC_SOLVE_TOL and ds < TC_SOLVE_TOL, (dp, ds)
    assert dp <= 2.0 * ds + 1e-6, (dp, ds)


def test_pair_kernel_rejects_what_it_cannot_plan(gpu_lib):
    """d = 2,048 at k = 32 has no pair plan (rank 1's Y slice would need 1,024
    TMEM columns): an explicit request for the pair kernel says so instead of
    running another kernel."""
    stored, _, _ = _parts([300, 300], 2048, 5, "bf16")
    with B.LocalPower(stored, dtype="bf16") as lp:
        B.lp_set_tuning(lp.ctx, kernel="pair")
        with pytest.raises(B.LPError) as e:
            lp.power_step(32, O.orth(np.random.default_rng(1).standard_normal((2048, 32))))
        assert e.value.status == B.LP_ERR_UNSUPPORTED


def test_pair_kernel_is_deterministic_for_every_ring_depth(gpu_lib):
    """Each issuer's accumulation chain and the epilogue's sum over issuers run in
    a fixed order: a solve repeats bit for bit.  A smaller ring deals units to
    fewer issuers (another summation order), within the same bar of the oracle."""
    sizes = [3000, 2500, 1777]
    stored, exact, _ = _parts(sizes, 512, 31, "bf16")
    y0 = np.random.default_rng(32).standard_normal((512, 16))
    sched = [2, 1]
    ref = O.localpower(exact, 16, sched, "sign", y0)["Z"]
    with B.LocalPower(stored, dtype="bf16") as lp:
        for ring in (0, 2, 3):
            B.lp_set_tuning(lp.ctx, ring_units=ring, kernel="pair")
            Z1, _, st = lp.solve(16, sched, "sign", y0)
            Z2, _, _ = lp.solve(16, sched, "sign", y0)
            assert st["path"] == TC_PAIR
            assert np.array_equal(Z1, Z2), ring
            assert O.subspace_dist(Z1, ref) < TC_SOLVE_TOL, ring


def test_pair_kernel_timeout_reports_and_the_context_recovers(gpu_lib):
    """Failure detection without a GPU fault: the test hook makes rank 0's
    producer wait, after its first ring fill, on a barrier that nothing
    completes, with a limit of 200,000 cycles.  The wait runs out, the kernel
    raises both ranks' abort flags, drains its copies and MMAs and returns; the
    solve reports LP_ERR_TIMEOUT, and the next solve on the same context (hook
    off) matches the oracle."""
    sizes = [256, 256]              # 4 tiles: 4 CTA pairs of 8 ring units each
    d, k = 1024, 16
    stored, exact, _ = _parts(sizes, d, 9, "bf16")
    y0 = np.random.default_rng(10).standard_normal((d, k))
    sched = [2, 1]
    ref = O.localpower(exact, k, sched, "sign", y0)["Z"]
    with B.LocalPower(stored, dtype="bf16") as lp:
        B.lp_set_tuning(lp.ctx, kernel="pair", test_stall_cycles=200_000)
        with pytest.raises(B.LPError) as e:
            lp.solve(k, sched, "sign", y0)
        assert e.value.status == B.LP_ERR_TIMEOUT
        B.lp_set_tuning(lp.ctx, kernel="pair")
        Z, _, st = lp.solve(k, sched, "sign", y0)
        assert st["path"] == TC_PAIR
    assert O.subspace_dist(Z, ref) < TC_SOLVE_TOL
