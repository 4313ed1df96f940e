"""Diagnostics of the method on the GPU, through the C ABI, against the FP64
oracle: the local-approximation measure eta of Def. 2 (lp_eta) and an
iteration rank r above the target rank k (Alg. 1 input r >= k).

Tolerances: lp_eta forms every M_i with the solve's own step kernels (FP32
accumulation over s_i rows; tensor-core paths for BF16 and hi/lo planes) and
measures ||M_i - M||_2, which is eta ||M||_2, so the relative error of a
deviation norm is the step's relative error divided by eta: 1e-4 for the FP32
kernels and 1e-3 for the tensor-core paths at the eta of these inputs (0.1 - 0.5).
"""
import numpy as np
import pytest

import oracle as O
import synth
from paper_2002_08014_gb300 import binding as B

pytestmark = pytest.mark.gpu


def _stored(sizes, d, seed, dtype):
    lam = 10.0 * 0.9 ** np.arange(1, min(40, d) + 1)
    A = synth.spiked_rows(sum(sizes), d, lam, 0.3, seed, threads=4)
    A32 = synth.split_rows(A, sizes)
    if dtype == "f32":
        return A32, A32, None
    if dtype == "bf16":
        bits = [synth.f32_to_bf16_bits(a) for a in A32]
        return bits, [("bf16", b) for b in bits], None
    if dtype == "f32_bf16x2":
        planes = [synth.f32_to_bf16x2_planes(a) for a in A32]
        return A32, [O.decode_bf16(h) + O.decode_bf16(l) for h, l in planes], None
    codes, scales = zip(*[synth.f32_to_e4m3_rowscaled(a) for a in A32])
    return list(codes), [("e4m3", c, s) for c, s in zip(codes, scales)], list(scales)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f32_bf16x2", "e4m3"])
@pytest.mark.parametrize("sizes,d", [
    ([900, 1300, 700, 1100], 48),      # Lanczos runs d steps: exact up to rounding
    ([2000, 2600, 1800], 300),         # 256 Lanczos steps < d
    ([500, 40, 777, 1200, 333], 130),  # uneven, d not a multiple of 16
])
def test_eta_matches_oracle(gpu_lib, dtype, sizes, d):
    stored, exact, scales = _stored(sizes, d, 500 + d, dtype)
    want, want_norms = O.eta(exact)
    with B.LocalPower(stored, dtype=dtype, row_scales=scales) as lp:
        got, norms = lp.eta()
    tol = 1e-4 if dtype in ("f32", "e4m3") else 1e-3
    assert 0.05 < want < 2.0
    assert abs(got - want) <= tol * want, (got, want)
    np.testing.assert_allclose(norms, want_norms, rtol=tol)


def test_eta_closed_form_on_gpu(gpu_lib):
    """Rows of partition i all equal x_i e_i: ||M_i - M||_2 = max((1 - p_i) x_i^2,
    max_{j != i} p_j x_j^2), ||M||_2 = max_j p_j x_j^2 (every value exact in FP32)."""
    xs, sizes = (2.0, 0.5, 1.5, 1.0), (3, 10, 7, 12)
    d = len(xs) + 2
    parts = [np.tile((np.eye(d)[i] * x).astype(np.float32), (s, 1)) for i, (x, s) in enumerate(zip(xs, sizes))]
    p = np.array(sizes, dtype=np.float64) / sum(sizes)
    x2 = np.array(xs) ** 2
    want = [max((1 - p[i]) * x2[i], max(p[j] * x2[j] for j in range(len(xs)) if j != i)) for i in range(len(xs))]
    normM = float(np.max(p * x2))
    with B.LocalPower(parts) as lp:
        e, norms = lp.eta()
    np.testing.assert_allclose(norms[:-1], want, rtol=1e-6)
    assert abs(norms[-1] - normM) <= 1e-6 * normM
    assert abs(e - max(want) / normM) <= 1e-6 * e


def test_eta_leaves_the_solve_alone_and_respects_the_budget(gpu_lib):
    sizes, d, k = [64] * 16, 1024, 8
    A, _, _ = _stored(sizes, d, 77, "f32")
    Y0 = synth.gaussian_start(d, k, 78)
    with B.LocalPower(A, hbm_budget_bytes=48 << 20) as lp:
        Z1, s1, st1 = lp.solve(k, [2, 2, 1], "sign", Y0, ritz=True)
        with pytest.raises(B.LPError) as e:     # 17 d x d matrices do not fit 48 MB
            lp.eta()
        assert e.value.status == B.LP_ERR_OOM
        Z2, s2, st2 = lp.result(k)
        assert np.array_equal(Z1, Z2) and np.array_equal(s1, s2)
        assert st1["kernel_launches"] == st2["kernel_launches"]
    with B.LocalPower(A) as lp:
        Z1, s1, _ = lp.solve(k, [2, 2, 1], "sign", Y0, ritz=True)
        e, _ = lp.eta()
        Z2, s2, _ = lp.result(k)
        assert np.array_equal(Z1, Z2) and np.array_equal(s1, s2)
    assert e > 0.5      # 64 rows per worker against d = 1024: the local matrices are far from M


@pytest.mark.parametrize("agg", ["sign", "opt"])
def test_iteration_rank_above_target(gpu_lib, agg):
    """A solve with iteration rank r > k is a solve of rank r; its first k Ritz
    vectors estimate U_k.  Parity with the oracle's r-column run, and at p = 1 the
    r-column span contains the k-column one (same leading start columns)."""
    sizes, d, k, r = [3000, 2500, 3500], 80, 4, 8
    A, _, _ = _stored(sizes, d, 81, "f32")
    Y0 = synth.gaussian_start(d, r, 82)
    sched = [4] * 6 + [1] * 2
    ref = O.localpower(A, r, sched, agg, Y0)
    ref_ritz, ref_sigma = O.ritz(A, ref["Z"])
    V, _ = O.top_k_truth(A, k)
    with B.LocalPower(A) as lp:
        Zr, sr, _ = lp.solve(r, sched, agg, Y0, ritz=True)
        assert O.subspace_dist(Zr, ref["Z"]) < 1e-6
        np.testing.assert_allclose(sr, ref_sigma, rtol=1e-5)
        assert O.subspace_dist(Zr[:, :k], ref_ritz[:, :k]) < 1e-5
        Zk, _, _ = lp.solve(k, sched, agg, Y0[:, :k])
        assert O.subspace_dist(Zr[:, :k], V) <= O.subspace_dist(Zk, V) * 1.01 + 1e-7
        Zk1, _, _ = lp.solve(k, [1] * 5, agg, Y0[:, :k])
        Zr1, _, _ = lp.solve(r, [1] * 5, agg, Y0)
        assert np.linalg.norm(Zk1 - Zr1 @ (Zr1.T @ Zk1), 2) < 1e-5
