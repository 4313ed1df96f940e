"""LP_FLAG_KXK_FP64: the k x k work in FP64 (the CholQR2 Gram and Cholesky, the
Procrustes SVD of eq. (3), the Rayleigh-Ritz eigen-solve) against the FP64
oracle, through the C ABI.

The d x k work stays FP32 in this mode, so on well-conditioned blocks it meets
the same bars as the default mode.  What the FP64 Gram adds is range: CholQR2
squares the condition number of Y in its Gram matrix, so an FP32 Gram loses
positive definiteness near kappa(Y) = u32^(-1/2) ~ 4e3, while an FP64 Gram of
FP32 products (each exact in FP64) keeps it to kappa ~ u64^(-1/2) ~ 7e7.  The
subspace of Z = Y L^{-T} is then limited by the FP32 triangular solve: a
backward error of ~k u32 |L| per row moves span(Z) by O(u32 kappa)."""
import numpy as np
import pytest

import oracle as O
from paper_2002_08014_gb300 import binding as B
from tests.test_parity_gpu import TC_SOLVE_TOL, _parts, _relF

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.mark.parametrize("d,k,batch", [(100, 5, 3), (1024, 16, 4), (257, 32, 2), (9, 1, 5), (2048, 32, 1)])
def test_orth_fp64_matches_oracle(gpu_lib, d, k, batch):
    rng = np.random.default_rng(d + k)
    Y = rng.standard_normal((batch, d, k)) @ np.diag(np.linspace(1.0, 30.0, k))
    ctx = B.lp_create(0)
    try:
        Z = B.lp_orth(ctx, Y, kxk_fp64=True)
    finally:
        B.lp_destroy(ctx)
    for b in range(batch):
        assert np.abs(Z[b].T @ Z[b] - np.eye(k)).max() < 1e-5
        ref = O.orth(Y[b])
        assert np.abs(Z[b] - ref).max() < 2e-5
        assert O.subspace_dist(Z[b], ref) < 1e-6


@pytest.mark.parametrize("kappa", [1e5, 1e6])
def test_orth_fp64_gram_keeps_ill_conditioned_blocks(gpu_lib, kappa):
    """Y = U diag(geomspace(1, 1/kappa)) V^T at d = 2,048, k = 32: past the FP32
    Gram's breakdown.  The FP64 mode returns an orthonormal basis whose span is
    within u32 kappa of span(Y) (Y as the device stores it, in FP32)."""
    rng = np.random.default_rng(int(np.log10(kappa)))
    d, k = 2048, 32
    Uq = O.orth(rng.standard_normal((d, k)))
    Vq = O.orth(rng.standard_normal((k, k)))
    Y = (Uq @ np.diag(np.geomspace(1.0, 1.0 / kappa, k)) @ Vq.T)[None]
    ctx = B.lp_create(0)
    try:
        Z = B.lp_orth(ctx, Y, kxk_fp64=True)[0]
    finally:
        B.lp_destroy(ctx)
    assert np.abs(Z.T @ Z - np.eye(k)).max() < 1e-5
    ref = O.orth(Y[0].astype(np.float32).astype(np.float64))
    dist = O.subspace_dist(Z, ref)
    assert dist < U32 * kappa, dist


@pytest.mark.parametrize("d,k,m,base", [(100, 5, 4, 0), (513, 16, 7, 3), (64, 32, 3, 2), (2048, 32, 5, 1)])
def test_align_opt_fp64_matches_oracle(gpu_lib, d, k, m, base):
    """The Procrustes aligners D_i = U V^T of C = Z_i^T Z_b (eq. (3)) with the
    k x k SVD in FP64, element-wise against the oracle's SVD."""
    rng = np.random.default_rng(11 * d + k)
    Zb = O.orth(rng.standard_normal((d, k)))
    Zs, Ys = [], []
    for _ in range(m):
        Q = O.orth(rng.standard_normal((k, k)))
        Zi = O.orth(Zb @ Q + 0.05 * rng.standard_normal((d, k)))
        Zs.append(Zi)
        Ys.append(Zi @ np.diag(np.linspace(3, 1, k)) + 0.01 * rng.standard_normal((d, k)))
    Zs[base] = Zb
    sizes = [100] * m
    sizes[base] = 150
    w = np.array(sizes, float) / sum(sizes)
    ctx = B.lp_create(0)
    try:
        Y, D = B.lp_align_aggregate(ctx, "opt", base, w, np.stack(Ys), np.stack(Zs), kxk_fp64=True)
    finally:
        B.lp_destroy(ctx)
    assert _relF(Y, O.aggregate(Ys, Zs, sizes, "opt")) < 5e-6
    for i in range(m):
        Dref = np.eye(k) if i == base else O.align("opt", Zs[i], Zb)
        assert np.abs(D[i] - Dref).max() < 1e-5
        assert np.abs(D[i].T @ D[i] - np.eye(k)).max() < 1e-5


@pytest.mark.parametrize("dtype,agg", [("f32", "sign"), ("f32", "opt"), ("bf16", "opt"), ("e4m3", "sign")])
def test_solve_fp64_kxk_matches_oracle_and_default_mode(gpu_lib, dtype, agg):
    """Whole solves with Ritz output in both k x k modes: each within its bar of
    the oracle (1e-6 for FP32 data, 1e-4 for reduced precision) and the Ritz
    values within 1e-5 of the oracle's.  The two modes differ only in the rounding
    of the k x k work, which the small eigengap here (lambda_k / lambda_{k+1} about
    1.09 on the FP32 data) amplifies in each independently; the subspace distance
    is a metric, so the two bars put them within twice the bar of each other."""
    sizes = [3000, 2200, 4100]
    d, k = 512, 24
    stored, exact, scales = _parts(sizes, d, 41, dtype)
    y0 = np.random.default_rng(42).standard_normal((d, k))
    sched = [3, 3, 2, 1]
    ref = O.localpower(exact, k, sched, agg, y0)
    Zr, sr = O.ritz(exact, ref["Z"])
    tol = 1e-6 if dtype == "f32" else TC_SOLVE_TOL
    with B.LocalPower(stored, dtype=dtype, row_scales=scales) as lp:
        Z64, s64, _ = lp.solve(k, sched, agg, y0, ritz=True, kxk_fp64=True)
        Z32, s32, _ = lp.solve(k, sched, agg, y0, ritz=True)
    assert O.subspace_dist(Z64, Zr) < tol
    assert O.subspace_dist(Z32, Zr) < tol
    assert O.subspace_dist(Z64, Z32) < 2 * tol
    assert np.allclose(s64, sr, rtol=1e-5, atol=0)
