"""FP8-E4M3 storage with FP32 row scales on the tensor cores (the streaming
kernel that widens the codes to FP16 in shared memory and factors the scales
out: Y = Q^T diag(s^2) Q Z), against the FP64 oracle on code x scale, through
the C ABI.  Same bars as the other tensor-core paths (1e-5 per step, 1e-4 per
solve)."""
import numpy as np
import pytest

import oracle as O
import synth
from paper_2002_08014_gb300 import binding as B
from tests.test_parity_gpu import TC_SOLVE_TOL, TC_STEP_TOL, _parts, _relF

pytestmark = pytest.mark.gpu

SIMT, TC_STREAM = 0, 2


def _scaled_elementwise_ok(Y, ref, exact, Z, c=1e-5):
    """After the common round-toward-zero scale, every entry within c of its own
    dot products' absolute sum (|A|^T |A| |Z|) / s."""
    a = O.as_f64(exact)
    alpha = float(np.vdot(Y, ref) / np.vdot(Y, Y))
    bound = c * (np.abs(a).T @ (np.abs(a) @ np.abs(Z))) / a.shape[0]
    return 0.0 <= alpha - 1.0 <= 400 * 2.0 ** -23 and bool((np.abs(alpha * Y - ref) <= bound).all())


@pytest.mark.parametrize("sizes,d,k", [
    ([2000, 1500, 2333], 2048, 32),   # the precision workload's width and rank (4-CTA clusters split d)
    ([700, 333], 2048, 16),
    ([300, 129, 77], 1000, 12),       # ragged d and tiles, one CTA per slice
    ([1200], 64, 4),
])
def test_fp8_tensor_core_step_matches_oracle(gpu_lib, sizes, d, k):
    codes, exact, scales = _parts(sizes, d, 900 + d + k, "e4m3")
    rng = np.random.default_rng(d + k)
    Z = O.orth(rng.standard_normal((d, k)))
    with B.LocalPower(codes, dtype="e4m3", row_scales=scales) as lp:
        Y = lp.power_step(k, Z, shared=True)
        y0 = rng.standard_normal((d, k))
        _, _, st = lp.solve(k, [1], "sign", y0)
        assert st["path"] == TC_STREAM
    for i, P in enumerate(exact):
        ref = O.local_step(P, Z)
        assert _relF(Y[i], ref) < TC_STEP_TOL, (i, _relF(Y[i], ref))
        assert _scaled_elementwise_ok(Y[i], ref, P, Z), i


def test_fp8_rows_with_widely_different_scales(gpu_lib):
    """Row scales spread over twelve orders of magnitude: W is scaled by
    s_r^2 / max s^2 before it becomes an FP16 operand, so nothing overflows and
    the small rows' (negligible) contributions do not disturb the result."""
    sizes = [900, 700]
    d, k = 512, 8
    rng = np.random.default_rng(5)
    A = synth.spiked_rows(sum(sizes), d, 10.0 * 0.8 ** np.arange(1, 17), 0.3, 6, threads=4)
    A *= (10.0 ** rng.uniform(-6, 6, sum(sizes)))[:, None].astype(np.float32)
    parts = synth.split_rows(A, sizes)
    codes, scales = zip(*[synth.f32_to_e4m3_rowscaled(p) for p in parts])
    exact = [("e4m3", c, s) for c, s in zip(codes, scales)]
    Z = O.orth(rng.standard_normal((d, k)))
    with B.LocalPower(list(codes), dtype="e4m3", row_scales=list(scales)) as lp:
        Y = lp.power_step(k, Z, shared=True)
    for i, P in enumerate(exact):
        ref = O.local_step(P, Z)
        assert np.isfinite(Y[i]).all()
        assert _relF(Y[i], ref) < TC_STEP_TOL, (i, _relF(Y[i], ref))


def test_fp8_tensor_core_and_simt_solves_agree_with_the_oracle(gpu_lib):
    sizes = [1500, 1700, 1333]
    d, k = 1024, 16
    codes, exact, scales = _parts(sizes, d, 77, "e4m3")
    y0 = synth.gaussian_start(d, k, 78)
    sched = [4, 4, 2, 1, 1]
    ref = O.localpower(exact, k, sched, "opt", y0)["Z"]
    with B.LocalPower(codes, dtype="e4m3", row_scales=scales) as lp:
        B.lp_solve(lp.ctx, k, sched, "opt", y0, 0, 0)
        Zt, _, st = lp.result(k)
        assert st["path"] == TC_STREAM
        B.lp_solve(lp.ctx, k, sched, "opt", y0, 0, B.LP_FLAG_SIMT)
        Zs, _, st2 = lp.result(k)
        assert st2["path"] == SIMT
    assert O.subspace_dist(Zt, ref) < TC_SOLVE_TOL
    assert O.subspace_dist(Zs, ref) < 1e-6
