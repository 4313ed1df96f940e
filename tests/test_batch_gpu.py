"""The batch runner (lp_batch_*): independent instances of different shapes and
dtypes, each with its step kernel chosen by the autotuner, solved by one CUDA
graph launch.  Each instance must match the FP64 oracle run on its own data,
and replaying the graph must reproduce the first launch bit for bit."""
import numpy as np
import pytest

import oracle as O
import synth
from paper_2002_08014_gb300 import binding as B

pytestmark = pytest.mark.gpu

TC_SOLVE_TOL = 1e-4


def _instance(seed, n, d, k, m, dtype):
    lam = 0.85 ** np.arange(1, d + 1)
    A = synth.spiked_rows(n, d, lam, 0.0, seed, threads=4)
    A32 = synth.split_rows(A, synth.partition_sizes(n, m))
    scales = None
    if dtype == "bf16":
        stored = [synth.f32_to_bf16_bits(a) for a in A32]
        exact = [O.decode_bf16(b) for b in stored]
    elif dtype == "f32_bf16x2":
        stored = A32
        exact = [O.decode_bf16(h) + O.decode_bf16(l) for h, l in (synth.f32_to_bf16x2_planes(a) for a in A32)]
    elif dtype == "e4m3":
        stored, scales = map(list, zip(*[synth.f32_to_e4m3_rowscaled(a) for a in A32]))
        exact = [O.decode_e4m3(c, sc) for c, sc in zip(stored, scales)]
    else:
        stored, exact = A32, A32
    return stored, exact, synth.gaussian_start(d, k, seed + 1), scales


SHAPES = [(4000, 64, 4, 4, "bf16"), (30000, 256, 16, 8, "bf16"), (12000, 700, 32, 6, "bf16"),
          (6000, 128, 8, 16, "f32"), (20000, 512, 16, 5, "f32_bf16x2"), (2500, 90, 8, 32, "bf16"),
          (5000, 200, 8, 6, "e4m3")]
SCHED = [4] * 5


def test_batch_matches_oracle_and_replays_exactly(gpu_lib):
    inst = [_instance(500 + i, *s) for i, s in enumerate(SHAPES)]
    with B.Batch() as bt:
        for (stored, _, y0, scales), shape in zip(inst, SHAPES):
            bt.add(stored, y0.shape[1], SCHED, "sign", y0, dtype=shape[4], row_scales=scales, refine_rounds=2)
        assert len(bt) == len(SHAPES)
        bt.autotune()
        bt.solve()
        first = [bt.result(i) for i in range(len(SHAPES))]
        bt.solve()
        second = [bt.result(i) for i in range(len(SHAPES))]
    for (Z1, s1, st1), (Z2, s2, st2) in zip(first, second):
        assert np.array_equal(Z1, Z2) and np.array_equal(s1, s2)
        assert st1["kernel_launches"] == st2["kernel_launches"]
        assert st1["rounds"] == len(SCHED) + 2
    for (stored, exact, y0, _), shape, (Z, sig, st) in zip(inst, SHAPES, first):
        ref = O.localpower(exact, y0.shape[1], SCHED + [1, 1], "sign", y0)
        tol = 1e-6 if shape[4] in ("f32", "e4m3") else TC_SOLVE_TOL
        assert O.subspace_dist(Z, ref["Z"]) < tol, shape


def test_batch_rejects_bad_input(gpu_lib):
    stored, _, y0, _ = _instance(600, 3000, 64, 8, 4, "f32")
    with B.Batch(hbm_budget_bytes=1 << 20) as bt:
        with pytest.raises(B.LPError) as e:
            bt.add(stored, 8, SCHED, "sign", y0)
        assert e.value.status == B.LP_ERR_OOM
    with B.Batch() as bt:
        with pytest.raises(B.LPError) as e:
            bt.solve()
        assert e.value.status == B.LP_ERR_STATE
        with pytest.raises(B.LPError) as e:
            bt.add(stored, 0, SCHED, "sign", y0)
        assert e.value.status == B.LP_ERR_INVALID
