"""The batch runner (lp_batch_*): independent instances of different shapes and
dtypes solved by one CUDA graph launch.  Instances sharing d, dtype, k, the
schedule, the aggregator and the flags form a group whose every step kind is
one launch over all of them (the group's step kernel chosen by the
autotuner).  Each instance must match the FP64 oracle run on its own data, the
same solve on a context of its own within the same bar, and replaying the
graph must reproduce the first launch bit for bit."""
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
        # k above the smallest partition's row count: rejected at add, with its reason
        small = [stored[0][:5]] + list(stored[1:])
        with pytest.raises(B.LPError) as e:
            bt.add(small, 8, SCHED, "sign", y0)
        assert e.value.status == B.LP_ERR_INVALID and "k exceeds" in str(e.value)
        assert len(bt) == 0


def _uneven_sizes(n, m, seed):
    """m partition sizes summing to n, uneven, the largest not first."""
    w = np.random.default_rng(seed).uniform(0.5, 2.0, m)
    w[0] = 0.3
    s_ = np.maximum(np.floor(w / w.sum() * n).astype(int), 40)
    s_[-1] += n - s_.sum()
    return [int(x) for x in s_]


def _grouped_instance(seed, n, d, k, m, dtype):
    # a factor-3 eigengap at k and a schedule long enough to converge to the top-k
    # subspace: the comparison then measures arithmetic, not the sensitivity of an
    # unconverged iterate (a 15% gap at k after 13 steps amplified the tensor
    # cores' FP32 rounding to 3.5e-4 on one instance, alone and grouped alike)
    lam = 0.9 ** np.arange(1, d + 1)
    lam[:k] *= 3.0
    A = synth.spiked_rows(n, d, lam, 0.0, seed, threads=4)
    A32 = synth.split_rows(A, _uneven_sizes(n, m, seed))
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


# (group, dtype, d, k, agg, instances as (n, m)): each group's instances share
# every launch parameter; n and m differ within a group.
GROUPS = [
    ("bf16", 256, 16, "sign", [(9000, 5), (3000, 4), (20000, 9), (1500, 6)]),
    ("bf16", 256, 16, "opt", [(7000, 7), (2500, 3)]),
    ("f32", 128, 8, "opt", [(6000, 4), (4000, 8), (900, 3)]),
    ("f32_bf16x2", 512, 32, "sign", [(8000, 6), (5000, 4)]),
    ("e4m3", 200, 8, "sign", [(5000, 6), (3500, 5), (2000, 4)]),
]
GSCHED = [4, 4, 4, 2]


@pytest.mark.parametrize("tune", [False, True])
def test_batch_groups_match_oracle_alone_and_replay(gpu_lib, tune):
    """Several instances per group (uneven n and m, the base not first, both
    aggregators, every storage type), Ritz output: each instance within its bar
    of the oracle (1e-6 FP32 and FP8 on the SIMT kernel's FP32 arithmetic,
    1e-4 on the tensor cores), its Ritz values within 1e-5 of the oracle's, the
    same solve on a context of its own within the same bar, and a replay bit
    for bit."""
    inst, meta = [], []
    for gi, (dtype, d, k, agg, members) in enumerate(GROUPS):
        for j, (n, m) in enumerate(members):
            inst.append(_grouped_instance(700 + 10 * gi + j, n, d, k, m, dtype))
            meta.append((dtype, d, k, agg))
    with B.Batch() as bt:
        for (stored, _, y0, scales), (dtype, d, k, agg) in zip(inst, meta):
            bt.add(stored, k, GSCHED, agg, y0, dtype=dtype, row_scales=scales, refine_rounds=2)
        if tune:
            bt.autotune()
        bt.solve()
        assert bt.groups() == len(GROUPS)
        first = [bt.result(i) for i in range(len(inst))]
        bt.solve()
        second = [bt.result(i) for i in range(len(inst))]
    for (Z1, s1, st1), (Z2, s2, st2) in zip(first, second):
        assert np.array_equal(Z1, Z2) and np.array_equal(s1, s2)
        assert st1["rounds"] == len(GSCHED) + 2 and st1["local_steps"] == sum(GSCHED) + 2
    for (stored, exact, y0, scales), (dtype, d, k, agg), (Z, sig, st) in zip(inst, meta, first):
        tol = 1e-6 if dtype in ("f32", "e4m3") and st["path"] == 0 else TC_SOLVE_TOL
        ref = O.localpower(exact, k, GSCHED + [1, 1], agg, y0)
        Zr, sr = O.ritz(exact, ref["Z"])
        assert O.subspace_dist(Z, Zr) < tol, (dtype, d, k, agg, O.subspace_dist(Z, Zr))
        assert np.allclose(sig, sr, rtol=1e-5, atol=0), (dtype, d, k)
        assert st["n"] == sum(O.as_f64(p).shape[0] for p in exact) and st["m"] == len(exact)
        with B.LocalPower(stored, dtype=dtype, row_scales=scales) as lp:
            if tune:
                B.lp_autotune(lp.ctx, k)
            Za, _, _ = lp.solve(k, GSCHED, agg, y0, refine_rounds=2, ritz=True)
        assert O.subspace_dist(Z, Za) < tol


def test_batch_group_of_one_is_the_lone_solve(gpu_lib):
    """A group with one instance runs the ordinary launch sequence on the same
    rows, so it reproduces the solve on a context of its own bit for bit."""
    stored, _, y0, _ = _grouped_instance(901, 12000, 256, 16, 6, "bf16")
    with B.Batch() as bt:
        bt.add(stored, 16, GSCHED, "sign", y0, dtype="bf16", refine_rounds=1)
        bt.solve()
        Zb, sb, _ = bt.result(0)
        assert bt.groups() == 1
    with B.LocalPower(stored, dtype="bf16") as lp:
        Za, sa, _ = lp.solve(16, GSCHED, "sign", y0, refine_rounds=1, ritz=True)
    assert np.array_equal(Zb, Za) and np.array_equal(sb, sa)


def test_batch_adding_after_a_solve_regroups(gpu_lib):
    """An instance added after a solve joins its group at the next solve; the
    earlier instances' results stay within the bar of the oracle."""
    a = _grouped_instance(910, 6000, 128, 8, 4, "f32")
    c = _grouped_instance(911, 3000, 128, 8, 5, "f32")
    with B.Batch() as bt:
        bt.add(a[0], 8, GSCHED, "sign", a[2])
        bt.solve()
        assert bt.groups() == 1
        bt.result(0)
        bt.add(c[0], 8, GSCHED, "sign", c[2])
        assert bt.groups() == 0
        bt.solve()
        assert bt.groups() == 1
        outs = [bt.result(i) for i in range(2)]
    for (_, exact, y0, _), (Z, _, _) in zip([a, c], outs):
        ref = O.localpower(exact, 8, GSCHED, "sign", y0)
        assert O.subspace_dist(Z, O.ritz(exact, ref["Z"])[0]) < 1e-6


def test_batch_rejects_trace_flag(gpu_lib):
    stored, _, y0, _ = _instance(602, 3000, 64, 8, 4, "f32")
    with B.Batch() as bt:
        with pytest.raises(B.LPError) as e:
            bt.add(stored, 8, SCHED, "sign", y0, flags=B.LP_FLAG_RITZ | B.LP_FLAG_TRACE)
        assert e.value.status == B.LP_ERR_INVALID
