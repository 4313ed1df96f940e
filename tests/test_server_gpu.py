"""The request server (lp_server_*): continuous batching of independent solves.

Each request is solved in its own context on its own stream, so its result
must not depend on what else is on the device: a request solved alone and the
same request solved while others run give identical bits.  Results are also
checked against the FP64 oracle, admission against the HBM budget, and error
isolation (one failing request leaves the others untouched)."""
import time

import numpy as np
import pytest

import oracle as O
import synth
from paper_2002_08014_gb300 import binding as B

pytestmark = pytest.mark.gpu

TC_SOLVE_TOL = 1e-4


def _request(seed, n, d, k, m, dtype="bf16"):
    lam = 0.85 ** np.arange(1, d + 1)
    A = synth.spiked_rows(n, d, lam, 0.0, seed, threads=4)
    sizes = synth.partition_sizes(n, m)
    A32 = synth.split_rows(A, sizes)
    if dtype == "bf16":
        stored = [synth.f32_to_bf16_bits(a) for a in A32]
        exact = [O.decode_bf16(b) for b in stored]
    else:
        stored, exact = A32, A32
    return stored, exact, synth.gaussian_start(d, k, seed + 1)


SHAPES = [(3000, 64, 4, 4), (20000, 300, 16, 8), (9000, 1000, 32, 5), (2500, 90, 8, 32), (40000, 512, 16, 16)]
SCHED = [4] * 6


def _drain(srv, ids, timeout=120.0):
    got, t0 = set(), time.time()
    while len(got) < len(ids):
        got.update(srv.progress())
        if time.time() - t0 > timeout:
            raise TimeoutError("server did not finish")
        time.sleep(0.0005)
    return got


def test_alone_and_in_the_mix_give_identical_results(gpu_lib):
    reqs = [_request(100 + i, *shape) for i, shape in enumerate(SHAPES)]
    alone = []
    with B.Server(max_active=1) as srv:
        for stored, _, y0 in reqs:
            k = y0.shape[1]
            rid = srv.submit(stored, k, SCHED, "sign", y0, dtype="bf16", refine_rounds=2)
            _drain(srv, [rid])
            alone.append(srv.result(rid))
    with B.Server(max_active=8) as srv:
        ids = [srv.submit(stored, y0.shape[1], SCHED, "sign", y0, dtype="bf16", refine_rounds=2)
               for stored, _, y0 in reqs]
        info = srv.query()
        assert info["queued"] + info["active"] + info["completed"] == len(reqs)
        _drain(srv, ids)
        mixed = [srv.result(rid) for rid in ids]
    for (Za, sa, _), (Zm, sm, _) in zip(alone, mixed):
        assert np.array_equal(Za, Zm) and np.array_equal(sa, sm)
    for (stored, exact, y0), (Z, sig, st) in zip(reqs, mixed):
        k = y0.shape[1]
        ref = O.localpower(exact, k, SCHED + [1, 1], "sign", y0)
        assert O.subspace_dist(Z, ref["Z"]) < TC_SOLVE_TOL
        assert st["rounds"] == len(SCHED) + 2


def test_admission_respects_the_hbm_budget(gpu_lib):
    reqs = [_request(200 + i, 30000, 256, 8, 6, "f32") for i in range(4)]
    budget = 96 << 20    # room for about two of these requests at a time
    with B.Server(hbm_budget_bytes=budget, max_active=8) as srv:
        ids = [srv.submit(stored, 8, SCHED, "opt", y0, dtype="f32") for stored, _, y0 in reqs]
        peak_active = 0
        got, t0 = set(), time.time()
        while len(got) < len(ids):
            got.update(srv.progress())
            info = srv.query()
            peak_active = max(peak_active, info["active"])
            assert info["hbm_in_use"] <= budget
            assert time.time() - t0 < 120
        assert 1 <= peak_active < len(ids)
        assert srv.query()["hbm_peak"] <= budget
        outs = [srv.result(rid) for rid in ids]
    for (stored, exact, y0), (Z, _, _) in zip(reqs, outs):
        ref = O.localpower(exact, 8, SCHED, "opt", y0)
        assert O.subspace_dist(Z, ref["Z"]) < 1e-6


def test_failures_stay_with_their_request(gpu_lib):
    good = _request(300, 5000, 128, 8, 4, "f32")
    bad_parts = [p.copy() for p in good[0]]
    bad_parts[2][7, 3] = np.nan
    with B.Server(max_active=4) as srv:
        with pytest.raises(B.LPError) as e:   # malformed: k above a partition's rows
            srv.submit([p[:5] for p in good[0]], 8, SCHED, "sign", good[2], dtype="f32")
        assert e.value.status == B.LP_ERR_INVALID
        with B.Server(hbm_budget_bytes=1 << 20) as tiny:
            with pytest.raises(B.LPError) as e:
                tiny.submit(good[0], 8, SCHED, "sign", good[2], dtype="f32")
            assert e.value.status == B.LP_ERR_OOM
        ids = [srv.submit(good[0], 8, SCHED, "sign", good[2], dtype="f32"),
               srv.submit(bad_parts, 8, SCHED, "sign", good[2], dtype="f32"),
               srv.submit(good[0], 8, SCHED, "sign", good[2], dtype="f32")]
        _drain(srv, ids)
        Z0, _, _ = srv.result(ids[0])
        with pytest.raises(B.LPError) as e:
            srv.result(ids[1])
        assert e.value.status == B.LP_ERR_NUMERIC
        Z2, _, _ = srv.result(ids[2])
        with pytest.raises(B.LPError) as e:   # already fetched
            srv.result(ids[0])
        assert e.value.status == B.LP_ERR_STATE
    assert np.array_equal(Z0, Z2)


def test_fp8_requests_with_row_scales(gpu_lib):
    """FP8-E4M3 requests carry one FP32 scale per row; each result matches the
    oracle on code x scale (SIMT FP32 arithmetic: the FP32 bar)."""
    lam = 0.85 ** np.arange(1, 129)
    reqs = []
    for i, (n, d, k, m) in enumerate([(6000, 128, 8, 4), (9000, 96, 5, 6)]):
        A = synth.spiked_rows(n, d, lam[:d], 0.0, 700 + i, threads=4)
        A32 = synth.split_rows(A, synth.partition_sizes(n, m))
        codes, scales = map(list, zip(*[synth.f32_to_e4m3_rowscaled(a) for a in A32]))
        reqs.append((codes, scales, [O.decode_e4m3(c, s_) for c, s_ in zip(codes, scales)],
                     synth.gaussian_start(d, k, 710 + i)))
    with B.Server(max_active=4) as srv:
        ids = [srv.submit(c, y0.shape[1], SCHED, "opt", y0, dtype="e4m3", row_scales=sc) for c, sc, _, y0 in reqs]
        _drain(srv, ids)
        outs = [srv.result(rid) for rid in ids]
    for (_, _, exact, y0), (Z, _, _) in zip(reqs, outs):
        ref = O.localpower(exact, y0.shape[1], SCHED, "opt", y0)
        assert O.subspace_dist(Z, ref["Z"]) < 1e-6


def test_pitched_device_rows(gpu_lib):
    """A request can name rows and the first d columns of a wider device pool."""
    torch = pytest.importorskip("torch")
    lam = 0.85 ** np.arange(1, 257)
    pool = synth.spiked_rows(6000, 256, lam, 0.0, 400, threads=4)
    bits = synth.f32_to_bf16_bits(pool)
    dev = torch.from_numpy(bits.view(np.int16)).cuda()
    d, k, sizes = 100, 8, [1500, 2500, 2000]
    offs = np.cumsum([0] + sizes[:-1])
    parts_dev = [dev[o:o + s] for o, s in zip(offs, sizes)]
    y0 = synth.gaussian_start(d, k, 401)
    with B.Server(max_active=2) as srv:
        rid = srv.submit(parts_dev, k, SCHED, "sign", y0, dtype="bf16", row_pitch=256, d=d)
        _drain(srv, [rid])
        Z, _, _ = srv.result(rid)
    exact = [O.decode_bf16(np.ascontiguousarray(bits[o:o + s, :d])) for o, s in zip(offs, sizes)]
    ref = O.localpower(exact, k, SCHED, "sign", y0)
    assert O.subspace_dist(Z, ref["Z"]) < TC_SOLVE_TOL
