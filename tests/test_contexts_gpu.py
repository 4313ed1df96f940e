"""Several contexts in one process whose solves use the same kernel
instantiation with different shared-memory plans.  The per-function limit on
dynamic shared memory is raised once to the device's maximum, so a context
planned later (smaller plan) cannot lower it under an earlier context's
captured solve graph: replaying that graph reproduces its first result bit for
bit."""
import numpy as np
import pytest

import oracle as O
from paper_2002_08014_gb300 import binding as B
from tests.test_parity_gpu import TC_SOLVE_TOL, _parts

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,kernel,d_big,d_small,k", [
    ("bf16", "stream", 1024, 128, 8),     # step_tcs_kernel<8, 1>: ring and Z stage sized by d
    ("bf16", "pair", 1024, 192, 16),      # step_pair_kernel<16, 1>
    ("f32", None, 1000, 96, 8),           # the SIMT step kernels
    ("e4m3", None, 1024, 256, 8),         # step_tcs8_kernel<8>
])
def test_graph_replay_after_another_context_planned(gpu_lib, dtype, kernel, d_big, d_small, k):
    sched = [2, 2, 1]
    a_st, a_ex, a_sc = _parts([3000, 2000], d_big, 51, dtype)
    b_st, b_ex, b_sc = _parts([2500, 1500], d_small, 52, dtype)
    ya = np.random.default_rng(53).standard_normal((d_big, k))
    yb = np.random.default_rng(54).standard_normal((d_small, k))
    with B.LocalPower(a_st, dtype=dtype, row_scales=a_sc) as la, \
            B.LocalPower(b_st, dtype=dtype, row_scales=b_sc) as lb:
        if kernel:
            B.lp_set_tuning(la.ctx, kernel=kernel)
            B.lp_set_tuning(lb.ctx, kernel=kernel)
        Za1, _, sta = la.solve(k, sched, "sign", ya)     # A plans, captures its graph and runs it
        Zb1, _, stb = lb.solve(k, sched, "sign", yb)     # B plans the same kernel with less shared memory
        Za2, _, sta2 = la.solve(k, sched, "sign", ya)    # A replays its graph
        Zb2, _, _ = lb.solve(k, sched, "sign", yb)
    assert sta["path"] == stb["path"] == sta2["path"]
    assert np.array_equal(Za1, Za2) and np.array_equal(Zb1, Zb2)
    tol = 1e-6 if sta["path"] == 0 else TC_SOLVE_TOL
    assert O.subspace_dist(Za1, O.localpower(a_ex, k, sched, "sign", ya)["Z"]) < tol
    assert O.subspace_dist(Zb1, O.localpower(b_ex, k, sched, "sign", yb)["Z"]) < tol
