"""The allocation-free power step (for callers that cannot allocate device
memory: its scratch is a fixed array inside the library) must give what the
context-based lp_power_step gives, call after call.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.  It passes alone in a fresh
process as well as after the other tests (the static array carries no state a
call depends on)."""
import numpy as np
import pytest

import oracle as O
import synth
from paper_2002_08014_gb300 import binding as B

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("sizes,d,k", [
    ([700, 333, 1000, 59], 256, 16),
    ([5000, 3333, 4100, 777], 1024, 16),   # the d = 1,024 pipelined kernel (bulk copies on bounded waits)
])
def test_static_scratch_step_matches_context_step_twice(gpu_lib, sizes, d, k):
    torch = pytest.importorskip("torch")
    A = synth.spiked_rows(sum(sizes), d, 4.0 * 0.8 ** np.arange(1, 9), 0.3, 77, threads=4)
    parts = synth.split_rows(A, sizes)
    dev = torch.device("cuda", 0)
    A_dev = torch.from_numpy(A).to(dev)
    stream = torch.cuda.Stream(device=dev)
    rng = np.random.default_rng(5)
    with B.LocalPower(parts) as lp:
        for call in range(2):  # two calls in a row, the second on a different Z
            Z = O.orth(rng.standard_normal((d, k)))
            ref = lp.power_step(k, Z, shared=True)                     # existing entry point
            z_dev = torch.from_numpy(Z).to(dev)
            y_dev = torch.full((len(sizes), d, k), float("nan"), dtype=torch.float64, device=dev)
            with torch.cuda.stream(stream):
                B.lp_power_step_static(A_dev, sizes, k, z_dev, y_dev, stream=stream)
            stream.synchronize()
            Y = y_dev.cpu().numpy()
            assert np.isfinite(Y).all()   # a wait that gave up would have set y to NaN
            for i in range(len(sizes)):
                assert _rel(Y[i], ref[i]) < 2e-6, (call, i, _rel(Y[i], ref[i]))


def test_static_scratch_rejects_oversized_problems(gpu_lib):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    d, k, m = 1024, 32, 512        # m * d * k * 4 bytes of padded Y alone exceed the 32 MiB array
    A = torch.zeros((m * 40, d), dtype=torch.float32, device=dev)
    z = torch.zeros((d, k), dtype=torch.float64, device=dev)
    y = torch.zeros((m, d, k), dtype=torch.float64, device=dev)
    with pytest.raises(B.LPError) as e:
        B.lp_power_step_static(A, [40] * m, k, z, y)
    assert e.value.status == B.LP_ERR_INVALID
    assert "scratch" in B.lp_last_error(None)
