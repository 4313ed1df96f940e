"""The synthetic workloads: shapes, spectra, schedules and seeds.

They stand in for the paper's LIBSVM datasets (Sec. 5 and Table 4: n from 506
to 581,012, d from 6 to 780, k = 5, about 1,000 rows per node), which are not
used here.  Rows are spiked Gaussian (see ``spiked``).

  plain   n=4,000      d=100   k=5   m=4    p=4, T=20          lam_j = 0.8^j (j=1..d), sigma = 0.1
  fp32    n=1,000,000  d=1,024 k=16  m=64   p = 8,4,2,1 (10 rounds each), then 10 more rounds at p = 1
                                            (T = 50, 160 local steps: the decaying schedule alone stops
                                            at dist ~1.4e-4 to the top-16 subspace with sign-fixing)
                                            lam_j = 10*0.9^j (j<=32), noise variance 0.1
  lowprec n=4,000,000  d=2,048 k=32  m=128  p=4, T=30, then 3 refinement rounds
                                            lam_j = j^-1.5 (j<=k), 0.5*j^-1.5 (k<j<=4k), noise variance 1e-3
"""
from __future__ import annotations

import numpy as np

from .spiked import gaussian_start, partition_sizes, spiked_rows

SEED_BASE = 2002_08014 * 10


def _decay(p0: int, per: int) -> list[int]:
    out, p = [], p0
    while p >= 1:
        out += [p] * per
        p //= 2
    return out


CONFIGS = {
    "plain": dict(index=0, n=4_000, d=100, k=5, m=4, schedule=[4] * 20, aggs=("sign", "opt", "identity"),
                  lam=lambda d, k: 0.8 ** np.arange(1, d + 1), noise_sigma=0.1, dtype="f32"),
    "fp32": dict(index=1, n=1_000_000, d=1024, k=16, m=64, schedule=_decay(8, 10) + [1] * 10, aggs=("sign", "opt"),
                 lam=lambda d, k: 10.0 * 0.9 ** np.arange(1, 33), noise_sigma=float(np.sqrt(0.1)), dtype="f32"),
    "lowprec": dict(index=2, n=4_000_000, d=2048, k=32, m=128, schedule=[4] * 30, refine_rounds=3,
                    aggs=("sign",),
                    lam=lambda d, k: np.concatenate([np.arange(1, k + 1) ** -1.5,
                                                     0.5 * np.arange(k + 1, 4 * k + 1) ** -1.5]),
                    noise_sigma=float(np.sqrt(1e-3)), dtype="bf16"),
}


def config_schedule(name: str) -> list[int]:
    c = CONFIGS[name]
    return list(c["schedule"]) + [1] * int(c.get("refine_rounds", 0))


def make_config_data(name: str, n: int | None = None, m: int | None = None, threads: int | None = None):
    """(A as float32 n x d, partition sizes, Y_0) for a named workload.

    ``n``/``m`` override the row and partition counts (same spectrum, same seeds),
    which gives smaller cases with the workload's structure.
    """
    c = CONFIGS[name]
    n = c["n"] if n is None else int(n)
    m = c["m"] if m is None else int(m)
    seed = SEED_BASE + c["index"]
    lam = c["lam"](c["d"], c["k"])
    A = spiked_rows(n, c["d"], lam, c["noise_sigma"], seed, threads=threads)
    sizes = partition_sizes(n, m)
    Y0 = gaussian_start(c["d"], c["k"], seed)
    return A, sizes, Y0
