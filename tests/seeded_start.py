"""Test-side implementation of the start block that lp_solve_seeded draws:
SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) on counters, the top 53 bits as a uniform in [0, 1),
and the Box-Muller transform on consecutive pairs.  Written from the published
definitions, independently of the library's C implementation."""
import math

import numpy as np

_MASK = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15


def splitmix64_at(seed: int, counter: int) -> int:
    """The (counter + 1)-th output of SplitMix64 whose state starts at `seed`."""
    z = (seed + (counter + 1) * _GAMMA) & _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def seeded_start(seed: int, d: int, k: int) -> np.ndarray:
    """d x k N(0,1) block, row-major entries 2q (cosine) and 2q + 1 (sine) from counters 2q, 2q + 1."""
    n = d * k
    out = np.empty(n)
    for q in range((n + 1) // 2):
        u1 = (splitmix64_at(seed, 2 * q) >> 11) * 2.0 ** -53
        u2 = (splitmix64_at(seed, 2 * q + 1) >> 11) * 2.0 ** -53
        r = math.sqrt(-2.0 * math.log1p(-u1))
        out[2 * q] = r * math.cos(2.0 * math.pi * u2)
        if 2 * q + 1 < n:
            out[2 * q + 1] = r * math.sin(2.0 * math.pi * u2)
    return out.reshape(d, k)
