"""Spiked-Gaussian rows, Gaussian start blocks and row partitions.

The data model: each row is a = U diag(sqrt(lam)) g + sigma e, with U a random
orthonormal d x q matrix, g ~ N(0, I_q) and e ~ N(0, I_d).  The rows are iid, so
cutting them into contiguous blocks gives the same distribution as the paper's
shuffle-then-partition (Sec. 5, Settings).

Determinism: every row block of BLOCK_ROWS rows draws from its own
``SeedSequence(seed, spawn_key=(stream, block))``, so the bytes do not depend on
the number of threads used to make them.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

BLOCK_ROWS = 8192

# Sub-stream identifiers (independent SeedSequence spawn keys).
STREAM_U = 1
STREAM_ROWS = 2
STREAM_START = 3


def _rng(seed: int, *key: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(int(seed), spawn_key=tuple(int(x) for x in key))))


def partition_sizes(n: int, m: int) -> list[int]:
    """Row counts s_i of m contiguous partitions of n rows: floor(n/m) + [i < n mod m]."""
    if m < 1 or n < m:
        raise ValueError(f"need 1 <= m <= n, got n={n}, m={m}")
    q, r = divmod(n, m)
    return [q + (1 if i < r else 0) for i in range(m)]


def split_rows(A: np.ndarray, sizes) -> list[np.ndarray]:
    """Contiguous row blocks of A with the given sizes (views, no copy)."""
    out, o = [], 0
    for s in sizes:
        out.append(A[o:o + s])
        o += s
    if o != A.shape[0]:
        raise ValueError("partition sizes do not add up to the row count")
    return out


def haar_columns(d: int, q: int, seed: int) -> np.ndarray:
    """d x q matrix with orthonormal columns, Haar distributed (QR of a Gaussian
    with the signs of diag(R) moved into Q, Mezzadri 2007)."""
    G = _rng(seed, STREAM_U).standard_normal((d, q))
    Q, R = np.linalg.qr(G)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s


def spiked_rows(n: int, d: int, lam, noise_sigma: float, seed: int,
                out_dtype=np.float32, threads: int | None = None, U: np.ndarray | None = None) -> np.ndarray:
    """n x d row-major matrix of spiked-Gaussian rows (see module docstring).

    lam: the q spike variances lam_1..lam_q (q <= d).  The rows are made in
    FP64 and rounded once to ``out_dtype`` (round-to-nearest-even for float32).
    """
    lam = np.asarray(lam, dtype=np.float64)
    q = lam.shape[0]
    if q > d:
        raise ValueError("more spikes than dimensions")
    if U is None:
        U = haar_columns(d, q, seed)
    B = np.ascontiguousarray((U * np.sqrt(lam)).T)  # q x d: row-vector form g^T (U diag(sqrt lam))^T
    out = np.empty((n, d), dtype=out_dtype)
    nblk = (n + BLOCK_ROWS - 1) // BLOCK_ROWS

    def one(b: int) -> None:
        r0 = b * BLOCK_ROWS
        r1 = min(n, r0 + BLOCK_ROWS)
        rng = _rng(seed, STREAM_ROWS, b)
        g = rng.standard_normal((r1 - r0, q))
        e = rng.standard_normal((r1 - r0, d))
        blk = g @ B
        blk += noise_sigma * e
        out[r0:r1] = blk  # one rounding to out_dtype

    if threads is None:
        threads = min(32, os.cpu_count() or 1)
    if threads <= 1 or nblk == 1:
        for b in range(nblk):
            one(b)
    else:
        with ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(one, range(nblk)))
    return out


def gaussian_start(d: int, k: int, seed: int) -> np.ndarray:
    """The standard Gaussian d x k start block Y_0 (Alg. 1, initialisation), FP64
    row-major.  Both sides orthonormalise it themselves."""
    return np.ascontiguousarray(_rng(seed, STREAM_START).standard_normal((d, k)))
