"""Encoders for the reduced-precision stored forms of the data matrix.

These make the bytes a caller would hand to the library (BF16, or FP8-E4M3 with
one FP32 scale per row).  They are input preparation, not part of LocalPower;
the oracle decodes the stored bytes with its own decoder and never re-encodes.

* BF16: the top 16 bits of the FP32 pattern after round-to-nearest-even.
* BF16x2 planes of FP32 data: hi = BF16(a), lo = BF16(a - hi), both RNE; a - hi
  is exact in FP32, so the stored matrix hi + lo is within 2^-17 |a| of a.
* FP8-E4M3 (the OCP "FN" variant: bias 7, no infinities, max 448):
  scale_r = max_j |a_rj| / 448 in FP32 (1 for an all-zero row), then
  q_rj = E4M3(a_rj / scale_r) with round-to-nearest-even and saturation to
  +-448 (satfinite).
"""
from __future__ import annotations

import numpy as np

E4M3_MAX = 448.0


def f32_to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """FP32 array -> uint16 BF16 bit patterns (round to nearest even, NaN kept quiet)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    u = x.view(np.uint32)
    lsb = (u >> np.uint32(16)) & np.uint32(1)
    r = (u + np.uint32(0x7FFF) + lsb) >> np.uint32(16)
    nan = np.isnan(x)
    if nan.any():
        r = np.where(nan, (u >> np.uint32(16)) | np.uint32(0x40), r)
    return r.astype(np.uint16)


def f32_to_bf16x2_planes(x: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """FP32 array -> (hi, lo) uint16 BF16 bit patterns with hi = BF16(x), lo = BF16(x - hi)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    hi = f32_to_bf16_bits(x)
    hi_val = (hi.astype(np.uint32) << np.uint32(16)).view(np.float32)
    lo = f32_to_bf16_bits((x - hi_val).astype(np.float32))
    return hi, lo


def _e4m3_positive_table() -> np.ndarray:
    """Values of the finite non-negative E4M3 codes 0..126, ascending."""
    vals = np.empty(127, dtype=np.float64)
    for c in range(127):
        e, m = c >> 3, c & 7
        vals[c] = (m / 8.0) * 2.0 ** -6 if e == 0 else (1.0 + m / 8.0) * 2.0 ** (e - 7)
    return vals


_E4M3_POS = _e4m3_positive_table()


def _e4m3_encode(y: np.ndarray) -> np.ndarray:
    """FP32 values (already scaled) -> E4M3 codes, RNE, satfinite."""
    a = np.abs(y.astype(np.float64))
    a = np.minimum(a, E4M3_MAX)
    hi = np.searchsorted(_E4M3_POS, a, side="left")          # first table value >= a
    hi = np.minimum(hi, 126)
    lo = np.maximum(hi - 1, 0)
    vhi, vlo = _E4M3_POS[hi], _E4M3_POS[lo]
    exact = vhi == a
    dlo, dhi = a - vlo, vhi - a
    pick_hi = (dhi < dlo) | ((dhi == dlo) & ((hi & 1) == 0))
    code = np.where(exact, hi, np.where(pick_hi, hi, lo)).astype(np.uint8)
    sign = (np.signbit(y) & (code != 0)).astype(np.uint8) << np.uint8(7)
    return code | sign


def f32_to_e4m3_rowscaled(x: np.ndarray, block_rows: int = 4096):
    """FP32 n x d -> (uint8 codes n x d, float32 scales n)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    n, d = x.shape
    codes = np.empty((n, d), dtype=np.uint8)
    scales = np.empty(n, dtype=np.float32)
    for r0 in range(0, n, block_rows):
        blk = x[r0:r0 + block_rows]
        amax = np.max(np.abs(blk), axis=1)
        sc = (amax / np.float32(E4M3_MAX)).astype(np.float32)
        sc[sc == 0] = np.float32(1.0)
        scales[r0:r0 + block_rows] = sc
        codes[r0:r0 + block_rows] = _e4m3_encode((blk / sc[:, None]).astype(np.float32))
    return codes, scales
