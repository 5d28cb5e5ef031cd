"""Exact IEEE float32 arithmetic on the CPU for tests: numpy's float32 add, multiply and divide round to
nearest; the fused multiply-add is emulated here. The product of two floats is exact in double, the sum
is carried as a double pair (TwoSum), and the only case where rounding that pair to float32 differs from
rounding its leading double -- a leading part exactly halfway between two floats -- is settled by the sign
of the trailing part."""
from __future__ import annotations

import numpy as np


def fma32(a, b, c):
    a, b, c = (np.asarray(v, np.float32).astype(np.float64) for v in (a, b, c))
    p = a * b  # exact: two 24-bit significands
    s = p + c
    bb = s - p
    e = (p - (s - bb)) + (c - bb)  # TwoSum: s + e == p + c exactly
    r = s.astype(np.float32)  # s rounded to float32, ties to even
    d = s - r.astype(np.float64)  # exact (s and r are close)
    nb = np.where(d > 0, np.nextafter(r, np.float32(np.inf)), np.nextafter(r, np.float32(-np.inf)))
    gap = np.abs(nb.astype(np.float64) - r.astype(np.float64))
    mid = (d != 0) & (2.0 * np.abs(d) == gap)  # s lies exactly halfway between r and nb
    # at a midpoint the exact value p + c = s + e lies beyond it (towards nb) when e has the sign of d
    return np.where(mid & (e != 0) & (np.sign(e) == np.sign(d)), nb, r).astype(np.float32)
