"""CPU checks of the arithmetic arguments behind the cost kernel's exact shortcuts, restated from their
definitions with numpy's IEEE float32 arithmetic (round to nearest): where a shortcut claims that the
contract's float sequence always yields a value, that claim is brute-forced over the pixel range.

- Integer shift (rectified entries): floor(((x + h2) rounded + 0.5) rounded) = x + D, D = floor(h2 + 0.5),
  for every integer x < 2^15, whenever h2 + 0.5 lies more than 2^-23 (2^15 + |h2|) from every integer
  and |h2| < 2^20.
- Rectified row: with |h5| < 0.25, floor(((y + h5) rounded + 0.5) rounded) = y for every y < 2^15.
"""
from __future__ import annotations

import math

import numpy as np

X = np.arange(0, 1 << 15, dtype=np.float32)


def contract_column(h2: np.float32) -> np.ndarray:
    s = (X + h2).astype(np.float32)
    t = (s + np.float32(0.5)).astype(np.float32)
    return np.floor(t).astype(np.int64)


def shift_rule(h2: float):
    """(safe, D) as staged: the kernel's condition, evaluated in double on the float value of h2."""
    d = math.floor(h2 + 0.5)
    g = h2 + 0.5 - d
    return abs(h2) < 2.0 ** 20 and min(g, 1.0 - g) > 2.0 ** -23 * (32768.0 + abs(h2)), d


def _h2_values():
    rng = np.random.default_rng(1909)
    vals = list(rng.uniform(-4000, 4000, 3000)) + list(rng.uniform(-200, 200, 2000))
    # adversarial: just inside and just outside the margin around half-integers, at several magnitudes
    for k in (0.5, 3.5, 10.5, 100.5, 1000.5, -0.5, -250.5, 4000.5):
        m = 2.0 ** -23 * (32768.0 + abs(k))
        for off in (-3 * m, -1.01 * m, -0.99 * m, -1e-6, 0.0, 1e-6, 0.99 * m, 1.01 * m, 3 * m):
            vals.append(k + off)
    return np.unique(np.array(vals, dtype=np.float32))


def test_integer_shift_equals_the_contract_wherever_the_rule_allows_it():
    n_safe = n_unsafe_diff = 0
    for h2 in _h2_values():
        safe, d = shift_rule(float(h2))
        col = contract_column(h2)
        if safe:
            n_safe += 1
            assert np.array_equal(col, X.astype(np.int64) + d), float(h2)
        elif not np.array_equal(col, X.astype(np.int64) + d):
            n_unsafe_diff += 1
    assert n_safe > 4000
    # the margin is not vacuous: values it rejects near half-integers do round the other way somewhere
    assert n_unsafe_diff > 0


def test_rectified_row_is_the_reference_row():
    rng = np.random.default_rng(5)
    h5s = np.concatenate([rng.uniform(-0.25, 0.25, 200), [0.0, -0.0, 0.2499999, -0.2499999, 1e-30, -1e-30]])
    for h5 in h5s.astype(np.float32):
        if not abs(float(h5)) < 0.25:
            continue
        s = (X + h5).astype(np.float32)
        t = (s + np.float32(0.5)).astype(np.float32)
        assert np.array_equal(np.floor(t).astype(np.int64), X.astype(np.int64)), float(h5)
