"""CPU checks of the arithmetic arguments behind the cost kernel's exact shortcuts, restated from their
definitions with numpy's IEEE float32 arithmetic (round to nearest): where a shortcut claims that the
contract's float sequence always yields a value, that claim is brute-forced over the pixel range.

- Integer shift (rectified entries): floor(((x + h2) rounded + 0.5) rounded) = x + D, D = floor(h2 + 0.5),
  for every integer x < 2^15, whenever h2 + 0.5 lies more than 2^-23 (2^15 + |h2|) from every integer
  and |h2| < 2^20.
- Rectified row: with |h5| < 0.25, floor(((y + h5) rounded + 0.5) rounded) = y for every y < 2^15.
- The same two claims for the FP64 projection of FP64-precision contexts (shift_fp64), in IEEE double:
  the column is x + D when h2 + 0.5 is an integer or lies more than 2^-30 from every integer, and the row
  is y when |h5| < 0.49.
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


# ------------------------------------------------------------------- FP64 projection, integer shift

X64 = np.arange(0, 1 << 15, dtype=np.float64)


def fp64_projection_column(h2: float) -> np.ndarray:
    """The FP64 projection's column for H = [[1, 0, h2], [0, 1, h5], [0, 0, 1]], operation by operation in
    IEEE double (numpy rounds each operation to nearest): X = (1 x + 0 y) + h2, Wz = (0 x + 0 y) + 1,
    floor(X / Wz + 0.5)."""
    y = 7.0
    X = (1.0 * X64 + 0.0 * y) + h2
    W = (0.0 * X64 + 0.0 * y) + 1.0
    return np.floor(X / W + 0.5).astype(np.int64)


def fp64_shift_rule(h2: float):
    """(safe, D) as the kernel stages it (shift_fp64): |h2| < 2^20 and h2 + 0.5 an integer or more than 2^-30
    from every integer."""
    g = h2 + 0.5
    f = math.floor(g)
    r = g - f
    return abs(h2) < 2.0 ** 20 and (r == 0.0 or min(r, 1.0 - r) > 2.0 ** -30), int(f)


def _h2_values_fp64():
    rng = np.random.default_rng(1910)
    vals = list(rng.uniform(-4000, 4000, 3000)) + [k - 0.5 for k in range(-40, 41)]  # exact half-integers
    for k in (0.5, 3.5, 100.5, 1000.5, -0.5, -250.5, 4000.5, 2.0 ** 19 + 0.5):
        for off in (-2.0 ** -29, -2.0 ** -30 * 1.01, -2.0 ** -30 * 0.99, -2.0 ** -40, -2.0 ** -44, 2.0 ** -44,
                    2.0 ** -40, 2.0 ** -30 * 0.99, 2.0 ** -30 * 1.01, 2.0 ** -29):
            vals.append(k + off)
    return np.unique(np.array(vals, dtype=np.float64))


def test_fp64_integer_shift_equals_the_fp64_projection_wherever_the_rule_allows_it():
    n_safe = n_unsafe_diff = 0
    for h2 in _h2_values_fp64():
        safe, d = fp64_shift_rule(float(h2))
        col = fp64_projection_column(float(h2))
        if safe:
            n_safe += 1
            assert np.array_equal(col, X64.astype(np.int64) + d), float(h2)
        elif not np.array_equal(col, X64.astype(np.int64) + d):
            n_unsafe_diff += 1
    assert n_safe > 3000
    # the margin is not vacuous: values within 2^-30 of a half-integer (not on it) round the other way
    assert n_unsafe_diff > 0


def test_fp64_rectified_row_is_the_reference_row():
    rng = np.random.default_rng(6)
    for h5 in np.concatenate([rng.uniform(-0.49, 0.49, 200), [0.0, 0.4899999, -0.4899999]]):
        Y = (0.0 * 3.0 + 1.0 * X64) + float(h5)
        assert np.array_equal(np.floor(Y / 1.0 + 0.5).astype(np.int64), X64.astype(np.int64)), float(h5)
