"""Pins of the oracle's segment adjacency and adaptive smoothing weights (Eq. 2-3, Sec. III-D)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from synth.configs import make_workload


def test_grid_edge_counts_closed_form():
    """A jittered grid of R x C cells has (C-1)R + C(R-1) 4-connected edges and 2(C-1)(R-1) more
    diagonal ones (its boundaries are straight lines, so cells meet at every grid corner)."""
    for W, H, cell, seed in [(480, 270, 16, 3), (244, 138, 8, 5), (97, 61, 10, 7)]:
        lab, S = synth.grid_labels(W, H, cell, 3, seed)
        C, R = (W + cell - 1) // cell, (H + cell - 1) // cell
        frame = synth.View(*(np.zeros((H, W), np.uint8) for _ in range(3)))
        es, et, _ = oracle.adjacency(lab, S, frame, 1, 4)
        assert len(es) == (C - 1) * R + C * (R - 1)
        es8, et8, _ = oracle.adjacency(lab, S, frame, 1, 8)
        assert len(es8) == len(es) + 2 * (C - 1) * (R - 1)
        assert np.all(es < et) and np.all(np.diff(es.astype(np.int64) * S + et) > 0)  # sorted, unique


def test_beta_of_uniform_segments():
    """Segments of constant colour: beta = beta0 / (|dY| + |dCb| + |dCr|); equal colours hit the floor."""
    lab = np.zeros((4, 6), np.int32)
    lab[:, 3:] = 1
    lab[2:, :3] = 2
    Y = np.where(lab == 0, 10, np.where(lab == 1, 40, 10)).astype(np.uint16)
    U = np.where(lab == 1, 25, 20).astype(np.uint16)
    V = np.full_like(Y, 7)
    es, et, b = oracle.adjacency(lab, 3, synth.View(Y, U, V), 2, 4, beta0=70.0, min_diff=2.0)
    got = {(int(s), int(t)): float(x) for s, t, x in zip(es, et, b)}
    assert got == {(0, 1): pytest.approx(70.0 / 35.0), (0, 2): pytest.approx(70.0 / 2.0),
                   (1, 2): pytest.approx(70.0 / 35.0)}
    assert got[(0, 1)] == np.float32(2.0) and got[(0, 2)] == np.float32(35.0)


@pytest.mark.parametrize("conn", [4, 8])
def test_adjacency_against_numpy(conn):
    wl = make_workload("hd8", reduced=True)
    r = 3
    lab, S = wl.labels(r)
    v = wl.view(r)
    es, et, b = oracle.adjacency(lab, S, v, 2, conn, beta0=50.0, min_diff=1.0)
    pairs = [(lab[:, :-1], lab[:, 1:]), (lab[:-1, :], lab[1:, :])]
    if conn == 8:
        pairs += [(lab[:-1, :-1], lab[1:, 1:]), (lab[:-1, 1:], lab[1:, :-1])]
    keys = set()
    for a, c in pairs:
        m = a != c
        lo, hi = np.minimum(a[m], c[m]), np.maximum(a[m], c[m])
        keys |= set(zip(lo.tolist(), hi.tolist()))
    assert set(zip(es.tolist(), et.tolist())) == keys
    n = np.bincount(lab.ravel(), minlength=S).astype(np.float64)
    means = np.stack([np.bincount(lab.ravel(), weights=np.asarray(ch, np.float64).ravel(), minlength=S) / n
                      for ch in (v.Y, v.U, v.V)], 1)
    dist = np.abs(means[es] - means[et]).sum(1)
    np.testing.assert_allclose(b, 50.0 / np.maximum(dist, 1.0), rtol=1e-6)
