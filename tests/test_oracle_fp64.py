"""Pins of the oracle's FP64 projection mode (the sample position taken from the unrounded FP64
homography, Sec. III-C's T[.] evaluated in double precision instead of the FP32 contract).

The yardstick is exact rational arithmetic: every table entry is a double, hence an exact fraction, and
floor(u + 1/2) of the exact quotient is computed with Python's Fraction. The FP64 projection can differ
from it only where u + 1/2 lies within ~1e-12 of an integer; the rigs below are checked to stay clear of
that. The second rig is built so that every label's disparity lies 1e-7 below a half-integer, where the
FP32 contract rounds the other way: it pins the FP64 mode exactly where the two modes differ.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth


def _exact_sample(h, x, y, wv, hv):
    """(in view, ui, vi, distance of u + 1/2 and v + 1/2 to the nearest integer) in exact arithmetic."""
    F = [Fraction(float(e)) for e in h]
    X = F[0] * x + F[1] * y + F[2]
    Y = F[3] * x + F[4] * y + F[5]
    Wz = F[6] * x + F[7] * y + F[8]
    if Wz <= 0:
        return False, 0, 0, 1.0
    tu, tv = X / Wz + Fraction(1, 2), Y / Wz + Fraction(1, 2)
    ui, vi = math.floor(tu), math.floor(tv)
    gap = float(min(tu - ui, ui + 1 - tu, tv - vi, vi + 1 - tv))
    return 0 <= ui < wv and 0 <= vi < hv, ui, vi, gap


def _brute_volume(cams, views, ref, nbrs, H64, L, labels, S, penalty):
    """Cost volume with exact sample positions: per pixel the minimum over neighbours of the L1 colour
    distance (or the penalty), summed per segment. Returns (volume, smallest tie gap, in-view count)."""
    Hr, Wr = labels.shape
    vol = np.zeros((S, L), np.int64)
    gap_min, n_in = 1.0, 0
    ref_px = np.stack([np.asarray(a, np.int64) for a in (views[ref].Y, views[ref].U, views[ref].V)], -1)
    for y in range(Hr):
        for x in range(Wr):
            s = labels[y, x]
            for d in range(L):
                best = None
                for k, v in enumerate(nbrs):
                    ok, ui, vi, gap = _exact_sample(H64[k, d], x, y, cams[v].width, cams[v].height)
                    gap_min = min(gap_min, gap)
                    if ok:
                        n_in += 1
                        q = [int(np.asarray(a)[vi, ui]) for a in (views[v].Y, views[v].U, views[v].V)]
                        c = sum(abs(int(ref_px[y, x, ch]) - q[ch]) for ch in range(3))
                    else:
                        c = penalty
                    best = c if best is None else min(best, c)
                vol[s, d] += best
    return vol, gap_min, n_in


def _random_views(cams, seed):
    rng = np.random.default_rng(seed)
    return [synth.View(*(rng.integers(0, 256, (c.height, c.width), dtype=np.uint8) for _ in range(3)))
            for c in cams]


def _near_tie_rig(L=4):
    """Two cameras 0.1 m apart on the x axis with f = 100 px: sample u = x - 10 iz. The depths are chosen so
    that 10 iz_d = 10.5000001 + d, i.e. every disparity lies 1e-7 beyond a half-integer. Exactly,
    floor(u + 1/2) = x - 11 - d; the FP32 table rounds 10.5000001 to 10.5 and gives x - 10 - d."""
    f, B, W, H = 100.0, 0.1, 64, 16
    iz0, iz1 = (10.5000001) / (f * B), (10.5000001 + (L - 1)) / (f * B)
    cams = [synth.Camera(synth.intrinsics(f, W, H), np.eye(3), np.zeros(3), W, H),
            synth.Camera(synth.intrinsics(f, W, H), np.eye(3), -np.array([B, 0.0, 0.0]), W, H)]
    return cams, 1.0 / iz1, 1.0 / iz0


def test_fp64_table_is_the_table_before_its_rounding():
    cams = synth.arc_rig(3, 3.0, 8.0, 80.0, 48, 32, seed=5)
    t32 = oracle.homography_table(cams, 1, [0, 2], 5, 2.0, 5.0)
    t64 = oracle.homography_table_f64(cams, 1, [0, 2], 5, 2.0, 5.0)
    assert t64.dtype == np.float64 and t32.dtype == np.float32
    assert np.array_equal(t64.astype(np.float32), t32)
    iz = oracle.label_inv_depths(5, 2.0, 5.0)
    for k, v in enumerate([0, 2]):
        for d in range(5):
            assert np.array_equal(t64[k, d], oracle.homography_f64(cams[1], cams[v], iz[d]).ravel())
    with pytest.raises(TypeError):
        oracle.cost_volume(cams, _random_views(cams, 1), 1, 1, [0, 2], t64.astype(np.float16), 5,
                           np.zeros((32, 48), np.int32), 1, 765)


def test_fp64_volume_equals_exact_rational_volume_on_a_convergent_rig():
    """Convergent cameras 8 degrees apart (projective homographies with h6, h7 != 0)."""
    cams = synth.arc_rig(3, 3.0, 8.0, 80.0, 48, 32, seed=5)
    views = _random_views(cams, 2)
    lab, S = synth.grid_labels(48, 32, 8, 2, seed=3)
    L, nbrs = 5, [0, 2]
    H64 = oracle.homography_table_f64(cams, 1, nbrs, L, 2.0, 5.0)
    assert np.all(H64[:, :, 6] != 0.0)
    got = oracle.cost_volume(cams, views, 1, 1, nbrs, H64, L, lab, S, 765)
    want, gap, n_in = _brute_volume(cams, views, 1, nbrs, H64, L, lab, S, 765)
    assert gap > 1e-9  # no evaluation near enough to a tie for FP64 rounding to matter
    assert n_in > 0.3 * lab.size * L * len(nbrs)
    assert np.array_equal(got, want)


def test_fp64_volume_on_half_integer_disparities_where_fp32_rounds_the_other_way():
    cams, z_near, z_far = _near_tie_rig()
    views = _random_views(cams, 4)
    lab, S = synth.grid_labels(64, 16, 8, 1, seed=6)
    L = 4
    H64 = oracle.homography_table_f64(cams, 0, [1], L, z_near, z_far)
    H32 = oracle.homography_table(cams, 0, [1], L, z_near, z_far)
    got = oracle.cost_volume(cams, views, 1, 0, [1], H64, L, lab, S, 765)
    want, gap, _ = _brute_volume(cams, views, 0, [1], H64, L, lab, S, 765)
    assert gap > 1e-9
    assert np.array_equal(got, want)
    # the hand-derived sample column, x - 11 - d, for a few pixels and every label
    for d in range(L):
        for x, y in ((20, 3), (40, 9), (63, 15)):
            ok, ui, vi, _ = _exact_sample(H64[0, d], x, y, 64, 16)
            assert (ok, ui, vi) == (x - 11 - d >= 0, x - 11 - d, y)
    # the FP32 contract samples one column to the right on every label
    fp32 = oracle.cost_volume(cams, views, 1, 0, [1], H32, L, lab, S, 765)
    assert np.all(H32[0, :, 2] == -(10.5 + np.arange(L)).astype(np.float32))
    assert not np.array_equal(fp32, got)
    # every evaluation differs except those out of view in both modes (columns x < 10 + d)
    bad, tot = oracle.fp64_mismatch(cams, 0, [1], L, z_near, z_far)
    assert (bad, tot) == (sum((64 - 10 - d) * 16 for d in range(L)), 64 * 16 * L)


def test_fp64_centre_table_on_half_integer_disparities():
    """Centre table in the FP64 mode: the centre of each segment lands on column mx - 11 - d, exactly."""
    cams, z_near, z_far = _near_tie_rig()
    views = _random_views(cams, 7)
    lab, S = synth.grid_labels(64, 16, 8, 1, seed=6)
    lab1, _ = synth.grid_labels(64, 16, 5, 1, seed=8)
    L = 4
    H64 = oracle.homography_table_f64(cams, 0, [1], L, z_near, z_far)
    m, sp = oracle.centre_table(cams, views, 1, 0, [1], H64, L, [lab, lab1], S, 3, 765)
    ys, xs = np.mgrid[0:16, 0:64]
    Y0, Y1 = [np.stack([np.asarray(a, np.int64) for a in (v.Y, v.U, v.V)], -1) for v in views]
    for s in range(S):
        sel = lab == s
        n = int(sel.sum())
        mx = (2 * int(xs[sel].sum()) + n) // (2 * n)
        my = (2 * int(ys[sel].sum()) + n) // (2 * n)
        for d in range(L):
            ui, vi = mx - 11 - d, my
            if ui < 0:
                assert m[s, d, 0] == 9 * 765 and sp[s, d, 0] == -1
                continue
            want = 0
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    rx, ry, qx, qy = mx + dx, my + dy, ui + dx, vi + dy
                    if not (0 <= rx < 64 and 0 <= ry < 16 and 0 <= qx < 64 and 0 <= qy < 16):
                        want += 765
                    else:
                        want += int(np.abs(Y0[ry, rx] - Y1[qy, qx]).sum())
            assert m[s, d, 0] == want, (s, d)
            assert sp[s, d, 0] == lab1[vi, ui]


def test_fp64_behind_the_camera_is_out_of_view():
    """A camera at the reference centre looking backwards, R = diag(-1, 1, -1): every candidate plane is
    behind it (Wz < 0), although X / Wz falls inside its image. Every sample is out of view."""
    cams = synth.arc_rig(3, 3.0, 8.0, 80.0, 48, 32, seed=5)
    cr = cams[1]
    back = synth.Camera(cr.K.copy(), np.diag([-1.0, 1.0, -1.0]) @ cr.R, np.zeros(3), cr.width, cr.height)
    back.t = -back.R @ cr.centre
    cams = cams + [back]
    views = _random_views(cams, 9)
    lab, S = synth.grid_labels(48, 32, 8, 2, seed=3)
    H64 = oracle.homography_table_f64(cams, 1, [3], 3, 2.0, 5.0)
    x, y = 20, 10
    h = H64[0, 1]
    Wz = h[6] * x + h[7] * y + h[8]
    u = (h[0] * x + h[1] * y + h[2]) / Wz
    assert Wz < 0 and 0 <= math.floor(u + 0.5) < 48
    got = oracle.cost_volume(cams, views, 1, 1, [3], H64, 3, lab, S, 765)
    n = np.bincount(lab.ravel(), minlength=S).astype(np.int64)
    assert np.array_equal(got, np.repeat((n * 765)[:, None], 3, 1))
    want, _, n_in = _brute_volume(cams, views, 1, [3], H64, 3, lab, S, 765)
    assert n_in == 0 and np.array_equal(got, want)


@pytest.mark.parametrize("name,lo,hi", [("tiny", 0.0, 0.0), ("serving_small", 0.0, 0.0), ("hd8", 1e-3, 4e-3),
                                        ("uhd15", 5e-5, 2e-4)])
def test_fp32_contract_mismatch_fraction_per_workload(name, lo, hi):
    """The reported figure: the fraction of evaluations whose FP32-contract sample (or in/out decision)
    differs from the FP64 projection, on 20,000 seeded pixels of the first reference x every label x every
    neighbour. The 1920x1080 rectified rig concentrates it in the few (label, view) pairs whose disparity
    lies within FP32 resolution of a half-integer; the 3840x2160 convergent rig spreads it thinly. The
    FP64 projection mode has none by construction. Printed with -s."""
    from synth.configs import make_workload
    wl = make_workload(name)
    r = wl.ref_views[0]
    c = wl.cams[r]
    pix = np.random.default_rng(7).integers(0, c.width * c.height, 20000).astype(np.int32)
    bad, tot = oracle.fp64_mismatch(wl.cams, r, wl.neighbours(r), wl.n_labels, wl.z_near, wl.z_far, pix=pix)
    print(f"{name}: FP32-contract vs FP64-projection sample mismatch {bad} of {tot} = {bad / tot:.3e}")
    assert lo <= bad / tot <= hi
