"""Pins of the CPU oracle against facts fixed by the paper and by geometry, not by the oracle itself.

Each pin is chosen so that a plausible mistake in the oracle (a dropped term, a swapped x/y, a
wrong sign in the plane offset, a transposed rotation, a wrong tie-break or threshold comparison)
fails at least one of them:
  - candidate depths uniform in 1/z between z_far and z_near (Sec. IV-A);
  - the FP64 homography against an independent 3D back-project / transform / project path, for
    reference-camera planes and for centre-camera planes (Eq. 4's T[.], Sec. III-B);
  - the closed form of the homography for an identical-intrinsics, parallel-axes, x-baseline rig;
  - the whole cost volume against an independent FP64 ray path on every (segment, label) entry;
  - zero cost and correct winner at the true label of painted fronto-parallel planes (Eq. 4);
  - a duplicated reference view costs nothing; a view that sees nothing costs the penalty;
  - the temporal test at exact threshold boundaries, I-frame adoption and the channel modes
    (Sec. III-E, T_P = 3 and T_I = 1);
  - winner-take-all ties and adoption.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import oracle_runs
import synth
from synth.configs import label_depth, make_workload


# ------------------------------------------------------------------------------ independent paths

def _iz(d, L, zn, zf):
    return 1.0 / zf + d * ((1.0 / zn - 1.0 / zf) / (L - 1))


def _world_points_ref_plane(cam_r, z, xs, ys):
    """Back-project reference pixels onto the plane at camera depth z (ray through K^-1 (x, y, 1))."""
    rays = np.linalg.solve(cam_r.K, np.stack([xs, ys, np.ones_like(xs)]).reshape(3, -1).astype(np.float64))
    rays = rays / rays[2]
    Xr = rays * z
    return cam_r.R.T @ (Xr - cam_r.t[:, None])


def _world_points_centre_plane(cam_r, cam_c, z, xs, ys):
    """Intersect reference pixel rays with the plane at depth z in front of the centre camera."""
    rays = np.linalg.solve(cam_r.K, np.stack([xs, ys, np.ones_like(xs)]).reshape(3, -1).astype(np.float64))
    dw = cam_r.R.T @ rays
    C = cam_r.centre[:, None]
    # depth of a world point in the centre camera: e3 . (R_c X + t_c)
    rc = cam_c.R[2]
    lam = (z - cam_c.t[2] - rc @ C) / (rc @ dw)
    return C + lam * dw


def _project(cam, Xw):
    Xv = cam.R @ Xw + cam.t[:, None]
    uvw = cam.K @ Xv
    return uvw[0] / uvw[2], uvw[1] / uvw[2], Xv[2]


def _cost_fp64(wl, r, d, frame=0):
    """Independent per-pixel combined cost of label d via FP64 3D geometry, then segment sums."""
    cr = wl.cams[r]
    H, W = cr.height, cr.width
    ys, xs = np.mgrid[0:H, 0:W]
    z = 1.0 / _iz(d, wl.n_labels, wl.z_near, wl.z_far)
    Xw = _world_points_ref_plane(cr, z, xs.astype(np.float64), ys.astype(np.float64))
    ref = wl.view(r, frame)
    refc = [np.asarray(a, np.int64).ravel() for a in (ref.Y, ref.U, ref.V)]
    acc = None
    for v in wl.neighbours(r):
        cv = wl.cams[v]
        u, vv, zc = _project(cv, Xw)
        ui, vi = np.floor(u + 0.5), np.floor(vv + 0.5)
        inside = (zc > 0) & (ui >= 0) & (ui <= cv.width - 1) & (vi >= 0) & (vi <= cv.height - 1)
        uc, vc = np.where(inside, ui, 0).astype(np.int64), np.where(inside, vi, 0).astype(np.int64)
        img = wl.view(v, frame)
        c = np.zeros(H * W, np.int64)
        for a, plane in zip(refc, (img.Y, img.U, img.V)):
            c += np.abs(a - np.asarray(plane, np.int64)[vc, uc])
        c = np.where(inside, c, wl.oob_penalty)
        if acc is None:
            acc = c
        elif wl.combine == "min":
            acc = np.minimum(acc, c)
        else:
            acc = acc + c
    lab, S = wl.labels(r)
    return np.bincount(lab.ravel(), weights=acc.astype(np.float64), minlength=S).astype(np.int64)


# ------------------------------------------------------------------------------------------ depths

def test_label_depths_uniform_in_inverse_depth():
    L, zn, zf = 250, 1.0, 20.0
    iz = oracle.label_inv_depths(L, zn, zf)
    assert iz[0] == pytest.approx(1.0 / zf, rel=1e-15)
    assert iz[-1] == pytest.approx(1.0 / zn, rel=1e-14)
    steps = np.diff(iz)
    assert np.allclose(steps, (1.0 / zn - 1.0 / zf) / (L - 1), rtol=1e-9, atol=0)
    assert np.all(steps > 0)  # label 0 is the far plane


# -------------------------------------------------------------------------------------- homography

@pytest.mark.parametrize("rig", ["linear", "arc"])
def test_homography_matches_3d_path_reference_planes(rig):
    if rig == "linear":
        cams = synth.linear_rig(4, 0.1, 1500.0, 1920, 1080)
    else:
        cams = synth.arc_rig(5, 3.0, 8.0, 3000.0, 3840, 2160, seed=7)
    rng = np.random.default_rng(1)
    for r, v in [(0, 1), (1, 3), (2, 0)]:
        for z in [0.8, 2.5, 14.0]:
            Hm = oracle.homography_f64(cams[r], cams[v], 1.0 / z)
            xs = rng.uniform(0, cams[r].width - 1, 50)
            ys = rng.uniform(0, cams[r].height - 1, 50)
            u3, v3, _ = _project(cams[v], _world_points_ref_plane(cams[r], z, xs, ys))
            p = Hm @ np.stack([xs, ys, np.ones_like(xs)])
            np.testing.assert_allclose(p[0] / p[2], u3, rtol=0, atol=1e-7)
            np.testing.assert_allclose(p[1] / p[2], v3, rtol=0, atol=1e-7)


def test_homography_matches_3d_path_centre_planes():
    cams = synth.arc_rig(5, 3.0, 8.0, 3000.0, 3840, 2160, seed=11)
    rng = np.random.default_rng(2)
    c = 2
    for r, v in [(0, 1), (4, 2), (1, 3)]:
        for z in [1.0, 3.0, 12.0]:
            Hm = oracle.homography_f64(cams[r], cams[v], 1.0 / z, cam_c=cams[c])
            xs = rng.uniform(0, 3839, 40)
            ys = rng.uniform(0, 2159, 40)
            u3, v3, _ = _project(cams[v], _world_points_centre_plane(cams[r], cams[c], z, xs, ys))
            p = Hm @ np.stack([xs, ys, np.ones_like(xs)])
            np.testing.assert_allclose(p[0] / p[2], u3, rtol=0, atol=1e-6)
            np.testing.assert_allclose(p[1] / p[2], v3, rtol=0, atol=1e-6)


def test_homography_closed_form_for_x_baseline():
    """Identical K, R = I, centres on the x axis: H = [[1, 0, f (x_r - x_v) / z], [0, 1, 0], [0, 0, 1]]."""
    f = 1234.5
    cams = synth.linear_rig(3, 0.07, f, 640, 480)
    L, zn, zf = 16, 0.5, 9.0
    tab = oracle.homography_table(cams, 1, [0, 2], L, zn, zf)
    for k, v in enumerate([0, 2]):
        for d in range(L):
            iz = _iz(d, L, zn, zf)
            expect = np.array([1, 0, f * (cams[1].centre[0] - cams[v].centre[0]) * iz, 0, 1, 0, 0, 0, 1])
            np.testing.assert_allclose(tab[k, d], expect.astype(np.float32), rtol=2e-7, atol=2e-7)
            assert tab[k, d, 8] == 1.0 and tab[k, d, 6] == 0.0 and tab[k, d, 7] == 0.0


def test_centre_planes_equal_reference_planes_for_parallel_rig():
    """Sec. III-B: with parallel optical axes the two depth definitions coincide."""
    cams = synth.linear_rig(5, 0.1, 1500.0, 1920, 1080)
    a = oracle.homography_table(cams, 1, [0, 2, 4], 50, 1.0, 20.0, plane_mode=0)
    b = oracle.homography_table(cams, 1, [0, 2, 4], 50, 1.0, 20.0, plane_mode=1, centre=2)
    np.testing.assert_allclose(a, b, rtol=3e-7, atol=1e-6)


# ------------------------------------------------------------------------------------- cost volume

@pytest.mark.parametrize("name,combine", [("tiny", "min"), ("tiny", "sum"), ("uhd15", "min")])
def test_cost_volume_against_fp64_ray_path(name, combine):
    """Every (segment, label) entry of the oracle's FP32-contract volume equals the FP64 ray-path
    sum, except entries holding a pixel whose FP32 sample position differs from FP64's (rare)."""
    wl = make_workload(name, reduced=(name != "tiny"))
    wl.combine = combine
    r = wl.ref_views[0] if name == "tiny" else 7
    vol = oracle_runs.volume(wl, r)
    labels = range(wl.n_labels) if name == "tiny" else range(0, wl.n_labels, 6)
    n_eq = n_tot = 0
    for d in labels:
        ref = _cost_fp64(wl, r, d)
        eq = vol[:, d] == ref
        n_eq += int(eq.sum())
        n_tot += eq.size
        # where they differ, the difference is at most a few samples' worth
        bound = 4 * wl.oob_penalty * (len(wl.neighbours(r)) if combine == "sum" else 1)
        assert np.all(np.abs(vol[:, d].astype(np.int64) - ref) <= bound)
    assert n_eq / n_tot > 0.99, (n_eq, n_tot)


@pytest.mark.parametrize("name,combine", [("tiny", "min"), ("tiny", "sum"), ("uhd15", "min"), ("uhd15", "sum")])
def test_cost_entries_equal_the_volume_rows(name, combine):
    """The single-entry checker (or_cost_entries, used at sizes where the whole volume is too slow) returns,
    for every requested (segment, label) pair in any order, that entry of the volume, and the volume itself
    is pinned to the FP64 ray path above. Pairs are drawn so that segment and label indices differ (a
    swapped index or a wrong row stride would read another entry), with repeats, the last segment and the
    last label, and segments that own no pixel (cost 0)."""
    wl = make_workload(name, reduced=(name != "tiny"))
    wl.combine = combine
    r = wl.ref_views[-1]
    vol = oracle_runs.volume(wl, r)
    S, L = vol.shape
    rng = np.random.default_rng(7)
    seg = np.concatenate([rng.integers(0, S, 400), [S - 1, 0, S - 1], rng.integers(0, S, 5)]).astype(np.int32)
    lab = np.concatenate([rng.integers(0, L, 400), [L - 1, L - 1, 0], rng.integers(0, L, 5)]).astype(np.int32)
    got = oracle_runs.entries(wl, r, seg, lab)
    np.testing.assert_array_equal(got, vol[seg, lab])
    # a whole label column and a whole segment row
    col = oracle_runs.entries(wl, r, np.arange(S, dtype=np.int32), np.full(S, L // 2, np.int32))
    np.testing.assert_array_equal(col, vol[:, L // 2])
    row = oracle_runs.entries(wl, r, np.full(L, S // 3, np.int32), np.arange(L, dtype=np.int32))
    np.testing.assert_array_equal(row, vol[S // 3])


def test_cost_entries_against_fp64_ray_path():
    """or_cost_entries on whole label columns against the FP64 ray path directly (the same >99 % agreement
    the volume has; the rest differ only where an FP32 sample position differs from FP64's)."""
    wl = make_workload("tiny")
    r = wl.ref_views[0]
    lab, S = wl.labels(r)
    for d in (0, 17, wl.n_labels - 1):
        got = oracle_runs.entries(wl, r, np.arange(S, dtype=np.int32), np.full(S, d, np.int32)).astype(np.int64)
        ref = _cost_fp64(wl, r, d)
        assert np.mean(got == ref) > 0.99
        assert np.all(np.abs(got - ref) <= 4 * wl.oob_penalty)


def test_cost_entries_reject_out_of_range_pairs():
    wl = make_workload("tiny")
    r = wl.ref_views[0]
    lab, S = wl.labels(r)
    for seg, lb in (([S], [0]), ([-1], [0]), ([0], [wl.n_labels]), ([0], [-1])):
        with pytest.raises(RuntimeError):
            oracle_runs.entries(wl, r, np.array(seg, np.int32), np.array(lb, np.int32))


def _painted_tiny():
    wl = make_workload("tiny", painted=True)
    r = wl.ref_views[0]
    return wl, r


def _fully_matched_segments(wl, r, k, d):
    """Segments whose reference pixels all lie on plane k and each of whose pixels is seen on plane k,
    inside the image, by at least one neighbour at label d (FP64 3D path, generator plane ids)."""
    cr = wl.cams[r]
    H, W = cr.height, cr.width
    ys, xs = np.mgrid[0:H, 0:W]
    z = 1.0 / _iz(d, wl.n_labels, wl.z_near, wl.z_far)
    Xw = _world_points_ref_plane(cr, z, xs.astype(np.float64), ys.astype(np.float64))
    seen = np.zeros(H * W, bool)
    for v in wl.neighbours(r):
        cv = wl.cams[v]
        u, vv, zc = _project(cv, Xw)
        ui, vi = np.floor(u + 0.5), np.floor(vv + 0.5)
        inside = (zc > 0) & (ui >= 0) & (ui <= cv.width - 1) & (vi >= 0) & (vi <= cv.height - 1)
        pid = wl.view(v, aux=True).plane_id
        hit = np.zeros(H * W, bool)
        hit[inside] = pid[vi[inside].astype(int), ui[inside].astype(int)] == k
        seen |= hit
    on_k = (wl.view(r, aux=True).plane_id.ravel() == k) & seen
    lab, S = wl.labels(r)
    n = np.bincount(lab.ravel(), minlength=S)
    good = np.bincount(lab.ravel(), weights=on_k.astype(np.float64), minlength=S)
    return np.nonzero((n > 0) & (good == n))[0]


@pytest.mark.parametrize("k,d", [(0, 10), (1, 38)])
def test_zero_cost_and_wta_at_true_label_of_painted_planes(k, d):
    """Eq. 4 on an exact-correspondence scene: fronto-parallel plane k lies on label d, its texture
    is painted from the reference pixels, so a fully matched segment costs 0 at d; d is an
    unambiguous label (its rounded disparity differs from both neighbouring labels' in every view),
    so every other label costs more and the winner is d."""
    wl, r = _painted_tiny()
    assert abs(label_depth(d, wl.n_labels, wl.z_near, wl.z_far) - 1.0 / _iz(d, wl.n_labels, wl.z_near,
                                                                              wl.z_far)) < 1e-12
    for v in wl.neighbours(r):
        disp = lambda dd: 400.0 * (wl.cams[r].centre[0] - wl.cams[v].centre[0]) * _iz(dd, wl.n_labels, wl.z_near,
                                                                                     wl.z_far)
        rd = [math.floor(disp(dd) + 0.5) for dd in (d - 1, d, d + 1)]
        assert rd[0] != rd[1] and rd[2] != rd[1]
    segs = _fully_matched_segments(wl, r, k, d)
    assert len(segs) >= 10
    vol = oracle_runs.volume(wl, r)
    assert np.all(vol[segs, d] == 0)
    win = oracle.wta(vol)
    assert np.all(win[segs] == d)
    assert np.all(vol[segs][:, np.arange(wl.n_labels) != d] > 0)


def test_duplicated_reference_view_costs_nothing():
    wl = make_workload("tiny")
    r = wl.ref_views[0]
    cams = list(wl.cams) + [wl.cams[r]]
    views = wl.views() + [wl.view(r)]
    lab, S = wl.labels(r)
    H = oracle.homography_table(cams, r, [3], wl.n_labels, wl.z_near, wl.z_far)
    vol = oracle.cost_volume(cams, views, 1, r, [3], H, wl.n_labels, lab, S, 765)
    assert np.all(vol == 0)
    # with a sum over {duplicate, view 0} the volume equals that of view 0 alone
    H2 = oracle.homography_table(cams, r, [3, 0], wl.n_labels, wl.z_near, wl.z_far)
    v2 = oracle.cost_volume(cams, views, 1, r, [3, 0], H2, wl.n_labels, lab, S, 765, combine="sum")
    H0 = oracle.homography_table(cams, r, [0], wl.n_labels, wl.z_near, wl.z_far)
    v0 = oracle.cost_volume(cams, views, 1, r, [0], H0, wl.n_labels, lab, S, 765)
    np.testing.assert_array_equal(v2, v0)


def test_views_that_see_nothing_cost_the_penalty():
    """A camera at the reference centre looking backwards sees no candidate plane (Wz < 0), and a
    camera far to the side sees them outside its image: every sample is out of view."""
    wl = make_workload("tiny")
    r = wl.ref_views[0]
    cr = wl.cams[r]
    back = synth.Camera(cr.K.copy(), np.diag([-1.0, 1.0, -1.0]), np.zeros(3), cr.width, cr.height)
    back.t = -back.R @ cr.centre
    side = synth.Camera(cr.K.copy(), np.eye(3), -np.array([500.0, 0.0, 0.0]), cr.width, cr.height)
    cams = list(wl.cams) + [back, side]
    views = wl.views() + [wl.view(0), wl.view(2)]
    lab, S = wl.labels(r)
    n = np.bincount(lab.ravel(), minlength=S).astype(np.int64)
    H = oracle.homography_table(cams, r, [3, 4], wl.n_labels, wl.z_near, wl.z_far)
    vmin = oracle.cost_volume(cams, views, 1, r, [3, 4], H, wl.n_labels, lab, S, 765)
    np.testing.assert_array_equal(vmin, np.repeat((n * 765)[:, None], wl.n_labels, 1))
    vsum = oracle.cost_volume(cams, views, 1, r, [3, 4], H, wl.n_labels, lab, S, 100, combine="sum")
    np.testing.assert_array_equal(vsum, np.repeat((n * 200)[:, None], wl.n_labels, 1))


def test_listed_segments_only_touch_their_rows():
    wl = make_workload("tiny")
    r = wl.ref_views[0]
    full = oracle_runs.volume(wl, r)
    lst = np.array([3, 100, 101, 509], np.int32)
    part = oracle_runs.volume(wl, r, seg_list=lst, out=np.full_like(full, -7))
    np.testing.assert_array_equal(part[lst], full[lst])
    rest = np.setdiff1d(np.arange(full.shape[0]), lst)
    assert np.all(part[rest] == -7)


def test_fp64_mismatch_fraction_is_small_and_reported():
    """The FP32 contract picks a different nearest sample than FP64 only near .5 ties; this measures
    it (parity of the contract itself against FP64 is a reported figure, not an exact pin)."""
    wl = make_workload("tiny")
    r = wl.ref_views[0]
    bad, tot = oracle.fp64_mismatch(wl.cams, r, wl.neighbours(r), wl.n_labels, wl.z_near, wl.z_far)
    assert tot == 480 * 270 * 64 * 2
    print(f"tiny fp32-vs-fp64 sample mismatch fraction {bad / tot:.3e}")
    assert bad / tot < 1e-3


# ---------------------------------------------------------------------------------------- temporal

def _frames(seed, shape=(40, 56), hi=900):
    rng = np.random.default_rng(seed)
    return [synth.View(*(rng.integers(0, hi, shape).astype(np.uint16) for _ in range(3))) for _ in range(3)]


def _shift(view, dy=0, du=0, dv=0):
    return synth.View((view.Y.astype(np.int64) + dy).astype(np.uint16), (view.U.astype(np.int64) + du).astype(np.uint16),
                      (view.V.astype(np.int64) + dv).astype(np.uint16))


TP_8BIT, TI_8BIT = 3, 1  # Sec. III-E thresholds


def test_temporal_static_and_boundaries():
    lab, S = synth.grid_labels(56, 40, 8, 2, 5)
    a, b, _ = _frames(3)
    t_p, t_i = TP_8BIT * 4, TI_8BIT * 4  # thresholds scaled to 10-bit samples
    m, ch, n = oracle.temporal_mask(lab, S, a, a, None, 2, t_p, t_i, 0)
    assert np.all(m == 1) and n == 0
    # mean moved by exactly T: changed; by T - 1: unchanged
    m, ch, n = oracle.temporal_mask(lab, S, _shift(a, t_p), a, None, 2, t_p, t_i, 0)
    assert np.all(m == 0) and n == S and np.array_equal(ch, np.arange(S))
    m, _, _ = oracle.temporal_mask(lab, S, _shift(a, t_p - 1), a, None, 2, t_p, t_i, 0)
    assert np.all(m == 1)
    # sum moved by T*n - 1 (one pixel one step short): unchanged; a negative move counts the same
    cur = _shift(a, t_p)
    ys, xs = np.nonzero(lab == 5)
    cur.Y[ys[0], xs[0]] -= 1
    m, ch, n = oracle.temporal_mask(lab, S, cur, a, None, 2, t_p, t_i, 0)
    assert m[5] == 1 and np.all(np.delete(m, 5) == 0) and 5 not in ch and n == S - 1
    m, _, _ = oracle.temporal_mask(lab, S, _shift(a, -t_p), _shift(a, 0), None, 2, t_p, t_i, 0)
    assert np.all(m == 0)


def test_temporal_iframe_adoption_and_preference():
    lab, S = synth.grid_labels(56, 40, 8, 2, 6)
    a, b, _ = _frames(4)
    t_p, t_i = 12, 4
    # far from the previous frame, close to the I frame: adopt the I frame's depth
    m, _, n = oracle.temporal_mask(lab, S, _shift(b, t_i - 1), _shift(a, 300), b, 2, t_p, t_i, 0)
    assert np.all(m == 2) and n == 0
    m, _, n = oracle.temporal_mask(lab, S, _shift(b, t_i), _shift(a, 300), b, 2, t_p, t_i, 0)
    assert np.all(m == 0) and n == S
    # close to both: the previous P frame is preferred
    m, _, _ = oracle.temporal_mask(lab, S, b, b, b, 2, t_p, t_i, 0)
    assert np.all(m == 1)


def test_temporal_channel_modes_and_empty_segments():
    lab, S = synth.grid_labels(56, 40, 8, 2, 7)
    a, _, _ = _frames(5)
    cur = _shift(a, 0, du=50)
    m, _, _ = oracle.temporal_mask(lab, S, cur, a, None, 2, 12, 4, 0)
    assert np.all(m == 1)  # luma only: the chroma change is not seen
    m, _, _ = oracle.temporal_mask(lab, S, cur, a, None, 2, 12, 4, 1)
    assert np.all(m == 0)
    m, ch, n = oracle.temporal_mask(lab, S + 3, a, a, None, 2, 12, 4, 0)
    assert np.all(m[:S] == 1) and np.all(m[S:] == 0) and list(ch) == [S, S + 1, S + 2]


# --------------------------------------------------------------------------------------------- WTA

def test_wta_ties_smallest_label_and_adoption():
    cost = np.array([[5, 3, 3, 9], [1, 1, 1, 1], [7, 6, 5, 4], [0, 2, 0, 2]], np.int32)
    assert list(oracle.wta(cost)) == [1, 0, 3, 0]
    mask = np.array([0, 1, 2, 0], np.uint8)
    prev = np.array([9, 8, 7, 6], np.uint16)
    ifr = np.array([19, 18, 17, 16], np.uint16)
    assert list(oracle.wta(cost, mask, prev, ifr)) == [1, 8, 17, 0]
    out = oracle.wta(cost, seg_list=[2], out=np.full(4, 99, np.uint16))
    assert list(out) == [99, 99, 3, 99]


def test_depth_map_takes_label_depth():
    lab, S = synth.grid_labels(30, 20, 8, 2, 1)
    seg_label = (np.arange(S) * 7 % 50).astype(np.uint16)
    dm = oracle.depth_map(lab, S, seg_label, 50, 1.0, 20.0)
    expect = np.array([label_depth(int(seg_label[s]), 50, 1.0, 20.0) for s in lab.ravel()], np.float32)
    np.testing.assert_allclose(dm.ravel(), expect, rtol=1e-6)
