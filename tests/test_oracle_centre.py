"""Pins of the oracle's centre table (Eq. 4 at segment centres with a window, and the segment s' that
Eq. 5 needs), against facts fixed by geometry and by an independent FP64 implementation."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from synth.configs import make_workload
from test_oracle_pins import _iz, _project, _world_points_ref_plane


def _centres(lab, S):
    H, W = lab.shape
    ys, xs = np.mgrid[0:H, 0:W]
    n = np.bincount(lab.ravel(), minlength=S).astype(np.int64)
    sx = np.bincount(lab.ravel(), weights=xs.ravel().astype(np.float64), minlength=S).astype(np.int64)
    sy = np.bincount(lab.ravel(), weights=ys.ravel().astype(np.float64), minlength=S).astype(np.int64)
    nz = np.maximum(n, 1)
    return (2 * sx + n) // (2 * nz), (2 * sy + n) // (2 * nz), n


def _table_fp64(wl, r, nbrs, labels_views, window, d):
    """Independent FP64 version of one label's (m, s') for every segment."""
    lab, S = wl.labels(r)
    mx, my, n = _centres(lab, S)
    cr = wl.cams[r]
    z = 1.0 / _iz(d, wl.n_labels, wl.z_near, wl.z_far)
    Xw = _world_points_ref_plane(cr, z, mx.astype(np.float64), my.astype(np.float64))
    ref = wl.view(r)
    half = window // 2
    m = np.zeros((S, len(nbrs)), np.int64)
    sp = np.full((S, len(nbrs)), -1, np.int64)
    for k, v in enumerate(nbrs):
        cv = wl.cams[v]
        u, vv, zc = _project(cv, Xw)
        ui, vi = np.floor(u + 0.5).astype(np.int64), np.floor(vv + 0.5).astype(np.int64)
        inside = (zc > 0) & (ui >= 0) & (ui <= cv.width - 1) & (vi >= 0) & (vi <= cv.height - 1) & (n > 0)
        img = wl.view(v)
        for dy in range(-half, half + 1):
            for dx in range(-half, half + 1):
                rx, ry, qx, qy = mx + dx, my + dy, ui + dx, vi + dy
                ok = inside & (rx >= 0) & (rx < cr.width) & (ry >= 0) & (ry < cr.height) & (qx >= 0) & \
                    (qx < cv.width) & (qy >= 0) & (qy < cv.height)
                c = np.zeros(S, np.int64)
                for a, b in zip((ref.Y, ref.U, ref.V), (img.Y, img.U, img.V)):
                    av = np.asarray(a, np.int64)[np.where(ok, ry, 0), np.where(ok, rx, 0)]
                    bv = np.asarray(b, np.int64)[np.where(ok, qy, 0), np.where(ok, qx, 0)]
                    c += np.abs(av - bv)
                m[:, k] += np.where(ok, c, wl.oob_penalty)
        if labels_views[v] is not None:
            sp[:, k] = np.where(inside, labels_views[v][np.where(inside, vi, 0), np.where(inside, ui, 0)], -1)
    return m, sp


@pytest.mark.parametrize("name,window", [("tiny", 3), ("tiny", 5), ("uhd15", 3)])
def test_centre_table_against_fp64_path(name, window):
    wl = make_workload(name, reduced=(name != "tiny"))
    r = wl.ref_views[0] if name == "tiny" else 7
    nbrs = wl.neighbours(r)[:4]
    lab, S = wl.labels(r)
    labels_views = [wl.labels(v)[0] if v != 2 else None for v in range(wl.n_views)]
    labels_views[r] = lab
    H = oracle.homography_table(wl.cams, r, nbrs, wl.n_labels, wl.z_near, wl.z_far)
    m, sp = oracle.centre_table(wl.cams, wl.views(), wl.sample_bytes, r, nbrs, H, wl.n_labels, labels_views, S,
                                window, wl.oob_penalty)
    eq = tot = 0
    for d in range(0, wl.n_labels, 5):
        m64, sp64 = _table_fp64(wl, r, nbrs, labels_views, window, d)
        same = (m[:, d, :] == m64) & (sp[:, d, :] == sp64)
        eq += int(same.sum())
        tot += same.size
    assert eq / tot > 0.99, (eq, tot)


def test_centre_window_costs_zero_at_true_label_of_painted_planes():
    """Painted fronto-parallel planes on labels 10 and 38 (exact correspondence): segments whose whole
    centre window lies on the plane in the reference and in a neighbour that sees it there cost 0."""
    wl = make_workload("tiny", painted=True)
    r = wl.ref_views[0]
    lab, S = wl.labels(r)
    mx, my, n = _centres(lab, S)
    pid_r = wl.view(r, aux=True).plane_id
    nbrs = wl.neighbours(r)
    H = oracle.homography_table(wl.cams, r, nbrs, wl.n_labels, wl.z_near, wl.z_far)
    labels_views = [wl.labels(v)[0] for v in range(wl.n_views)]
    m, sp = oracle.centre_table(wl.cams, wl.views(), 1, r, nbrs, H, wl.n_labels, labels_views, S, 3, 765)
    found = 0
    for plane, d in ((0, 10), (1, 38)):
        z = 1.0 / _iz(d, wl.n_labels, wl.z_near, wl.z_far)
        for k, v in enumerate(nbrs):
            pid_v = wl.view(v, aux=True).plane_id
            cv = wl.cams[v]
            for s in range(S):
                x0, y0 = int(mx[s]), int(my[s])
                if not (1 <= x0 < 479 and 1 <= y0 < 269) or np.any(pid_r[y0 - 1:y0 + 2, x0 - 1:x0 + 2] != plane):
                    continue
                Xw = _world_points_ref_plane(wl.cams[r], z, np.array([float(x0)]), np.array([float(y0)]))
                u, vv, _ = _project(cv, Xw)
                ui, vi = int(np.floor(u[0] + 0.5)), int(np.floor(vv[0] + 0.5))
                if not (1 <= ui < cv.width - 1 and 1 <= vi < cv.height - 1):
                    continue
                if np.any(pid_v[vi - 1:vi + 2, ui - 1:ui + 2] != plane):
                    continue
                assert m[s, d, k] == 0, (plane, s, k)
                assert sp[s, d, k] == labels_views[v][vi, ui]
                found += 1
    assert found >= 50


def test_centre_table_border_and_empty_segments():
    wl = make_workload("tiny")
    r = wl.ref_views[0]
    lab, S0 = wl.labels(r)
    lab = lab.copy()
    lab[0, 0] = S0  # a one-pixel segment in the corner: its window sticks out by one row and column
    S = S0 + 2      # and segment S0 + 1 is empty
    nbrs = [0]
    H = oracle.homography_table(wl.cams, r, nbrs, wl.n_labels, wl.z_near, wl.z_far)
    labels_views = [wl.labels(0)[0], lab, None]
    m, sp = oracle.centre_table(wl.cams, wl.views(), 1, r, nbrs, H, wl.n_labels, labels_views, S, 3, 765)
    assert np.all(m[S0 + 1] == 9 * 765) and np.all(sp[S0 + 1] == -1)
    # at every label the corner window has at least 5 of its 9 pairs outside the reference image
    assert np.all(m[S0] >= 5 * 765)
    m1, _ = oracle.centre_table(wl.cams, wl.views(), 1, r, nbrs, H, wl.n_labels, labels_views, S, 1, 765)
    assert np.all(m1[S0 + 1] == 765)
    assert np.all(m1[S0] <= 765)  # a single in-image pair (or the penalty when out of view)
