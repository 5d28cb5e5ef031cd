"""CPU check of the FP32 cost kernel's tile cull (box_out_of_view), restated with exact IEEE float32
arithmetic: a (tile box, homography) pair that the corner test declares out of view must have every pixel
of the box out of view under the FP32 contract (Wz <= 0, or the rounded sample outside the image). Random
convergent rigs at 3840x2160 scale and a neighbour rotated 75 degrees (Wz = 0 crosses the image)."""
from __future__ import annotations

import math

import numpy as np

import oracle
import synth
from ieee32 import fma32

F = np.float32


def box_out_of_view(h, x0, x1, y0, y1, wv, hv, corners=4) -> bool:
    """corners=1 tests the first corner only: an unsound cull, to show that the check detects one."""
    m = F(2.0 ** -20)
    left = right = top = bottom = behind = True
    a = [F(abs(v)) for v in h]
    for k in range(corners):
        x = F(x1 if k & 1 else x0)
        y = F(y1 if k & 2 else y0)
        X = fma32(h[0], x, fma32(h[1], y, h[2]))
        Y = fma32(h[3], x, fma32(h[4], y, h[5]))
        Z = fma32(h[6], x, fma32(h[7], y, h[8]))
        sx = fma32(a[0], x, fma32(a[1], y, a[2]))
        sy = fma32(a[3], x, fma32(a[4], y, a[5]))
        sz = fma32(a[6], x, fma32(a[7], y, a[8]))
        tl, tr = F(X + Z), fma32(F(-wv), Z, X)
        tt, tb = F(Y + Z), fma32(F(-hv), Z, Y)
        left = left and tl < -m * F(F(sx + sz) + abs(tl))
        right = right and tr > m * F(F(sx + F(F(wv) * sz)) + abs(tr))
        top = top and tt < -m * F(F(sy + sz) + abs(tt))
        bottom = bottom and tb > m * F(F(sy + F(F(hv) * sz)) + abs(tb))
        behind = behind and Z < -m * F(sz + abs(Z))
    return bool(left or right or top or bottom or behind)


def in_view(h, xs, ys, wv, hv):
    """The FP32 contract's in-view decision per pixel."""
    X = fma32(h[0], xs, fma32(h[1], ys, h[2]))
    Y = fma32(h[3], xs, fma32(h[4], ys, h[5]))
    W = fma32(h[6], xs, fma32(h[7], ys, h[8]))
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        r = (F(1.0) / W).astype(F)
        fu = np.floor((X * r).astype(F) + F(0.5))
        fv = np.floor((Y * r).astype(F) + F(0.5))
    return (W > 0) & (fu >= 0) & (fu <= wv - 1) & (fv >= 0) & (fv <= hv - 1)


def _rotated(base, deg, C=(0.08, 0.0, 0.0)):
    a = math.radians(deg)
    R = np.array([[math.cos(a), 0.0, -math.sin(a)], [0.0, 1.0, 0.0], [math.sin(a), 0.0, math.cos(a)]])
    return synth.Camera(base.K.copy(), R, -R @ np.array(C), base.width, base.height)


def test_culled_boxes_are_out_of_view_at_every_pixel():
    rng = np.random.default_rng(20)
    W, H = 3840, 2160
    n_culled = n_kept = n_unsound = 0
    tables = []
    for _ in range(8):
        cams = synth.arc_rig(5, 3.0, float(rng.uniform(6, 40)), float(rng.uniform(800, 4000)), W, H,
                             seed=int(rng.integers(1 << 30)), roll_deg=5.0)
        tables.append((oracle.homography_table(cams, 2, [0, 1, 3, 4], 32, 0.8, 15.0), W, H))
    base = synth.Camera(synth.intrinsics(1200.0, W, H), np.eye(3), np.zeros(3), W, H)
    rot = [base, _rotated(base, 75.0), _rotated(base, 30.0)]
    tables.append((oracle.homography_table(rot, 0, [1, 2], 32, 0.5, 10.0), W, H))
    for table, wv, hv in tables:
        for _ in range(60):
            k, d = int(rng.integers(table.shape[0])), int(rng.integers(table.shape[1]))
            h = [F(v) for v in table[k, d]]
            bw, bh = int(rng.integers(1, 130)), int(rng.integers(1, 33))
            x0, y0 = int(rng.integers(0, W - bw)), int(rng.integers(0, H - bh))
            culled = box_out_of_view(h, x0, x0 + bw - 1, y0, y0 + bh - 1, wv, hv)
            xs, ys = np.meshgrid(np.arange(x0, x0 + bw, dtype=F), np.arange(y0, y0 + bh, dtype=F))
            inv = in_view(h, xs.ravel(), ys.ravel(), wv, hv)
            if culled:
                n_culled += 1
                assert not inv.any(), (k, d, x0, y0, bw, bh)
            else:
                n_kept += 1
            if box_out_of_view(h, x0, x0 + bw - 1, y0, y0 + bh - 1, wv, hv, corners=1) and inv.any():
                n_unsound += 1
    assert n_culled > 50 and n_kept > 50
    assert n_unsound > 0  # a one-corner test would cull boxes with pixels in view: the check sees that
