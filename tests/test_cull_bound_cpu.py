"""CPU check of the FP32 cost kernel's per-tile entry classes (box_class), restated with exact IEEE float32
arithmetic, on random convergent rigs at 3840x2160 scale and a neighbour rotated 75 degrees (Wz = 0 crosses
the image):
  - a (tile box, homography) pair the corner test declares out of view (kOut) has every pixel of the box out
    of view under the FP32 contract (Wz <= 0, or the rounded sample outside the image);
  - a pair declared in front (kFront) has Wz_f32 > 2^-92 at every pixel, so its reciprocal is that of a
    normal float and finite and positive;
  - a pair declared inside (kIn) has, in addition, every pixel's sample in view.
Variants that test one corner only, or drop the margin, are shown unsound by the same check."""
from __future__ import annotations

import math

import numpy as np

import oracle
import synth
from ieee32 import fma32

F = np.float32


def box_class(h, x0, x1, y0, y1, wv, hv, corners=4, edge=1) -> str:
    """'out', 'in', 'front' or 'general', as the kernel's box_class. corners=1 tests the first corner only,
    and edge=0 proves u <= wv and v <= hv where the kernel proves u <= wv - 1 and v <= hv - 1: unsound
    variants, to show that the check detects them."""
    m = F(2.0 ** -20)
    left = right = top = bottom = behind = True
    front = inside = True
    a = [F(abs(v)) for v in h]
    wv1, hv1 = F(wv - edge), F(hv - edge)
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
        left = left and tl < m * -F(F(sx + sz) + abs(tl))
        right = right and tr > m * F(F(sx + F(F(wv) * sz)) + abs(tr))
        top = top and tt < m * -F(F(sy + sz) + abs(tt))
        bottom = bottom and tb > m * F(F(sy + F(F(hv) * sz)) + abs(tb))
        behind = behind and Z < m * -F(sz + abs(Z))
        front = front and Z > max(F(m * F(sz + abs(Z))), F(2.0 ** -90))
        ir, ib = fma32(wv1, Z, F(-X)), fma32(hv1, Z, F(-Y))
        inside = (inside and X > F(m * F(sx + abs(X))) and Y > F(m * F(sy + abs(Y)))
                  and ir > F(m * F(F(sx + F(wv1 * sz)) + abs(ir))) and ib > F(m * F(F(sy + F(hv1 * sz)) + abs(ib))))
    if left or right or top or bottom or behind:
        return "out"
    if front:
        return "in" if inside else "front"
    return "general"


def box_out_of_view(h, x0, x1, y0, y1, wv, hv, corners=4) -> bool:
    return box_class(h, x0, x1, y0, y1, wv, hv, corners) == "out"


def wz32(h, xs, ys):
    return fma32(h[6], xs, fma32(h[7], ys, h[8]))


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


def _tables_and_boxes(seed, n_rigs=8, per_table=80):
    rng = np.random.default_rng(seed)
    W, H = 3840, 2160
    tables = []
    for _ in range(n_rigs):
        cams = synth.arc_rig(5, 3.0, float(rng.uniform(6, 40)), float(rng.uniform(800, 4000)), W, H,
                             seed=int(rng.integers(1 << 30)), roll_deg=5.0)
        tables.append(oracle.homography_table(cams, 2, [0, 1, 3, 4], 32, 0.8, 15.0))
    base = synth.Camera(synth.intrinsics(1200.0, W, H), np.eye(3), np.zeros(3), W, H)
    rot = [base, _rotated(base, 75.0), _rotated(base, 30.0)]
    tables.append(oracle.homography_table(rot, 0, [1, 2], 32, 0.5, 10.0))
    for table in tables:
        for _ in range(per_table):
            k, d = int(rng.integers(table.shape[0])), int(rng.integers(table.shape[1]))
            h = [F(v) for v in table[k, d]]
            bw, bh = int(rng.integers(1, 130)), int(rng.integers(1, 33))
            x0, y0 = int(rng.integers(0, W - bw)), int(rng.integers(0, H - bh))
            xs, ys = np.meshgrid(np.arange(x0, x0 + bw, dtype=F), np.arange(y0, y0 + bh, dtype=F))
            yield h, (x0, x0 + bw - 1, y0, y0 + bh - 1), xs.ravel(), ys.ravel(), W, H


def test_inside_and_front_boxes_hold_at_every_pixel():
    """kIn: every pixel in view with Wz_f32 > 2^-92; kFront: Wz_f32 > 2^-92 at every pixel. Most boxes of a
    convergent rig that are not out of view are inside, which is what makes the class worth having."""
    counts = {"in": 0, "front": 0, "general": 0, "out": 0}
    for h, box, xs, ys, wv, hv in _tables_and_boxes(21):
        cls = box_class(h, *box, wv, hv)
        counts[cls] += 1
        if cls in ("in", "front"):
            assert np.all(wz32(h, xs, ys) > F(2.0 ** -92)), (h, box)
        if cls == "in":
            assert in_view(h, xs, ys, wv, hv).all(), (h, box)
    assert counts["in"] > 200 and counts["front"] > 5 and counts["out"] > 50, counts


def _edge_boxes(seed):
    """Boxes whose last column samples just past the right edge of the view: u in (wv - 0.45, wv - 0.05) at
    that pixel, so it rounds to column wv (out of view) although u < wv."""
    for h, box, xs, ys, wv, hv in _tables_and_boxes(seed, per_table=40):
        y = float(box[2])
        x = np.arange(0, 3840, dtype=np.float64)
        hd = [float(v) for v in h]
        Z = hd[6] * x + hd[7] * y + hd[8]
        with np.errstate(divide="ignore", invalid="ignore"):
            u = (hd[0] * x + hd[1] * y + hd[2]) / Z
        hit = np.nonzero((Z > 0) & (u > wv - 0.45) & (u < wv - 0.05))[0]
        if len(hit) == 0:
            continue
        x1 = int(hit[0])
        x0 = max(0, x1 - 16)
        bx, by = np.meshgrid(np.arange(x0, x1 + 1, dtype=F), np.array([y], F))
        yield h, (x0, x1, int(y), int(y)), bx.ravel(), by.ravel(), wv, hv


def test_inside_class_with_one_corner_or_the_wrong_edge_is_caught():
    """The same check finds boxes that a one-corner test, or a test of u <= wv instead of u <= wv - 1, would
    wrongly call inside: the check can see an unsound classification, and the sound one passes on the very
    boxes built to sit at the view's edge."""
    bad_corner = bad_edge = n_edge = 0
    for h, box, xs, ys, wv, hv in _tables_and_boxes(22, per_table=120):
        if box_class(h, *box, wv, hv, corners=1) == "in" and not in_view(h, xs, ys, wv, hv).all():
            bad_corner += 1
    for h, box, xs, ys, wv, hv in _edge_boxes(23):
        n_edge += 1
        inv = in_view(h, xs, ys, wv, hv)
        assert not inv.all()
        assert box_class(h, *box, wv, hv) != "in"
        if box_class(h, *box, wv, hv, edge=0) == "in":
            bad_edge += 1
    assert bad_corner > 0 and bad_edge > 0, (bad_corner, bad_edge, n_edge)
