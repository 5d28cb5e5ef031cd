"""GPU parity of the superpixel segmentation (Sec. IV-C): the CUDA path equals the oracle's definition
bit for bit (labels are integers decided by exact integer arithmetic)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import synth
from synth.configs import make_workload

pytestmark = pytest.mark.gpu

ftv = pytest.importorskip("paper_1909_02294_gb300")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from gpu_runs import dev  # noqa: E402


def gpu_segment(frames, sb, bd, S, m, T, pitch_pad=0):
    sg = ftv.Segmenter([(np.asarray(f.Y).shape[1], np.asarray(f.Y).shape[0]) for f in frames], sb, bd, S, m, T)
    try:
        planes = []
        for f in frames:
            trip = []
            for a in (f.Y, f.U, f.V):
                a = np.asarray(a)
                if pitch_pad:
                    wide = np.zeros((a.shape[0], a.shape[1] + pitch_pad), a.dtype)
                    wide[:, : a.shape[1]] = a
                    trip.append(dev(wide)[:, : a.shape[1]])
                else:
                    trip.append(dev(a))
            planes.append(tuple(trip))
        labs = [torch.full(np.asarray(f.Y).shape, -7, dtype=torch.int32, device="cuda") for f in frames]
        ftv.ftv_superpixels(sg, planes, labs)
        assert ftv.ftv_segmenter_check(sg) == 0
        segs = ftv.ftv_segmenter_segments(sg)
        return [l.cpu().numpy() for l in labs], segs
    finally:
        sg.close()


def _strip(values, channel=0, bd=8):
    vals = np.asarray(values)
    planes = [np.zeros((1, len(vals)), np.uint16 if bd > 8 else np.uint8) for _ in range(3)]
    planes[channel][0] = vals
    return synth.View(*planes)


def test_worked_examples_on_the_gpu():
    """The hand-worked strips of the oracle pins, now through the CUDA path, which always applies the
    connectivity step. It leaves the first four unchanged (every label is one run). In the fifth, label 1
    holds {0, 1} and {4, 5}: equal sizes, so {0, 1} (named first) stays; {4, 5} (mean 800 in 1/16 units)
    touches label 0's {2, 3} (1040) and label 2's {6, 7, 8} (3200) and joins label 0."""
    cases = [
        (_strip([0, 0, 60, 60, 100, 100, 100, 100]), 1, 8, 4, 63, 1, [0, 0, 1, 1, 1, 1, 1, 1]),
        (_strip([0, 0, 60, 60, 100, 100, 100, 100], 2), 1, 8, 4, 64, 1, [0, 0, 0, 1, 1, 1, 1, 1]),
        (_strip([0, 0, 240, 240, 400, 400, 400, 400], 0, 10), 2, 10, 4, 63, 1, [0, 0, 1, 1, 1, 1, 1, 1]),
        (_strip([1, 0, 1, 10, 19, 29]), 1, 8, 3, 0, 2, [0, 0, 0, 0, 1, 1]),
        (_strip([50, 50, 60, 70, 50, 50, 200, 200, 200]), 1, 8, 3, 0, 2, [1, 1, 0, 0, 0, 0, 2, 2, 2]),
    ]
    for f, sb, bd, S, m, T, want in cases:
        (lab,), _ = gpu_segment([f], sb, bd, S, m, T)
        assert lab.ravel().tolist() == want
        assert lab.ravel().tolist() == oracle.superpixels(f, sb, bd, S, m, T).ravel().tolist()


@pytest.mark.parametrize("W,H,n,noise,S,m,T", [
    (333, 217, 20, 0, 8, 5, 10),
    (333, 217, 20, 8, 8, 5, 10),
    (301, 149, 12, 16, 13, 5, 4),
    (128, 96, 9, 12, 5, 0, 3),
    (250, 190, 15, 10, 9, 40, 6),
    (47, 29, 4, 20, 1, 5, 2),
    (200, 130, 10, 6, 64, 5, 5),
])
def test_parity_with_the_oracle_on_mosaics(W, H, n, noise, S, m, T):
    f = synth.mosaic(W, H, n, noise_sigma=noise, seed=W + S)
    (lab,), segs = gpu_segment([f], 1, 8, S, m, T)
    want = oracle.superpixels(f, 1, 8, S, m, T)
    assert segs == [oracle.grid_segments(W, H, S)]
    assert np.array_equal(lab, want)


@pytest.mark.parametrize("bd", [10, 12, 16])
def test_parity_at_high_bit_depths(bd):
    """10 bits takes the 32-bit colour path, 12 and 16 bits the 64-bit one."""
    f = synth.mosaic(257, 171, 14, bit_depth=bd, noise_sigma=3.0 * (1 << (bd - 8)), seed=bd)
    (lab,), _ = gpu_segment([f], 2, bd, 11, 5, 5)
    assert np.array_equal(lab, oracle.superpixels(f, 2, bd, 11, 5, 5))


def test_degenerate_sizes_and_padded_pitches():
    frames = [synth.mosaic(1, 1, 1, seed=1), synth.mosaic(1, 37, 3, noise_sigma=30, seed=2),
              synth.mosaic(41, 1, 3, noise_sigma=30, seed=3), synth.mosaic(9, 7, 2, noise_sigma=30, seed=4)]
    for f in frames:
        for S in (1, 3, 64):
            (lab,), segs = gpu_segment([f], 1, 8, S, 5, 3, pitch_pad=5)
            assert np.array_equal(lab, oracle.superpixels(f, 1, 8, S, 5, 3))
            assert lab.max() < segs[0]


def test_one_call_segments_images_of_different_sizes():
    wl = make_workload("tiny")
    frames = [wl.view(v) for v in range(wl.n_views)] + [synth.mosaic(190, 77, 8, noise_sigma=9, seed=7),
                                                         synth.mosaic(33, 250, 5, noise_sigma=9, seed=8)]
    labs, segs = gpu_segment(frames, 1, 8, 10, 5, 10)
    for f, lab, k in zip(frames, labs, segs):
        want = oracle.superpixels(f, 1, 8, 10, 5, 10)
        assert np.array_equal(lab, want)
        assert k == oracle.grid_segments(lab.shape[1], lab.shape[0], 10)


def test_full_hd_view_bit_exact():
    """One 1920x1080 10-bit view of the 8-view rig with the paper's m = 5 and 20,736 segments (S = 10)."""
    wl = make_workload("hd8")
    f = wl.view(0)
    (lab,), segs = gpu_segment([f], 2, wl.bit_depth, 10, 5, 10)
    assert segs == [20736]
    assert np.array_equal(lab, oracle.superpixels(f, 2, wl.bit_depth, 10, 5, 10))


def test_uhd_batch_properties():
    """Fifteen 3840x2160 views in one call (S = 13: 296 x 167 = 49,432 segments per view), beyond what
    the oracle finishes in seconds: every label in range and every non-empty label one 8-connected set,
    checked on the first and the last view."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    wl = make_workload("uhd15")
    frames = [wl.view(v) for v in range(wl.n_views)]
    labs, segs = gpu_segment(frames, 2, wl.bit_depth, 13, 5, 10)
    assert segs == [296 * 167] * len(frames)
    for lab in (labs[0], labs[-1]):
        H, W = lab.shape
        assert lab.min() >= 0 and lab.max() < segs[0]
        idx = np.arange(H * W).reshape(H, W)
        rows, cols = [], []
        for a, b in ((lab[:, :-1] == lab[:, 1:], (idx[:, :-1], idx[:, 1:])),
                     (lab[:-1] == lab[1:], (idx[:-1], idx[1:])),
                     (lab[:-1, :-1] == lab[1:, 1:], (idx[:-1, :-1], idx[1:, 1:])),
                     (lab[:-1, 1:] == lab[1:, :-1], (idx[:-1, 1:], idx[1:, :-1]))):
            rows.append(b[0][a])
            cols.append(b[1][a])
        r, c = np.concatenate(rows), np.concatenate(cols)
        g = coo_matrix((np.ones(len(r), np.int8), (r, c)), shape=(H * W, H * W))
        n_comp, _ = connected_components(g, directed=False)
        assert n_comp == len(np.unique(lab))


def test_superpixels_feed_the_cost_volume():
    """Segmentation -> segment index -> cost volume on the device: the volume over the GPU's superpixels
    equals the oracle's volume over the oracle's superpixels."""
    wl = make_workload("tiny")
    r = wl.ref_views[0]
    (lab_d_np,), (S,) = gpu_segment([wl.view(r)], 1, 8, 12, 5, 10)
    lab_o = oracle.superpixels(wl.view(r), 1, 8, 12, 5, 10)
    assert np.array_equal(lab_d_np, lab_o)
    ctx = ftv.ftv_depth_init(wl.cams, [r], wl.n_labels, wl.z_near, wl.z_far, sample_bytes=1, bit_depth=8,
                             oob_penalty=wl.oob_penalty, combine=ftv.FTV_COMBINE_MIN, max_segments=S)
    try:
        planes = [(dev(v.Y), dev(v.U), dev(v.V)) for v in wl.views()]
        cost = torch.empty((S, wl.n_labels), dtype=torch.int32, device="cuda")
        ftv.ftv_cost_volume(ctx, planes, [dev(lab_d_np)], [S], [cost])
        assert ftv.ftv_check(ctx) == 0
        nb = wl.neighbours(r)
        H = oracle.homography_table(wl.cams, r, nb, wl.n_labels, wl.z_near, wl.z_far)
        want = oracle.cost_volume(wl.cams, wl.views(), 1, r, nb, H, wl.n_labels, lab_o, S, wl.oob_penalty, "min")
        assert np.array_equal(cost.cpu().numpy(), want)
    finally:
        ctx.close()


def test_launch_count_accounting():
    f = synth.mosaic(64, 48, 5, noise_sigma=10, seed=9)
    sg = ftv.Segmenter([(64, 48)], 1, 8, 8, 5, 4)
    try:
        planes = [(dev(f.Y), dev(f.U), dev(f.V))]
        lab = torch.empty((48, 64), dtype=torch.int32, device="cuda")
        ftv.ftv_superpixels(sg, planes, [lab])
        n1 = ftv.ftv_segmenter_launch_count(sg)
        ftv.ftv_superpixels(sg, planes, [lab])
        assert ftv.ftv_segmenter_launch_count(sg) == 2 * n1 > 0
        assert ftv.ftv_segmenter_check(sg) == 0
    finally:
        sg.close()


def test_profiling_events_time_the_assignment_passes():
    f = synth.mosaic(640, 360, 20, noise_sigma=8, seed=11)
    sg = ftv.Segmenter([(640, 360)], 1, 8, 8, 5, 4)
    try:
        with pytest.raises(ftv.FtvError):
            ftv.ftv_segmenter_kernel_ms(sg)  # nothing timed yet
        ftv.ftv_segmenter_set_profiling(sg, True)
        lab = torch.empty((360, 640), dtype=torch.int32, device="cuda")
        ftv.ftv_superpixels(sg, [(dev(f.Y), dev(f.U), dev(f.V))], [lab])
        a, t = ftv.ftv_segmenter_kernel_ms(sg)
        assert 0 < 4 * a < t
        assert ftv.ftv_segmenter_check(sg) == 0
        assert np.array_equal(lab.cpu().numpy(), oracle.superpixels(f, 1, 8, 8, 5, 4))
    finally:
        sg.close()
