"""GPU parity: the CUDA cost volume, temporal mask and winner-take-all against the CPU oracle.

Integer outputs, so the bar is bit-exact everywhere. Small and reduced workloads are compared entry
by entry over whole volumes (they span many 1024-pixel tiles, several label blocks and a ragged last
tile); the full-size workloads, run in the launch configuration the benchmark times, are compared on
seeded samples of (segment, label) entries that the oracle computes one by one.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import oracle_runs
import synth
from synth.configs import make_workload

pytestmark = pytest.mark.gpu

ftv = pytest.importorskip("paper_1909_02294_gb300")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from gpu_runs import Run, dev  # noqa: E402


def _oracle_all(wl, combine=None, plane_mode=0, centre=0, nbr_lists=None, frame=0, penalty=None):
    out = []
    for i, r in enumerate(wl.ref_views):
        lab, S = wl.labels(r)
        nb = nbr_lists[i] if nbr_lists is not None else wl.neighbours(r)
        H = oracle.homography_table(wl.cams, r, nb, wl.n_labels, wl.z_near, wl.z_far, plane_mode=plane_mode,
                                    centre=centre)
        out.append(oracle.cost_volume(wl.cams, wl.views(frame), wl.sample_bytes, r, nb, H, wl.n_labels, lab, S,
                                      wl.oob_penalty if penalty is None else penalty, combine or wl.combine))
    return out


def _assert_equal(got, ref, what):
    got = got.cpu().numpy() if isinstance(got, torch.Tensor) else got
    bad = int((got != ref).sum())
    assert bad == 0, f"{what}: {bad} of {ref.size} entries differ"


@pytest.mark.parametrize("combine,penalty", [("min", None), ("sum", None), ("min", 100), ("sum", 100)])
def test_tiny_volume_wta_and_depth_bit_exact(combine, penalty):
    """penalty 100 is below the largest sample cost (765): the kernel's min keeps out-of-view samples."""
    wl = make_workload("tiny")
    if penalty is not None:
        wl.penalty = penalty
    run = Run(wl, combine=combine)
    costs = run.volumes()
    assert run.check() == 0
    ref = _oracle_all(wl, combine)
    _assert_equal(costs[0], ref[0], "tiny volume")
    S = run.S[0]
    win = torch.empty(S, dtype=torch.int16, device="cuda")
    depth = torch.empty((270, 480), dtype=torch.float32, device="cuda")
    ftv.ftv_wta_depth(run.ctx, 0, costs[0], S, win, labels_pix=run.labels[0], depth_map=depth)
    assert run.check() == 0
    w_ref = oracle.wta(ref[0])
    assert np.array_equal(win.cpu().numpy().view(np.uint16), w_ref)
    d_ref = oracle.depth_map(wl.labels(1)[0], S, w_ref, wl.n_labels, wl.z_near, wl.z_far)
    assert np.array_equal(depth.cpu().numpy(), d_ref)
    run.close()


@pytest.mark.parametrize("name", ["hd8", "uhd15", "temporal"])
def test_reduced_workloads_bit_exact(name):
    wl = make_workload(name, reduced=True)
    run = Run(wl)
    costs = run.volumes()
    assert run.check() == 0
    for c, ref, r in zip(costs, _oracle_all(wl), wl.ref_views):
        _assert_equal(c, ref, f"{wl.name} ref {r}")
    # the convergent rig's projective entries cull whole tiles; the rectified rig's never do
    culled = ftv.ftv_culled_evaluations(run.ctx)
    if name == "uhd15":
        assert 0 < culled < wl.evaluations()
    if name == "hd8":
        assert culled == 0
    run.close()


def test_serving_small_shape_bit_exact():
    wl = make_workload("serving_small")
    run = Run(wl)
    costs = run.volumes()
    assert run.check() == 0
    for c, ref in zip(costs, _oracle_all(wl)):
        _assert_equal(c, ref, "serving_small")
    run.close()


def test_sixteen_bit_samples_use_wide_texels():
    wl = make_workload("hd8", reduced=True)
    wl.bit_depth = 12  # 12-bit samples: packed as 16-bit fields
    wl.ref_views = [0, 5]
    run = Run(wl)
    costs = run.volumes()
    assert run.check() == 0
    for c, ref in zip(costs, _oracle_all(wl)):
        _assert_equal(c, ref, "12-bit")
    run.close()


def test_centre_planes_and_nearest_neighbour_views():
    wl = make_workload("uhd15", reduced=True)
    lists = [[1], [6, 8], [13]]  # the paper's set D: nearest left and right (one at the ends)
    run = Run(wl, plane_mode=1, centre=7, nbr_lists=lists)
    costs = run.volumes()
    assert run.check() == 0
    for c, ref in zip(costs, _oracle_all(wl, plane_mode=1, centre=7, nbr_lists=lists)):
        _assert_equal(c, ref, "centre planes")
    run.close()


def test_affine_and_out_of_view_homography_modes():
    """Cameras displaced along the optical axis give homographies with h6 = h7 = 0 and h8 != 1 (and
    h8 <= 0 for candidate planes behind the displaced camera): the kernel's affine and all-out paths."""
    wl = make_workload("tiny")
    base = wl.cams[1]
    for C in ([0.0, 0.0, 0.3], [0.02, 0.0, 1.0]):
        R = np.eye(3)
        wl.cams.append(synth.Camera(base.K.copy(), R, -R @ np.array(C), base.width, base.height))
    # a parallel camera with another focal length and a vertical offset: affine with unit scale but not
    # row-preserving (h0 != 1, h5 far from 0), next to the rectified views 0 and 2
    K2 = base.K.copy()
    K2[0, 0] *= 1.1
    K2[1, 1] *= 1.1
    wl.cams.append(synth.Camera(K2, np.eye(3), -np.array([0.03, 0.02, 0.0]), base.width, base.height))
    lists = [[0, 3, 4, 5, 2]]
    wl.nbr_views = {1: lists[0]}
    run = Run(wl, nbr_lists=lists)
    for combine in ("min", "sum"):
        run.close()
        run = Run(wl, nbr_lists=lists, combine=combine)
        costs = run.volumes()
        assert run.check() == 0
        ref = _oracle_all(wl, combine=combine, nbr_lists=lists)
        _assert_equal(costs[0], ref[0], f"affine modes ({combine})")
    H5 = oracle.homography_table(wl.cams, 1, [5, 0], wl.n_labels, wl.z_near, wl.z_far)
    assert np.all(H5[0, :, 8] == 1.0) and np.all(H5[0, :, 0] != 1.0)  # unit, not rectified
    assert np.all(H5[1, :, 0] == 1.0) and np.all(H5[1, :, 4] == 1.0) and np.all(H5[1, :, 3] == 0.0)  # rectified
    H = oracle.homography_table(wl.cams, 1, [3, 4], wl.n_labels, wl.z_near, wl.z_far)
    assert np.all(H[:, :, 6] == 0) and np.all(H[:, :, 7] == 0)
    assert np.any(H[0, :, 8] != 1.0) and np.any(H[1, :, 8] <= 0) and np.any(H[1, :, 8] > 0)
    run.close()


def test_rectified_shift_path_and_its_fallbacks():
    """Rectified neighbours take the kernel's integer-shift path (column x + D, row kept) when the view's
    pitch is the reference width and its height at least the reference height; a shorter view (rows
    beyond it out of view) and a narrower one (another pitch) keep the float sequence. All must equal
    the contract, with min and sum."""
    wl = make_workload("tiny")
    base = wl.cams[1]
    for C, (w, h) in (([0.037, 0.0, 0.0], (480, 200)), ([-0.021, 0.0, 0.0], (400, 270)),
                      ([0.013, 0.0, 0.0], (480, 300))):
        wl.cams.append(synth.Camera(base.K.copy(), np.eye(3), -np.array(C), w, h))
    lists = [[0, 3, 4, 5, 2]]
    for combine in ("min", "sum"):
        run = Run(wl, nbr_lists=lists, combine=combine)
        costs = run.volumes()
        assert run.check() == 0
        _assert_equal(costs[0], _oracle_all(wl, combine=combine, nbr_lists=lists)[0], f"shift path ({combine})")
        run.close()


def test_projective_entries_whose_denominator_changes_sign():
    """A neighbour rotated 75 degrees about the vertical axis: Wz = 0 crosses the reference image, so
    part of every candidate plane is behind it (the kernel's general entries with the guarded
    reciprocal); a 4-degree rotation keeps Wz > 0 everywhere (the kernel's far-from-zero entries)."""
    import math
    wl = make_workload("tiny")
    base = wl.cams[1]
    for deg in (75.0, 4.0):
        a = math.radians(deg)
        R = np.array([[math.cos(a), 0.0, -math.sin(a)], [0.0, 1.0, 0.0], [math.sin(a), 0.0, math.cos(a)]])
        C = np.array([0.08, 0.0, 0.0])
        wl.cams.append(synth.Camera(base.K.copy(), R, -R @ C, base.width, base.height))
    lists = [[3, 4, 0]]
    for combine in ("min", "sum"):
        run = Run(wl, nbr_lists=lists, combine=combine)
        costs = run.volumes()
        assert run.check() == 0
        _assert_equal(costs[0], _oracle_all(wl, combine=combine, nbr_lists=lists)[0], f"rotated views ({combine})")
        run.close()


def test_tile_cull_is_exact_in_every_combination():
    """Two neighbours rotated 75 and 4 degrees about the vertical axis (projective entries only, so the
    kernel's tile cull runs): tiles that no pixel of which can reach a view are decided without sampling,
    and the volume still equals the oracle's with the minimum over views under the penalty floor, with a
    penalty below the largest sample cost (culled samples then take the penalty explicitly), and with
    the sum."""
    import math
    wl = make_workload("tiny")
    base = wl.cams[1]
    for deg in (75.0, 4.0):
        a = math.radians(deg)
        R = np.array([[math.cos(a), 0.0, -math.sin(a)], [0.0, 1.0, 0.0], [math.sin(a), 0.0, math.cos(a)]])
        C = np.array([0.08, 0.0, 0.0])
        wl.cams.append(synth.Camera(base.K.copy(), R, -R @ C, base.width, base.height))
    lists = [[3, 4]]
    for combine, penalty in (("min", None), ("min", 100), ("sum", None)):
        run = Run(wl, nbr_lists=lists, combine=combine, penalty=penalty)
        costs = run.volumes()
        assert run.check() == 0
        assert ftv.ftv_culled_evaluations(run.ctx) > 0
        want = _oracle_all(wl, combine=combine, nbr_lists=lists, penalty=penalty)[0]
        _assert_equal(costs[0], want, f"culled tiles ({combine}, penalty {penalty})")
        run.close()


def test_listed_segments_leave_other_rows_untouched():
    wl = make_workload("hd8", reduced=True)
    run = Run(wl)
    rng = np.random.default_rng(3)
    lists, counts, host_lists = [], [], []
    for S in run.S:
        lst = np.sort(rng.choice(S, size=S // 7, replace=False)).astype(np.int32)
        host_lists.append(lst)
        pad = np.concatenate([lst, np.full(5, -1, np.int32)])  # capacity beyond the count is ignored
        lists.append(dev(pad))
        counts.append(dev(np.array([len(lst)], np.int32)))
    costs = run.volumes(seg_lists=lists, n_listed=counts, fill=-7)
    assert run.check() == 0
    full = _oracle_all(wl)
    for c, ref, lst in zip(costs, full, host_lists):
        got = c.cpu().numpy()
        _assert_equal(got[lst], ref[lst], "listed rows")
        rest = np.setdiff1d(np.arange(ref.shape[0]), lst)
        assert np.all(got[rest] == -7)
    run.close()


def test_cached_segment_index_and_determinism():
    wl = make_workload("hd8", reduced=True)
    run = Run(wl)
    a = [c.cpu().numpy() for c in run.volumes()]
    for i in range(len(wl.ref_views)):
        ftv.ftv_segment_index(run.ctx, i, run.labels[i], run.S[i])
    b = [c.cpu().numpy() for c in run.volumes(use_cache=True)]
    assert run.check() == 0
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    run.close()


def _tiny_with_labels(lab, S):
    wl = make_workload("tiny")
    wl._labels[1] = (np.ascontiguousarray(lab, np.int32), S)
    return wl


@pytest.mark.parametrize("case", ["one_segment", "pixel_segments", "empty_segments", "stripes"])
def test_degenerate_segmentations(case):
    H, W = 270, 480
    if case == "one_segment":
        lab, S = np.zeros((H, W), np.int32), 1
    elif case == "pixel_segments":
        lab = np.empty((H, W), np.int32)
        lab[:, :64] = np.arange(H * 64).reshape(H, 64)  # one-pixel segments
        lab[:, 64:] = H * 64 + np.arange(H * (W - 64)).reshape(H, W - 64) // 37  # 37-pixel runs
        S = int(lab.max()) + 1
    elif case == "empty_segments":
        lab, S0 = synth.grid_labels(W, H, 16, 3, 11)
        lab = lab * 3  # only every third id is used
        S = 3 * S0 + 5
    else:  # one segment per row: segments cut by every tile boundary
        lab, S = np.repeat(np.arange(H, dtype=np.int32)[:, None], W, 1), H
    wl = _tiny_with_labels(lab, S)
    run = Run(wl)
    costs = run.volumes()
    assert run.check() == 0
    _assert_equal(costs[0], _oracle_all(wl)[0], case)
    run.close()


def test_single_neighbour_and_single_label():
    wl = make_workload("tiny")
    wl.n_labels = 1
    run = Run(wl, nbr_lists=[[2]])
    costs = run.volumes()
    assert run.check() == 0
    ref = _oracle_all(wl, nbr_lists=[[2]])
    _assert_equal(costs[0], ref[0], "L=1, N=1")
    run.close()


def test_invalid_labels_and_overflow_are_reported_not_trapped():
    wl = make_workload("tiny")
    lab, S = wl.labels(1)
    bad = lab.copy()
    bad[5, 7] = S  # out of range
    bad[6, 8] = -1
    wl2 = _tiny_with_labels(bad, S)
    run = Run(wl2)
    run.volumes()
    assert run.check() == ftv.FTV_ERR_INVALID_ARG
    # the context stays usable and clean afterwards
    run.labels = [dev(lab)]
    c = run.volumes()
    assert run.check() == 0
    _assert_equal(c[0], _oracle_all(make_workload("tiny"))[0], "after invalid labels")
    run.close()
    # one segment of 129600 pixels with a penalty of 2^20 could overflow int32
    wl3 = _tiny_with_labels(np.zeros((270, 480), np.int32), 1)
    run = Run(wl3, penalty=1 << 20)
    run.volumes()
    assert run.check() == ftv.FTV_ERR_OVERFLOW
    run.close()


def test_samples_above_bit_depth_are_reported():
    wl = make_workload("tiny")
    wl.views()  # rendered with 8-bit samples ...
    wl.bit_depth = 7  # ... then declared as 7-bit: samples above 127 must be reported
    run = Run(wl)
    run.volumes()
    assert run.check() == ftv.FTV_ERR_INVALID_ARG
    run.close()


# ------------------------------------------------------------------------------------------ temporal

def test_temporal_mask_and_adoption_bit_exact():
    wl = make_workload("temporal", reduced=True)
    run = Run(wl)
    r = wl.ref_views[2]
    lab, S = wl.labels(r)
    labels = dev(lab)
    frames = [run.planes(f)[r] for f in range(3)]
    host = [wl.view(r, f) for f in range(3)]
    for mode in (0, 1):
        for cur, prev, ifr in [(1, 0, None), (2, 1, 0), (1, 1, None)]:
            mask = torch.empty(S, dtype=torch.uint8, device="cuda")
            changed = torch.empty(S, dtype=torch.int32, device="cuda")
            n = torch.empty(1, dtype=torch.int32, device="cuda")
            ftv.ftv_temporal_mask(run.ctx, 2, frames[cur], frames[prev], frames[ifr] if ifr is not None else None,
                                  labels, S, 12, 4, mode, mask, changed, n)
            assert run.check() == 0
            m_ref, ch_ref, n_ref = oracle.temporal_mask(lab, S, host[cur], host[prev],
                                                        host[ifr] if ifr is not None else None, 2, 12, 4, mode)
            assert np.array_equal(mask.cpu().numpy(), m_ref)
            assert int(n.item()) == n_ref
            assert np.array_equal(changed.cpu().numpy()[:n_ref], ch_ref)
    # masked WTA: listed (changed) segments get the argmin, others adopt
    mask = torch.empty(S, dtype=torch.uint8, device="cuda")
    changed = torch.empty(S, dtype=torch.int32, device="cuda")
    n = torch.empty(1, dtype=torch.int32, device="cuda")
    ftv.ftv_temporal_mask(run.ctx, 2, frames[1], frames[0], frames[0], labels, S, 12, 4, 0, mask, changed, n)
    costs = run.volumes(frame=1, seg_lists=[changed if i == 2 else None for i in range(len(wl.ref_views))],
                        n_listed=[n if i == 2 else None for i in range(len(wl.ref_views))], fill=0)
    prev_l = dev(np.arange(S, dtype=np.uint16) % wl.n_labels)
    ifr_l = dev((np.arange(S, dtype=np.uint16) * 3) % wl.n_labels)
    out = torch.full((S,), 999, dtype=torch.int16, device="cuda")
    ftv.ftv_wta_depth(run.ctx, 2, costs[2], S, out, mask=mask, prev_label=prev_l, iframe_label=ifr_l)
    assert run.check() == 0
    m_host = mask.cpu().numpy()
    vol_ref = np.zeros((S, wl.n_labels), np.int32)
    ch = changed.cpu().numpy()[: int(n.item())]
    if len(ch):
        vol_ref = oracle_runs.volume(wl, r, frame=1, seg_list=ch, out=vol_ref)
    w_ref = oracle.wta(vol_ref, m_host, prev_l.cpu().numpy(), ifr_l.cpu().numpy())
    assert np.array_equal(out.cpu().numpy().view(np.uint16), w_ref)
    run.close()


def test_temporal_mask_label_layouts_and_call_sequences():
    """Label maps the kernel's per-tile bins do not cover, called in sequence on one context whose segment
    count grows, shrinks and grows again (the decide pass leaves the sums zero for the next call): one label
    per pixel at random (a tile's labels span far more than its bins, so runs go to global memory
    directly), three segments of whole column bands (runs span every tile) and the workload's own map, in
    both channel modes. A call with a label outside [0, S) reports it, and the next call is exact again.
    Frames of the reduced temporal workload (244 x 138: ragged in both tile directions; Sec. III-E)."""
    wl = make_workload("temporal", reduced=True)
    run = Run(wl, max_segments=6000)
    r = wl.ref_views[2]
    frames = [run.planes(f)[r] for f in range(3)]
    host = [wl.view(r, f) for f in range(3)]
    lab0, S0 = wl.labels(r)
    Hh, W = lab0.shape
    rng = np.random.default_rng(11)
    rand = rng.integers(0, 5000, size=(Hh, W), dtype=np.int32)
    bands = np.repeat((np.arange(W, dtype=np.int32) * 3 // W)[None, :], Hh, axis=0)

    def check(lab, S, mode, cur, prev, ifr):
        mask = torch.empty(S, dtype=torch.uint8, device="cuda")
        changed = torch.empty(S, dtype=torch.int32, device="cuda")
        n = torch.empty(1, dtype=torch.int32, device="cuda")
        ftv.ftv_temporal_mask(run.ctx, 2, frames[cur], frames[prev], frames[ifr] if ifr is not None else None,
                              dev(lab), S, 12, 4, mode, mask, changed, n)
        assert run.check() == 0
        m_ref, ch_ref, n_ref = oracle.temporal_mask(lab, S, host[cur], host[prev],
                                                    host[ifr] if ifr is not None else None, 2, 12, 4, mode)
        assert np.array_equal(mask.cpu().numpy(), m_ref)
        assert int(n.item()) == n_ref
        assert np.array_equal(changed.cpu().numpy()[:n_ref], ch_ref)

    for lab, S in [(rand, 5000), (lab0, S0), (bands, 3), (rand, 5000), (lab0, S0)]:
        check(lab, S, 0, 1, 0, 0)
        check(lab, S, 1, 2, 1, None)
    bad = lab0.copy()
    bad[Hh // 2, W // 3] = S0
    mask = torch.empty(S0, dtype=torch.uint8, device="cuda")
    changed = torch.empty(S0, dtype=torch.int32, device="cuda")
    n = torch.empty(1, dtype=torch.int32, device="cuda")
    ftv.ftv_temporal_mask(run.ctx, 2, frames[1], frames[0], None, dev(bad), S0, 12, 4, 0, mask, changed, n)
    assert run.check() == ftv.FTV_ERR_INVALID_ARG
    check(lab0, S0, 0, 1, 0, 0)
    run.close()


def test_temporal_mask_after_adjacency_on_the_same_reference():
    """ftv_adjacency uses a reference's slot of the context's temporal sums as scratch: a temporal test of that
    reference right after it (and once more after that) still equals the oracle's (Sec. III-E)."""
    wl = make_workload("temporal", reduced=True)
    run = Run(wl)
    i, r = 2, wl.ref_views[2]
    lab, S = wl.labels(r)
    labels = dev(lab)
    frames = [run.planes(f)[r] for f in range(3)]
    host = [wl.view(r, f) for f in range(3)]
    cap = 8 * S + 64
    es = torch.zeros(cap, dtype=torch.int32, device="cuda")
    et = torch.zeros(cap, dtype=torch.int32, device="cuda")
    beta = torch.zeros(cap, dtype=torch.float32, device="cuda")
    ne = torch.zeros(1, dtype=torch.int32, device="cuda")
    for _ in range(2):
        ftv.ftv_adjacency(run.ctx, i, frames[1], labels, S, 4, 37.5, 1.5, es, et, beta, ne)
        for cur, prev in ((1, 0), (2, 1)):
            mask = torch.empty(S, dtype=torch.uint8, device="cuda")
            changed = torch.empty(S, dtype=torch.int32, device="cuda")
            n = torch.empty(1, dtype=torch.int32, device="cuda")
            ftv.ftv_temporal_mask(run.ctx, i, frames[cur], frames[prev], frames[0], labels, S, 12, 4, 1, mask,
                                  changed, n)
            assert run.check() == 0
            m_ref, ch_ref, n_ref = oracle.temporal_mask(lab, S, host[cur], host[prev], host[0], 2, 12, 4, 1)
            assert np.array_equal(mask.cpu().numpy(), m_ref)
            assert int(n.item()) == n_ref
            assert np.array_equal(changed.cpu().numpy()[:n_ref], ch_ref)
    run.close()


def test_temporal_mask_views_equals_the_oracle_per_reference():
    """Every reference of the reduced temporal workload in one ftv_temporal_mask_views call, two of them with
    other label maps (one label per pixel at random; five column bands), in both channel modes, with and
    without the I frame: each reference's mask, ordered list and count equal the oracle's (Sec. III-E). A
    repeated reference index is refused before anything runs."""
    wl = make_workload("temporal", reduced=True)
    run = Run(wl, max_segments=6000)
    R = len(wl.ref_views)
    planes = [run.planes(f) for f in range(3)]
    rng = np.random.default_rng(12)
    labs = []
    for i, r in enumerate(wl.ref_views):
        lab, S = wl.labels(r)
        if i == 1:
            lab, S = rng.integers(0, 4000, size=lab.shape, dtype=np.int32), 4000
        elif i == 4:
            lab, S = np.repeat((np.arange(lab.shape[1], dtype=np.int32) * 5 // lab.shape[1])[None, :], lab.shape[0],
                               axis=0), 5
        labs.append((np.ascontiguousarray(lab), S))
    labels_d = [dev(l) for l, _ in labs]
    Ss = [S for _, S in labs]
    for mode in (0, 1):
        for cur, prev, ifr in [(1, 0, 0), (2, 1, None)]:
            masks = [torch.empty(S, dtype=torch.uint8, device="cuda") for S in Ss]
            changed = [torch.empty(S, dtype=torch.int32, device="cuda") for S in Ss]
            ns = [torch.empty(1, dtype=torch.int32, device="cuda") for _ in Ss]
            ftv.ftv_temporal_mask_views(run.ctx, list(range(R)), [planes[cur][r] for r in wl.ref_views],
                                        [planes[prev][r] for r in wl.ref_views],
                                        [planes[ifr][r] for r in wl.ref_views] if ifr is not None else None,
                                        labels_d, Ss, 12, 4, mode, masks, changed, ns)
            assert run.check() == 0
            for i, r in enumerate(wl.ref_views):
                host = [wl.view(r, f) for f in range(3)]
                m_ref, ch_ref, n_ref = oracle.temporal_mask(labs[i][0], Ss[i], host[cur], host[prev],
                                                            host[ifr] if ifr is not None else None, 2, 12, 4, mode)
                assert np.array_equal(masks[i].cpu().numpy(), m_ref), (mode, i)
                assert int(ns[i].item()) == n_ref, (mode, i)
                assert np.array_equal(changed[i].cpu().numpy()[:n_ref], ch_ref), (mode, i)
    with pytest.raises(ftv.FtvError):
        ftv.ftv_temporal_mask_views(run.ctx, [0, 0], [planes[1][wl.ref_views[0]]] * 2, [planes[0][wl.ref_views[0]]] * 2,
                                    None, [labels_d[0]] * 2, [Ss[0]] * 2, 12, 4, 0, masks[:1] * 2, changed[:1] * 2,
                                    ns[:1] * 2)
    run.close()


def test_temporal_mask_views_more_references_than_one_launch_holds():
    """18 references of one context (more than the 16 one launch sequence takes, so the call makes two), each
    64 x 48 with its own random 10-bit frames and label map, in one ftv_temporal_mask_views call against the
    oracle per reference (Sec. III-E)."""
    import types
    from synth import linear_rig
    n, W, Hh, S = 18, 64, 48, 40
    cams = linear_rig(n, 0.02, 100.0, W, Hh)
    ctx = ftv.ftv_depth_init(cams, list(range(n)), 4, 1.0, 10.0, sample_bytes=2, bit_depth=10, max_segments=S)
    rng = np.random.default_rng(18)
    labs, host, dev_frames = [], [], []
    for r in range(n):
        labs.append(rng.integers(0, S, size=(Hh, W), dtype=np.int32) if r % 2 else
                    np.repeat(np.repeat(np.arange(S // 8 * 8, dtype=np.int32).reshape(S // 8, 8) % S, Hh // 5 + 1,
                                        axis=0)[:Hh], W // 8, axis=1)[:, :W].copy())
        frames = []
        for f in range(3):
            Y, U, V = (rng.integers(0, 1024, size=(Hh, W)).astype(np.uint16) for _ in range(3))
            frames.append(types.SimpleNamespace(Y=Y, U=U, V=V))
        host.append(frames)
        dev_frames.append([tuple(dev(a) for a in (v.Y, v.U, v.V)) for v in frames])
    for mode, ifr in ((0, 2), (1, None)):
        masks = [torch.empty(S, dtype=torch.uint8, device="cuda") for _ in range(n)]
        changed = [torch.empty(S, dtype=torch.int32, device="cuda") for _ in range(n)]
        ns = [torch.empty(1, dtype=torch.int32, device="cuda") for _ in range(n)]
        ftv.ftv_temporal_mask_views(ctx, list(range(n)), [dev_frames[r][1] for r in range(n)],
                                    [dev_frames[r][0] for r in range(n)],
                                    [dev_frames[r][ifr] for r in range(n)] if ifr is not None else None,
                                    [dev(l) for l in labs], [S] * n, 40, 20, mode, masks, changed, ns)
        assert ftv.ftv_check(ctx) == 0
        for r in range(n):
            m_ref, ch_ref, n_ref = oracle.temporal_mask(labs[r], S, host[r][1], host[r][0],
                                                        host[r][ifr] if ifr is not None else None, 2, 40, 20, mode)
            assert np.array_equal(masks[r].cpu().numpy(), m_ref), (mode, r)
            assert int(ns[r].item()) == n_ref, (mode, r)
            assert np.array_equal(changed[r].cpu().numpy()[:n_ref], ch_ref), (mode, r)
    ctx.close()


# ------------------------------------------------------------------------------------ full size, sampled

@pytest.mark.parametrize("name", ["hd8", "uhd15"])
def test_full_size_sampled_entries(name):
    wl = make_workload(name)
    run = Run(wl)
    costs = run.volumes()
    assert run.check() == 0
    rng = np.random.default_rng(7)
    for i, r in enumerate(wl.ref_views[:: 3 if name == "uhd15" else 2]):
        idx = wl.ref_views.index(r)
        S = run.S[idx]
        seg = rng.integers(0, S, 24).astype(np.int32)
        lab = rng.integers(0, wl.n_labels, 24).astype(np.int32)
        got = costs[idx][torch.from_numpy(seg).long().cuda(), torch.from_numpy(lab).long().cuda()].cpu().numpy()
        ref = oracle_runs.entries(wl, r, seg, lab)
        assert np.array_equal(got, ref), (name, r, got, ref)
        # the winner of sampled rows equals the argmin of the GPU's own full rows, checked on the host
        win = torch.empty(S, dtype=torch.int16, device="cuda")
        ftv.ftv_wta_depth(run.ctx, idx, costs[idx], S, win)
        rows = costs[idx][torch.from_numpy(seg).long().cuda()].cpu().numpy()
        assert np.array_equal(win.cpu().numpy().view(np.uint16)[seg], rows.argmin(1).astype(np.uint16))
    run.close()


def _random_views(cams, seed, bits=8):
    rng = np.random.default_rng(seed)
    hi = (1 << bits)
    dt = np.uint8 if bits <= 8 else np.uint16
    return [synth.View(*(rng.integers(0, hi, (c.height, c.width), dtype=dt) for _ in range(3))) for c in cams]


@pytest.mark.parametrize("combine,penalty", [("min", None), ("min", 100), ("sum", None)])
def test_thirty_two_neighbours_on_a_convergent_arc(combine, penalty):
    """FTV_MAX_NBRS = 32 neighbours of one reference on a convergent arc (projective entries): the per-label
    neighbour lists are built by one warp with one lane per neighbour, so the last lane is used; the label
    block is 512 / 32 = 16 labels."""
    W, H, L = 200, 120, 24
    cams = synth.arc_rig(33, 3.0, 3.0, 260.0, W, H, seed=5, roll_deg=2.0)
    views = _random_views(cams, 6)
    lab, S = synth.grid_labels(W, H, 9, 2, seed=7)
    nb = [v for v in range(33) if v != 16]
    comb = ftv.FTV_COMBINE_MIN if combine == "min" else ftv.FTV_COMBINE_SUM
    pen = 765 if penalty is None else penalty
    ctx = ftv.ftv_depth_init(cams, [16], L, 0.8, 15.0, sample_bytes=1, bit_depth=8, oob_penalty=pen, combine=comb,
                             max_segments=S)
    assert ftv.ftv_get_launch_shape(ctx)["max_label_block"] == 16
    cost = torch.empty((S, L), dtype=torch.int32, device="cuda")
    ftv.ftv_cost_volume(ctx, [(dev(v.Y), dev(v.U), dev(v.V)) for v in views], [dev(lab)], [S], [cost])
    assert ftv.ftv_check(ctx) == 0
    Ht = oracle.homography_table(cams, 16, nb, L, 0.8, 15.0)
    want = oracle.cost_volume(cams, views, 1, 16, nb, Ht, L, lab, S, pen, combine)
    _assert_equal(cost, want, f"32 neighbours ({combine}, penalty {pen})")
    ctx.close()


def test_maximum_label_count():
    """FTV_MAX_LABELS = 4096 candidate depths on a small linear rig (64 label blocks of 64 per tile)."""
    W, H, L = 96, 40, ftv.FTV_MAX_LABELS
    cams = synth.linear_rig(3, 0.05, 120.0, W, H)
    views = _random_views(cams, 8, bits=10)
    lab, S = synth.grid_labels(W, H, 8, 1, seed=9)
    ctx = ftv.ftv_depth_init(cams, [1], L, 0.5, 20.0, sample_bytes=2, bit_depth=10, max_segments=S)
    cost = torch.empty((S, L), dtype=torch.int32, device="cuda")
    ftv.ftv_cost_volume(ctx, [(dev(v.Y), dev(v.U), dev(v.V)) for v in views], [dev(lab)], [S], [cost])
    win = torch.empty(S, dtype=torch.int16, device="cuda")
    ftv.ftv_wta_depth(ctx, 0, cost, S, win)
    assert ftv.ftv_check(ctx) == 0
    Ht = oracle.homography_table(cams, 1, [0, 2], L, 0.5, 20.0)
    want = oracle.cost_volume(cams, views, 2, 1, [0, 2], Ht, L, lab, S, 3 * 1023)
    _assert_equal(cost, want, "4096 labels")
    assert np.array_equal(win.cpu().numpy().view(np.uint16), oracle.wta(want))
    ctx.close()
