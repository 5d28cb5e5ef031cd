"""CPU-side checks of the C-ABI library: it loads, exports what include/ftv.h declares, forms the same
FP32 homography table as the oracle bit for bit, and rejects bad arguments before touching a device."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import synth
from synth.configs import make_workload

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ftv():
    import __graft_entry__
    __graft_entry__._load_builder().build()
    import paper_1909_02294_gb300 as ftv
    return ftv


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"FTV_API\s+[\w\s\*]+?\b(ftv_\w+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol(ftv):
    names = _declared()
    assert {"ftv_depth_init", "ftv_cost_volume", "ftv_temporal_mask", "ftv_wta_depth"} <= names
    lib = ctypes.CDLL(ftv.ftv.LIB_PATH)
    for n in sorted(names):
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
    assert set(ftv.ftv.EXPORTED) <= names


@pytest.mark.parametrize("name,reduced", [("tiny", False), ("hd8", False), ("uhd15", False), ("uhd15", True),
                                          ("serving_small", False)])
def test_homography_table_bit_identical_to_oracle(ftv, name, reduced):
    wl = make_workload(name, reduced=reduced)
    for i, r in enumerate(wl.ref_views[:4]):
        mine = ftv.ftv_compute_homographies(wl.cams, wl.ref_views, i, wl.n_labels, wl.z_near, wl.z_far)
        ref = oracle.homography_table(wl.cams, r, wl.neighbours(r), wl.n_labels, wl.z_near, wl.z_far)
        assert mine.shape == ref.shape
        assert np.array_equal(mine.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("name,reduced", [("tiny", False), ("hd8", False), ("uhd15", False)])
def test_fp64_homography_table_bit_identical_to_oracle(ftv, name, reduced):
    """The FP64 projection mode's table (before the FP32 rounding), computed by the library's host code,
    equals the oracle's byte for byte, and rounds to the FP32 table."""
    wl = make_workload(name, reduced=reduced)
    for i, r in enumerate(wl.ref_views[:4]):
        mine = ftv.ftv_compute_homographies_f64(wl.cams, wl.ref_views, i, wl.n_labels, wl.z_near, wl.z_far)
        ref = oracle.homography_table_f64(wl.cams, r, wl.neighbours(r), wl.n_labels, wl.z_near, wl.z_far)
        assert mine.dtype == np.float64 and mine.shape == ref.shape
        assert mine.tobytes() == ref.tobytes()
        f32 = ftv.ftv_compute_homographies(wl.cams, wl.ref_views, i, wl.n_labels, wl.z_near, wl.z_far)
        assert np.array_equal(mine.astype(np.float32).view(np.uint32), f32.view(np.uint32))
    r0 = wl.ref_views[0]
    two = wl.neighbours(r0)[:2]
    lists = [two] + [wl.neighbours(r)[:1] for r in wl.ref_views[1:]]
    mine = ftv.ftv_compute_homographies_f64(wl.cams, wl.ref_views, 0, 7, wl.z_near, wl.z_far, nbr_lists=lists,
                                            plane_mode=ftv.FTV_PLANES_CENTRE, centre_view=1)
    ref = oracle.homography_table_f64(wl.cams, r0, two, 7, wl.z_near, wl.z_far, plane_mode=1, centre=1)
    assert mine.tobytes() == ref.tobytes()


def test_homography_table_centre_planes_and_neighbour_lists(ftv):
    wl = make_workload("uhd15", reduced=True)
    lists = [[1, 2], [6, 8, 0], [13]]
    for i, r in enumerate(wl.ref_views):
        mine = ftv.ftv_compute_homographies(wl.cams, wl.ref_views, i, 33, 0.8, 15.0, nbr_lists=lists,
                                            plane_mode=ftv.FTV_PLANES_CENTRE, centre_view=7)
        ref = oracle.homography_table(wl.cams, r, lists[i], 33, 0.8, 15.0, plane_mode=1, centre=7)
        assert np.array_equal(mine.view(np.uint32), ref.view(np.uint32))


def test_init_rejects_bad_arguments_before_any_device_call(ftv):
    wl = make_workload("tiny")
    good = dict(sample_bytes=1, bit_depth=8, max_segments=600)
    bad_cases = [
        dict(n_labels=0), dict(z_near=0.0), dict(z_far=0.4), dict(sample_bytes=3), dict(bit_depth=9),
        dict(max_segments=0), dict(plane_mode=1, centre_view=7), dict(combine=5), dict(ref_views=[1, 1]),
        dict(nbr_lists=[[1]]),
    ]
    for case in bad_cases:
        kw = dict(good)
        args = dict(cams=wl.cams, ref_views=[1], n_labels=64, z_near=0.5, z_far=10.0)
        for k in list(case):
            if k in args:
                args[k] = case.pop(k)
        kw.update(case)
        with pytest.raises(ftv.FtvError) as e:
            ftv.ftv_depth_init(args["cams"], args["ref_views"], args["n_labels"], args["z_near"], args["z_far"], **kw)
        assert e.value.code == 1, case
    bad_cam = synth.Camera(wl.cams[0].K.copy(), wl.cams[0].R, wl.cams[0].t, 480, 270)
    bad_cam.K[2, 0] = 0.1
    with pytest.raises(ftv.FtvError) as e:
        ftv.ftv_depth_init([bad_cam] + wl.cams[1:], [1], 64, 0.5, 10.0, **good)
    assert e.value.code == 1
    assert ftv.ftv_status_str(4).startswith("segment cost")


@pytest.mark.parametrize("sizes,sb,bd,S,m,T", [
    ([], 1, 8, 8, 5, 10),              # no image
    ([(0, 5)], 1, 8, 8, 5, 10),        # empty width
    ([(40000, 5)], 1, 8, 8, 5, 10),    # wider than FTV_MAX_DIM
    ([(64, 48)], 3, 8, 8, 5, 10),      # sample size
    ([(64, 48)], 1, 9, 8, 5, 10),      # 9 bits in one byte
    ([(64, 48)], 2, 0, 8, 5, 10),      # no bits
    ([(64, 48)], 1, 8, 0, 5, 10),      # grid step 0
    ([(64, 48)], 1, 8, 65, 5, 10),     # grid step above FTV_SEG_MAX_STEP
    ([(64, 48)], 1, 8, 8, -1, 10),     # negative compactness
    ([(64, 48)], 1, 8, 8, 256, 10),    # compactness above 255
    ([(64, 48)], 1, 8, 8, 5, 0),       # no pass
    ([(64, 48)], 1, 8, 8, 5, 65),      # too many passes
    ([(32767, 32767), (32767, 32767), (32767, 32767)], 2, 10, 8, 5, 10),  # 2^31 pixels or more
])
def test_segmenter_rejects_bad_configurations_on_the_host(ftv, sizes, sb, bd, S, m, T):
    with pytest.raises(ftv.FtvError) as e:
        ftv.Segmenter(sizes, sb, bd, S, m, T)
    assert e.value.code == ftv.FTV_ERR_INVALID_ARG


def test_label_split_by_reciprocal_multiply_is_exact_at_every_label_count():
    """The centre table splits an entry index j < L * N into (neighbour, label) with
    umulhi(j, ceil(2^32 / L)) instead of j / L. Its error term grows with j and first shows just below a
    multiple of L, so checking j = kL - 1 and kL for every k up to N and every L up to the limits covers
    every j the kernel can see."""
    hdr = open(os.path.join(ROOT, "include", "ftv.h")).read()
    nbrs = int(re.search(r"#define FTV_MAX_NBRS (\d+)", hdr).group(1))
    max_labels = int(re.search(r"#define FTV_MAX_LABELS (\d+)", hdr).group(1))
    for L in range(2, max_labels + 1):
        magic = ((1 << 32) + L - 1) // L
        k = np.arange(1, nbrs + 1, dtype=np.uint64)
        j = np.concatenate([k * L - 1, (k - 1) * L]).astype(np.uint64)
        got = (j * np.uint64(magic)) >> np.uint64(32)
        assert np.array_equal(got, j // np.uint64(L)), L


def test_job_footprint_on_the_host(ftv):
    """ftv_job_footprint needs no device: it grows with the segment count, an FP64-precision stream adds
    exactly its FP64 homography tables (8 bytes x 9 per neighbour and label of every reference), and an
    invalid configuration is refused."""
    wl = make_workload("hd8")
    S = max(wl.labels(r)[1] for r in wl.ref_views)
    args = (wl.cams, wl.ref_views, wl.n_labels, wl.z_near, wl.z_far)
    kw = dict(sample_bytes=wl.sample_bytes, bit_depth=wl.bit_depth, max_segments=S)
    a = ftv.ftv_job_footprint(*args, S, **kw)
    b = ftv.ftv_job_footprint(*args, S + 1000, **kw)
    assert 0 < a < b
    c = ftv.ftv_job_footprint(*args, S, precision=ftv.FTV_PRECISION_FP64, **kw)
    nbrs = sum(len(wl.neighbours(r)) for r in wl.ref_views)
    assert c - a == nbrs * wl.n_labels * 9 * 8
    # more than the views' input planes and the int32 cost volume alone
    inputs = sum(3 * cm.width * cm.height * wl.sample_bytes for cm in wl.cams)
    assert a > inputs + len(wl.ref_views) * S * wl.n_labels * 4
    with pytest.raises(ftv.FtvError):
        ftv.ftv_job_footprint(*args, -1, **kw)
    with pytest.raises(ftv.FtvError):
        ftv.ftv_job_footprint(wl.cams, wl.ref_views, 0, wl.z_near, wl.z_far, S, **kw)


def test_static_temporal_mask_refuses_tensors_on_another_device(ftv, monkeypatch):
    """The allocation-free temporal test runs on its label map's device; an output or a frame on another
    device is refused on the host before the library is called (no launch)."""
    import torch

    class Fake:
        def __init__(self, device):
            self.device = torch.device(device)

        def data_ptr(self):
            return 4096

        def stride(self, k):
            return 16

        def element_size(self):
            return 2

    called = []
    monkeypatch.setattr(ftv.ftv.lib, "ftv_temporal_mask_static", lambda *a: called.append(a) or 0, raising=False)
    frame = (Fake("cuda:0"), Fake("cuda:0"), Fake("cuda:0"))
    for odd in ("mask", "frame", "status"):
        mask = Fake("cuda:1" if odd == "mask" else "cuda:0")
        cur = (Fake("cuda:1"), frame[1], frame[2]) if odd == "frame" else frame
        status = Fake("cuda:1") if odd == "status" else None
        with pytest.raises(ftv.FtvError) as e:
            ftv.ftv_temporal_mask_static(16, 8, 2, cur, frame, None, Fake("cuda:0"), 4, 12, 4, 0, mask,
                                         Fake("cuda:0"), Fake("cuda:0"), status=status)
        assert e.value.code == ftv.FTV_ERR_INVALID_ARG
    assert called == []


def test_binding_constants_match_the_header(ftv):
    txt = open(os.path.join(ROOT, "include", "ftv.h")).read()
    for name in ("FTV_MAX_VIEWS", "FTV_MAX_NBRS", "FTV_MAX_LABELS", "FTV_MAX_DIM", "FTV_STATIC_MAX_SEGMENTS",
                 "FTV_MAX_BATCH_CHUNKS"):
        m = re.search(r"#define\s+" + name + r"\s+(\d+)", txt)
        assert m and int(m.group(1)) == getattr(ftv, name), name
    codes = dict(re.findall(r"(FTV_(?:OK|ERR_\w+))\s*=\s*(\d+)", txt))
    for name, value in codes.items():
        assert getattr(ftv, name) == int(value), name
