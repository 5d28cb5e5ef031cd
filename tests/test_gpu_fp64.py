"""GPU parity of the FP64 projection mode (FTV_PRECISION_FP64): sample positions from the unrounded
homography in IEEE double, as the oracle's FP64 mode computes them (Sec. III-C's T[.]; the paper fixes no
precision). The kernel evaluates each tile in an FP32 local frame with a rigorous error bound and redoes
in FP64 the evaluations near a rounding boundary; whatever path an evaluation takes, the volume must
equal the oracle's FP64-mode volume bit for bit.
"""
from __future__ import annotations

import math

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

from gpu_runs import Run, dev  # noqa: E402

FP64 = ftv.FTV_PRECISION_FP64


def _oracle_fp64(wl, combine=None, nbr_lists=None, plane_mode=0, centre=0, penalty=None, frame=0):
    out = []
    for i, r in enumerate(wl.ref_views):
        lab, S = wl.labels(r)
        nb = nbr_lists[i] if nbr_lists is not None else wl.neighbours(r)
        H = oracle.homography_table_f64(wl.cams, r, nb, wl.n_labels, wl.z_near, wl.z_far, plane_mode=plane_mode,
                                        centre=centre)
        out.append(oracle.cost_volume(wl.cams, wl.views(frame), wl.sample_bytes, r, nb, H, wl.n_labels, lab, S,
                                      wl.oob_penalty if penalty is None else penalty, combine or wl.combine))
    return out


def _assert_equal(got, ref, what):
    got = got.cpu().numpy() if isinstance(got, torch.Tensor) else got
    bad = int((got != ref).sum())
    assert bad == 0, f"{what}: {bad} of {ref.size} entries differ"


def _near_tie(W=256, H=48, L=8, wide=False):
    """Two cameras 0.1 m apart, f = 100 px; depths put every label's disparity 1e-7 beyond a half-integer
    (10 iz_d = 10.5000001 + d), where the FP32 contract rounds the other way. wide: the neighbour image is 8
    columns wider (its principal point 4 px further right, so the offsets stay 1e-7 beyond half-integers)."""
    f, B = 100.0, 0.1
    Wv = W + 8 if wide else W
    cams = [synth.Camera(synth.intrinsics(f, W, H), np.eye(3), np.zeros(3), W, H),
            synth.Camera(synth.intrinsics(f, Wv, H), np.eye(3), -np.array([B, 0.0, 0.0]), Wv, H)]
    rng = np.random.default_rng(11)
    views = [synth.View(*(rng.integers(0, 256, (H, c.width), dtype=np.uint8) for _ in range(3))) for c in cams]
    lab, S = synth.grid_labels(W, H, 8, 2, seed=12)
    return cams, views, lab, S, L, 1.0 / ((10.5000001 + L - 1) / (f * B)), 1.0 / (10.5000001 / (f * B))


def test_fp64_tables_equal_the_oracle_tables():
    for name, reduced, pm in (("tiny", False, 0), ("hd8", True, 0), ("uhd15", True, 1)):
        wl = make_workload(name, reduced=reduced)
        run = Run(wl, plane_mode=pm, centre=wl.n_views // 2, precision=FP64)
        for i, r in enumerate(wl.ref_views):
            got = ftv.ftv_get_homographies_f64(run.ctx, i)
            want = oracle.homography_table_f64(wl.cams, r, wl.neighbours(r), wl.n_labels, wl.z_near, wl.z_far,
                                               plane_mode=pm, centre=wl.n_views // 2)
            assert got.tobytes() == want.tobytes(), (name, r)
            assert np.array_equal(ftv.ftv_get_homographies(run.ctx, i), want.astype(np.float32))
        run.close()


@pytest.mark.parametrize("name,reduced,combine", [("tiny", False, "min"), ("tiny", False, "sum"),
                                                  ("hd8", True, "min"), ("uhd15", True, "min"),
                                                  ("temporal", True, "min")])
def test_fp64_volumes_bit_exact(name, reduced, combine):
    wl = make_workload(name, reduced=reduced)
    run = Run(wl, combine=combine, precision=FP64)
    costs = run.volumes()
    assert run.check() == 0
    want = _oracle_fp64(wl, combine=combine)
    for i in range(len(wl.ref_views)):
        _assert_equal(costs[i], want[i], f"{name} ref {wl.ref_views[i]} ({combine})")
    run.close()


@pytest.mark.parametrize("combine,wide", [("min", False), ("sum", False), ("min", True), ("sum", True)])
def test_fp64_on_half_integer_disparities(combine, wide):
    """Every evaluation lies 1e-7 from a rounding boundary, far inside the FP32 bound, and the volume differs
    from the FP32 contract's. With equal image widths every entry is an exact FP64 integer shift (its offset
    is more than 2^-30 from a half-integer): nothing is recomputed. With a wider neighbour image the shift
    does not apply (the neighbour's row pitch differs), and every evaluation goes through the FP64 path."""
    cams, views, lab, S, L, zn, zf = _near_tie(wide=wide)
    comb = ftv.FTV_COMBINE_MIN if combine == "min" else ftv.FTV_COMBINE_SUM
    vols = {}
    for prec in (ftv.FTV_PRECISION_FP32, FP64):
        ctx = ftv.ftv_depth_init(cams, [0], L, zn, zf, sample_bytes=1, bit_depth=8, oob_penalty=765, combine=comb,
                                 max_segments=S, precision=prec)
        cost = torch.empty((S, L), dtype=torch.int32, device="cuda")
        ftv.ftv_cost_volume(ctx, [(dev(v.Y), dev(v.U), dev(v.V)) for v in views], [dev(lab)], [S], [cost])
        assert ftv.ftv_check(ctx) == 0
        vols[prec] = cost.cpu().numpy()
        if prec == FP64:
            n_rec, n_cull = ftv.ftv_fp64_recomputed(ctx), ftv.ftv_culled_evaluations(ctx)
            if wide:
                assert n_rec + n_cull == lab.size * L and n_rec > 0.9 * lab.size * L
            else:
                assert n_rec == 0
        else:
            assert ftv.ftv_fp64_recomputed(ctx) == 0
        ctx.close()
    H64 = oracle.homography_table_f64(cams, 0, [1], L, zn, zf)
    H32 = oracle.homography_table(cams, 0, [1], L, zn, zf)
    assert np.array_equal(vols[FP64], oracle.cost_volume(cams, views, 1, 0, [1], H64, L, lab, S, 765, combine))
    assert np.array_equal(vols[ftv.FTV_PRECISION_FP32], oracle.cost_volume(cams, views, 1, 0, [1], H32, L, lab, S,
                                                                           765, combine))
    assert not np.array_equal(vols[FP64], vols[ftv.FTV_PRECISION_FP32])


def _rotated(base, deg, C=(0.08, 0.0, 0.0)):
    a = math.radians(deg)
    R = np.array([[math.cos(a), 0.0, -math.sin(a)], [0.0, 1.0, 0.0], [math.sin(a), 0.0, math.cos(a)]])
    return synth.Camera(base.K.copy(), R, -R @ np.array(C), base.width, base.height)


@pytest.mark.parametrize("combine,penalty", [("min", None), ("min", 100), ("sum", None)])
def test_fp64_rotated_behind_and_axial_cameras(combine, penalty):
    """Neighbours rotated 75 degrees (Wz = 0 crosses the reference image: entries without an error bound,
    all evaluations in FP64), 4 degrees (bounded entries), a camera looking backwards from the reference
    centre (every plane behind it: culled), and two cameras displaced along the optical axis (affine
    entries, h8 <= 0 for planes behind one of them)."""
    wl = make_workload("tiny")
    base = wl.cams[1]
    wl.cams.append(_rotated(base, 75.0))
    wl.cams.append(_rotated(base, 4.0))
    back = synth.Camera(base.K.copy(), np.diag([-1.0, 1.0, -1.0]), np.zeros(3), base.width, base.height)
    back.t = -back.R @ base.centre
    wl.cams.append(back)
    for C in ([0.0, 0.0, 0.3], [0.02, 0.0, 1.0]):
        wl.cams.append(synth.Camera(base.K.copy(), np.eye(3), -np.array(C), base.width, base.height))
    lists = [[3, 4, 5, 6, 7, 0]]
    run = Run(wl, nbr_lists=lists, combine=combine, penalty=penalty, precision=FP64)
    costs = run.volumes()
    assert run.check() == 0
    assert ftv.ftv_fp64_recomputed(run.ctx) > 0 and ftv.ftv_culled_evaluations(run.ctx) > 0
    want = _oracle_fp64(wl, combine=combine, nbr_lists=lists, penalty=penalty)[0]
    _assert_equal(costs[0], want, f"rotated/behind/axial ({combine}, {penalty})")
    run.close()


def test_fp64_listed_segments_leave_other_rows_untouched():
    wl = make_workload("hd8", reduced=True)
    run = Run(wl, precision=FP64)
    full = run.volumes()
    rng = np.random.default_rng(3)
    lists, counts = [], []
    for S in run.S:
        sel = np.sort(rng.choice(S, S // 7, replace=False)).astype(np.int32)
        lists.append(dev(sel))
        counts.append(torch.tensor([len(sel)], dtype=torch.int32, device="cuda"))
    part = run.volumes(seg_lists=lists, n_listed=counts, fill=-5, use_cache=True)
    assert run.check() == 0
    for f, p, sel in zip(full, part, lists):
        f, p, sel = f.cpu().numpy(), p.cpu().numpy(), sel.cpu().numpy()
        assert np.array_equal(p[sel], f[sel])
        rest = np.setdiff1d(np.arange(f.shape[0]), sel)
        assert np.all(p[rest] == -5)
    run.close()


def test_fp64_streams_in_a_batch_and_mixed_precision_refused():
    """A batch of FP64-precision streams gives the winner-take-all labels of the oracle's FP64 volumes
    (I frame); a batch that mixes FP32 and FP64 streams is refused on the host."""
    wl = make_workload("temporal", reduced=True)
    S = [wl.labels(r)[1] for r in wl.ref_views]
    ctxs = {}
    for prec in (FP64, ftv.FTV_PRECISION_FP32):
        c = ftv.ftv_depth_init(wl.cams, wl.ref_views, wl.n_labels, wl.z_near, wl.z_far, sample_bytes=wl.sample_bytes,
                               bit_depth=wl.bit_depth, oob_penalty=wl.oob_penalty, max_segments=max(S), precision=prec)
        ftv.ftv_stream_init(c, [dev(wl.labels(r)[0]) for r in wl.ref_views], S, 12, 4, 0)
        ctxs[prec] = c
    planes = [(dev(v.Y), dev(v.U), dev(v.V)) for v in wl.views(0)]
    out = [torch.zeros(s, dtype=torch.int16, device="cuda") for s in S]

    def job(c):
        return {"ctx": c, "planes": planes, "frame_type": ftv.FTV_FRAME_I, "label_out": out, "depth_out": None}

    b = ftv.ftv_batch_create(2, 32, 32)
    assert ftv.ftv_batch_prepare(b, [job(ctxs[FP64]), job(ctxs[ftv.FTV_PRECISION_FP32])]) == ftv.FTV_ERR_INVALID_ARG
    assert ftv.ftv_batch_prepare(b, [job(ctxs[FP64])]) == 0
    ftv.ftv_batch_launch(b)
    assert ftv.ftv_batch_wait(b) == 0
    want = _oracle_fp64(wl)
    for i in range(len(wl.ref_views)):
        assert np.array_equal(out[i].cpu().numpy().view(np.uint16), oracle.wta(want[i]))
    b.close()
    for c in ctxs.values():
        c.close()


@pytest.mark.parametrize("name", ["hd8", "uhd15"])
def test_fp64_full_size_sampled_entries(name):
    """Full-size workloads in the benchmark's launch configuration: sampled (segment, label) entries
    against the oracle's FP64 entries, and how many whole-volume entries differ from the FP32 contract."""
    wl = make_workload(name)
    run = Run(wl, precision=FP64)
    costs = run.volumes()
    assert run.check() == 0
    rec = ftv.ftv_fp64_recomputed(run.ctx)
    run32 = Run(wl)
    costs32 = run32.volumes()
    differ = sum(int((a != b).sum()) for a, b in zip(costs, costs32))
    total = sum(c.numel() for c in costs)
    print(f"{name}: FP64-mode entries differing from the FP32 contract {differ} of {total}; "
          f"evaluations recomputed in FP64 {rec}")
    run32.close()
    rng = np.random.default_rng(17)
    for r in wl.ref_views[:: 3 if name == "uhd15" else 2]:
        idx = wl.ref_views.index(r)
        seg = rng.integers(0, run.S[idx], 24).astype(np.int32)
        lab = rng.integers(0, wl.n_labels, 24).astype(np.int32)
        got = costs[idx][torch.from_numpy(seg).long().cuda(), torch.from_numpy(lab).long().cuda()].cpu().numpy()
        lm, S = wl.labels(r)
        H = oracle.homography_table_f64(wl.cams, r, wl.neighbours(r), wl.n_labels, wl.z_near, wl.z_far)
        want = oracle.cost_entries(wl.cams, wl.views(), wl.sample_bytes, r, wl.neighbours(r), H, wl.n_labels, lm, S,
                                   wl.oob_penalty, seg, lab, combine=wl.combine)
        assert np.array_equal(got, want), (name, r)
    run.close()


def test_fp64_centre_table():
    for case in ("tiny", "near_tie"):
        if case == "tiny":
            wl = make_workload("tiny")
            cams, views, r, nb, L = wl.cams, wl.views(), wl.ref_views[0], wl.neighbours(wl.ref_views[0]), wl.n_labels
            labels = [wl.labels(v)[0] for v in range(wl.n_views)]
            S, zn, zf, pen = wl.labels(r)[1], wl.z_near, wl.z_far, wl.oob_penalty
        else:
            cams, views, lab, S, L, zn, zf = _near_tie()
            r, nb, pen = 0, [1], 765
            labels = [lab, synth.grid_labels(256, 48, 5, 1, seed=13)[0]]
        ctx = ftv.ftv_depth_init(cams, [r], L, zn, zf, nbr_lists=[nb], sample_bytes=1, bit_depth=8, oob_penalty=pen,
                                 max_segments=S, precision=FP64)
        m = torch.empty((S, L, len(nb)), dtype=torch.int32, device="cuda")
        sp = torch.empty_like(m)
        ftv.ftv_centre_table(ctx, [(dev(v.Y), dev(v.U), dev(v.V)) for v in views], [dev(l) for l in labels], [S], 3,
                             [m], [sp])
        assert ftv.ftv_check(ctx) == 0
        H = oracle.homography_table_f64(cams, r, nb, L, zn, zf)
        mo, spo = oracle.centre_table(cams, views, 1, r, nb, H, L, labels, S, 3, pen)
        assert np.array_equal(m.cpu().numpy(), mo), case
        assert np.array_equal(sp.cpu().numpy(), spo), case
        ctx.close()
