"""Whole-volume GPU parity at the benchmark workloads' full sizes, with the CPU oracle run on every host core
as the checker (tests/oracle_runs.py: volume_all_cores).

  - every reference of the 1920x1080 8-view workload (20736 segments x 250 labels each) and two of the
    3840x2160 15-view workload (49432 x 400): every entry of the cost volume (Eq. 4 summed over the segment,
    min over the neighbouring views) and the winner-take-all labels, in the default launch shape (the one
    the autotuner keeps for both on GB300); a whole 1080p reference in the FP64 projection mode;
  - the whole 30-frame 1920x1080 8-view temporal sequence through the stream/batch path: per frame and
    reference the temporal mask, the ordered list of re-estimated segments and the labels, against the
    oracle's I/P procedure of Sec. III-E (I frames at frames 0 and 15, P frames between).
Integer outputs: bit-exact.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import oracle_runs
from synth.configs import make_workload

pytestmark = pytest.mark.gpu

ftv = pytest.importorskip("paper_1909_02294_gb300")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from gpu_runs import Run, dev, from_device_pointer  # noqa: E402

T_P, T_I = 12, 4  # the paper's 8-bit T_P = 3, T_I = 1 scaled to 10-bit samples


@pytest.mark.parametrize("name,refs", [("hd8", [0, 1, 2, 3, 4, 5, 6, 7]), ("uhd15", [0, 7])])
def test_whole_reference_volume_at_full_size(name, refs):
    """Every reference of the 1080p workload and an end and the middle reference of the 4K arc (the most
    and the fewest culled tiles), each whole volume computed in one launch with all references."""
    wl = make_workload(name)
    run = Run(wl)
    costs = run.volumes()
    assert run.check() == 0
    for ref in refs:
        idx = wl.ref_views.index(ref)
        S = run.S[idx]
        got = costs[idx].cpu().numpy()
        want = oracle_runs.volume_all_cores(wl, ref)
        assert got.shape == want.shape == (S, wl.n_labels)
        bad = np.argwhere(got != want)
        assert len(bad) == 0, (name, ref, len(bad), bad[:5].tolist())
        win = torch.empty(S, dtype=torch.int16, device="cuda")
        ftv.ftv_wta_depth(run.ctx, idx, costs[idx], S, win)
        assert run.check() == 0
        assert np.array_equal(win.cpu().numpy().view(np.uint16), oracle.wta(want))
    run.close()


def test_whole_reference_volume_at_full_size_fp64_projection():
    """FP64 projection mode on a whole 1080p reference (integer-shift entries, the local frame and its tie
    test), against the oracle's FP64 mode."""
    wl = make_workload("hd8")
    run = Run(wl, precision=ftv.FTV_PRECISION_FP64)
    costs = run.volumes()
    assert run.check() == 0
    for ref in (4,):
        idx = wl.ref_views.index(ref)
        H64 = oracle.homography_table_f64(wl.cams, ref, wl.neighbours(ref), wl.n_labels, wl.z_near, wl.z_far)
        want = oracle_runs.volume_all_cores(wl, ref, table_=H64)
        got = costs[idx].cpu().numpy()
        assert np.array_equal(got, want), (ref, int((got != want).sum()))
    run.close()


def test_temporal_sequence_at_full_size_through_the_stream_path():
    wl = make_workload("temporal")
    n_frames, i_frames = wl.n_frames, {0, 15}
    S = [wl.labels(r)[1] for r in wl.ref_views]
    ctx = ftv.ftv_depth_init(wl.cams, wl.ref_views, wl.n_labels, wl.z_near, wl.z_far, sample_bytes=wl.sample_bytes,
                             bit_depth=wl.bit_depth, oob_penalty=wl.oob_penalty, max_segments=max(S))
    ftv.ftv_stream_init(ctx, [dev(wl.labels(r)[0]) for r in wl.ref_views], S, T_P, T_I, ftv.FTV_TM_Y_ONLY)
    out = [torch.zeros(s, dtype=torch.int16, device="cuda") for s in S]
    batch = ftv.ftv_batch_create(1, len(wl.ref_views), wl.n_views)
    tables = {r: oracle_runs.table(wl, r) for r in wl.ref_views}
    prev_lab, i_lab = {}, {}
    prev_f = i_f = None
    changed_total = 0
    for f in range(n_frames):
        ftype = ftv.FTV_FRAME_I if f in i_frames else ftv.FTV_FRAME_P
        views = wl.views(f)
        planes = [(dev(v.Y), dev(v.U), dev(v.V)) for v in views]
        assert ftv.ftv_batch_prepare(batch, [{"ctx": ctx, "planes": planes, "frame_type": ftype,
                                              "label_out": out}]) == 0
        ftv.ftv_batch_replay(batch)
        assert ftv.ftv_batch_wait(batch) == 0
        for i, r in enumerate(wl.ref_views):
            lab, s_r = wl.labels(r)
            if ftype == ftv.FTV_FRAME_I:
                mask = np.zeros(s_r, np.uint8)
                changed = np.arange(s_r, dtype=np.int32)
            else:
                mask, changed, _ = oracle.temporal_mask(lab, s_r, views[r], wl.view(r, prev_f), wl.view(r, i_f),
                                                        wl.sample_bytes, T_P, T_I, ftv.FTV_TM_Y_ONLY)
            vol = oracle_runs.volume_all_cores(wl, r, frame=f, seg_list=changed, table_=tables[r], views=views)
            if ftype == ftv.FTV_FRAME_I:
                labels = oracle.wta(vol)
                i_lab[r] = labels.copy()
            else:
                labels = oracle.wta(vol, mask, prev_lab[r], i_lab[r])
            prev_lab[r] = labels.copy()
            m_ptr, n_ptr = ftv.ftv_stream_mask(ctx, i)
            n_got = int(from_device_pointer(n_ptr, 1, "<i4")[0])
            assert n_got == len(changed), (f, r)
            assert np.array_equal(from_device_pointer(m_ptr, s_r, "|u1"), mask), (f, r)
            assert np.array_equal(from_device_pointer(ftv.ftv_stream_changed(ctx, i), n_got, "<i4"), changed), (f, r)
            got = out[i].cpu().numpy().view(np.uint16)
            assert np.array_equal(got, labels), (f, r, int((got != labels).sum()))
            if ftype == ftv.FTV_FRAME_P:
                changed_total += len(changed)
        prev_f = f
        if ftype == ftv.FTV_FRAME_I:
            i_f = f
        if f > 0 and f - 1 != i_f:
            wl.drop_frame(f - 1)
    # the workload re-estimates a minority of segments per P frame (about 15 % by construction)
    p_frames = n_frames - len(i_frames)
    assert 0.03 < changed_total / (p_frames * sum(S)) < 0.4
    batch.close()
    ctx.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_temporal_mask_at_full_size(mode):
    """ftv_temporal_mask on two 1920x1080 references of the temporal workload (20736 segments: the mask is
    decided and the list compacted over many blocks), frame 1 against frame 0 as the previous P and as the
    I frame, and without an I frame: mask, ordered list and count equal the oracle's (Sec. III-E)."""
    wl = make_workload("temporal")
    run = Run(wl)
    for i in (0, 5):
        r = wl.ref_views[i]
        lab, S = wl.labels(r)
        labels = dev(lab)
        cur = [dev(a) for a in (wl.view(r, 1).Y, wl.view(r, 1).U, wl.view(r, 1).V)]
        prev = [dev(a) for a in (wl.view(r, 0).Y, wl.view(r, 0).U, wl.view(r, 0).V)]
        for with_i in (True, False):
            mask = torch.empty(S, dtype=torch.uint8, device="cuda")
            changed = torch.empty(S, dtype=torch.int32, device="cuda")
            n = torch.empty(1, dtype=torch.int32, device="cuda")
            ftv.ftv_temporal_mask(run.ctx, i, cur, prev, prev if with_i else None, labels, S, T_P, T_I, mode, mask,
                                  changed, n)
            assert run.check() == 0
            m_ref, ch_ref, n_ref = oracle.temporal_mask(lab, S, wl.view(r, 1), wl.view(r, 0),
                                                        wl.view(r, 0) if with_i else None, wl.sample_bytes, T_P, T_I,
                                                        mode)
            assert S > 4096 and 0 < n_ref < S
            assert int(n.item()) == n_ref
            assert np.array_equal(mask.cpu().numpy(), m_ref)
            assert np.array_equal(changed.cpu().numpy()[:n_ref], ch_ref)
    run.close()
