"""GPU parity of the batched / served form: camera streams with resident temporal state, many jobs
per launch, captured-graph replay.

Reference: the oracle run frame by frame as Sec. III-E describes (I frame: every segment estimated;
P frame: temporal test against the previous P and the I frame, cost only for changed segments,
winner-take-all for those, adoption for the others). Integer outputs: bit-exact.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from synth import configs
from synth.configs import make_workload

pytestmark = pytest.mark.gpu

ftv = pytest.importorskip("paper_1909_02294_gb300")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from gpu_runs import dev  # noqa: E402

T_P, T_I = 12, 4  # the paper's 8-bit thresholds (3, 1) scaled to 10-bit samples


def _streams():
    a = make_workload("temporal", reduced=True)  # 8 views 244x138, 40 labels, moving planes
    b = configs._temporal(configs.BASE_SEED + 41, W=320, H=180, f=250.0, L=24, refs=[0, 2, 4], n_frames=4,
                          name="temporal_b")
    return [a, b]


class Stream:
    def __init__(self, wl, mode=0):
        self.wl = wl
        self.S = [wl.labels(r)[1] for r in wl.ref_views]
        self.ctx = ftv.ftv_depth_init(wl.cams, wl.ref_views, wl.n_labels, wl.z_near, wl.z_far,
                                      sample_bytes=wl.sample_bytes, bit_depth=wl.bit_depth,
                                      oob_penalty=wl.oob_penalty, max_segments=max(self.S))
        labels = [dev(wl.labels(r)[0]) for r in wl.ref_views]
        ftv.ftv_stream_init(self.ctx, labels, self.S, T_P, T_I, mode)
        self.out = [torch.zeros(s, dtype=torch.int16, device="cuda") for s in self.S]
        self.depth = [torch.zeros((wl.cams[r].height, wl.cams[r].width), dtype=torch.float32, device="cuda")
                      for r in wl.ref_views]

    def job(self, frame, frame_type, depth=False):
        planes = [(dev(v.Y), dev(v.U), dev(v.V)) for v in self.wl.views(frame)]
        return {"ctx": self.ctx, "planes": planes, "frame_type": frame_type, "label_out": self.out,
                "depth_out": self.depth if depth else None}

    def labels(self):
        return [o.cpu().numpy().view(np.uint16).copy() for o in self.out]


class OracleStream:
    """The paper's I/P procedure on the CPU oracle."""

    def __init__(self, wl, mode=0):
        self.wl, self.mode = wl, mode
        self.prev_frame = self.i_frame = None
        self.prev = {}
        self.ilab = {}

    def step(self, frame, frame_type):
        wl = self.wl
        out = []
        for r in wl.ref_views:
            lab, S = wl.labels(r)
            H = oracle.homography_table(wl.cams, r, wl.neighbours(r), wl.n_labels, wl.z_near, wl.z_far)
            if frame_type == ftv.FTV_FRAME_I:
                mask = np.zeros(S, np.uint8)
                changed = np.arange(S, dtype=np.int32)
            else:
                mask, changed, _ = oracle.temporal_mask(lab, S, wl.view(r, frame), wl.view(r, self.prev_frame),
                                                        wl.view(r, self.i_frame), wl.sample_bytes, T_P, T_I, self.mode)
            vol = np.zeros((S, wl.n_labels), np.int32)
            if len(changed):
                vol = oracle.cost_volume(wl.cams, wl.views(frame), wl.sample_bytes, r, wl.neighbours(r), H,
                                         wl.n_labels, lab, S, wl.oob_penalty, seg_list=changed, out=vol)
            if frame_type == ftv.FTV_FRAME_I:
                labels = oracle.wta(vol)
                self.ilab[r] = labels.copy()
            else:
                labels = oracle.wta(vol, mask, self.prev[r], self.ilab[r])
            self.prev[r] = labels.copy()
            out.append(labels)
        self.prev_frame = frame
        if frame_type == ftv.FTV_FRAME_I:
            self.i_frame = frame
        return out


def _run(batch, jobs, replay=False):
    assert ftv.ftv_batch_prepare(batch, jobs) == 0
    (ftv.ftv_batch_replay if replay else ftv.ftv_batch_launch)(batch)
    assert ftv.ftv_batch_wait(batch) == 0


SCHEDULE = [(0, 0), (1, 1), (2, 1), (3, 1)]  # (frame, type): I then P frames


def test_batched_streams_match_oracle_frame_by_frame():
    wls = _streams()
    streams = [Stream(w) for w in wls]
    refs = [OracleStream(w) for w in wls]
    batch = ftv.ftv_batch_create(4, 32, 32)
    for frame, ftype in SCHEDULE:
        _run(batch, [s.job(frame, ftype, depth=(k == 0)) for k, s in enumerate(streams)])
        for s, o in zip(streams, refs):
            got = s.labels()
            want = o.step(frame, ftype)
            for r, (g, w) in enumerate(zip(got, want)):
                assert np.array_equal(g, w), (s.wl.name, frame, r, int((g != w).sum()))
        # per-pixel depth of the first stream's references
        s0 = streams[0]
        for r_i, r in enumerate(s0.wl.ref_views):
            lab, S = s0.wl.labels(r)
            want_d = oracle.depth_map(lab, S, refs[0].prev[r], s0.wl.n_labels, s0.wl.z_near, s0.wl.z_far)
            assert np.array_equal(s0.depth[r_i].cpu().numpy(), want_d)
    assert ftv.ftv_batch_launch_count(batch) == 10 * len(SCHEDULE)
    batch.close()
    for s in streams:
        s.ctx.close()


def test_results_identical_alone_in_the_mix_and_replayed():
    wls = _streams()
    # alone: one stream per batch, direct launches
    alone = []
    for w in wls:
        s = Stream(w)
        b = ftv.ftv_batch_create(1, 16, 16)
        res = []
        for frame, ftype in SCHEDULE:
            _run(b, [s.job(frame, ftype)])
            res.append(s.labels())
        alone.append(res)
        b.close()
        s.ctx.close()
    # in the mix, through the captured graph (the first replay captures, later ones replay)
    streams = [Stream(w) for w in wls]
    b = ftv.ftv_batch_create(4, 32, 32)
    mixed = [[], []]
    for frame, ftype in SCHEDULE:
        _run(b, [s.job(frame, ftype) for s in streams], replay=True)
        for k, s in enumerate(streams):
            mixed[k].append(s.labels())
    for k in range(2):
        for fa, fb in zip(alone[k], mixed[k]):
            for a, c in zip(fa, fb):
                assert np.array_equal(a, c)
    # a batch whose staging block is in use reports busy instead of racing
    assert ftv.ftv_batch_prepare(b, [streams[0].job(0, 0)]) in (0, ftv.FTV_ERR_BUSY)
    b.close()
    for s in streams:
        s.ctx.close()


def test_batch_argument_errors():
    w = _streams()[0]
    s = Stream(w)
    b = ftv.ftv_batch_create(1, 16, 16)
    # a P frame before any I frame
    assert ftv.ftv_batch_prepare(b, [s.job(1, ftv.FTV_FRAME_P)]) == ftv.FTV_ERR_STATE
    # the same stream twice in one batch
    b2 = ftv.ftv_batch_create(2, 32, 32)
    assert ftv.ftv_batch_prepare(b2, [s.job(0, 0), s.job(0, 0)]) == ftv.FTV_ERR_INVALID_ARG
    # over capacity
    b3 = ftv.ftv_batch_create(1, 2, 16)
    assert ftv.ftv_batch_prepare(b3, [s.job(0, 0)]) == ftv.FTV_ERR_BUSY
    assert ftv.ftv_stream_footprint(s.ctx, s.S) > 0
    for x in (b, b2, b3):
        x.close()
    s.ctx.close()


def test_chunked_cost_launches_give_identical_results():
    """The batch's cost work split over several persistent launches (a scheduling aid for serving) gives
    the same labels as one launch, launched directly or through the captured graph."""
    wls = _streams()
    results = {}
    for chunks, replay in ((1, False), (5, True), (16, False)):
        streams = [Stream(w) for w in wls]
        b = ftv.ftv_batch_create(4, 32, 32)
        ftv.ftv_batch_set_chunks(b, chunks)
        res = []
        for frame, ftype in SCHEDULE:
            _run(b, [s.job(frame, ftype) for s in streams], replay=replay)
            res.append([s.labels() for s in streams])
        assert ftv.ftv_batch_launch_count(b) == (9 + chunks) * len(SCHEDULE)
        results[chunks] = res
        for bad in (0, ftv.FTV_MAX_BATCH_CHUNKS + 1):
            with pytest.raises(ftv.FtvError):
                ftv.ftv_batch_set_chunks(b, bad)
        b.close()
        for s in streams:
            s.ctx.close()
    for chunks in (5, 16):
        for fa, fb in zip(results[1], results[chunks]):
            for sa, sb in zip(fa, fb):
                for a, c in zip(sa, sb):
                    assert np.array_equal(a, c), chunks


def _poll_until_done(batch, ticket, limit_s=60.0):
    import time
    t0 = time.time()
    while True:
        rc, st = ftv.ftv_batch_poll(batch, ticket)
        if rc == 0:
            return st
        assert rc == ftv.FTV_ERR_BUSY, rc
        assert time.time() - t0 < limit_s, "ticket did not complete"
        time.sleep(1e-3)


def test_ticketed_batch_reports_each_job_on_its_own():
    """ftv_batch_submit / flush / poll: three streams in one launch, one of whose label maps holds a label
    outside [0, S) (made on the host). Only that job's ticket reports FTV_ERR_INVALID_ARG, frame after frame;
    the other two equal the oracle's I/P procedure (Sec. III-E)."""
    wls = _streams()
    good = [Stream(w) for w in wls]
    bad_wl = make_workload("temporal", reduced=True)
    lab_bad = [bad_wl.labels(r)[0].copy() for r in bad_wl.ref_views]
    S_bad = [bad_wl.labels(r)[1] for r in bad_wl.ref_views]
    lab_bad[1][3, 5] = S_bad[1]  # one pixel of reference 1 labelled S
    bad_ctx = ftv.ftv_depth_init(bad_wl.cams, bad_wl.ref_views, bad_wl.n_labels, bad_wl.z_near, bad_wl.z_far,
                                 sample_bytes=bad_wl.sample_bytes, bit_depth=bad_wl.bit_depth,
                                 oob_penalty=bad_wl.oob_penalty, max_segments=max(S_bad))
    ftv.ftv_stream_init(bad_ctx, [dev(l) for l in lab_bad], S_bad, T_P, T_I, 0)
    bad_out = [torch.zeros(s, dtype=torch.int16, device="cuda") for s in S_bad]
    refs = [OracleStream(w) for w in wls]
    batch = ftv.ftv_batch_create(4, 64, 64)
    for frame, ftype in SCHEDULE:
        tickets, jobs = [], []  # the jobs' device buffers must stay valid until their tickets complete
        for s in good:
            jobs.append(s.job(frame, ftype))
            rc, t = ftv.ftv_batch_submit(batch, jobs[-1])
            assert rc == 0 and t > 0
            tickets.append(t)
        planes = [(dev(v.Y), dev(v.U), dev(v.V)) for v in bad_wl.views(frame)]
        rc, t_bad = ftv.ftv_batch_submit(batch, {"ctx": bad_ctx, "planes": planes, "frame_type": ftype,
                                                 "label_out": bad_out})
        assert rc == 0
        # a second frame of a queued stream waits for the next launch; a queued ticket is pending
        assert ftv.ftv_batch_submit(batch, good[0].job(frame, ftype))[0] == ftv.FTV_ERR_BUSY
        assert ftv.ftv_batch_poll(batch, t_bad)[0] == ftv.FTV_ERR_BUSY
        assert ftv.ftv_batch_flush(batch) == 0
        assert _poll_until_done(batch, t_bad) == ftv.FTV_ERR_INVALID_ARG
        for t in tickets:
            assert _poll_until_done(batch, t) == 0
        for s, o in zip(good, refs):
            for r, (g, w) in enumerate(zip(s.labels(), o.step(frame, ftype))):
                assert np.array_equal(g, w), (s.wl.name, frame, r)
        assert ftv.ftv_batch_wait(batch) == ftv.FTV_ERR_INVALID_ARG  # the OR over the launch's jobs
    # unknown tickets
    assert ftv.ftv_batch_poll(batch, 0)[0] == ftv.FTV_ERR_INVALID_ARG
    assert ftv.ftv_batch_poll(batch, 10 ** 9)[0] == ftv.FTV_ERR_INVALID_ARG
    assert ftv.ftv_batch_flush(batch) == 0  # nothing queued
    batch.close()
    bad_ctx.close()
    for s in good:
        s.ctx.close()


def test_ticketed_admission_by_footprint():
    """A batch with an HBM budget admits jobs while the footprints (ftv_job_footprint) of the queued and
    in-flight jobs fit: with room for one stream's footprint, a second job waits (FTV_ERR_BUSY) until the
    first has completed, and a budget below one job's footprint refuses it outright."""
    wls = _streams()
    streams = [Stream(w) for w in wls]
    fp = [ftv.ftv_job_footprint(w.cams, w.ref_views, w.n_labels, w.z_near, w.z_far, max(s.S),
                                sample_bytes=w.sample_bytes, bit_depth=w.bit_depth, max_segments=max(s.S))
          for w, s in zip(wls, streams)]
    batch = ftv.ftv_batch_create(4, 64, 64)
    ftv.ftv_batch_set_budget(batch, max(fp) + min(fp) // 2)
    j0, j1 = streams[0].job(0, 0), streams[1].job(0, 0)  # kept alive until their tickets complete
    rc, t0 = ftv.ftv_batch_submit(batch, j0)
    assert rc == 0
    assert ftv.ftv_batch_submit(batch, j1)[0] == ftv.FTV_ERR_BUSY  # queued + new > budget
    assert ftv.ftv_batch_flush(batch) == 0
    assert _poll_until_done(batch, t0) == 0
    rc, t1 = ftv.ftv_batch_submit(batch, j1)  # the first has completed: room again
    assert rc == 0
    assert ftv.ftv_batch_flush(batch) == 0
    assert _poll_until_done(batch, t1) == 0
    ftv.ftv_batch_set_budget(batch, min(fp) - 1)
    assert ftv.ftv_batch_submit(batch, streams[0].job(1, 1))[0] == ftv.FTV_ERR_OUT_OF_MEMORY
    batch.close()
    for s in streams:
        s.ctx.close()


def test_job_footprint_covers_the_device_allocations():
    """The device memory taken by creating a stream's context and resident state is what ftv_job_footprint
    states for them (its input-frame part excluded), up to the allocator's rounding of each allocation."""
    wl = make_workload("hd8")
    S = [wl.labels(r)[1] for r in wl.ref_views]
    fp = ftv.ftv_job_footprint(wl.cams, wl.ref_views, wl.n_labels, wl.z_near, wl.z_far, max(S),
                               sample_bytes=wl.sample_bytes, bit_depth=wl.bit_depth, max_segments=max(S))
    input_bytes = sum(3 * c.width * c.height * wl.sample_bytes for c in wl.cams)
    labels = [dev(wl.labels(r)[0]) for r in wl.ref_views]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    ctx = ftv.ftv_depth_init(wl.cams, wl.ref_views, wl.n_labels, wl.z_near, wl.z_far, sample_bytes=wl.sample_bytes,
                             bit_depth=wl.bit_depth, oob_penalty=wl.oob_penalty, max_segments=max(S))
    ftv.ftv_stream_init(ctx, labels, [max(S)] * len(S), T_P, T_I, 0)
    torch.cuda.synchronize()
    used = free0 - torch.cuda.mem_get_info()[0]
    n_allocs = 10 + 10 * len(S) + 3 + 11 * len(S)
    assert fp - input_bytes <= used + (2 << 20), (fp - input_bytes, used)
    assert used <= fp - input_bytes + n_allocs * (2 << 20), (fp - input_bytes, used)
    ctx.close()


def test_stream_state_checkpoint_and_resume():
    """A stream's resident state saved after an I and two P frames and loaded into a fresh stream of the same
    shape: the next P frame gives the oracle's labels on both the original and the restored stream. A
    checkpoint of another shape, or a short buffer, is refused."""
    wls = _streams()
    w = wls[0]
    a = Stream(w)
    o = OracleStream(w)
    batch = ftv.ftv_batch_create(2, 32, 32)
    for frame, ftype in SCHEDULE[:3]:
        _run(batch, [a.job(frame, ftype)])
        o.step(frame, ftype)
    buf = ftv.ftv_stream_state_save(a.ctx)
    torch.cuda.synchronize()
    b = Stream(w)
    ftv.ftv_stream_state_load(b.ctx, buf)
    frame, ftype = SCHEDULE[3]
    want = o.step(frame, ftype)
    for s in (a, b):
        _run(batch, [s.job(frame, ftype)])
        for r, (g, x) in enumerate(zip(s.labels(), want)):
            assert np.array_equal(g, x), r
    other = Stream(wls[1])
    with pytest.raises(ftv.FtvError):
        ftv.ftv_stream_state_load(other.ctx, buf)
    with pytest.raises(ftv.FtvError):
        ftv.ftv_stream_state_load(b.ctx, buf[: buf.numel() // 2])
    batch.close()
    for s in (a, b, other):
        s.ctx.close()
