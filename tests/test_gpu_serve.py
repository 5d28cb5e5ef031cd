"""The serving loop: continuous batching gives the oracle's labels on a mix of the serving workload's three
stream shapes, the same labels as plain per-job launches per stream and frame, and keeps in-stream order
under admission limits."""
from __future__ import annotations

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

ftv = pytest.importorskip("paper_1909_02294_gb300")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1909_02294_gb300 import serve  # noqa: E402

import oracle  # noqa: E402
import oracle_runs  # noqa: E402
from synth.configs import serving_streams_reduced  # noqa: E402


def _oracle_labels(wl, seqs, n_frames, gop):
    """The paper's I/P procedure (Sec. III-E) on the CPU oracle for one stream's frames, in order: luma-only
    temporal test against the previous and the I frame (T_P = 12, T_I = 4 for 10-bit samples), costs of the
    changed segments only, winner-take-all, adoption of the reused segments' labels."""
    out, prev_lab, i_lab = [], {}, {}
    prev_f = i_f = None
    for seq in seqs:
        f, is_i = seq % n_frames, seq % gop == 0
        labels_f = []
        for r in wl.ref_views:
            lab, S = wl.labels(r)
            if is_i:
                mask, changed = np.zeros(S, np.uint8), np.arange(S, dtype=np.int32)
            else:
                mask, changed, _ = oracle.temporal_mask(lab, S, wl.view(r, f), wl.view(r, prev_f), wl.view(r, i_f),
                                                        wl.sample_bytes, serve.T_P_10BIT, serve.T_I_10BIT,
                                                        ftv.FTV_TM_Y_ONLY)
            vol = oracle_runs.volume_all_cores(wl, r, frame=f, seg_list=changed)
            labels = oracle.wta(vol) if is_i else oracle.wta(vol, mask, prev_lab[r], i_lab[r])
            if is_i:
                i_lab[r] = labels.copy()
            prev_lab[r] = labels.copy()
            labels_f.append(labels)
        out.append(labels_f)
        prev_f = f
        if is_i:
            i_f = f
    return out


def test_served_mix_of_three_shapes_equals_the_oracle(monkeypatch):
    """Six streams, two of each serving shape (reduced sizes), 30 Poisson requests through the served path
    (ticketed submissions, captured-graph launches, three slots); the arc-rig shape is made to count as heavy,
    so its batches take the chunked low-priority path. Every stream's labels, frame by frame, equal the
    oracle's I/P procedure."""
    monkeypatch.setattr(serve, "HEAVY_EVALS", 5e7)
    wls = serving_streams_reduced(2)
    n_frames, gop = 3, 3
    streams = [serve.Stream(w, n_frames, gop, torch.device("cuda"), keep_labels=True) for w in wls]
    assert any(s.heavy for s in streams) and not all(s.heavy for s in streams)
    trace = serve.poisson_trace(len(streams), 30, 3000.0, 11)
    res = serve.run_served(streams, trace, slots=3, budget_bytes=1 << 30)
    assert res["jobs"] == 30
    for sid, (s, w) in enumerate(zip(streams, wls)):
        seqs = sorted(r.seq for r in trace if r.sid == sid)
        assert len(s.history) == len(seqs)
        want = _oracle_labels(w, seqs, n_frames, gop)
        for k, (got_f, want_f) in enumerate(zip(s.history, want)):
            for r, (g, x) in enumerate(zip(got_f, want_f)):
                assert np.array_equal(g, x), (w.name, seqs[k], r, int((g != x).sum()))
    for s in streams:
        s.close()


@pytest.mark.parametrize("budget_gb", [8.0, 0.15])
def test_served_equals_plain_per_stream(budget_gb):
    kw = dict(per_shape=2, gop=4, n_frames=3, keep_labels=True, shapes=["s540", "s1080"])
    a = serve.make_streams(**kw)
    trace = serve.poisson_trace(len(a), 24, 4000.0, 3)
    res_a = serve.run_served(a, trace, slots=3, budget_bytes=int(budget_gb * (1 << 30)))
    b = serve.make_streams(**kw)
    res_b = serve.run_plain(b, serve.poisson_trace(len(b), 24, 4000.0, 3))
    for sa, sb in zip(a, b):
        assert len(sa.history) == len(sb.history) > 0
        for fa, fb in zip(sa.history, sb.history):
            for x, y in zip(fa, fb):
                assert np.array_equal(x, y)
    assert res_a["jobs"] == res_b["jobs"] == 24
    assert res_a["batches"] <= 24
    for s in a + b:
        s.close()


def test_sequence_runner_reports_skipped_fraction():
    from synth.configs import make_workload
    res = serve.run_sequence(make_workload("temporal", reduced=True), 4, 4)
    assert res["frames"] == 4 and res["depth_maps"] == 32
    assert 0.0 < res["changed_fraction_p_frames"] < 1.0


def test_tuned_launch_shapes_serve_the_same_labels(tmp_path, monkeypatch):
    """Streams whose contexts take the autotuner's launch shape (one tuning per stream shape, cached in a
    JSON file) give the same labels as streams with the default shape."""
    monkeypatch.setenv("FTV_TUNE_CACHE", str(tmp_path / "shapes.json"))
    kw = dict(per_shape=2, gop=3, n_frames=2, keep_labels=True, shapes=["s540"])
    a = serve.make_streams(**kw, tune=True)
    chosen = serve.tune_streams(a)  # the second time from the cache
    assert all(v["source"] == "cache" for v in chosen.values()) and len(chosen) == 1
    b = serve.make_streams(**kw)
    for streams in (a, b):
        serve.run_plain(streams, serve.poisson_trace(len(streams), 8, 4000.0, 5))
    for sa, sb in zip(a, b):
        assert len(sa.history) == len(sb.history) > 0
        for fa, fb in zip(sa.history, sb.history):
            for x, y in zip(fa, fb):
                assert np.array_equal(x, y)
    for s in a + b:
        s.close()
