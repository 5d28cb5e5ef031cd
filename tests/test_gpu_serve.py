"""The serving loop: continuous batching gives the same labels as plain per-job launches, per stream
and frame, and keeps in-stream order under admission limits."""
from __future__ import annotations

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

ftv = pytest.importorskip("paper_1909_02294_gb300")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1909_02294_gb300 import serve  # noqa: E402


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
