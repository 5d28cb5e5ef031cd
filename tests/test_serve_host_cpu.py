"""Host logic of the serving loop (paper_1909_02294_gb300/serve.py), no GPU: the request trace and the
throughput / latency statistics."""
from __future__ import annotations

import numpy as np
import pytest


@pytest.fixture(scope="module")
def serve():
    import __graft_entry__
    __graft_entry__._load_builder().build()
    from paper_1909_02294_gb300 import serve
    return serve


def test_poisson_trace_keeps_stream_order_and_rate(serve):
    reqs = serve.poisson_trace(5, 4000, 200.0, seed=3)
    t = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(t) >= 0)
    seqs = {}
    for r in reqs:
        assert r.seq == seqs.get(r.sid, 0)  # each stream's requests in order, numbered from 0
        seqs[r.sid] = r.seq + 1
    assert set(seqs) == set(range(5)) and sum(seqs.values()) == 4000
    assert abs(len(reqs) / t[-1] - 200.0) < 20.0  # mean rate within 10 %
    assert all(r.arrival == 0.0 for r in serve.poisson_trace(3, 50, 0.0, seed=1))  # capacity runs


class _Cam:
    def __init__(self, w, h):
        self.width, self.height = w, h


class _WL:
    def __init__(self, w, h):
        self.cams = [_Cam(w, h)]


class _Stream:
    def __init__(self, w, h, refs):
        self.wl, self.n_refs = _WL(w, h), refs


def test_stats_count_depth_maps_and_percentiles(serve):
    streams = [_Stream(960, 540, 3), _Stream(1920, 1080, 8)]
    reqs = []
    for i in range(100):
        r = serve.Request(i, i % 2, i // 2, arrival=0.01 * i)
        r.done = r.arrival + (0.002 if r.sid == 0 else 0.020)
        reqs.append(r)
    st = serve._stats(streams, reqs)
    assert st["jobs"] == 100 and st["depth_maps"] == 50 * 3 + 50 * 8
    span = reqs[-1].done - reqs[0].arrival
    assert st["wall_s"] == pytest.approx(span)
    assert st["depth_maps_per_s"] == pytest.approx(550 / span)
    assert st["p50_ms"] == pytest.approx(11.0) and st["p99_ms"] == pytest.approx(20.0)
    assert st["p99_ms_by_shape"] == {"1920x1080": pytest.approx(20.0), "960x540": pytest.approx(2.0)}
