"""Host logic of the launch-shape tuner (paper_1909_02294_gb300/tune.py): job-class keys, the candidate
grid and the JSON cache, with the library's shape calls replaced by a fake (no GPU)."""
from __future__ import annotations

import json

import numpy as np
import pytest


@pytest.fixture(scope="module")
def tune():
    import __graft_entry__
    __graft_entry__._load_builder().build()
    from paper_1909_02294_gb300 import tune
    return tune


class _Cam:
    def __init__(self, w, h):
        self.width, self.height = w, h


class FakeLib:
    """Stands in for the ftv binding: a context with limits (64, 4) and a timing table."""

    def __init__(self, best=(32, 3)):
        self.shape = {"label_block": 63, "ctas_per_sm": 4, "max_label_block": 64, "max_ctas_per_sm": 4}
        self.best = best
        self.tuned = 0
        self.set_calls = []

    def ftv_get_launch_shape(self, ctx):
        return dict(self.shape)

    def ftv_set_launch_shape(self, ctx, lb, ct):
        assert 1 <= lb <= 64 and 0 <= ct <= 4
        self.set_calls.append((lb, ct))
        self.shape["label_block"], self.shape["ctas_per_sm"] = lb, ct

    def ftv_autotune(self, ctx, planes, labels, S, costs, lbs, cts, reps):
        self.tuned += 1
        ms = np.array([[1.0 + abs(a - self.best[0]) + abs(b - self.best[1]) for b in cts] for a in lbs], np.float32)
        i, j = np.unravel_index(np.argmin(ms), ms.shape)
        self.ftv_set_launch_shape(ctx, lbs[i], cts[j])
        return lbs[i], cts[j], ms


def test_job_class_keys_are_canonical_and_distinguish_classes(tune):
    cams = [_Cam(1920, 1080)] * 3
    k1 = tune.job_class(cams, [0, 1], [2, 2], 250, 2, 10, 0, 0, "GB300")
    k2 = tune.job_class(list(cams), (0, 1), (2, 2), 250, 2, 10, 0, 0, "GB300")
    assert k1 == k2 and json.loads(k1)["labels"] == 250
    for other in (tune.job_class(cams, [0, 1], [2, 2], 400, 2, 10, 0, 0, "GB300"),
                  tune.job_class(cams, [0, 1], [2, 2], 250, 2, 10, 0, 1, "GB300"),
                  tune.job_class(cams, [0, 1], [2, 2], 250, 2, 10, 0, 0, "B200"),
                  tune.job_class([_Cam(960, 540)] * 3, [0, 1], [2, 2], 250, 2, 10, 0, 0, "GB300")):
        assert other != k1


def test_candidate_grid_respects_the_limits(tune):
    assert tune.candidates({"max_label_block": 64, "max_ctas_per_sm": 4}) == ([64, 32, 16, 8], [4, 3, 2])
    assert tune.candidates({"max_label_block": 36, "max_ctas_per_sm": 2}) == ([36, 32, 18, 16, 8], [2, 1])
    assert tune.candidates({"max_label_block": 1, "max_ctas_per_sm": 1}) == ([1], [1])


def test_tune_once_then_apply_from_cache(tune, tmp_path, monkeypatch):
    fake = FakeLib(best=(16, 3))
    monkeypatch.setattr(tune, "ftv", fake)
    path = str(tmp_path / "sub" / "shapes.json")
    rec = tune.apply_or_tune(None, "classA", None, None, None, None, cache_path=path)
    assert rec["source"] == "tuned" and (rec["label_block"], rec["ctas_per_sm"]) == (16, 3) and fake.tuned == 1
    assert json.load(open(path))["classA"]["label_block"] == 16
    fake.shape.update(label_block=63, ctas_per_sm=4)
    rec = tune.apply_or_tune(None, "classA", None, None, None, None, cache_path=path)
    assert rec["source"] == "cache" and fake.tuned == 1 and fake.set_calls[-1] == (16, 3)
    # another class tunes and is added beside the first
    tune.apply_or_tune(None, "classB", None, None, None, None, cache_path=path)
    assert set(json.load(open(path))) == {"classA", "classB"} and fake.tuned == 2


def test_cached_shapes_outside_the_limits_are_tuned_again(tune, tmp_path, monkeypatch):
    fake = FakeLib(best=(32, 4))
    monkeypatch.setattr(tune, "ftv", fake)
    path = str(tmp_path / "shapes.json")
    tune.save(path, {"k": {"label_block": 200, "ctas_per_sm": 4}})
    rec = tune.apply_or_tune(None, "k", None, None, None, None, cache_path=path)
    assert rec["source"] == "tuned" and rec["label_block"] == 32
    assert tune.apply_or_tune(None, "new", None, None, None, None, cache_path=path, tune=False) is None
    rec = tune.apply_or_tune(None, "k2", None, None, None, None, cache_path=path, write=False)
    assert rec["source"] == "tuned" and "k2" not in json.load(open(path))


def test_unreadable_cache_counts_as_empty(tune, tmp_path):
    p = tmp_path / "bad.json"
    p.write_text("{not json")
    assert tune.load(str(p)) == {}
    assert tune.load(str(tmp_path / "missing.json")) == {}
