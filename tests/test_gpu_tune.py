"""Launch shapes and the autotuner on the GPU: every (label block, CTAs per SM) shape gives the oracle's
volume bit for bit; the autotuner keeps its fastest candidate; the JSON cache round-trips."""
from __future__ import annotations

import json

import numpy as np
import pytest
import torch

import oracle
from synth.configs import make_workload

pytestmark = pytest.mark.gpu

ftv = pytest.importorskip("paper_1909_02294_gb300")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from gpu_runs import Run  # noqa: E402
from paper_1909_02294_gb300 import tune  # noqa: E402


def _oracle(wl):
    out = []
    for r in wl.ref_views:
        lab, S = wl.labels(r)
        H = oracle.homography_table(wl.cams, r, wl.neighbours(r), wl.n_labels, wl.z_near, wl.z_far)
        out.append(oracle.cost_volume(wl.cams, wl.views(), wl.sample_bytes, r, wl.neighbours(r), H, wl.n_labels, lab,
                                      S, wl.oob_penalty, wl.combine))
    return out


@pytest.mark.parametrize("name,reduced", [("tiny", False), ("hd8", True), ("uhd15", True)])
def test_every_launch_shape_gives_the_oracle_volume(name, reduced):
    wl = make_workload(name, reduced=reduced)
    run = Run(wl)
    want = _oracle(wl)
    shape = ftv.ftv_get_launch_shape(run.ctx)
    m, occ = shape["max_label_block"], shape["max_ctas_per_sm"]
    assert shape["label_block"] <= m and shape["ctas_per_sm"] == occ >= 1
    for lb in sorted({1, 7, max(1, m // 2), m}):
        for ct in sorted({1, occ}):
            ftv.ftv_set_launch_shape(run.ctx, lb, ct)
            got = ftv.ftv_get_launch_shape(run.ctx)
            assert got["label_block"] <= lb and got["ctas_per_sm"] == ct
            costs = run.volumes()
            assert run.check() == 0
            for c, w in zip(costs, want):
                assert np.array_equal(c.cpu().numpy(), w), (name, lb, ct)
    for bad in ((0, 0), (m + 1, 0), (1, occ + 1), (1, -1)):
        with pytest.raises(ftv.FtvError):
            ftv.ftv_set_launch_shape(run.ctx, *bad)
    run.close()


def test_autotune_keeps_its_fastest_candidate_and_caches_it(tmp_path):
    wl = make_workload("hd8", reduced=True)
    run = Run(wl)
    L = wl.n_labels
    costs = [torch.empty((S, L), dtype=torch.int32, device="cuda") for S in run.S]
    occ = ftv.ftv_get_launch_shape(run.ctx)["max_ctas_per_sm"]
    lbs, cts = [32, 16, 8], sorted({occ, 1}, reverse=True)
    lb, ct, ms = ftv.ftv_autotune(run.ctx, run.planes(), run.labels, run.S, costs, lbs, cts, reps=2)
    assert ms.shape == (3, len(cts)) and np.all(ms > 0)
    i, j = np.unravel_index(int(np.argmin(ms)), ms.shape)
    assert (lb, ct) == (lbs[i], cts[j])
    shape = ftv.ftv_get_launch_shape(run.ctx)
    assert shape["label_block"] <= lb and shape["ctas_per_sm"] == ct
    for c, w in zip(costs, _oracle(wl)):
        assert np.array_equal(c.cpu().numpy(), w)
    # the JSON cache: tuned once, applied from the cache the second time
    key = tune.job_class(wl.cams, wl.ref_views, [len(wl.neighbours(r)) for r in wl.ref_views], L, wl.sample_bytes,
                         wl.bit_depth, 0, 0, torch.cuda.get_device_name())
    path = str(tmp_path / "shapes.json")
    rec = tune.apply_or_tune(run.ctx, key, run.planes(), None, run.S, costs, cache_path=path, reps=1)
    assert rec["source"] == "tuned" and key in json.load(open(path))
    ftv.ftv_set_launch_shape(run.ctx, 1, 1)
    rec2 = tune.apply_or_tune(run.ctx, key, run.planes(), None, run.S, costs, cache_path=path)
    assert rec2["source"] == "cache" and rec2["label_block"] == rec["label_block"]
    assert ftv.ftv_get_launch_shape(run.ctx)["ctas_per_sm"] == rec["ctas_per_sm"]
    run.close()
