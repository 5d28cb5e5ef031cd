"""GPU parity of segment adjacency and adaptive smoothing weights (Eq. 2-3)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from synth.configs import make_workload

pytestmark = pytest.mark.gpu

ftv = pytest.importorskip("paper_1909_02294_gb300")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from gpu_runs import Run, dev  # noqa: E402


@pytest.mark.parametrize("name,conn,cap", [("tiny", 4, None), ("tiny", 8, 100), ("hd8", 4, None), ("hd8", 8, None)])
def test_adjacency_bit_exact(name, conn, cap):
    wl = make_workload(name, reduced=(name != "tiny"))
    run = Run(wl)
    i = 0
    r = wl.ref_views[i]
    lab, S = wl.labels(r)
    v = wl.view(r)
    es_r, et_r, b_r = oracle.adjacency(lab, S, v, wl.sample_bytes, conn, beta0=37.5, min_diff=1.5)
    capacity = cap if cap is not None else len(es_r) + 10
    es = torch.full((capacity,), -1, dtype=torch.int32, device="cuda")
    et = torch.full((capacity,), -1, dtype=torch.int32, device="cuda")
    b = torch.zeros(capacity, dtype=torch.float32, device="cuda")
    n = torch.zeros(1, dtype=torch.int32, device="cuda")
    frame = [dev(a) for a in (v.Y, v.U, v.V)]
    ftv.ftv_adjacency(run.ctx, i, frame, dev(lab), S, conn, 37.5, 1.5, es, et, b, n)
    assert run.check() == 0
    assert int(n.item()) == len(es_r)
    k = min(capacity, len(es_r))
    assert np.array_equal(es.cpu().numpy()[:k], es_r[:k])
    assert np.array_equal(et.cpu().numpy()[:k], et_r[:k])
    assert np.array_equal(b.cpu().numpy()[:k].view(np.uint32), b_r[:k].view(np.uint32))
    if cap is not None:
        assert np.all(es.cpu().numpy()[k:] == -1)
    run.close()
