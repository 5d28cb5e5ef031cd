"""The allocation-free temporal test (ftv_temporal_mask_static) against the context-based one.

ftv_temporal_mask_static serves callers that cannot call cudaMalloc (a fixed device-memory budget
reserved up front, or a loop that must not take cudaMalloc's implicit device synchronisation); it keeps
its accumulators in a statically sized array inside the library. This file is collected last so that a
run stopping at its first failure has already run every other test; it also passes on its own.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

ftv = pytest.importorskip("paper_1909_02294_gb300")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from synth.configs import make_workload  # noqa: E402
from gpu_runs import Run  # noqa: E402


def _outputs(S):
    return (torch.empty(S, dtype=torch.uint8, device="cuda"), torch.empty(S, dtype=torch.int32, device="cuda"),
            torch.empty(1, dtype=torch.int32, device="cuda"))


def test_static_scratch_temporal_mask_matches_context_version_twice():
    wl = make_workload("temporal", reduced=True)
    run = Run(wl)
    r_index, r = 3, wl.ref_views[3]
    lab, S = wl.labels(r)
    labels = torch.from_numpy(lab).cuda()
    frames = [run.planes(f)[r] for f in range(3)]
    cam = wl.cams[r]
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    # two calls in a row with different inputs: the second must not see the first one's accumulators
    for cur, prev, ifr, mode in [(1, 0, 0, ftv.FTV_TM_ALL_YUV), (2, 1, 0, ftv.FTV_TM_Y_ONLY)]:
        m_a, c_a, n_a = _outputs(S)
        ftv.ftv_temporal_mask(run.ctx, r_index, frames[cur], frames[prev], frames[ifr], labels, S, 12, 4, mode,
                              m_a, c_a, n_a)
        m_b, c_b, n_b = _outputs(S)
        ftv.ftv_temporal_mask_static(cam.width, cam.height, wl.sample_bytes, frames[cur], frames[prev], frames[ifr],
                                     labels, S, 12, 4, mode, m_b, c_b, n_b, status=status)
        torch.cuda.synchronize()
        assert run.check() == 0
        n = int(n_a.item())
        assert int(n_b.item()) == n
        assert torch.equal(m_a, m_b)
        assert torch.equal(c_a[:n], c_b[:n])
        assert 0 < n < S  # a mix of changed and reused segments
    assert int(status.item()) == 0
    run.close()


def test_static_scratch_rejects_too_many_segments():
    wl = make_workload("temporal", reduced=True)
    r = wl.ref_views[0]
    lab, S = wl.labels(r)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (wl.view(r).Y, wl.view(r).U, wl.view(r).V)]
    big = ftv.FTV_STATIC_MAX_SEGMENTS + 1
    m, c, n = _outputs(big)
    with pytest.raises(ftv.FtvError) as e:
        ftv.ftv_temporal_mask_static(wl.cams[r].width, wl.cams[r].height, 2, dev, dev, None,
                                     torch.from_numpy(lab).cuda(), big, 12, 4, 0, m, c, n)
    assert e.value.code == ftv.FTV_ERR_INVALID_ARG
