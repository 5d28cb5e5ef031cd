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


def test_static_scratch_without_status_word_and_with_a_bad_label():
    """Without a caller status word (d_status NULL) the results are unchanged; with one pixel labelled S the
    call reports the bad label in the caller's word and leaves that pixel out, as the context version does."""
    wl = make_workload("temporal", reduced=True)
    run = Run(wl)
    r_index, r = 2, wl.ref_views[2]
    lab, S = wl.labels(r)
    frames = [run.planes(f)[r] for f in range(2)]
    cam = wl.cams[r]
    bad = lab.copy()
    bad[4, 9] = S
    for lab_k, expect_bad in ((lab, False), (bad, True)):
        labels = torch.from_numpy(lab_k).cuda()
        m_a, c_a, n_a = _outputs(S)
        ftv.ftv_temporal_mask(run.ctx, r_index, frames[1], frames[0], None, labels, S, 12, 4, ftv.FTV_TM_ALL_YUV,
                              m_a, c_a, n_a)
        assert run.check() == (ftv.FTV_ERR_INVALID_ARG if expect_bad else 0)
        for with_status in (False, True):
            status = torch.zeros(1, dtype=torch.int32, device="cuda") if with_status else None
            m_b, c_b, n_b = _outputs(S)
            ftv.ftv_temporal_mask_static(cam.width, cam.height, wl.sample_bytes, frames[1], frames[0], None, labels, S,
                                         12, 4, ftv.FTV_TM_ALL_YUV, m_b, c_b, n_b, status=status)
            torch.cuda.synchronize()
            n = int(n_a.item())
            assert int(n_b.item()) == n
            assert torch.equal(m_a, m_b) and torch.equal(c_a[:n], c_b[:n])
            if with_status:
                assert (int(status.item()) & 1) == (1 if expect_bad else 0)  # the bad-label bit
    run.close()


def test_static_scratch_refuses_host_memory_before_launching():
    """A label map in host memory (not memory of the current device) is refused with FTV_ERR_INVALID_ARG by
    the argument check, before anything is launched."""
    import ctypes
    wl = make_workload("temporal", reduced=True)
    r = wl.ref_views[0]
    lab, S = wl.labels(r)
    planes = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (wl.view(r).Y, wl.view(r).U, wl.view(r).V)]
    host_labels = torch.from_numpy(lab).pin_memory()
    m, c, n = _outputs(S)
    cp = (ctypes.c_void_p * 3)(*[t.data_ptr() for t in planes])
    pitch = (ctypes.c_int64 * 3)(*[t.stride(0) * t.element_size() for t in planes])
    rc = ftv.ftv.lib.ftv_temporal_mask_static(wl.cams[r].width, wl.cams[r].height, 2, cp, pitch, cp, pitch, None,
                                              None, host_labels.data_ptr(), S, 12, 4, 0, m.data_ptr(), c.data_ptr(),
                                              n.data_ptr(), None, torch.cuda.current_stream().cuda_stream)
    assert rc == ftv.FTV_ERR_INVALID_ARG


def test_static_entry_odd_width_and_unaligned_planes_equal_the_oracle():
    """A view 243 pixels wide (odd: the kernel loads its two columns one sample at a time and clamps the second
    one at the right edge) whose planes start one sample past a 4-byte boundary, in both channel modes, with
    and without the I frame: mask, ordered list and count equal the oracle's (Sec. III-E)."""
    import types
    import oracle
    wl = make_workload("temporal", reduced=True)
    r = wl.ref_views[3]
    lab, S = wl.labels(r)
    H, W = lab.shape[0], lab.shape[1] - 1
    labels = torch.from_numpy(np.ascontiguousarray(lab[:, 1:])).cuda()
    host = []
    dev_planes = []
    for fr in range(3):
        v = wl.view(r, fr)
        host.append(types.SimpleNamespace(Y=v.Y[:, 1:], U=v.U[:, 1:], V=v.V[:, 1:]))
        # full-width device planes, sliced one column in: the base is 2 bytes past a 4-byte boundary
        dev_planes.append(tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda()[:, 1:] for a in (v.Y, v.U, v.V)))
    assert dev_planes[0][0].data_ptr() % 4 == 2
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for cur, prev, ifr, mode in [(1, 0, 0, ftv.FTV_TM_ALL_YUV), (2, 1, None, ftv.FTV_TM_Y_ONLY),
                                 (2, 0, 1, ftv.FTV_TM_Y_ONLY)]:
        m, c, n = _outputs(S)
        ftv.ftv_temporal_mask_static(W, H, 2, dev_planes[cur], dev_planes[prev],
                                     dev_planes[ifr] if ifr is not None else None, labels, S, 12, 4, mode, m, c, n,
                                     status=status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        m_ref, ch_ref, n_ref = oracle.temporal_mask(np.ascontiguousarray(lab[:, 1:]), S, host[cur], host[prev],
                                                    host[ifr] if ifr is not None else None, 2, 12, 4, mode)
        assert np.array_equal(m.cpu().numpy(), m_ref)
        assert int(n.item()) == n_ref
        assert np.array_equal(c.cpu().numpy()[:n_ref], ch_ref)
