"""GPU parity of the centre table (Eq. 4 at segment centres with the Eq. 5 correspondence s')."""
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


@pytest.mark.parametrize("name,window,drop", [("tiny", 3, None), ("tiny", 5, 0), ("hd8", 3, 2), ("uhd15", 3, 1),
                                              ("hd8@12", 3, None)])
def test_centre_table_bit_exact(name, window, drop):
    """8-bit (tiny), 10-bit (hd8, uhd15) and, declared as 12-bit, the wide 16-bit-field texels."""
    wl = make_workload(name.split("@")[0], reduced=(name != "tiny"))
    if name.endswith("@12"):
        wl.bit_depth = 12
        wl.ref_views = [0, 5]
    run = Run(wl)
    labels_h = [wl.labels(v)[0] for v in range(wl.n_views)]
    if drop is not None and drop not in wl.ref_views:
        labels_h[drop] = None  # a neighbour without a segmentation: s' = -1 there
    labels_d = [dev(l) if l is not None else None for l in labels_h]
    L = wl.n_labels
    ms, sps = [], []
    for i, r in enumerate(wl.ref_views):
        n = len(wl.neighbours(r))
        ms.append(torch.empty((run.S[i], L, n), dtype=torch.int32, device="cuda"))
        sps.append(torch.empty((run.S[i], L, n), dtype=torch.int32, device="cuda"))
    ftv.ftv_centre_table(run.ctx, run.planes(), labels_d, run.S, window, ms, sps)
    assert run.check() == 0
    for i, r in enumerate(wl.ref_views):
        H = oracle.homography_table(wl.cams, r, wl.neighbours(r), L, wl.z_near, wl.z_far)
        m, sp = oracle.centre_table(wl.cams, wl.views(), wl.sample_bytes, r, wl.neighbours(r), H, L, labels_h,
                                    run.S[i], window, wl.oob_penalty)
        assert np.array_equal(ms[i].cpu().numpy(), m), (name, r)
        assert np.array_equal(sps[i].cpu().numpy(), sp), (name, r)
    run.close()


@pytest.mark.parametrize("window", [1, 3, 15])
def test_centre_table_single_neighbour_empty_segments_and_window_limits(window):
    """One neighbour (the kernel's label/neighbour split has a special case there), the smallest, the paper's
    and the largest window, a one-pixel segment in the corner (its window leaves the image) and an empty
    segment."""
    wl = make_workload("tiny")
    r = wl.ref_views[0]
    lab, S0 = wl.labels(r)
    lab = lab.copy()
    lab[0, 0] = S0
    S = S0 + 2
    run = Run(wl, nbr_lists=[[0]], max_segments=S)
    labels_h = [wl.labels(v)[0] for v in range(wl.n_views)]
    labels_h[r] = lab
    L = wl.n_labels
    m = torch.empty((S, L, 1), dtype=torch.int32, device="cuda")
    sp = torch.empty((S, L, 1), dtype=torch.int32, device="cuda")
    ftv.ftv_centre_table(run.ctx, run.planes(), [dev(l) for l in labels_h], [S], window, [m], [sp])
    assert run.check() == 0
    H = oracle.homography_table(wl.cams, r, [0], L, wl.z_near, wl.z_far)
    mo, spo = oracle.centre_table(wl.cams, wl.views(), wl.sample_bytes, r, [0], H, L, labels_h, S, window,
                                  wl.oob_penalty)
    assert np.array_equal(m.cpu().numpy(), mo)
    assert np.array_equal(sp.cpu().numpy(), spo)
    assert np.all(mo[S0 + 1] == window * window * wl.oob_penalty)
    run.close()
