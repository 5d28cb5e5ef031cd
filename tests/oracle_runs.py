"""Helpers that run the CPU oracle over a synthetic workload (tests and benchmark baseline only)."""
from __future__ import annotations

import numpy as np

import oracle


def table(wl, r: int, plane_mode: int = 0, centre: int = 0) -> np.ndarray:
    return oracle.homography_table(wl.cams, r, wl.neighbours(r), wl.n_labels, wl.z_near, wl.z_far,
                                   plane_mode=plane_mode, centre=centre)


def volume(wl, r: int, frame: int = 0, seg_list=None, plane_mode: int = 0, centre: int = 0,
           out=None) -> np.ndarray:
    lab, S = wl.labels(r)
    H = table(wl, r, plane_mode, centre)
    return oracle.cost_volume(wl.cams, wl.views(frame), wl.sample_bytes, r, wl.neighbours(r), H, wl.n_labels,
                              lab, S, wl.oob_penalty, wl.combine, seg_list=seg_list, out=out)


def entries(wl, r: int, seg, lab, frame: int = 0) -> np.ndarray:
    lm, S = wl.labels(r)
    H = table(wl, r)
    return oracle.cost_entries(wl.cams, wl.views(frame), wl.sample_bytes, r, wl.neighbours(r), H, wl.n_labels,
                               lm, S, wl.oob_penalty, seg, lab, combine=wl.combine)
