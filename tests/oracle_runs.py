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


def volume_all_cores(wl, r: int, frame: int = 0, seg_list=None, out=None, table_=None, threads: int = 0,
                     views=None) -> np.ndarray:
    """The same oracle volume, its segment rows split over every host core: threads run or_cost_volume on
    disjoint row lists into one output (the oracle keeps no global state and ctypes releases the GIL while
    it runs). Rows outside seg_list keep out's values, as in volume()."""
    import concurrent.futures as cf
    import os
    lab, S = wl.labels(r)
    H = table(wl, r) if table_ is None else table_
    if out is None:
        out = np.zeros((S, wl.n_labels), np.int32)
    rows = np.arange(S, dtype=np.int32) if seg_list is None else np.ascontiguousarray(seg_list, np.int32)
    if len(rows) == 0:
        return out
    vs = wl.views(frame) if views is None else views
    n = threads or max(1, os.cpu_count() or 1)
    parts = [p for p in np.array_split(rows, min(len(rows), 4 * n)) if len(p)]

    def run(part):
        oracle.cost_volume(wl.cams, vs, wl.sample_bytes, r, wl.neighbours(r), H, wl.n_labels, lab, S,
                           wl.oob_penalty, wl.combine, seg_list=part, out=out)

    with cf.ThreadPoolExecutor(n) as ex:
        list(ex.map(run, parts))
    return out
