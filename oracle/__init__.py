"""Python access to the plain CPU oracle (ftv_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the benchmark's CPU
baseline leg, never by the library. It shares no code with the CUDA path. Each wrapper takes numpy
arrays and follows the function of the same name in ftv_oracle.c, which cites the paper passage it
implements.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ftv_oracle.c")
_LIB = os.path.join(_HERE, "libftv_oracle.so")
_lib = None

COMBINE = {"min": 0, "sum": 1}


def build(force: bool = False) -> str:
    """Compile the oracle with strict IEEE single/double arithmetic (no contraction, no fast math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-frounding-math", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Cam(ctypes.Structure):
    _fields_ = [("K", ctypes.c_double * 9), ("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class Img(ctypes.Structure):
    _fields_ = [("Y", ctypes.c_void_p), ("U", ctypes.c_void_p), ("V", ctypes.c_void_p),
                ("pitch", ctypes.c_int64)]


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        for name in ["or_label_inv_depths", "or_homography_f64", "or_homography_table", "or_homography_table_f64",
                     "or_cost_volume",
                     "or_cost_entries", "or_fp64_mismatch", "or_temporal_mask", "or_wta", "or_depth_map",
                     "or_centre_table", "or_adjacency", "or_snic", "or_connectivity", "or_superpixels"]:
            getattr(_lib, name).restype = ctypes.c_int
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def cams_array(cams):
    arr = (Cam * len(cams))()
    for i, c in enumerate(cams):
        arr[i].K[:] = [float(v) for v in np.asarray(c.K, np.float64).ravel()]
        arr[i].R[:] = [float(v) for v in np.asarray(c.R, np.float64).ravel()]
        arr[i].t[:] = [float(v) for v in np.asarray(c.t, np.float64).ravel()]
        arr[i].width, arr[i].height = int(c.width), int(c.height)
    return arr


def _imgs(views):
    keep = []
    arr = (Img * len(views))()
    for i, v in enumerate(views):
        Y, U, V = (np.ascontiguousarray(a) for a in (v.Y, v.U, v.V))
        keep += [Y, U, V]
        arr[i].Y, arr[i].U, arr[i].V = Y.ctypes.data, U.ctypes.data, V.ctypes.data
        arr[i].pitch = Y.shape[1]
    return arr, keep


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def label_inv_depths(L: int, z_near: float, z_far: float) -> np.ndarray:
    out = np.empty(L, np.float64)
    _check(_load().or_label_inv_depths(ctypes.c_int(L), ctypes.c_double(z_near), ctypes.c_double(z_far),
                                       _p(out)), "label_inv_depths")
    return out


def homography_f64(cam_r, cam_v, iz: float, cam_c=None) -> np.ndarray:
    a = cams_array([cam_r, cam_v] + ([cam_c] if cam_c is not None else []))
    H = np.empty(9, np.float64)
    cc = ctypes.byref(a[2]) if cam_c is not None else None
    _check(_load().or_homography_f64(ctypes.byref(a[0]), ctypes.byref(a[1]), cc, ctypes.c_double(iz), _p(H)),
           "homography_f64")
    return H.reshape(3, 3)


def homography_table(cams, ref: int, nbrs, L: int, z_near: float, z_far: float, plane_mode: int = 0,
                     centre: int = 0) -> np.ndarray:
    nb = np.ascontiguousarray(nbrs, np.int32)
    out = np.empty((len(nb), L, 9), np.float32)
    _check(_load().or_homography_table(cams_array(cams), ctypes.c_int(len(cams)), ctypes.c_int(ref),
                                       ctypes.c_int(len(nb)), _p(nb), ctypes.c_int(L), ctypes.c_double(z_near),
                                       ctypes.c_double(z_far), ctypes.c_int(plane_mode), ctypes.c_int(centre),
                                       _p(out)), "homography_table")
    return out


def homography_table_f64(cams, ref: int, nbrs, L: int, z_near: float, z_far: float, plane_mode: int = 0,
                         centre: int = 0) -> np.ndarray:
    """The same table kept in FP64 (before the rounding to FP32): the FP64 projection's homographies."""
    nb = np.ascontiguousarray(nbrs, np.int32)
    out = np.empty((len(nb), L, 9), np.float64)
    _check(_load().or_homography_table_f64(cams_array(cams), ctypes.c_int(len(cams)), ctypes.c_int(ref),
                                           ctypes.c_int(len(nb)), _p(nb), ctypes.c_int(L), ctypes.c_double(z_near),
                                           ctypes.c_double(z_far), ctypes.c_int(plane_mode), ctypes.c_int(centre),
                                           _p(out)), "homography_table_f64")
    return out


def _tables(H):
    """(FP32 table, FP64 table) arguments for a table H: a float32 table selects the FP32 contract, a
    float64 table (homography_table_f64) the FP64 projection. Any other type is refused, not cast."""
    H = np.asarray(H)
    if H.dtype == np.float32:
        return np.ascontiguousarray(H), None
    if H.dtype == np.float64:
        return None, np.ascontiguousarray(H)
    raise TypeError(f"homography table must be float32 or float64, not {H.dtype}")


def cost_volume(cams, views, sample_bytes: int, ref: int, nbrs, H: np.ndarray, L: int, labels: np.ndarray,
                S: int, penalty: int, combine: str = "min", seg_list=None, out: np.ndarray | None = None):
    """int32 [S][L] cost volume of reference `ref`; rows of unlisted segments keep `out`'s values. H is
    the FP32 table (FP32 contract) or the FP64 table (FP64 projection)."""
    nb = np.ascontiguousarray(nbrs, np.int32)
    imgs, keep = _imgs(views)
    lab = np.ascontiguousarray(labels, np.int32)
    Hc, H64 = _tables(H)
    if out is None:
        out = np.zeros((S, L), np.int32)
    sl = np.ascontiguousarray(seg_list, np.int32) if seg_list is not None else None
    _check(_load().or_cost_volume(cams_array(cams), ctypes.c_int(len(cams)), imgs, ctypes.c_int(sample_bytes),
                                  ctypes.c_int(ref), ctypes.c_int(len(nb)), _p(nb), _p(Hc), _p(H64),
                                  ctypes.c_int(L), _p(lab), ctypes.c_int(S), ctypes.c_int(penalty), ctypes.c_int(COMBINE[combine]),
                                  _p(sl), ctypes.c_int(len(sl) if sl is not None else 0), _p(out)), "cost_volume")
    return out


def cost_entries(cams, views, sample_bytes: int, ref: int, nbrs, H: np.ndarray, L: int, labels: np.ndarray,
                 S: int, penalty: int, seg, lab, combine: str = "min") -> np.ndarray:
    nb = np.ascontiguousarray(nbrs, np.int32)
    imgs, keep = _imgs(views)
    lm = np.ascontiguousarray(labels, np.int32)
    Hc, H64 = _tables(H)
    sg = np.ascontiguousarray(seg, np.int32)
    lb = np.ascontiguousarray(lab, np.int32)
    out = np.empty(len(sg), np.int32)
    _check(_load().or_cost_entries(cams_array(cams), ctypes.c_int(len(cams)), imgs, ctypes.c_int(sample_bytes),
                                   ctypes.c_int(ref), ctypes.c_int(len(nb)), _p(nb), _p(Hc), _p(H64),
                                   ctypes.c_int(L), _p(lm), ctypes.c_int(S), ctypes.c_int(penalty),
                                   ctypes.c_int(COMBINE[combine]),
                                   ctypes.c_int(len(sg)), _p(sg), _p(lb), _p(out)), "cost_entries")
    return out


def fp64_mismatch(cams, ref: int, nbrs, L: int, z_near: float, z_far: float, pix=None, plane_mode: int = 0,
                  centre: int = 0) -> tuple[int, int]:
    nb = np.ascontiguousarray(nbrs, np.int32)
    px = np.ascontiguousarray(pix, np.int32) if pix is not None else None
    out = np.zeros(2, np.int64)
    _check(_load().or_fp64_mismatch(cams_array(cams), ctypes.c_int(len(cams)), ctypes.c_int(ref),
                                    ctypes.c_int(len(nb)), _p(nb), ctypes.c_int(L), ctypes.c_double(z_near),
                                    ctypes.c_double(z_far), ctypes.c_int(plane_mode), ctypes.c_int(centre),
                                    ctypes.c_int(len(px) if px is not None else 0), _p(px), _p(out)),
           "fp64_mismatch")
    return int(out[0]), int(out[1])


def temporal_mask(labels: np.ndarray, S: int, cur, prev, iframe, sample_bytes: int, t_p: int, t_i: int,
                  mode: int):
    """Returns (mask uint8 [S], changed list int32, n_changed)."""
    lab = np.ascontiguousarray(labels, np.int32)
    H, W = lab.shape
    im, keep = _imgs([cur, prev] + ([iframe] if iframe is not None else []))
    mask = np.empty(S, np.uint8)
    ch = np.empty(max(S, 1), np.int32)
    n = ctypes.c_int32(0)
    _check(_load().or_temporal_mask(ctypes.c_int(W), ctypes.c_int(H), _p(lab), ctypes.c_int(S),
                                    ctypes.byref(im[0]), ctypes.byref(im[1]),
                                    ctypes.byref(im[2]) if iframe is not None else None,
                                    ctypes.c_int(sample_bytes), ctypes.c_int(t_p), ctypes.c_int(t_i),
                                    ctypes.c_int(mode), _p(mask), _p(ch), ctypes.byref(n)), "temporal_mask")
    return mask, ch[: n.value].copy(), n.value


def wta(cost: np.ndarray, mask=None, prev_label=None, iframe_label=None, seg_list=None,
        out: np.ndarray | None = None) -> np.ndarray:
    c = np.ascontiguousarray(cost, np.int32)
    S, L = c.shape
    if out is None:
        out = np.zeros(S, np.uint16)
    m = np.ascontiguousarray(mask, np.uint8) if mask is not None else None
    pl = np.ascontiguousarray(prev_label, np.uint16) if prev_label is not None else None
    il = np.ascontiguousarray(iframe_label, np.uint16) if iframe_label is not None else None
    sl = np.ascontiguousarray(seg_list, np.int32) if seg_list is not None else None
    _check(_load().or_wta(_p(c), ctypes.c_int(S), ctypes.c_int(L), _p(m), _p(pl), _p(il), _p(sl),
                          ctypes.c_int(len(sl) if sl is not None else 0), _p(out)), "wta")
    return out


def depth_map(labels: np.ndarray, S: int, seg_label: np.ndarray, L: int, z_near: float, z_far: float):
    lab = np.ascontiguousarray(labels, np.int32)
    H, W = lab.shape
    sl = np.ascontiguousarray(seg_label, np.uint16)
    out = np.empty((H, W), np.float32)
    _check(_load().or_depth_map(ctypes.c_int(W), ctypes.c_int(H), _p(lab), ctypes.c_int(S), _p(sl),
                                ctypes.c_int(L), ctypes.c_double(z_near), ctypes.c_double(z_far), _p(out)),
           "depth_map")
    return out


def centre_table(cams, views, sample_bytes: int, ref: int, nbrs, H: np.ndarray, L: int, labels_views, S: int,
                 window: int, penalty: int):
    """(m int32 [S][L][N], s' int32 [S][L][N]) of or_centre_table; labels_views[v] is view v's int32
    [H][W] label map or None (labels_views[ref] is required). H: FP32 or FP64 table, as in cost_volume."""
    nb = np.ascontiguousarray(nbrs, np.int32)
    imgs, keep = _imgs(views)
    Hc, H64 = _tables(H)
    labs = [np.ascontiguousarray(l, np.int32) if l is not None else None for l in labels_views]
    lp = (ctypes.c_void_p * len(labs))(*[l.ctypes.data if l is not None else None for l in labs])
    m = np.empty((S, L, len(nb)), np.int32)
    sp = np.empty((S, L, len(nb)), np.int32)
    _check(_load().or_centre_table(cams_array(cams), ctypes.c_int(len(cams)), imgs, ctypes.c_int(sample_bytes),
                                   ctypes.c_int(ref), ctypes.c_int(len(nb)), _p(nb), _p(Hc), _p(H64),
                                   ctypes.c_int(L), lp,
                                   ctypes.c_int(S), ctypes.c_int(window), ctypes.c_int(penalty), _p(m), _p(sp)),
           "centre_table")
    return m, sp


def adjacency(labels: np.ndarray, S: int, frame, sample_bytes: int, connectivity: int = 4, beta0: float = 1.0,
              min_diff: float = 1.0, cap: int | None = None):
    """(edge_s int32, edge_t int32, beta float32) of or_adjacency, edges in increasing (s, t) order."""
    lab = np.ascontiguousarray(labels, np.int32)
    H, W = lab.shape
    im, keep = _imgs([frame])
    cap = cap if cap is not None else 4 * H * W + 1
    es = np.empty(cap, np.int32)
    et = np.empty(cap, np.int32)
    bt = np.empty(cap, np.float32)
    n = ctypes.c_int32(0)
    _check(_load().or_adjacency(ctypes.c_int(W), ctypes.c_int(H), _p(lab), ctypes.c_int(S), ctypes.byref(im[0]),
                                ctypes.c_int(sample_bytes), ctypes.c_int(connectivity), ctypes.c_double(beta0),
                                ctypes.c_double(min_diff), ctypes.c_int(cap), _p(es), _p(et), _p(bt),
                                ctypes.byref(n)), "adjacency")
    k = min(n.value, cap)
    return es[:k].copy(), et[:k].copy(), bt[:k].copy()


def grid_segments(W: int, H: int, S: int) -> int:
    """Number of grid cells (= labels) of the S x S seed grid: ceil(W / S) * ceil(H / S)."""
    return -(-W // S) * -(-H // S)


def snic(frame, sample_bytes: int, bit_depth: int, S: int, m: int) -> np.ndarray:
    """int32 [H][W] labels of or_snic (sequential SNIC, the paper's segmentation)."""
    H, W = np.asarray(frame.Y).shape
    im, keep = _imgs([frame])
    out = np.empty((H, W), np.int32)
    _check(_load().or_snic(ctypes.c_int(W), ctypes.c_int(H), ctypes.byref(im[0]), ctypes.c_int(sample_bytes),
                           ctypes.c_int(bit_depth), ctypes.c_int(S), ctypes.c_int(m), _p(out)), "snic")
    return out


def connectivity(labels: np.ndarray, K: int, frame, sample_bytes: int) -> np.ndarray:
    """or_connectivity applied to a copy of labels (int32 [H][W], values in [0, K)), colours from frame."""
    lab = np.array(labels, np.int32, order="C", copy=True)
    H, W = lab.shape
    im, keep = _imgs([frame])
    _check(_load().or_connectivity(ctypes.c_int(W), ctypes.c_int(H), _p(lab), ctypes.c_int(K), ctypes.byref(im[0]),
                                   ctypes.c_int(sample_bytes)), "connectivity")
    return lab


def superpixels(frame, sample_bytes: int, bit_depth: int, S: int, m: int, iterations: int,
                connect: bool = True) -> np.ndarray:
    """int32 [H][W] labels of or_superpixels (the data-parallel reformulation the GPU computes)."""
    H, W = np.asarray(frame.Y).shape
    im, keep = _imgs([frame])
    out = np.empty((H, W), np.int32)
    _check(_load().or_superpixels(ctypes.c_int(W), ctypes.c_int(H), ctypes.byref(im[0]),
                                  ctypes.c_int(sample_bytes), ctypes.c_int(bit_depth), ctypes.c_int(S),
                                  ctypes.c_int(m), ctypes.c_int(iterations), ctypes.c_int(1 if connect else 0),
                                  _p(out)), "superpixels")
    return out
