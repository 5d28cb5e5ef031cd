"""Thin Python binding of the C ABI in include/ftv.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does nothing but convert
arguments: torch CUDA tensors become device pointers, the current torch stream becomes the
ftv_stream, and non-zero status codes become FtvError. All computation happens in libftv.so's CUDA
kernels; if the shared library is missing this module raises at import, there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("FTV_LIBRARY") or os.path.join(_HERE, "libftv.so")

FTV_OK = 0
FTV_ERR_INVALID_ARG, FTV_ERR_OUT_OF_MEMORY, FTV_ERR_CUDA, FTV_ERR_OVERFLOW = 1, 2, 3, 4
FTV_ERR_TIMEOUT, FTV_ERR_BUSY, FTV_ERR_STATE, FTV_ERR_CHECKED = 5, 6, 7, 8
STATUS = {0: "ok", 1: "invalid argument", 2: "out of device memory", 3: "CUDA error",
          4: "segment cost may overflow int32", 5: "device wait timed out", 6: "busy", 7: "call out of order"}
FTV_PLANES_REF, FTV_PLANES_CENTRE = 0, 1
FTV_COMBINE_MIN, FTV_COMBINE_SUM = 0, 1
FTV_TM_Y_ONLY, FTV_TM_ALL_YUV = 0, 1
FTV_MASK_CHANGED, FTV_MASK_REUSE_P, FTV_MASK_REUSE_I = 0, 1, 2
FTV_PRECISION_FP32, FTV_PRECISION_FP64 = 0, 1
FTV_MAX_VIEWS, FTV_MAX_NBRS, FTV_MAX_LABELS, FTV_MAX_DIM = 64, 32, 4096, 32767  # include/ftv.h


class FtvError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS.get(code, code)} ({code})")
        self.code = code


class ftv_camera(ctypes.Structure):
    _fields_ = [("K", ctypes.c_double * 9), ("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class ftv_config(ctypes.Structure):
    _fields_ = [("n_views", ctypes.c_int32), ("cams", ctypes.POINTER(ftv_camera)),
                ("n_refs", ctypes.c_int32), ("ref_views", ctypes.POINTER(ctypes.c_int32)),
                ("nbr_offsets", ctypes.POINTER(ctypes.c_int32)), ("nbr_views", ctypes.POINTER(ctypes.c_int32)),
                ("n_labels", ctypes.c_int32), ("z_near", ctypes.c_double), ("z_far", ctypes.c_double),
                ("plane_mode", ctypes.c_int32), ("centre_view", ctypes.c_int32),
                ("sample_bytes", ctypes.c_int32), ("bit_depth", ctypes.c_int32),
                ("oob_penalty", ctypes.c_int32), ("combine", ctypes.c_int32),
                ("max_segments", ctypes.c_int32), ("precision", ctypes.c_int32)]


class ftv_segmenter_config(ctypes.Structure):
    _fields_ = [("n_images", ctypes.c_int32), ("widths", ctypes.POINTER(ctypes.c_int32)),
                ("heights", ctypes.POINTER(ctypes.c_int32)), ("sample_bytes", ctypes.c_int32),
                ("bit_depth", ctypes.c_int32), ("grid_step", ctypes.c_int32), ("compactness", ctypes.c_int32),
                ("iterations", ctypes.c_int32)]


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run __graft_entry__.build() (nvcc, sm_103a)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {
        "ftv_depth_init": [ctypes.POINTER(ftv_config), ctypes.POINTER(vp)],
        "ftv_depth_destroy": [vp],
        "ftv_get_homographies": [vp, i32, vp],
        "ftv_get_homographies_f64": [vp, i32, vp],
        "ftv_compute_homographies": [ctypes.POINTER(ftv_config), i32, vp],
        "ftv_compute_homographies_f64": [ctypes.POINTER(ftv_config), i32, vp],
        "ftv_get_neighbours": [vp, i32, vp, vp],
        "ftv_get_label_depths": [vp, vp],
        "ftv_segment_index": [vp, i32, vp, i32, vp],
        "ftv_cost_volume": [vp, vp, vp, vp, vp, vp, vp, vp, vp],
        "ftv_temporal_mask": [vp, i32, vp, vp, vp, vp, vp, vp, vp, i32, i32, i32, i32, vp, vp, vp, vp],
        "ftv_temporal_mask_views": [vp, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, i32, i32, i32, vp, vp, vp, vp],
        "ftv_wta_depth": [vp, i32, vp, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp],
        "ftv_check": [vp, vp],
        "ftv_culled_evaluations": [vp, vp, vp],
        "ftv_fp64_recomputed": [vp, vp, vp],
        "ftv_set_launch_shape": [vp, i32, i32],
        "ftv_get_launch_shape": [vp, vp, vp, vp, vp],
        "ftv_autotune": [vp, vp, vp, vp, vp, vp, vp, i32, vp, i32, i32, vp, vp, vp, vp],
        "ftv_set_profiling": [vp, i32],
        "ftv_stream_init": [vp, vp, vp, i32, i32, i32, vp],
        "ftv_stream_footprint": [vp, vp, vp],
        "ftv_stream_labels": [vp, i32, vp],
        "ftv_stream_mask": [vp, i32, vp, vp],
        "ftv_stream_changed": [vp, i32, vp],
        "ftv_stream_state_bytes": [vp, vp],
        "ftv_stream_state_save": [vp, vp, i64, vp],
        "ftv_stream_state_load": [vp, vp, i64, vp],
        "ftv_reciprocal_check": [vp, vp],
        "ftv_centre_table": [vp, vp, vp, vp, vp, i32, vp, vp, vp],
        "ftv_adjacency": [vp, i32, vp, vp, vp, i32, i32, ctypes.c_double, ctypes.c_double, i32, vp, vp, vp, vp,
                          vp],
        "ftv_batch_create": [i32, i32, i32, vp],
        "ftv_batch_destroy": [vp],
        "ftv_batch_prepare": [vp, vp, i32],
        "ftv_batch_launch": [vp, vp],
        "ftv_batch_replay": [vp, vp],
        "ftv_batch_set_chunks": [vp, i32],
        "ftv_batch_query": [vp],
        "ftv_batch_wait": [vp],
        "ftv_job_footprint": [ctypes.POINTER(ftv_config), i32, vp],
        "ftv_batch_set_budget": [vp, i64],
        "ftv_batch_submit": [vp, vp, vp],
        "ftv_batch_flush": [vp, vp],
        "ftv_batch_poll": [vp, ctypes.c_uint64, vp],
        "ftv_temporal_mask_static": [i32, i32, i32, vp, vp, vp, vp, vp, vp, vp, i32, i32, i32, i32, vp, vp, vp, vp,
                                     vp],
        "ftv_last_kernel_ms": [vp, vp],
        "ftv_segmenter_init": [ctypes.POINTER(ftv_segmenter_config), vp],
        "ftv_segmenter_segments": [vp, vp],
        "ftv_superpixels": [vp, vp, vp, vp, vp],
        "ftv_segmenter_check": [vp, vp],
        "ftv_segmenter_destroy": [vp],
        "ftv_segmenter_set_profiling": [vp, i32],
        "ftv_segmenter_kernel_ms": [vp, vp, vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.ftv_batch_launch_count.argtypes = [vp]
    lib.ftv_batch_launch_count.restype = i64
    lib.ftv_launch_count.argtypes = [vp]
    lib.ftv_launch_count.restype = i64
    lib.ftv_segmenter_launch_count.argtypes = [vp]
    lib.ftv_segmenter_launch_count.restype = i64
    lib.ftv_status_str.argtypes = [ctypes.c_int]
    lib.ftv_status_str.restype = ctypes.c_char_p
    return lib


lib = _load()

EXPORTED = ["ftv_depth_init", "ftv_depth_destroy", "ftv_compute_homographies", "ftv_get_homographies",
            "ftv_get_homographies_f64", "ftv_compute_homographies_f64", "ftv_fp64_recomputed", "ftv_set_launch_shape", "ftv_get_launch_shape",
            "ftv_autotune", "ftv_get_neighbours",
            "ftv_get_label_depths", "ftv_segment_index", "ftv_cost_volume", "ftv_temporal_mask", "ftv_temporal_mask_views",
            "ftv_wta_depth", "ftv_check", "ftv_culled_evaluations", "ftv_launch_count", "ftv_status_str", "ftv_set_profiling",
            "ftv_last_kernel_ms", "ftv_temporal_mask_static", "ftv_stream_init", "ftv_stream_footprint",
            "ftv_stream_labels", "ftv_stream_mask", "ftv_stream_changed", "ftv_stream_state_bytes", "ftv_stream_state_save",
            "ftv_stream_state_load", "ftv_reciprocal_check", "ftv_centre_table", "ftv_adjacency", "ftv_batch_create", "ftv_batch_destroy", "ftv_batch_prepare", "ftv_batch_launch",
            "ftv_batch_replay", "ftv_batch_query", "ftv_batch_wait", "ftv_batch_launch_count", "ftv_batch_set_chunks",
            "ftv_job_footprint", "ftv_batch_set_budget", "ftv_batch_submit", "ftv_batch_flush", "ftv_batch_poll",
            "ftv_segmenter_init", "ftv_segmenter_segments", "ftv_superpixels", "ftv_segmenter_check",
            "ftv_segmenter_launch_count", "ftv_segmenter_destroy", "ftv_segmenter_set_profiling",
            "ftv_segmenter_kernel_ms"]


def _ok(code: int, where: str) -> None:
    if code != FTV_OK:
        raise FtvError(code, where)


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _arr(ctype, values):
    values = list(values)
    return (ctype * max(1, len(values)))(*values)


def camera_struct(cam) -> ftv_camera:
    c = ftv_camera()
    c.K[:] = [float(v) for v in np.asarray(cam.K, np.float64).ravel()]
    c.R[:] = [float(v) for v in np.asarray(cam.R, np.float64).ravel()]
    c.t[:] = [float(v) for v in np.asarray(cam.t, np.float64).ravel()]
    c.width, c.height = int(cam.width), int(cam.height)
    return c


@dataclass
class Context:
    """Owns an ftv_ctx handle (ftv_depth_destroy on close)."""
    handle: int
    n_refs: int
    n_labels: int
    ref_views: list

    def close(self) -> None:
        if self.handle:
            ftv_depth_destroy(self)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _config(cams, ref_views, n_labels, z_near, z_far, nbr_lists, plane_mode, centre_view, sample_bytes,
            bit_depth, oob_penalty, combine, max_segments, precision=FTV_PRECISION_FP32):
    cam_arr = (ftv_camera * len(cams))(*[camera_struct(c) for c in cams])
    refs = _arr(ctypes.c_int32, ref_views)
    cfg = ftv_config()
    cfg.n_views, cfg.cams = len(cams), ctypes.cast(cam_arr, ctypes.POINTER(ftv_camera))
    cfg.n_refs, cfg.ref_views = len(ref_views), ctypes.cast(refs, ctypes.POINTER(ctypes.c_int32))
    keep = [cam_arr, refs]
    if nbr_lists is not None:
        offs = [0]
        flat = []
        for lst in nbr_lists:
            flat += list(lst)
            offs.append(len(flat))
        o, f = _arr(ctypes.c_int32, offs), _arr(ctypes.c_int32, flat)
        keep += [o, f]
        cfg.nbr_offsets = ctypes.cast(o, ctypes.POINTER(ctypes.c_int32))
        cfg.nbr_views = ctypes.cast(f, ctypes.POINTER(ctypes.c_int32))
    cfg.n_labels, cfg.z_near, cfg.z_far = n_labels, z_near, z_far
    cfg.plane_mode, cfg.centre_view = plane_mode, centre_view
    cfg.sample_bytes, cfg.bit_depth, cfg.oob_penalty = sample_bytes, bit_depth, oob_penalty
    cfg.combine, cfg.max_segments, cfg.precision = combine, max_segments, precision
    return cfg, keep


def ftv_depth_init(cams, ref_views, n_labels: int, z_near: float, z_far: float, *, nbr_lists=None,
                   plane_mode: int = FTV_PLANES_REF, centre_view: int = 0, sample_bytes: int = 1,
                   bit_depth: int = 8, oob_penalty: int = -1, combine: int = FTV_COMBINE_MIN,
                   max_segments: int = 1, precision: int = FTV_PRECISION_FP32) -> Context:
    cfg, keep = _config(cams, ref_views, n_labels, z_near, z_far, nbr_lists, plane_mode, centre_view, sample_bytes,
                        bit_depth, oob_penalty, combine, max_segments, precision)
    h = ctypes.c_void_p()
    _ok(lib.ftv_depth_init(ctypes.byref(cfg), ctypes.byref(h)), "ftv_depth_init")
    return Context(h.value, len(ref_views), n_labels, list(ref_views))


def ftv_compute_homographies(cams, ref_views, ref_index: int, n_labels: int, z_near: float, z_far: float, *,
                             nbr_lists=None, plane_mode: int = FTV_PLANES_REF, centre_view: int = 0) -> np.ndarray:
    """Host-only FP32 homography table [n_nbrs][n_labels][9] of reference ref_index."""
    cfg, keep = _config(cams, ref_views, n_labels, z_near, z_far, nbr_lists, plane_mode, centre_view, 1, 8, -1,
                        FTV_COMBINE_MIN, 1)
    ref = ref_views[ref_index]
    n = len(nbr_lists[ref_index]) if nbr_lists is not None else len(cams) - 1
    out = np.empty((n, n_labels, 9), np.float32)
    _ok(lib.ftv_compute_homographies(ctypes.byref(cfg), ref_index, out.ctypes.data), "ftv_compute_homographies")
    return out


def ftv_compute_homographies_f64(cams, ref_views, ref_index: int, n_labels: int, z_near: float, z_far: float, *,
                                 nbr_lists=None, plane_mode: int = FTV_PLANES_REF, centre_view: int = 0) -> np.ndarray:
    """Host-only FP64 homography table [n_nbrs][n_labels][9] of reference ref_index (before the FP32 rounding)."""
    cfg, keep = _config(cams, ref_views, n_labels, z_near, z_far, nbr_lists, plane_mode, centre_view, 1, 8, -1,
                        FTV_COMBINE_MIN, 1)
    n = len(nbr_lists[ref_index]) if nbr_lists is not None else len(cams) - 1
    out = np.empty((n, n_labels, 9), np.float64)
    _ok(lib.ftv_compute_homographies_f64(ctypes.byref(cfg), ref_index, out.ctypes.data),
        "ftv_compute_homographies_f64")
    return out


def ftv_depth_destroy(ctx: Context) -> None:
    _ok(lib.ftv_depth_destroy(ctx.handle), "ftv_depth_destroy")


def ftv_get_homographies(ctx: Context, ref_index: int) -> np.ndarray:
    n = ctypes.c_int32()
    _ok(lib.ftv_get_neighbours(ctx.handle, ref_index, ctypes.byref(n), None), "ftv_get_neighbours")
    out = np.empty((n.value, ctx.n_labels, 9), np.float32)
    _ok(lib.ftv_get_homographies(ctx.handle, ref_index, out.ctypes.data), "ftv_get_homographies")
    return out


def ftv_get_homographies_f64(ctx: Context, ref_index: int) -> np.ndarray:
    """The FP64 table before its rounding (the FP64 projection's homographies)."""
    n = ctypes.c_int32()
    _ok(lib.ftv_get_neighbours(ctx.handle, ref_index, ctypes.byref(n), None), "ftv_get_neighbours")
    out = np.empty((n.value, ctx.n_labels, 9), np.float64)
    _ok(lib.ftv_get_homographies_f64(ctx.handle, ref_index, out.ctypes.data), "ftv_get_homographies_f64")
    return out


def ftv_get_neighbours(ctx: Context, ref_index: int) -> list[int]:
    n = ctypes.c_int32()
    _ok(lib.ftv_get_neighbours(ctx.handle, ref_index, ctypes.byref(n), None), "ftv_get_neighbours")
    out = np.empty(max(1, n.value), np.int32)
    _ok(lib.ftv_get_neighbours(ctx.handle, ref_index, ctypes.byref(n), out.ctypes.data), "ftv_get_neighbours")
    return [int(v) for v in out[: n.value]]


def ftv_get_label_depths(ctx: Context) -> np.ndarray:
    out = np.empty(ctx.n_labels, np.float32)
    _ok(lib.ftv_get_label_depths(ctx.handle, out.ctypes.data), "ftv_get_label_depths")
    return out


def ftv_segment_index(ctx: Context, ref_index: int, labels, n_segments: int, stream=None) -> None:
    _ok(lib.ftv_segment_index(ctx.handle, ref_index, _ptr(labels), n_segments, _stream(stream)),
        "ftv_segment_index")


def ftv_cost_volume(ctx: Context, planes, labels, n_segments, costs, seg_lists=None, n_listed=None,
                    stream=None) -> None:
    """planes: per view a (Y, Cb, Cr) triple of 2-D CUDA tensors (uint8 or uint16, any row pitch);
    labels: per reference an int32 [H][W] tensor or None (reuse the cached index);
    costs: per reference an int32 [S][L] tensor; seg_lists/n_listed: optional per-reference device
    list and one-element int32 length tensor."""
    ptrs, pitches = [], []
    for trip in planes:
        for t in trip:
            ptrs.append(_ptr(t))
            pitches.append(int(t.stride(0)) * t.element_size())
    R = ctx.n_refs
    p_arr = _arr(ctypes.c_void_p, ptrs)
    pitch_arr = _arr(ctypes.c_int64, pitches)
    lab_arr = _arr(ctypes.c_void_p, [_ptr(l) if l is not None else None for l in labels]) if labels is not None else None
    nseg = _arr(ctypes.c_int32, n_segments) if n_segments is not None else None
    sl = _arr(ctypes.c_void_p, [_ptr(x) for x in seg_lists]) if seg_lists is not None else None
    nl = _arr(ctypes.c_void_p, [_ptr(x) for x in n_listed]) if n_listed is not None else None
    c_arr = _arr(ctypes.c_void_p, [_ptr(c) for c in costs])
    assert len(costs) == R
    _ok(lib.ftv_cost_volume(ctx.handle, p_arr, pitch_arr, lab_arr, nseg, sl, nl, c_arr, _stream(stream)),
        "ftv_cost_volume")


def ftv_set_launch_shape(ctx: Context, label_block: int, ctas_per_sm: int = 0) -> None:
    _ok(lib.ftv_set_launch_shape(ctx.handle, int(label_block), int(ctas_per_sm)), "ftv_set_launch_shape")


def ftv_get_launch_shape(ctx: Context) -> dict:
    """{'label_block', 'ctas_per_sm', 'max_label_block', 'max_ctas_per_sm'} of the context's cost kernel."""
    v = [ctypes.c_int32() for _ in range(4)]
    _ok(lib.ftv_get_launch_shape(ctx.handle, *[ctypes.byref(x) for x in v]), "ftv_get_launch_shape")
    return dict(zip(("label_block", "ctas_per_sm", "max_label_block", "max_ctas_per_sm"), (x.value for x in v)))


def ftv_autotune(ctx: Context, planes, labels, n_segments, costs, label_blocks, ctas, reps: int = 3,
                 stream=None) -> tuple[int, int, np.ndarray]:
    """Times the cost kernel for every (label block, CTAs per SM) candidate on these inputs and keeps the
    fastest on the context. Returns (label_block, ctas_per_sm, ms [len(label_blocks)][len(ctas)])."""
    ptrs, pitches = [], []
    for trip in planes:
        for t in trip:
            ptrs.append(_ptr(t))
            pitches.append(int(t.stride(0)) * t.element_size())
    lab_arr = _arr(ctypes.c_void_p, [_ptr(l) if l is not None else None for l in labels]) if labels is not None else None
    nseg = _arr(ctypes.c_int32, n_segments) if n_segments is not None else None
    c_arr = _arr(ctypes.c_void_p, [_ptr(c) for c in costs])
    lbs, cts = _arr(ctypes.c_int32, list(label_blocks)), _arr(ctypes.c_int32, list(ctas))
    ms = np.zeros((len(label_blocks), len(ctas)), np.float32)
    b_lb, b_ct = ctypes.c_int32(), ctypes.c_int32()
    _ok(lib.ftv_autotune(ctx.handle, _arr(ctypes.c_void_p, ptrs), _arr(ctypes.c_int64, pitches), lab_arr, nseg,
                         c_arr, lbs, len(label_blocks), cts, len(ctas), int(reps), _stream(stream),
                         ms.ctypes.data, ctypes.byref(b_lb), ctypes.byref(b_ct)), "ftv_autotune")
    return b_lb.value, b_ct.value, ms


def _trip(planes):
    if planes is None:
        return None, None
    ptrs = _arr(ctypes.c_void_p, [_ptr(t) for t in planes])
    pitches = _arr(ctypes.c_int64, [int(t.stride(0)) * t.element_size() if t is not None else 0 for t in planes])
    return ptrs, pitches


def ftv_temporal_mask(ctx: Context, ref_index: int, cur, prev, iframe, labels, n_segments: int, t_p: int, t_i: int,
                      mode: int, mask, changed_list, n_changed, stream=None) -> None:
    cp, cpi = _trip(cur)
    pp, ppi = _trip(prev)
    ip, ipi = _trip(iframe)
    _ok(lib.ftv_temporal_mask(ctx.handle, ref_index, cp, cpi, pp, ppi, ip, ipi, _ptr(labels), n_segments, t_p, t_i,
                              mode, _ptr(mask), _ptr(changed_list), _ptr(n_changed), _stream(stream)),
        "ftv_temporal_mask")


def ftv_temporal_mask_views(ctx: Context, ref_indices, cur, prev, iframe, labels, n_segments, t_p: int, t_i: int,
                            mode: int, masks, changed_lists, n_changed, stream=None) -> None:
    """ftv_temporal_mask for several references in one launch sequence: cur, prev (and iframe, or None) are
    lists of (Y, Cb, Cr) plane triples, one per reference; labels, n_segments, masks, changed_lists and
    n_changed are per-reference lists."""
    n = len(ref_indices)
    cp, cpi = _trip([t for trip in cur for t in trip])
    pp, ppi = _trip([t for trip in prev for t in trip])
    ip, ipi = _trip([t for trip in iframe for t in trip]) if iframe is not None else (None, None)
    _ok(lib.ftv_temporal_mask_views(ctx.handle, n, _arr(ctypes.c_int32, ref_indices), cp, cpi, pp, ppi, ip, ipi,
                                    _arr(ctypes.c_void_p, [_ptr(t) for t in labels]),
                                    _arr(ctypes.c_int32, n_segments), t_p, t_i, mode,
                                    _arr(ctypes.c_void_p, [_ptr(t) for t in masks]),
                                    _arr(ctypes.c_void_p, [_ptr(t) for t in changed_lists]),
                                    _arr(ctypes.c_void_p, [_ptr(t) for t in n_changed]), _stream(stream)),
        "ftv_temporal_mask_views")


def ftv_wta_depth(ctx: Context, ref_index: int, cost, n_segments: int, label_out, *, mask=None, prev_label=None,
                  iframe_label=None, seg_list=None, n_listed=None, labels_pix=None, depth_map=None,
                  stream=None) -> None:
    _ok(lib.ftv_wta_depth(ctx.handle, ref_index, _ptr(cost), n_segments, _ptr(mask), _ptr(prev_label),
                          _ptr(iframe_label), _ptr(seg_list), _ptr(n_listed), _ptr(label_out), _ptr(labels_pix),
                          _ptr(depth_map), _stream(stream)), "ftv_wta_depth")


def ftv_check(ctx: Context, stream=None) -> int:
    """Wait for the stream and return the context's device status code (0 = clean)."""
    return int(lib.ftv_check(ctx.handle, _stream(stream)))


def ftv_culled_evaluations(ctx: Context, stream=None) -> int:
    """Evaluations of the most recent ftv_cost_volume call decided without sampling (whole tile out of
    a neighbour's view); waits for the stream."""
    n = ctypes.c_int64()
    _ok(lib.ftv_culled_evaluations(ctx.handle, _stream(stream), ctypes.byref(n)), "ftv_culled_evaluations")
    return int(n.value)


def ftv_fp64_recomputed(ctx: Context, stream=None) -> int:
    """Evaluations of the most recent ftv_cost_volume call of an FP64-precision context that were computed
    in double precision (near a rounding boundary, or no error bound); waits for the stream."""
    n = ctypes.c_int64()
    _ok(lib.ftv_fp64_recomputed(ctx.handle, _stream(stream), ctypes.byref(n)), "ftv_fp64_recomputed")
    return int(n.value)


def ftv_launch_count(ctx: Context) -> int:
    return int(lib.ftv_launch_count(ctx.handle))


def ftv_status_str(code: int) -> str:
    return lib.ftv_status_str(code).decode()


def ftv_set_profiling(ctx: Context, enable: bool) -> None:
    _ok(lib.ftv_set_profiling(ctx.handle, 1 if enable else 0), "ftv_set_profiling")


def ftv_last_kernel_ms(ctx: Context) -> float:
    ms = ctypes.c_float()
    _ok(lib.ftv_last_kernel_ms(ctx.handle, ctypes.byref(ms)), "ftv_last_kernel_ms")
    return float(ms.value)


FTV_STATIC_MAX_SEGMENTS = 65536


def ftv_temporal_mask_static(width: int, height: int, sample_bytes: int, cur, prev, iframe, labels, n_segments: int,
                             t_p: int, t_i: int, mode: int, mask, changed_list, n_changed, status=None,
                             stream=None) -> None:
    """The temporal test without a context and without any device allocation (statically sized scratch
    inside the library, at most FTV_STATIC_MAX_SEGMENTS segments). Runs on the label map's device; every
    tensor argument must be on that device."""
    import torch
    args = [t for trip in (cur, prev, iframe) if trip is not None for t in trip if t is not None]
    args += [t for t in (mask, changed_list, n_changed, status) if t is not None]
    if any(getattr(t, "device", None) != labels.device for t in args):
        raise FtvError(FTV_ERR_INVALID_ARG, "ftv_temporal_mask_static: tensors on different devices")
    cp, cpi = _trip(cur)
    pp, ppi = _trip(prev)
    ip, ipi = _trip(iframe)
    with torch.cuda.device(labels.device):
        _ok(lib.ftv_temporal_mask_static(width, height, sample_bytes, cp, cpi, pp, ppi, ip, ipi, _ptr(labels),
                                         n_segments, t_p, t_i, mode, _ptr(mask), _ptr(changed_list), _ptr(n_changed),
                                         _ptr(status), _stream(stream)), "ftv_temporal_mask_static")


FTV_FRAME_I, FTV_FRAME_P = 0, 1


class ftv_frame_job(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("d_planes", ctypes.c_void_p), ("pitch_bytes", ctypes.c_void_p),
                ("frame_type", ctypes.c_int32), ("d_label_out", ctypes.c_void_p), ("d_depth_out", ctypes.c_void_p)]


def ftv_stream_init(ctx: Context, labels, n_segments, t_p: int, t_i: int, mode: int, stream=None) -> None:
    """Make ctx a camera stream with static label maps labels[r] (int32 [H][W] device tensors)."""
    lab = _arr(ctypes.c_void_p, [_ptr(l) for l in labels])
    ns = _arr(ctypes.c_int32, n_segments)
    _ok(lib.ftv_stream_init(ctx.handle, lab, ns, t_p, t_i, mode, _stream(stream)), "ftv_stream_init")


def ftv_stream_footprint(ctx: Context, n_segments) -> int:
    out = ctypes.c_int64()
    _ok(lib.ftv_stream_footprint(ctx.handle, _arr(ctypes.c_int32, n_segments), ctypes.byref(out)),
        "ftv_stream_footprint")
    return int(out.value)


def ftv_stream_labels(ctx: Context, ref_index: int) -> int:
    p = ctypes.c_void_p()
    _ok(lib.ftv_stream_labels(ctx.handle, ref_index, ctypes.byref(p)), "ftv_stream_labels")
    return int(p.value)


def ftv_stream_mask(ctx: Context, ref_index: int) -> tuple[int, int]:
    """(device pointer of the uint8 mask [S], device pointer of the int32 changed count)."""
    m, n = ctx_void(), ctx_void()
    _ok(lib.ftv_stream_mask(ctx.handle, ref_index, ctypes.byref(m), ctypes.byref(n)), "ftv_stream_mask")
    return int(m.value), int(n.value)


def ftv_stream_changed(ctx: Context, ref_index: int) -> int:
    """Device pointer of the int32 list of segments the last frame re-estimated (length: ftv_stream_mask)."""
    p = ctypes.c_void_p()
    _ok(lib.ftv_stream_changed(ctx.handle, ref_index, ctypes.byref(p)), "ftv_stream_changed")
    return int(p.value)


def ftv_stream_state_save(ctx: Context, stream=None):
    """Checkpoint of the stream's resident temporal state as a pinned uint8 tensor (valid after a sync)."""
    import torch
    n = ctypes.c_int64()
    _ok(lib.ftv_stream_state_bytes(ctx.handle, ctypes.byref(n)), "ftv_stream_state_bytes")
    buf = torch.empty(int(n.value), dtype=torch.uint8).pin_memory()
    _ok(lib.ftv_stream_state_save(ctx.handle, buf.data_ptr(), buf.numel(), _stream(stream)), "ftv_stream_state_save")
    return buf


def ftv_stream_state_load(ctx: Context, buf, stream=None) -> None:
    """Restore a checkpoint (from ftv_stream_state_save) into a stream of the same shape."""
    _ok(lib.ftv_stream_state_load(ctx.handle, buf.data_ptr(), buf.numel(), _stream(stream)), "ftv_stream_state_load")


def ctx_void():
    return ctypes.c_void_p()


class Batch:
    """Owns an ftv_batch handle."""

    def __init__(self, max_jobs: int, max_units: int, max_views: int):
        h = ctypes.c_void_p()
        _ok(lib.ftv_batch_create(max_jobs, max_units, max_views, ctypes.byref(h)), "ftv_batch_create")
        self.handle = h.value

    def close(self) -> None:
        if self.handle:
            _ok(lib.ftv_batch_destroy(self.handle), "ftv_batch_destroy")
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ftv_batch_create(max_jobs: int, max_units: int, max_views: int) -> Batch:
    return Batch(max_jobs, max_units, max_views)


def _frame_jobs(jobs):
    keep = []
    arr = (ftv_frame_job * max(1, len(jobs)))()
    for k, j in enumerate(jobs):
        ptrs, pitches = [], []
        for trip in j["planes"]:
            for t in trip:
                ptrs.append(_ptr(t))
                pitches.append(int(t.stride(0)) * t.element_size())
        pa, pi = _arr(ctypes.c_void_p, ptrs), _arr(ctypes.c_int64, pitches)
        lo = _arr(ctypes.c_void_p, [_ptr(t) for t in j["label_out"]]) if j.get("label_out") is not None else None
        do = _arr(ctypes.c_void_p, [_ptr(t) for t in j["depth_out"]]) if j.get("depth_out") is not None else None
        keep += [pa, pi, lo, do]
        arr[k].ctx = j["ctx"].handle
        arr[k].d_planes = ctypes.cast(pa, ctypes.c_void_p)
        arr[k].pitch_bytes = ctypes.cast(pi, ctypes.c_void_p)
        arr[k].frame_type = j["frame_type"]
        arr[k].d_label_out = ctypes.cast(lo, ctypes.c_void_p) if lo is not None else None
        arr[k].d_depth_out = ctypes.cast(do, ctypes.c_void_p) if do is not None else None
    return arr, keep


def ftv_batch_prepare(batch: Batch, jobs) -> int:
    """jobs: list of dicts {ctx, planes (per view (Y, Cb, Cr) tensors), frame_type, label_out (list or
    None), depth_out (list or None)}. Returns the status code (FTV_ERR_BUSY while the batch is in use)."""
    arr, keep = _frame_jobs(jobs)
    return int(lib.ftv_batch_prepare(batch.handle, arr, len(jobs)))


def ftv_job_footprint(cams, ref_views, n_labels: int, z_near: float, z_far: float, n_segments_max: int = 0, *,
                      nbr_lists=None, sample_bytes: int = 1, bit_depth: int = 8, max_segments: int = 1,
                      precision: int = FTV_PRECISION_FP32) -> int:
    """Device bytes of one camera stream of this configuration: context, resident stream state and one
    input frame (host only)."""
    cfg, keep = _config(cams, ref_views, n_labels, z_near, z_far, nbr_lists, FTV_PLANES_REF, 0, sample_bytes,
                        bit_depth, -1, FTV_COMBINE_MIN, max_segments, precision)
    out = ctypes.c_int64()
    _ok(lib.ftv_job_footprint(ctypes.byref(cfg), n_segments_max, ctypes.byref(out)), "ftv_job_footprint")
    return int(out.value)


def ftv_batch_set_budget(batch: Batch, budget_bytes: int) -> None:
    _ok(lib.ftv_batch_set_budget(batch.handle, int(budget_bytes)), "ftv_batch_set_budget")


def ftv_batch_submit(batch: Batch, job) -> tuple[int, int]:
    """Queue one job (a dict as in ftv_batch_prepare). Returns (status, ticket); status FTV_ERR_BUSY means
    not admitted now (retry after a ticket completes)."""
    arr, keep = _frame_jobs([job])
    t = ctypes.c_uint64()
    rc = int(lib.ftv_batch_submit(batch.handle, arr, ctypes.byref(t)))
    return rc, int(t.value)


def ftv_batch_flush(batch: Batch, stream=None) -> int:
    """Launch the queued jobs; returns the status (FTV_ERR_BUSY while the previous launch runs)."""
    return int(lib.ftv_batch_flush(batch.handle, _stream(stream)))


def ftv_batch_poll(batch: Batch, ticket: int) -> tuple[int, int]:
    """Non-blocking: (FTV_OK, the job's own status) once it completed, (FTV_ERR_BUSY, -1) while pending."""
    st = ctypes.c_int32(-1)
    rc = int(lib.ftv_batch_poll(batch.handle, ctypes.c_uint64(ticket), ctypes.byref(st)))
    return rc, int(st.value)


def ftv_batch_launch(batch: Batch, stream=None) -> None:
    _ok(lib.ftv_batch_launch(batch.handle, _stream(stream)), "ftv_batch_launch")


def ftv_batch_replay(batch: Batch, stream=None) -> None:
    _ok(lib.ftv_batch_replay(batch.handle, _stream(stream)), "ftv_batch_replay")


FTV_MAX_BATCH_CHUNKS = 16


def ftv_batch_set_chunks(batch: Batch, chunks: int) -> None:
    _ok(lib.ftv_batch_set_chunks(batch.handle, chunks), "ftv_batch_set_chunks")


def ftv_batch_query(batch: Batch) -> int:
    return int(lib.ftv_batch_query(batch.handle))


def ftv_batch_wait(batch: Batch) -> int:
    return int(lib.ftv_batch_wait(batch.handle))


def ftv_batch_launch_count(batch: Batch) -> int:
    return int(lib.ftv_batch_launch_count(batch.handle))


def ftv_reciprocal_check() -> tuple[int, bool]:
    """(mismatching inputs of the Newton-Raphson reciprocal on this device, whether the kernel uses it)."""
    n, used = ctypes.c_int64(), ctypes.c_int32()
    _ok(lib.ftv_reciprocal_check(ctypes.byref(n), ctypes.byref(used)), "ftv_reciprocal_check")
    return int(n.value), bool(used.value)


def ftv_centre_table(ctx: Context, planes, labels_views, n_segments, window: int, m_out, sprime_out,
                     stream=None) -> None:
    """planes as in ftv_cost_volume; labels_views: per view an int32 [H][W] tensor or None;
    m_out / sprime_out: per reference int32 [S][L][N] tensors."""
    ptrs, pitches = [], []
    for trip in planes:
        for t in trip:
            ptrs.append(_ptr(t))
            pitches.append(int(t.stride(0)) * t.element_size())
    _ok(lib.ftv_centre_table(ctx.handle, _arr(ctypes.c_void_p, ptrs), _arr(ctypes.c_int64, pitches),
                             _arr(ctypes.c_void_p, [_ptr(l) for l in labels_views]), _arr(ctypes.c_int32, n_segments),
                             window, _arr(ctypes.c_void_p, [_ptr(t) for t in m_out]),
                             _arr(ctypes.c_void_p, [_ptr(t) for t in sprime_out]), _stream(stream)), "ftv_centre_table")


def ftv_adjacency(ctx: Context, ref_index: int, frame, labels, n_segments: int, connectivity: int, beta0: float,
                  min_diff: float, edge_s, edge_t, beta, n_edges, stream=None) -> None:
    """frame: (Y, Cb, Cr) tensors; edge_s/edge_t int32, beta float32 tensors of equal capacity;
    n_edges: one-element int32 tensor receiving the edge count."""
    fp, fpi = _trip(frame)
    _ok(lib.ftv_adjacency(ctx.handle, ref_index, fp, fpi, _ptr(labels), n_segments, connectivity, beta0, min_diff,
                          int(edge_s.numel()) if edge_s is not None else 0, _ptr(edge_s), _ptr(edge_t), _ptr(beta),
                          _ptr(n_edges), _stream(stream)), "ftv_adjacency")


FTV_SEG_MAX_IMAGES, FTV_SEG_MAX_STEP = 4096, 64


class Segmenter:
    """Owns an ftv_segmenter handle (superpixel segmentation of a fixed set of image sizes)."""

    def __init__(self, sizes, sample_bytes: int, bit_depth: int, grid_step: int, compactness: int = 5,
                 iterations: int = 10):
        """sizes: list of (width, height)."""
        self.sizes = [(int(w), int(h)) for w, h in sizes]
        ws = _arr(ctypes.c_int32, [w for w, _ in self.sizes])
        hs = _arr(ctypes.c_int32, [h for _, h in self.sizes])
        cfg = ftv_segmenter_config(len(self.sizes), ws, hs, sample_bytes, bit_depth, grid_step, compactness,
                                   iterations)
        h = ctypes.c_void_p()
        _ok(lib.ftv_segmenter_init(ctypes.byref(cfg), ctypes.byref(h)), "ftv_segmenter_init")
        self.handle = h.value

    def close(self) -> None:
        if self.handle:
            _ok(lib.ftv_segmenter_destroy(self.handle), "ftv_segmenter_destroy")
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ftv_segmenter_init(sizes, sample_bytes: int, bit_depth: int, grid_step: int, compactness: int = 5,
                       iterations: int = 10) -> Segmenter:
    return Segmenter(sizes, sample_bytes, bit_depth, grid_step, compactness, iterations)


def ftv_segmenter_segments(sg: Segmenter) -> list[int]:
    out = np.empty(len(sg.sizes), np.int32)
    _ok(lib.ftv_segmenter_segments(sg.handle, out.ctypes.data), "ftv_segmenter_segments")
    return [int(v) for v in out]


def ftv_superpixels(sg: Segmenter, planes, labels, stream=None) -> None:
    """planes: per image a (Y, Cb, Cr) triple of 2-D CUDA tensors (uint8 or uint16, any row pitch);
    labels: per image a dense int32 [H][W] CUDA tensor."""
    ptrs, pitches = [], []
    for trip in planes:
        for t in trip:
            ptrs.append(_ptr(t))
            pitches.append(int(t.stride(0)) * t.element_size())
    _ok(lib.ftv_superpixels(sg.handle, _arr(ctypes.c_void_p, ptrs), _arr(ctypes.c_int64, pitches),
                            _arr(ctypes.c_void_p, [_ptr(l) for l in labels]), _stream(stream)), "ftv_superpixels")


def ftv_segmenter_check(sg: Segmenter, stream=None) -> int:
    """Wait for the stream and return the segmenter's device status code (0 = clean)."""
    return int(lib.ftv_segmenter_check(sg.handle, _stream(stream)))


def ftv_segmenter_launch_count(sg: Segmenter) -> int:
    return int(lib.ftv_segmenter_launch_count(sg.handle))


def ftv_segmenter_destroy(sg: Segmenter) -> None:
    sg.close()


def ftv_segmenter_set_profiling(sg: Segmenter, enable: bool) -> None:
    _ok(lib.ftv_segmenter_set_profiling(sg.handle, 1 if enable else 0), "ftv_segmenter_set_profiling")


def ftv_segmenter_kernel_ms(sg: Segmenter) -> tuple[float, float]:
    """(mean assignment-pass launch ms, whole-call device ms) of the most recent timed call."""
    a, t = ctypes.c_float(), ctypes.c_float()
    _ok(lib.ftv_segmenter_kernel_ms(sg.handle, ctypes.byref(a), ctypes.byref(t)), "ftv_segmenter_kernel_ms")
    return float(a.value), float(t.value)
