"""Helpers that run the CUDA library on a synthetic workload through the C ABI (GPU tests only)."""
from __future__ import annotations

import numpy as np
import torch

import paper_1909_02294_gb300 as ftv


def dev(a, device="cuda"):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device)


class Run:
    def __init__(self, wl, *, combine=None, plane_mode=0, centre=0, nbr_lists=None, max_segments=None,
                 penalty=None, precision=ftv.FTV_PRECISION_FP32):
        self.wl = wl
        self.combine = combine or wl.combine
        self.S = [wl.labels(r)[1] for r in wl.ref_views]
        self.nbr_lists = nbr_lists
        self.ctx = ftv.ftv_depth_init(
            wl.cams, wl.ref_views, wl.n_labels, wl.z_near, wl.z_far, nbr_lists=nbr_lists, plane_mode=plane_mode,
            centre_view=centre, sample_bytes=wl.sample_bytes, bit_depth=wl.bit_depth,
            oob_penalty=wl.oob_penalty if penalty is None else penalty,
            combine=ftv.FTV_COMBINE_MIN if self.combine == "min" else ftv.FTV_COMBINE_SUM,
            max_segments=max_segments or max(self.S), precision=precision)
        self.labels = [dev(wl.labels(r)[0]) for r in wl.ref_views]

    def planes(self, frame=0):
        return [(dev(v.Y), dev(v.U), dev(v.V)) for v in self.wl.views(frame)]

    def volumes(self, frame=0, seg_lists=None, n_listed=None, fill=None, use_cache=False, planes=None):
        L = self.wl.n_labels
        costs = [torch.full((S, L), fill, dtype=torch.int32, device="cuda") if fill is not None
                 else torch.empty((S, L), dtype=torch.int32, device="cuda") for S in self.S]
        ftv.ftv_cost_volume(self.ctx, planes if planes is not None else self.planes(frame),
                            None if use_cache else self.labels, None if use_cache else self.S, costs,
                            seg_lists=seg_lists, n_listed=n_listed)
        return costs

    def check(self) -> int:
        return ftv.ftv_check(self.ctx)

    def close(self):
        self.ctx.close()


class _DeviceArray:
    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 3}


def from_device_pointer(ptr: int, n: int, typestr: str) -> np.ndarray:
    """Host copy of n elements at a device pointer the library returned (typestr: '|u1', '<i4', '<u2')."""
    if n == 0:
        return np.zeros(0, np.dtype(typestr))
    return torch.as_tensor(_DeviceArray(ptr, (n,), typestr), device="cuda").cpu().numpy().copy()
