"""Seeded synthetic multiview inputs: camera rigs, layered-plane scenes, grid label maps.

Input generation only, shared by the CUDA library's tests and benchmark and by the CPU oracle's
tests. It holds none of the depth estimator's arithmetic (no plane homography, no matching cost,
no temporal test): it ray-casts textured planes into each camera (``ftv_synth.c``) and cuts each
reference view into a jittered grid of segments. The paper's multiview test sequences (Table I)
are not available, so these scenes stand in for them, shaped like the paper's workloads:
a few to 15 cameras, 480x270 to 3840x2160, YCbCr 4:4:4 (8-bit) or 10-bit 4:2:0 upsampled to 4:4:4,
tens of thousands of segments of 10-16 px cells (the paper uses segments of about 20 samples and up
to 100k segments per HD view).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ftv_synth.c")
_LIB = os.path.join(_HERE, "libftv_synth.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the ray-caster into synth/libftv_synth.so (plain C, pthreads)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-pthread", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Cam(ctypes.Structure):
    _fields_ = [("K", ctypes.c_double * 9), ("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class _Plane(ctypes.Structure):
    _fields_ = [("p0", ctypes.c_double * 3), ("e1", ctypes.c_double * 3), ("e2", ctypes.c_double * 3),
                ("half1", ctypes.c_double), ("half2", ctypes.c_double), ("texel", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("mode", ctypes.c_int32), ("pad", ctypes.c_int32)]


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.syn_render.restype = ctypes.c_int
        _lib.syn_grid_labels.restype = ctypes.c_int
    return _lib


# --------------------------------------------------------------------------------------------- rigs

@dataclass
class Camera:
    """Pinhole camera, X_cam = R X_world + t, pixel centres at integer coordinates."""
    K: np.ndarray
    R: np.ndarray
    t: np.ndarray
    width: int
    height: int

    @property
    def centre(self) -> np.ndarray:
        return -self.R.T @ self.t

    def as_struct(self) -> _Cam:
        c = _Cam()
        c.K[:] = [float(v) for v in np.asarray(self.K, np.float64).ravel()]
        c.R[:] = [float(v) for v in np.asarray(self.R, np.float64).ravel()]
        c.t[:] = [float(v) for v in np.asarray(self.t, np.float64).ravel()]
        c.width, c.height = int(self.width), int(self.height)
        return c


def intrinsics(f: float, width: int, height: int) -> np.ndarray:
    return np.array([[f, 0.0, (width - 1) / 2.0], [0.0, f, (height - 1) / 2.0], [0.0, 0.0, 1.0]])


def linear_rig(n: int, spacing: float, f: float, width: int, height: int) -> list[Camera]:
    """Cameras on the world x axis, parallel optical axes (R = I), centred on x = 0."""
    cams = []
    for i in range(n):
        C = np.array([(i - (n - 1) / 2.0) * spacing, 0.0, 0.0])
        R = np.eye(3)
        cams.append(Camera(intrinsics(f, width, height), R, -R @ C, width, height))
    return cams


def _rot_z(a: float) -> np.ndarray:
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def arc_rig(n: int, radius: float, step_deg: float, f: float, width: int, height: int, seed: int,
            focal_jitter: float = 0.03, roll_deg: float = 2.0) -> list[Camera]:
    """Convergent cameras on a horizontal arc around the world origin, each aimed at the origin,
    with a seeded per-camera roll in [-roll_deg, roll_deg] and focal f * (1 + U[-j, j])."""
    rng = np.random.default_rng(seed)
    cams = []
    for i in range(n):
        th = math.radians((i - (n - 1) / 2.0) * step_deg)
        C = np.array([radius * math.sin(th), 0.0, -radius * math.cos(th)])
        fwd = -C / np.linalg.norm(C)
        right = np.array([math.cos(th), 0.0, math.sin(th)])
        down = np.cross(fwd, right)
        R = np.stack([right, down, fwd])
        roll = math.radians(rng.uniform(-roll_deg, roll_deg))
        R = _rot_z(roll) @ R
        fi = f * (1.0 + rng.uniform(-focal_jitter, focal_jitter))
        cams.append(Camera(intrinsics(fi, width, height), R, -R @ C, width, height))
    return cams


# ------------------------------------------------------------------------------------------- scenes

@dataclass
class Plane:
    p0: np.ndarray
    e1: np.ndarray
    e2: np.ndarray
    half1: float = 0.0  # <= 0: unbounded
    half2: float = 0.0
    texel: float = 0.01
    seed: int = 0
    mode: int = 0  # 0 world texture, 1 painted from the paint camera (exact-correspondence scenes)
    velocity: np.ndarray = field(default_factory=lambda: np.zeros(3))  # world shift per frame

    def as_struct(self, frame: int = 0) -> _Plane:
        p = _Plane()
        p.p0[:] = [float(v) for v in self.p0]
        p.e1[:] = [float(v) for v in self.e1]
        p.e2[:] = [float(v) for v in self.e2]
        p.half1, p.half2, p.texel = float(self.half1), float(self.half2), float(self.texel)
        p.seed, p.mode = int(self.seed) & (2**64 - 1), int(self.mode)
        return p


def fronto_plane(cam: Camera, z: float, half: float = 0.0, centre_xy=(0.0, 0.0), **kw) -> Plane:
    """A plane parallel to `cam`'s image plane at camera depth z (centre offset in camera x/y)."""
    Rt = cam.R.T
    C = cam.centre
    p0 = C + Rt @ np.array([centre_xy[0], centre_xy[1], z])
    return Plane(p0=p0, e1=Rt[:, 0].copy(), e2=Rt[:, 1].copy(), half1=half, half2=half, **kw)


def slanted_plane(cam: Camera, z: float, tilt_deg: float, azimuth_deg: float, half: float,
                  centre_xy=(0.0, 0.0), **kw) -> Plane:
    """A bounded plane centred at camera depth z whose normal is tilted from the optical axis."""
    Rt = cam.R.T
    C = cam.centre
    a, b = math.radians(tilt_deg), math.radians(azimuth_deg)
    n = np.array([math.sin(a) * math.cos(b), math.sin(a) * math.sin(b), -math.cos(a)])
    e1 = np.cross(n, np.array([0.0, 1.0, 0.0]))
    if np.linalg.norm(e1) < 1e-9:
        e1 = np.array([1.0, 0.0, 0.0])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(n, e1)
    e2 /= np.linalg.norm(e2)
    p0 = C + Rt @ np.array([centre_xy[0], centre_xy[1], z])
    return Plane(p0=p0, e1=Rt @ e1, e2=Rt @ e2, half1=half, half2=half, **kw)


@dataclass
class View:
    Y: np.ndarray
    U: np.ndarray
    V: np.ndarray
    depth: np.ndarray | None = None
    plane_id: np.ndarray | None = None


def render(cam: Camera, planes: list[Plane], *, bit_depth: int = 8, frame: int = 0,
           noise_sigma: float = 0.0, specular_frac: float = 0.0, noise_seed: int = 0,
           chroma420: bool = False, paint: Camera | None = None, aux: bool = False,
           threads: int | None = None) -> View:
    """Ray-cast `planes` into `cam`. Samples are uint8 when bit_depth <= 8, else uint16."""
    lib = _load()
    W, H = cam.width, cam.height
    Y = np.empty((H, W), np.uint16)
    U = np.empty_like(Y)
    V = np.empty_like(Y)
    depth = np.empty((H, W), np.float32) if aux else None
    pid = np.empty((H, W), np.int32) if aux else None
    arr = (_Plane * max(1, len(planes)))(*[p.as_struct() for p in planes])
    offs = np.array([p.velocity * frame for p in planes], np.float64).reshape(-1) if planes else np.zeros(3)
    offs = np.ascontiguousarray(offs)
    c = cam.as_struct()
    pc = paint.as_struct() if paint is not None else None
    th = threads if threads is not None else min(64, os.cpu_count() or 1)
    rc = lib.syn_render(ctypes.byref(c), ctypes.byref(pc) if pc is not None else None,
                        ctypes.c_int(len(planes)), arr, offs.ctypes.data_as(ctypes.c_void_p),
                        ctypes.c_int(bit_depth), ctypes.c_double(noise_sigma),
                        ctypes.c_double(specular_frac), ctypes.c_uint64(noise_seed & (2**64 - 1)),
                        ctypes.c_int(1 if chroma420 else 0),
                        Y.ctypes.data_as(ctypes.c_void_p), U.ctypes.data_as(ctypes.c_void_p),
                        V.ctypes.data_as(ctypes.c_void_p),
                        depth.ctypes.data_as(ctypes.c_void_p) if aux else None,
                        pid.ctypes.data_as(ctypes.c_void_p) if aux else None, ctypes.c_int(th))
    if rc != 0:
        raise RuntimeError(f"syn_render failed ({rc})")
    if bit_depth <= 8:
        Y, U, V = Y.astype(np.uint8), U.astype(np.uint8), V.astype(np.uint8)
    return View(Y, U, V, depth, pid)


def grid_labels(width: int, height: int, cell: int, jitter: int, seed: int) -> tuple[np.ndarray, int]:
    """Jittered grid segmentation: returns (int32 [H][W] label map, segment count)."""
    lib = _load()
    lab = np.empty((height, width), np.int32)
    n = lib.syn_grid_labels(ctypes.c_int(width), ctypes.c_int(height), ctypes.c_int(cell),
                            ctypes.c_int(jitter), ctypes.c_uint64(seed & (2**64 - 1)),
                            lab.ctypes.data_as(ctypes.c_void_p))
    if n < 0:
        raise ValueError("bad grid parameters")
    return lab, int(n)


def mosaic(width: int, height: int, n_regions: int, *, bit_depth: int = 8, noise_sigma: float = 0.0,
           seed: int = 0) -> View:
    """Piecewise-constant (Y, Cb, Cr) image: the Voronoi cells of n_regions uniformly drawn sites, each
    with a uniform random colour, plus rounded N(0, noise_sigma^2) noise clamped to the sample range.
    plane_id holds each pixel's cell (the ground-truth regions for segmentation quality)."""
    rng = np.random.default_rng(seed)
    vmax = (1 << bit_depth) - 1
    sx = rng.uniform(0, width, n_regions)
    sy = rng.uniform(0, height, n_regions)
    col = rng.integers(0, vmax + 1, (n_regions, 3))
    ys, xs = np.mgrid[0:height, 0:width]
    rid = np.zeros((height, width), np.int32)
    best = np.full((height, width), np.inf)
    for k in range(n_regions):
        d = (xs - sx[k]) ** 2 + (ys - sy[k]) ** 2
        closer = d < best
        best[closer] = d[closer]
        rid[closer] = k
    dtype = np.uint8 if bit_depth <= 8 else np.uint16
    planes = []
    for c in range(3):
        v = col[rid, c].astype(np.float64)
        if noise_sigma > 0:
            v = v + np.rint(rng.normal(0.0, noise_sigma, v.shape))
        planes.append(np.clip(v, 0, vmax).astype(dtype))
    return View(planes[0], planes[1], planes[2], None, rid)


from .configs import Workload, make_workload, CONFIG_NAMES  # noqa: E402,F401
