"""The five benchmark workloads as seeded synthetic scenes, plus reduced variants for parity tests.

Workloads (seed = 190902294 + index):
  tiny      3 views 480x270 uint8 4:4:4, linear rig 5 cm apart, f = 400 px, 4 planes (2 fronto-parallel
            on label planes, 2 slanted), 16 px grid cells +-3 px jitter (510 segments), 64 labels in 1/z
            on [0.5, 10] m, reference = centre view, min over views, penalty 3*255.
  hd8       8 views 1920x1080, 10-bit 4:2:0 upsampled to 4:4:4 in uint16, linear rig 10 cm apart,
            f = 1500 px, 12 planes, Gaussian noise sigma 2 LSB, 10 px cells (20736 segments),
            250 labels on [1, 20] m, all 8 views are references, neighbours = the 7 others.
  uhd15     15 views 3840x2160 10-bit 4:4:4, convergent arc of radius 3 m with cameras 8 degrees
            apart, roll +-2 degrees, focal 3000 px +-3 %, 20 planes, 10 % specular-noise pixels,
            13 px cells (49432 segments), 400 labels on [0.8, 15] m, all 15 references.
  temporal  the hd8 rig over 30 frames: static background planes and 3 foreground planes translating
            4 px/frame; sensor noise re-drawn per frame.
  serving   stream shapes: 960x540 / 3 views / 64 labels, the hd8 shape and the uhd15 shape.

Plane depths on "label planes" use the label spacing of the workload (uniform in 1/z): that is scene
layout, chosen so that a plane lies exactly on one candidate depth.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import (Camera, Plane, View, arc_rig, fronto_plane, grid_labels, linear_rig, render,
               slanted_plane)

BASE_SEED = 190902294
CONFIG_NAMES = ["tiny", "hd8", "uhd15", "temporal", "serving_small"]


def label_depth(d: int, n_labels: int, z_near: float, z_far: float) -> float:
    """Depth of candidate plane d when candidates are uniform in 1/z and d = 0 is the far plane."""
    a, b = 1.0 / z_far, 1.0 / z_near
    return 1.0 / (a + d * (b - a) / (n_labels - 1))


@dataclass
class Workload:
    name: str
    cams: list[Camera]
    ref_views: list[int]
    n_labels: int
    z_near: float
    z_far: float
    bit_depth: int
    planes: list[Plane]
    cell: int
    jitter: int = 3
    nbr_views: dict | None = None  # ref -> list of neighbour views; None = all other views
    combine: str = "min"
    penalty: int = -1  # < 0: 3 * (2^bit_depth - 1)
    noise_sigma: float = 0.0
    specular_frac: float = 0.0
    chroma420: bool = False
    seed: int = BASE_SEED
    paint_view: int | None = None  # painted-texture scenes: camera whose pixels carry the texture
    n_frames: int = 1
    _views: dict = field(default_factory=dict, repr=False)
    _labels: dict = field(default_factory=dict, repr=False)

    @property
    def n_views(self) -> int:
        return len(self.cams)

    @property
    def sample_bytes(self) -> int:
        return 1 if self.bit_depth <= 8 else 2

    @property
    def oob_penalty(self) -> int:
        return self.penalty if self.penalty >= 0 else 3 * ((1 << self.bit_depth) - 1)

    def neighbours(self, r: int) -> list[int]:
        if self.nbr_views is not None and r in self.nbr_views:
            return list(self.nbr_views[r])
        return [v for v in range(self.n_views) if v != r]

    def view(self, v: int, frame: int = 0, aux: bool = False) -> View:
        key = (v, frame, aux)
        if key not in self._views:
            paint = self.cams[self.paint_view] if self.paint_view is not None else None
            self._views[key] = render(self.cams[v], self.planes, bit_depth=self.bit_depth, frame=frame,
                                      noise_sigma=self.noise_sigma, specular_frac=self.specular_frac,
                                      noise_seed=self.seed * 1000003 + 7919 * v + 104729 * frame,
                                      chroma420=self.chroma420, paint=paint, aux=aux)
        return self._views[key]

    def views(self, frame: int = 0) -> list[View]:
        return [self.view(v, frame) for v in range(self.n_views)]

    def drop_frame(self, frame: int) -> None:
        for k in [k for k in self._views if k[1] == frame]:
            del self._views[k]

    def labels(self, r: int) -> tuple[np.ndarray, int]:
        """Label map of reference view r (static over frames) and its segment count."""
        if r not in self._labels:
            c = self.cams[r]
            self._labels[r] = grid_labels(c.width, c.height, self.cell, self.jitter, self.seed + 31 * r)
        return self._labels[r]

    def evaluations(self) -> int:
        """pixel x label x neighbour-view evaluations of one full cost-volume pass."""
        return sum(self.cams[r].width * self.cams[r].height * self.n_labels * len(self.neighbours(r))
                   for r in self.ref_views)


def _texel(z: float, f: float, px: float = 1.5) -> float:
    return px * z / f


def _tiny(seed: int, painted: bool = False) -> Workload:
    f, W, H = 400.0, 480, 270
    cams = linear_rig(3, 0.05, f, W, H)
    L, zn, zf = 64, 0.5, 10.0
    ref = cams[1]
    rng = np.random.default_rng(seed)
    mode = 1 if painted else 0
    # background: unbounded fronto-parallel plane on label 10; a bounded square on label 38. Both labels
    # are unambiguous for this rig: their rounded disparities differ from those of the adjacent labels.
    z_bg, z_fg = label_depth(10, L, zn, zf), label_depth(38, L, zn, zf)
    planes = [
        fronto_plane(ref, z_bg, 0.0, texel=_texel(z_bg, f), seed=seed + 1, mode=mode),
        fronto_plane(ref, z_fg, 0.22, centre_xy=(-0.18, -0.05), texel=_texel(z_fg, f), seed=seed + 2,
                     mode=mode),
        slanted_plane(ref, 1.6, float(rng.uniform(20, 40)), float(rng.uniform(0, 360)), 0.3,
                      centre_xy=(0.75, 0.1), texel=_texel(1.6, f), seed=seed + 3, mode=mode),
        slanted_plane(ref, 0.65, float(rng.uniform(20, 40)), float(rng.uniform(0, 360)), 0.08,
                      centre_xy=(0.12, 0.12), texel=_texel(0.65, f), seed=seed + 4, mode=mode),
    ]
    return Workload("tiny", cams, [1], L, zn, zf, 8, planes, cell=16, seed=seed,
                    paint_view=1 if painted else None, penalty=765)


def _layered(ref: Camera, f: float, n_planes: int, zmin: float, zmax: float, z_bg: float, seed: int,
             rng: np.random.Generator, mode: int = 0) -> list[Plane]:
    planes = [fronto_plane(ref, z_bg, 0.0, texel=_texel(z_bg, f), seed=seed + 1, mode=mode)]
    fov_x = ref.width / (2 * f)
    fov_y = ref.height / (2 * f)
    for k in range(1, n_planes):
        z = float(math.exp(rng.uniform(math.log(zmin), math.log(zmax))))
        cx = float(rng.uniform(-0.8, 0.8)) * fov_x * z
        cy = float(rng.uniform(-0.8, 0.8)) * fov_y * z
        half = float(rng.uniform(0.08, 0.22)) * fov_x * z
        if rng.uniform() < 0.4:
            planes.append(fronto_plane(ref, z, half, centre_xy=(cx, cy), texel=_texel(z, f),
                                       seed=seed + 1 + k, mode=mode))
        else:
            planes.append(slanted_plane(ref, z, float(rng.uniform(10, 40)), float(rng.uniform(0, 360)),
                                        half, centre_xy=(cx, cy), texel=_texel(z, f), seed=seed + 1 + k,
                                        mode=mode))
    return planes


def _hd8(seed: int, W: int = 1920, H: int = 1080, f: float = 1500.0, L: int = 250,
         refs: list[int] | None = None, name: str = "hd8") -> Workload:
    cams = linear_rig(8, 0.10, f, W, H)
    rng = np.random.default_rng(seed)
    ref = cams[3]
    planes = _layered(ref, f, 12, 1.5, 12.0, 18.0, seed, rng)
    return Workload(name, cams, refs if refs is not None else list(range(8)), L, 1.0, 20.0, 10, planes,
                    cell=10 if W >= 1920 else 8, seed=seed,
                    noise_sigma=2.0, chroma420=True)


def _uhd15(seed: int, W: int = 3840, H: int = 2160, f: float = 3000.0, L: int = 400,
           refs: list[int] | None = None, cell: int = 13, name: str = "uhd15") -> Workload:
    cams = arc_rig(15, 3.0, 8.0, f, W, H, seed)
    rng = np.random.default_rng(seed + 17)
    centre = cams[7]
    # depths measured from the centre camera, which sits 3 m from the arc centre
    planes = _layered(centre, f, 20, 1.5, 9.0, 12.0, seed, rng)
    return Workload(name, cams, refs if refs is not None else list(range(15)), L, 0.8, 15.0, 10, planes,
                    cell=cell, seed=seed, specular_frac=0.10)


def _temporal(seed: int, W: int = 1920, H: int = 1080, f: float = 1500.0, L: int = 250,
              refs: list[int] | None = None, n_frames: int = 30, name: str = "temporal") -> Workload:
    cams = linear_rig(8, 0.10, f, W, H)
    rng = np.random.default_rng(seed)
    ref = cams[3]
    planes = _layered(ref, f, 9, 4.0, 12.0, 18.0, seed, rng)
    # three textured foreground planes translating 4 px/frame in the image (world shift 4 z / f)
    fov_x, fov_y = W / (2 * f), H / (2 * f)
    for k, (z, a, b) in enumerate([(2.0, -0.55, -0.1), (2.6, 0.2, 0.35), (3.2, 0.6, -0.4)]):
        planes.append(Plane(p0=np.array([a * fov_x * z, b * fov_y * z, z]), e1=np.array([1.0, 0.0, 0.0]),
                            e2=np.array([0.0, 1.0, 0.0]), half1=0.107 * z, half2=0.107 * z,
                            texel=_texel(z, f), seed=seed + 100 + k,
                            velocity=np.array([4.0 * z / f, 0.0, 0.0])))
    wl = Workload(name, cams, refs if refs is not None else list(range(8)), L, 1.0, 20.0, 10, planes,
                  cell=10 if W >= 1920 else 8, seed=seed, noise_sigma=2.0,
                  chroma420=True, n_frames=n_frames)
    return wl


def _serving_small(seed: int) -> Workload:
    cams = linear_rig(3, 0.10, 750.0, 960, 540)
    rng = np.random.default_rng(seed)
    planes = _layered(cams[1], 750.0, 8, 1.5, 12.0, 18.0, seed, rng)
    return Workload("serving_small", cams, [0, 1, 2], 64, 1.0, 20.0, 10, planes, cell=10, seed=seed)


def _movers(cam: Camera, f: float, seed: int, coverage: float = 0.05) -> list[Plane]:
    """Three textured planes parallel to `cam`'s image plane that translate 4 px/frame along its x axis
    (world shift 4 z / f per frame), each covering about `coverage` of the image."""
    fov_x, fov_y = cam.width / (2 * f), cam.height / (2 * f)
    out = []
    for k, (z, a, b) in enumerate([(2.0, -0.55, -0.1), (2.6, 0.2, 0.35), (3.2, 0.6, -0.4)]):
        half = 0.5 * math.sqrt(coverage * 4 * fov_x * fov_y) * z
        p = fronto_plane(cam, z, half, centre_xy=(a * fov_x * z, b * fov_y * z), texel=_texel(z, f),
                         seed=seed + 100 + k)
        p.velocity = cam.R.T @ np.array([4.0 * z / f, 0.0, 0.0])
        out.append(p)
    return out


def serving_streams(per_shape: int = 4) -> list[Workload]:
    """Camera streams of the serving workload: per_shape streams of each of 960x540 / 3 views / 64 labels,
    1920x1080 / 8 views / 250 labels and 3840x2160 / 15 views / 400 labels (10-bit 4:4:4 in uint16),
    each a seeded plane scene with three moving planes and sensor noise (sigma 2 LSB), so that about
    15 % of the segments change from frame to frame."""
    streams = []
    for i in range(per_shape):
        seed = BASE_SEED + 4 + 1000 * (i + 1)
        cams = linear_rig(3, 0.10, 750.0, 960, 540)
        rng = np.random.default_rng(seed)
        planes = _layered(cams[1], 750.0, 8, 4.0, 12.0, 18.0, seed, rng) + _movers(cams[1], 750.0, seed)
        streams.append(Workload(f"s540_{i}", cams, [0, 1, 2], 64, 1.0, 20.0, 10, planes, cell=10, seed=seed,
                                noise_sigma=2.0))
    for i in range(per_shape):
        seed = BASE_SEED + 4 + 1000 * (i + 1) + 1
        streams.append(_temporal(seed, name=f"s1080_{i}"))
    for i in range(per_shape):
        seed = BASE_SEED + 4 + 1000 * (i + 1) + 2
        wl = _uhd15(seed, name=f"s2160_{i}")
        wl.planes = wl.planes + _movers(wl.cams[7], 3000.0, seed)
        wl.noise_sigma = 2.0
        wl.specular_frac = 0.0  # per-frame specular flicker would mark most segments as changed
        streams.append(wl)
    return streams


def serving_streams_reduced(per_shape: int = 1) -> list[Workload]:
    """The serving workload's three stream shapes at sizes the CPU oracle finishes in seconds (parity tests):
    per_shape streams each of a 3-view linear rig (320x180, 64 labels), an 8-view linear rig (244x138, 40
    labels, references 0, 3 and 7) and the 15-view convergent arc (390x218, 24 labels, references 0, 7
    and 14), each with moving planes and sensor noise, 10-bit 4:4:4 in uint16."""
    streams = []
    for i in range(per_shape):
        seed = BASE_SEED + 5 + 1000 * (i + 1)
        cams = linear_rig(3, 0.10, 250.0, 320, 180)
        rng = np.random.default_rng(seed)
        planes = _layered(cams[1], 250.0, 8, 4.0, 12.0, 18.0, seed, rng) + _movers(cams[1], 250.0, seed)
        streams.append(Workload(f"r540_{i}", cams, [0, 1, 2], 64, 1.0, 20.0, 10, planes, cell=8, seed=seed,
                                noise_sigma=2.0))
    for i in range(per_shape):
        seed = BASE_SEED + 5 + 1000 * (i + 1) + 1
        streams.append(_temporal(seed, W=244, H=138, f=190.0, L=40, refs=[0, 3, 7], name=f"r1080_{i}"))
    for i in range(per_shape):
        seed = BASE_SEED + 5 + 1000 * (i + 1) + 2
        wl = _uhd15(seed, W=390, H=218, f=304.0, L=24, refs=[0, 7, 14], cell=7, name=f"r2160_{i}")
        wl.planes = wl.planes + _movers(wl.cams[7], 304.0, seed)
        wl.noise_sigma = 2.0
        wl.specular_frac = 0.0
        streams.append(wl)
    return streams


def make_workload(name: str, reduced: bool = False, painted: bool = False) -> Workload:
    """Build a named workload. `reduced` gives a small variant of the same structure (rig type,
    bit depth, chroma handling, noise, all references) that the CPU oracle finishes in seconds while
    still spanning many kernel tiles with a ragged tail."""
    seed = BASE_SEED + (CONFIG_NAMES.index(name) if name in CONFIG_NAMES else 97)
    if name == "tiny":
        return _tiny(seed, painted=painted)
    if name == "hd8":
        if reduced:
            return _hd8(seed, W=244, H=138, f=190.0, L=40, name="hd8_reduced")
        return _hd8(seed)
    if name == "uhd15_half":  # the uhd15 rig and scene at 1920x1080 (profiling-sized)
        return _uhd15(BASE_SEED + 2, W=1920, H=1080, f=1500.0, cell=13, name="uhd15_half")
    if name == "uhd15":
        if reduced:
            return _uhd15(seed, W=390, H=218, f=304.0, L=48, refs=[0, 7, 14], cell=7, name="uhd15_reduced")
        return _uhd15(seed)
    if name == "temporal":
        if reduced:
            return _temporal(seed, W=244, H=138, f=190.0, L=40, n_frames=4, name="temporal_reduced")
        return _temporal(seed)
    if name == "serving_small":
        return _serving_small(seed)
    raise KeyError(name)
