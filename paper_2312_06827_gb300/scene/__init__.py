"""Seeded synthetic scenes (inputs only; no denoiser arithmetic).

``render_frame(cfg, t)`` returns one frame of the procedural scene as FP32 numpy arrays:

=============  ==============  ==================================================
key            shape           meaning
=============  ==============  ==================================================
``noisy``      [H, W, 3]       radiance x Exp(1) per pixel, clamped to [0, 20]
``gt``         [H, W, 3]       noise-free radiance (same clamp)
``gbuf_nz``    [H, W, 4]       world unit normal (xyz) + linear view-axis depth
``motion``     [H, W, 2]       p_cur - p_prev in pixels
``roughness``  [H, W]          per object, never within 0.01 of 0.2
``albedo``     [H, W, 3]       per object, U[0.1, 0.9]
``shadow_*``   [H, W]          shadow channel of a spherical light: 1-sample visibility
                               (``shadow_noisy``), 64-sample visibility (``shadow_gt``),
                               the light's angular diameter in degrees (``shadow_angle``)
=============  ==============  ==================================================

Options: ``roughness`` (one value for every surface), ``rough_noise`` (noise amplitude scaled
by the roughness), ``moving_light`` (the light circles), ``light_radius`` (shadow channel).

The named workloads below are the denoiser's test and benchmark scenes: 6 spheres at 128x128
with a 0.5 px/frame pan; 40 spheres with one sphere moving 8 px/frame at 1080p and 4K; and the
32-stream uneven-resolution batch (8 streams each of 640x360, 1280x720, 1920x1080, 2560x1440,
per-stream seeds 1..32).
"""
from __future__ import annotations

import ctypes
import dataclasses
import threading

import numpy as np

from .. import _build

_lib = None
_lock = threading.Lock()


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_int), ("height", ctypes.c_int), ("n_spheres", ctypes.c_int),
        ("moving_sphere", ctypes.c_int), ("pan_px_per_frame", ctypes.c_double),
        ("moving_px_per_frame", ctypes.c_double), ("vfov_deg", ctypes.c_double),
        ("max_radiance", ctypes.c_double), ("seed", ctypes.c_uint64), ("stream", ctypes.c_uint64),
        ("roughness", ctypes.c_double), ("rough_noise", ctypes.c_int), ("moving_light", ctypes.c_int),
        ("light_radius", ctypes.c_double),
    ]


@dataclasses.dataclass(frozen=True)
class SceneConfig:
    width: int
    height: int
    n_spheres: int = 6
    moving_sphere: bool = False
    pan_px_per_frame: float = 0.5
    moving_px_per_frame: float = 8.0
    vfov_deg: float = 45.0
    max_radiance: float = 20.0
    seed: int = 0
    stream: int = 0
    roughness: float = -1.0          # < 0: drawn per object; else every surface's roughness
    rough_noise: bool = False        # noise factor 1 + roughness (Exp(1) - 1)
    moving_light: bool = False       # the light circles over the scene
    light_radius: float = 0.75       # spherical light of the shadow channel

    @property
    def pixels(self) -> int:
        return self.width * self.height


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build_scene()
            L = ctypes.CDLL(str(path))
            fp = ctypes.POINTER(ctypes.c_float)
            L.scene_render_frame.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_int, fp, fp, fp, fp, fp, fp]
            L.scene_render_frame.restype = ctypes.c_int
            L.scene_render_shadow.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_int, fp, fp, fp]
            L.scene_render_shadow.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


SHADOW_KEYS = ("shadow_noisy", "shadow_gt", "shadow_angle")


def _c(cfg: SceneConfig) -> _Cfg:
    return _Cfg(cfg.width, cfg.height, cfg.n_spheres, int(cfg.moving_sphere), cfg.pan_px_per_frame,
                cfg.moving_px_per_frame, cfg.vfov_deg, cfg.max_radiance, cfg.seed, cfg.stream,
                float(cfg.roughness), int(cfg.rough_noise), int(cfg.moving_light), float(cfg.light_radius))


def render_frame(cfg: SceneConfig, frame: int, want=("noisy", "gt", "gbuf_nz", "motion", "roughness", "albedo")):
    H, W = cfg.height, cfg.width
    shapes = {"noisy": (H, W, 3), "gt": (H, W, 3), "gbuf_nz": (H, W, 4), "motion": (H, W, 2),
              "roughness": (H, W), "albedo": (H, W, 3), "shadow_noisy": (H, W), "shadow_gt": (H, W),
              "shadow_angle": (H, W)}
    out = {k: np.empty(shapes[k], np.float32) for k in want}
    c = _c(cfg)
    main = [k for k in want if k not in SHADOW_KEYS]
    if main or not want:
        rc = lib().scene_render_frame(ctypes.byref(c), int(frame), _ptr(out.get("noisy")), _ptr(out.get("gt")),
                                      _ptr(out.get("gbuf_nz")), _ptr(out.get("motion")),
                                      _ptr(out.get("roughness")), _ptr(out.get("albedo")))
        if rc != 0:
            raise ValueError(f"scene_render_frame rejected {cfg}")
    if any(k in SHADOW_KEYS for k in want):
        rc = lib().scene_render_shadow(ctypes.byref(c), int(frame), _ptr(out.get("shadow_noisy")),
                                       _ptr(out.get("shadow_gt")), _ptr(out.get("shadow_angle")))
        if rc != 0:
            raise ValueError(f"scene_render_shadow rejected {cfg}")
    return out


def sequence(cfg: SceneConfig, n_frames: int, want=("noisy", "gbuf_nz", "motion", "roughness")):
    return [render_frame(cfg, t, want) for t in range(n_frames)]


# Named workloads (sizes, sphere counts, motion and seeds of the denoiser's test/bench scenes).
C0_128 = SceneConfig(128, 128, n_spheres=6, moving_sphere=False, seed=0)
C1_1080P = SceneConfig(1920, 1080, n_spheres=40, moving_sphere=True, seed=0)
C2_4K = SceneConfig(3840, 2160, n_spheres=40, moving_sphere=True, seed=0)
C0_FRAMES, C1_FRAMES, C2_FRAMES, C3_FRAMES = 4, 60, 30, 16


def batch_streams():
    """The 32 uneven streams: 8 each of 640x360, 1280x720, 1920x1080, 2560x1440, seeds 1..32."""
    sizes = [(640, 360), (1280, 720), (1920, 1080), (2560, 1440)]
    out = []
    for i in range(32):
        w, h = sizes[i // 8]
        out.append(SceneConfig(w, h, n_spheres=40, moving_sphere=True, seed=1 + i, stream=i))
    return out
