"""FP64 CPU oracle of the variance-guided denoiser (ctypes wrapper over ``svgf_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()`` and by the
benchmark's CPU-baseline leg, never by the product path.  It shares no code with the CUDA
library.  All arrays are converted to C-contiguous float64 before the call.

Functions follow the paper's stages (section numbers of "Hybrid-Rendering Techniques in GPU"):
``tonemap`` / ``inverse_tonemap`` (Sec. 3.4), ``clamp`` (Sec. 3.1), ``reproject`` and
``temporal`` (Sec. 2, Sec. 3 step 4), ``atrous`` (Sec. 2 Fig. 1, Sec. 3 step 5, Sec. 3.2,
Sec. 3.3), ``denoise_frame`` / ``Sequence`` (the whole frame).  The whole-frame composition is
pinned by its closed form with the edge functions off on a static scene (the history is the
pass-0 output, the output the inverse map of the last pass).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading
from pathlib import Path

import numpy as np

_DIR = Path(__file__).resolve().parent
_SRC = _DIR / "svgf_oracle.c"
_LIB = _DIR / "liboracle.so"
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> Path:
    if force or not _LIB.exists() or _SRC.stat().st_mtime > _LIB.stat().st_mtime:
        tmp = _LIB.with_suffix(f".tmp{os.getpid()}.so")
        cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               "-o", str(tmp), str(_SRC), "-lm"]
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stdout)
        os.replace(tmp, _LIB)
    return _LIB


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("alpha", ctypes.c_double), ("alpha_moments", ctypes.c_double),
        ("clamp_gamma", ctypes.c_double), ("atrous_iters", ctypes.c_int),
        ("sigma_z", ctypes.c_double), ("sigma_n", ctypes.c_double), ("sigma_l", ctypes.c_double),
        ("separable", ctypes.c_int), ("clamp_enable", ctypes.c_int),
        ("adaptive_start", ctypes.c_int), ("roughness_threshold", ctypes.c_double),
        ("tonemap", ctypes.c_int), ("luma_k", ctypes.c_double), ("inv_weight", ctypes.c_double),
        ("inverse_mode", ctypes.c_int), ("history_from_pass", ctypes.c_int),
        ("depth_rel_tol", ctypes.c_double), ("normal_cos_tol", ctypes.c_double),
        ("disocclusion_weight", ctypes.c_double), ("max_history", ctypes.c_int),
        ("min_temporal_frames", ctypes.c_int), ("spatial_var_radius", ctypes.c_int),
        ("eps", ctypes.c_double), ("rectify_mode", ctypes.c_int),
        ("iter_by_roughness", ctypes.c_int), ("iter_rough_t0", ctypes.c_double),
        ("iter_rough_t1", ctypes.c_double), ("iter_count0", ctypes.c_int),
        ("iter_count1", ctypes.c_int),
    ]


@dataclasses.dataclass
class OracleConfig:
    alpha: float = 0.2
    alpha_moments: float = 0.2
    clamp_gamma: float = 1.0
    atrous_iters: int = 5
    sigma_z: float = 1.0
    sigma_n: float = 128.0
    sigma_l: float = 4.0
    separable: bool = False
    clamp_enable: bool = True
    adaptive_start: bool = True
    roughness_threshold: float = 0.2
    tonemap: bool = True
    luma_k: float = 1.0
    inv_weight: float = 1.0
    inverse_mode: int = 0          # 0 exact, 1 paper-literal
    history_from_pass: int = 0
    depth_rel_tol: float = 0.1
    normal_cos_tol: float = 0.9
    disocclusion_weight: float = 1e-4
    max_history: int = 255
    min_temporal_frames: int = 4
    spatial_var_radius: int = 3
    eps: float = 1e-10
    rectify_mode: int = 0          # 0 variance colour clamping, 1 variance colour clipping
    iter_by_roughness: bool = False
    iter_rough_t0: float = 0.0
    iter_rough_t1: float = 0.05
    iter_count0: int = 0
    iter_count1: int = 1

    def _c(self) -> _Cfg:
        return _Cfg(
            float(self.alpha), float(self.alpha_moments), float(self.clamp_gamma),
            int(self.atrous_iters), float(self.sigma_z), float(self.sigma_n), float(self.sigma_l),
            int(self.separable), int(self.clamp_enable), int(self.adaptive_start),
            float(self.roughness_threshold), int(self.tonemap), float(self.luma_k),
            float(self.inv_weight), int(self.inverse_mode), int(self.history_from_pass),
            float(self.depth_rel_tol), float(self.normal_cos_tol), float(self.disocclusion_weight),
            int(self.max_history), int(self.min_temporal_frames), int(self.spatial_var_radius),
            float(self.eps), int(self.rectify_mode), int(self.iter_by_roughness),
            float(self.iter_rough_t0), float(self.iter_rough_t1), int(self.iter_count0),
            int(self.iter_count1))


_D = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(str(build()))
            i, l, P, C = ctypes.c_int, ctypes.c_long, _D, ctypes.POINTER(_Cfg)
            sig = {
                "ora_threads": ([], i),
                "ora_luma": ([P], ctypes.c_double),
                "ora_atrous_taps": ([i], i),
                "ora_tonemap": ([l, P, P, C], None),
                "ora_inverse_tonemap": ([l, P, P, C], None),
                "ora_depth_gradient": ([i, i, P, P], None),
                "ora_atrous_5x5": ([i, i, i, P, P, P, P, C], None),
                "ora_atrous_separable": ([i, i, i, P, P, P, P, C], None),
                "ora_atrous": ([i, i, i, P, P, P, P, C], None),
                "ora_clamp": ([i, i, P, P, P, C], None),
                "ora_reproject": ([i, i, P, P, P, P, P, i, P, P, P, P, C], None),
                "ora_temporal": ([i, i, P, P, P, P, P, P, i, P, P, P, C], None),
                "ora_denoise_frame": ([i, i, P, P, P, P, P, P, P, i, P, P, P, P, C], None),
                "ora_kpn_param_count": ([], i),
                "ora_kpn_forward": ([i, i, i, P, P, P, P, P, P], None),
                "ora_kpn_forward_q": ([i, i, i, P, P, P, P, P, P, i], None),
                "ora_kpn_loss": ([i, i, i, P, P, P, P], ctypes.c_double),
                "ora_kpn_grad": ([i, i, i, P, P, P, P, P], ctypes.c_double),
                "ora_kpn_grad_q": ([i, i, i, P, P, P, P, P, i], ctypes.c_double),
                "ora_bf16_round": ([l, P, P], None),
                "ora_kpn_features": ([i, i, P, P, P, P], None),
                "ora_kpn_conv": ([i, i, i, P, i, P, P, i, P], None),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != tuple(shape):
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def _p(a):
    return None if a is None else a.ctypes.data_as(_D)


def luma(rgb) -> np.ndarray:
    rgb = _f64(rgb)
    flat = rgb.reshape(-1, 3)
    return np.array([lib().ora_luma(_p(np.ascontiguousarray(flat[i]))) for i in range(flat.shape[0])]
                    ).reshape(rgb.shape[:-1])


def threads() -> int:
    """OpenMP threads the oracle's loops run on."""
    return lib().ora_threads()


def atrous_taps(separable: bool) -> int:
    return lib().ora_atrous_taps(int(separable))


def tonemap(rgb, cfg: OracleConfig = None):
    cfg = cfg or OracleConfig()
    a = _f64(rgb)
    out = np.empty_like(a)
    lib().ora_tonemap(a.size // 3, _p(a), _p(out), ctypes.byref(cfg._c()))
    return out


def inverse_tonemap(rgb, cfg: OracleConfig = None):
    cfg = cfg or OracleConfig()
    a = _f64(rgb)
    out = np.empty_like(a)
    lib().ora_inverse_tonemap(a.size // 3, _p(a), _p(out), ctypes.byref(cfg._c()))
    return out


def depth_gradient(gbuf):
    g = _f64(gbuf)
    H, W = g.shape[:2]
    out = np.empty((H, W, 2))
    lib().ora_depth_gradient(W, H, _p(g), _p(out))
    return out


def atrous(cv, gbuf, roughness, it: int, cfg: OracleConfig = None, mode: str = None):
    """One a-trous iteration. mode: None (per cfg.separable), '5x5' or 'separable'."""
    cfg = cfg or OracleConfig()
    cv = _f64(cv)
    H, W = cv.shape[:2]
    g = _f64(gbuf, (H, W, 4))
    r = _f64(roughness, (H, W)) if roughness is not None else None
    out = np.empty((H, W, 4))
    fn = {None: lib().ora_atrous, "5x5": lib().ora_atrous_5x5,
          "separable": lib().ora_atrous_separable}[mode]
    fn(W, H, int(it), _p(cv), _p(g), _p(r), _p(out), ctypes.byref(cfg._c()))
    return out


def clamp(cur_tm, hist, cfg: OracleConfig = None):
    cfg = cfg or OracleConfig()
    c = _f64(cur_tm)
    H, W = c.shape[:2]
    h = _f64(hist, (H, W, 3))
    out = np.empty((H, W, 3))
    lib().ora_clamp(W, H, _p(c), _p(h), _p(out), ctypes.byref(cfg._c()))
    return out


def reproject(gbuf, prev_gbuf, motion, hist_rgb, hist_mom, has_history=True, cfg: OracleConfig = None):
    cfg = cfg or OracleConfig()
    g = _f64(gbuf)
    H, W = g.shape[:2]
    pg = _f64(prev_gbuf, (H, W, 4)) if prev_gbuf is not None else None
    mv = _f64(motion, (H, W, 2))
    hr = _f64(hist_rgb, (H, W, 3))
    hm = _f64(hist_mom, (H, W, 3))
    rgb, mom, valid, margin = np.empty((H, W, 3)), np.empty((H, W, 3)), np.empty((H, W)), np.empty((H, W))
    lib().ora_reproject(W, H, _p(g), _p(pg), _p(mv), _p(hr), _p(hm), int(bool(has_history)),
                        _p(rgb), _p(mom), _p(valid), _p(margin), ctypes.byref(cfg._c()))
    return rgb, mom, valid.astype(bool), margin


def temporal(noisy, gbuf, prev_gbuf, motion, hist_rgb, hist_mom, has_history=True,
             cfg: OracleConfig = None):
    """Returns (cv [H,W,4] = accumulated colour + variance, moments [H,W,3], margin [H,W])."""
    cfg = cfg or OracleConfig()
    nz = _f64(noisy)
    H, W = nz.shape[:2]
    g = _f64(gbuf, (H, W, 4))
    pg = _f64(prev_gbuf, (H, W, 4)) if prev_gbuf is not None else None
    mv = _f64(motion, (H, W, 2))
    hr = _f64(hist_rgb, (H, W, 3)) if hist_rgb is not None else np.zeros((H, W, 3))
    hm = _f64(hist_mom, (H, W, 3)) if hist_mom is not None else np.zeros((H, W, 3))
    cv, mom, margin = np.empty((H, W, 4)), np.empty((H, W, 3)), np.empty((H, W))
    lib().ora_temporal(W, H, _p(nz), _p(g), _p(pg), _p(mv), _p(hr), _p(hm), int(bool(has_history)),
                       _p(cv), _p(mom), _p(margin), ctypes.byref(cfg._c()))
    return cv, mom, margin


class Sequence:
    """Runs the oracle frame by frame, holding the temporal state (colour history, moments and
    the previous G-buffer) the way a renderer would."""

    def __init__(self, width: int, height: int, cfg: OracleConfig = None):
        self.W, self.H = width, height
        self.cfg = cfg or OracleConfig()
        self.reset()

    def reset(self):
        self.hist_rgb = np.zeros((self.H, self.W, 3))
        self.hist_mom = np.zeros((self.H, self.W, 3))
        self.prev_gbuf = None
        self.has_history = False

    def step(self, noisy, gbuf, motion, roughness):
        H, W = self.H, self.W
        nz = _f64(noisy, (H, W, 3))
        g = _f64(gbuf, (H, W, 4))
        mv = _f64(motion, (H, W, 2))
        r = _f64(roughness, (H, W))
        hr_next, hm_next = np.empty((H, W, 3)), np.empty((H, W, 3))
        out, margin = np.empty((H, W, 4)), np.empty((H, W))
        lib().ora_denoise_frame(W, H, _p(nz), _p(g), _p(self.prev_gbuf), _p(mv), _p(r),
                                _p(self.hist_rgb), _p(self.hist_mom), int(self.has_history),
                                _p(hr_next), _p(hm_next), _p(out), _p(margin),
                                ctypes.byref(self.cfg._c()))
        self.hist_rgb, self.hist_mom, self.prev_gbuf = hr_next, hm_next, g
        self.has_history = True
        self.margin = margin
        return out


# ----------------------------------------------------------------------- learned part

KPN_CIN = (10, 32, 32, 32)
KPN_COUT = (32, 32, 32, 25)


def kpn_param_count() -> int:
    return lib().ora_kpn_param_count()


def kpn_unflatten(params):
    """Flat parameters -> [(W [co, 9, ci], b [co]) for the 4 layers]."""
    out, k = [], 0
    for ci, co in zip(KPN_CIN, KPN_COUT):
        w = np.asarray(params[k:k + co * 9 * ci]).reshape(co, 9, ci)
        k += co * 9 * ci
        b = np.asarray(params[k:k + co])
        k += co
        out.append((w, b))
    return out


def bf16_round(a):
    """Each value rounded to FP32 and then to the nearest BF16 (ties to even), as float64."""
    x = _f64(a)
    out = np.empty_like(x)
    lib().ora_bf16_round(x.size, _p(x), _p(out))
    return out


def kpn_forward(feat, c0, params, quant: bool = False):
    """feat [B, H, W, 10], c0 [B, H, W, 3] -> (K [B, H, W, 25], c1, c2 [B, H, W, 3]).
    quant: BF16 weights, activations (the rounding mode of the tensor-core path), FP64 sums."""
    f = _f64(feat)
    B, H, W = f.shape[:3]
    c = _f64(c0, (B, H, W, 3))
    prm = _f64(params, (kpn_param_count(),))
    K, c1, c2 = np.empty((B, H, W, 25)), np.empty((B, H, W, 3)), np.empty((B, H, W, 3))
    lib().ora_kpn_forward_q(B, H, W, _p(f), _p(c), _p(prm), _p(K), _p(c1), _p(c2), int(bool(quant)))
    return K, c1, c2


def kpn_loss(feat, c0, target, params) -> float:
    f = _f64(feat)
    B, H, W = f.shape[:3]
    return lib().ora_kpn_loss(B, H, W, _p(f), _p(_f64(c0, (B, H, W, 3))), _p(_f64(target, (B, H, W, 3))),
                              _p(_f64(params, (kpn_param_count(),))))


def kpn_grad(feat, c0, target, params, quant: bool = False):
    """(loss, flat gradient) of the mean squared error of c2 against target.  quant: BF16 weights,
    activations and data gradients (the rounding mode of the tensor-core path), FP64 sums."""
    f = _f64(feat)
    B, H, W = f.shape[:3]
    g = np.empty(kpn_param_count())
    loss = lib().ora_kpn_grad_q(B, H, W, _p(f), _p(_f64(c0, (B, H, W, 3))), _p(_f64(target, (B, H, W, 3))),
                                _p(_f64(params, (kpn_param_count(),))), _p(g), int(bool(quant)))
    return loss, g


def kpn_features(cv, gbuf, albedo):
    """cv [H, W, 4] (pass-0 tone-mapped colour and variance), gbuf [H, W, 4], albedo [H, W, 3]
    -> features [H, W, 10]."""
    c = _f64(cv)
    H, W = c.shape[:2]
    f = np.empty((H, W, 10))
    lib().ora_kpn_features(W, H, _p(c), _p(_f64(gbuf, (H, W, 4))), _p(_f64(albedo, (H, W, 3))), _p(f))
    return f


def kpn_conv(x, w, b):
    """One 3x3 layer: x [B, H, W, ci], w [co, 9, ci], b [co] -> z [B, H, W, co] (zero padding)."""
    xx = _f64(x)
    B, H, W, ci = xx.shape
    ww = _f64(w)
    co = ww.shape[0]
    z = np.empty((B, H, W, co))
    lib().ora_kpn_conv(B, H, W, _p(xx), ci, _p(ww), _p(_f64(b, (co,))), co, _p(z))
    return z
