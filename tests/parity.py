"""Helpers for the GPU-vs-oracle parity tests (not a test module).

Tolerances:
  * FP32 path, colour: max relative error 1e-5 in tone-mapped space,
    rel = |g - o| / max(|o|, 1e-3), where g and o are mapped by the FP64 forward tone map when
    the pipeline tone-maps (the inverse map amplifies FP32 rounding by up to 1/(1 - luma) ~ 21x
    at HDR 20 and the forward map takes that back out).
  * Variance: |g - o| / max(|o|, l^2) <= VAR_TOL, l the luminance of the (tone-mapped) colour
    of the same pixel.  The variance is a difference of second moments, mu2 - mu1^2, so FP32
    cancellation leaves an absolute error of order eps * l^2 however small the variance is; after
    five a-trous passes it is ~1e-6 l^2 and a plain relative error would measure only that
    cancellation.
  * Decision-flip candidates (oracle margin < 1e-5 in a reprojection threshold test) must be at
    most 0.01 % of the pixels; the pixels within their influence radius are excluded from the
    bound (their error is reported separately).
"""
from __future__ import annotations

import numpy as np
from scipy import ndimage

import oracle

COLOUR_TOL = 1e-5
VAR_TOL = 1e-5
LUMA = np.array([0.2126, 0.7152, 0.0722])
MARGIN = 1e-5


def oracle_config(c) -> oracle.OracleConfig:
    """The oracle's configuration with the GPU config's FP32 values (so that thresholds are the
    same numbers on both sides)."""
    f32 = lambda v: float(np.float32(v))
    return oracle.OracleConfig(
        alpha=f32(c.alpha), alpha_moments=f32(c.alpha_moments), clamp_gamma=f32(c.clamp_gamma),
        atrous_iters=c.atrous_iters, sigma_z=f32(c.sigma_z), sigma_n=f32(c.sigma_n),
        sigma_l=f32(c.sigma_l), separable=c.spatial_mode == 1, clamp_enable=bool(c.clamp_enable),
        adaptive_start=bool(c.adaptive_start), roughness_threshold=f32(c.roughness_threshold),
        tonemap=bool(c.tonemap), luma_k=f32(c.luma_k), inv_weight=f32(c.inv_weight),
        inverse_mode=c.inverse_mode, history_from_pass=c.history_from_pass,
        depth_rel_tol=f32(c.depth_rel_tol), normal_cos_tol=f32(c.normal_cos_tol),
        disocclusion_weight=f32(c.disocclusion_weight), max_history=c.max_history,
        min_temporal_frames=c.min_temporal_frames, spatial_var_radius=c.spatial_var_radius,
        eps=f32(c.eps), rectify_mode=c.rectify_mode, iter_by_roughness=bool(c.iter_by_roughness),
        iter_rough_t0=f32(c.iter_rough_t0), iter_rough_t1=f32(c.iter_rough_t1),
        iter_count0=c.iter_count0, iter_count1=c.iter_count1)


def influence_radius(c) -> int:
    """Pixels a changed input can reach through the temporal 7x7 window and the a-trous passes."""
    r = max(3, c.spatial_var_radius) + 1
    lvl = 1 if c.adaptive_start else 0
    for i in range(c.atrous_iters):
        r += 2 * (1 << (i + lvl)) + 1
    return r


def flip_candidates(margin: np.ndarray) -> np.ndarray:
    return margin < MARGIN


def excluded_mask(flags: np.ndarray, c) -> np.ndarray:
    if not flags.any():
        return flags
    r = influence_radius(c)
    return ndimage.binary_dilation(flags, structure=np.ones((3, 3), bool), iterations=r)


def tm64(rgb, c):
    rgb = np.asarray(rgb, np.float64)
    if not c.tonemap:
        return rgb
    return oracle.tonemap(rgb.reshape(-1, 3), oracle_config(c)).reshape(rgb.shape)


def colour_err(g, o, c=None, mapped=False):
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    if mapped:
        g, o = tm64(g, c), tm64(o, c)
    return np.abs(g - o) / np.maximum(np.abs(o), 1e-3)


def var_err(g, o, rgb_tm):
    """rgb_tm: the oracle's tone-mapped colour of the same pixels (sets the l^2 scale)."""
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    l2 = (np.asarray(rgb_tm, np.float64) @ LUMA) ** 2
    return np.abs(g - o) / np.maximum(np.maximum(np.abs(o), l2), 1e-12)


def report(name, cerr, verr, flags, excl):
    keep = ~excl
    ce = float(cerr[keep].max()) if keep.any() else 0.0
    ve = float(verr[keep].max()) if keep.any() else 0.0
    frac = float(flags.mean())
    inside = f", in excluded zone {float(cerr[excl].max()):.3e}" if excl.any() else ""
    print(f"[parity] {name}: colour max rel {ce:.3e}, variance max rel {ve:.3e}, "
          f"flip candidates {int(flags.sum())} ({frac:.2e}){inside}")
    return ce, ve, frac
