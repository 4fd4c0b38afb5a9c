"""Helpers for the GPU-vs-oracle parity tests (not a test module).

Tolerances:
  * FP32 path, colour: max relative error 1e-5 in tone-mapped space,
    rel = |g - o| / max(|o|, 1e-3), where g and o are mapped by the FP64 forward tone map when
    the pipeline tone-maps (the inverse map amplifies FP32 rounding by up to 1/(1 - luma) ~ 21x
    at HDR 20 and the forward map takes that back out).
  * Variance, one stage given the oracle's input: relative to the value itself,
    |g - o| / max(|o|, 1e-10 l^2) <= VAR_TOL = 1e-5, l the luminance of the (tone-mapped) colour
    of the same pixel.  The floor only catches variances the FP64 oracle computes as a
    cancelling difference of equal moments (of order 1e-16 l^2 where the GPU's central-form
    moments give 0); the scenes' variances lie orders of magnitude above it (median ~1e-5 l^2
    after the fifth pass).
  * Variance of the temporal stage (the moment difference for n >= 4, the 7x7 weighted estimate
    for n < 4): |g - o| <= VAR_TOL |o| + 8 u l sqrt(|o|), u = 2^-24.  The estimate is a weighted
    variance of FP32 luminances, each carrying up to ~3 u l of rounding the FP64 oracle does not
    have; a perturbation d of the samples moves a weighted variance v by at most 2 sqrt(v) max|d|
    (Cauchy-Schwarz), so no FP32 evaluation can be value-relative where v is near (u l)^2.  The
    a-trous passes (positive weighted sums, no such difference) keep the plain value-relative bar.
  * Variance at the end of a free-running sequence (each side carrying its own history and
    passes): SEQ_VAR_TOL = 5e-5, same measure.  The luminance weights of a pass have the
    sensitivity |d log w / d l| = 1 / (sigma_l sqrt(g(var))), which in the last pass is about
    l / (4 * 3.7e-3 l), i.e. ~70 per unit of relative colour change; the ~1e-7 relative colour
    differences the stages legitimately carry forward in FP32 therefore reach the final
    variance at ~1e-5 (measured up to 1.6e-5 at 1080p).
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
SEQ_VAR_TOL = 5e-5
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
    """Relative variance error, |g - o| / max(|o|, 1e-10 l^2); rgb_tm: the oracle's tone-mapped
    colour of the same pixels (l)."""
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    l2 = (np.asarray(rgb_tm, np.float64) @ LUMA) ** 2
    return np.abs(g - o) / np.maximum(np.maximum(np.abs(o), 1e-10 * l2), 1e-30)


U32 = 2.0 ** -24


def var_err_est(g, o, rgb_tm):
    """Variance error of the temporal stage's estimate, scaled so that <= VAR_TOL is the bound
    |g - o| <= VAR_TOL |o| + 8 u l sqrt(|o|)."""
    g = np.asarray(g, np.float64)
    o = np.abs(np.asarray(o, np.float64))
    l = np.abs(np.asarray(rgb_tm, np.float64) @ LUMA)
    return np.abs(g - o) / np.maximum(o + 8 * U32 * l * np.sqrt(o) / VAR_TOL, 1e-30)


def var_err_l2(g, o, rgb_tm):
    """Variance error on the l^2 scale, |g - o| / max(|o|, l^2): for the binary shadow channel,
    whose collapsed variances (1e-10 and below) carry the FP32 exponent-underflow error its own
    bar accounts for."""
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
