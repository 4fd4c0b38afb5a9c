"""The seeded input generator (no denoiser arithmetic): determinism, the noise model's mean,
the roughness options, the moving light and the shadow channel's statistics."""
import numpy as np
import pytest

from paper_2312_06827_gb300 import scene

STATIC = dict(n_spheres=10, moving_sphere=False, pan_px_per_frame=0.0, seed=5)


def test_frames_are_deterministic_and_noise_changes_per_frame():
    sc = scene.SceneConfig(64, 48, **STATIC)
    a, b = scene.render_frame(sc, 3), scene.render_frame(sc, 3)
    assert all(np.array_equal(a[k], b[k]) for k in a)
    c = scene.render_frame(sc, 4)
    assert np.array_equal(a["gt"], c["gt"]) and not np.array_equal(a["noisy"], c["noisy"])
    assert np.abs(c["motion"]).max() < 1e-9      # static camera and objects (re-projection rounding only)


def test_noise_has_unit_mean_factor():
    sc = scene.SceneConfig(48, 32, **STATIC)
    gt = scene.render_frame(sc, 0, want=("gt",))["gt"].astype(np.float64)
    acc = np.zeros_like(gt)
    n = 400
    for t in range(n):
        acc += scene.render_frame(sc, t, want=("noisy",))["noisy"]
    ok = (gt > 0.01) & (gt < 0.5)              # far from the HDR clamp
    ratio = (acc / n)[ok] / gt[ok]
    assert abs(ratio.mean() - 1.0) < 0.02       # Exp(1): mean 1, std 1 -> 0.05 per pixel
    assert 0.8 < np.std(ratio) * np.sqrt(n) < 1.2


def test_roughness_override_and_roughness_scaled_noise():
    sc = scene.SceneConfig(64, 48, roughness=0.0, rough_noise=True, **STATIC)
    fr = scene.render_frame(sc, 1, want=("noisy", "gt", "roughness"))
    assert np.all(fr["roughness"] == 0.0)
    assert np.array_equal(fr["noisy"], fr["gt"])    # a mirror-smooth surface is noise-free
    sc = scene.SceneConfig(64, 48, roughness=0.5, rough_noise=True, **STATIC)
    half = scene.render_frame(sc, 1, want=("noisy", "gt"))
    full = scene.render_frame(scene.SceneConfig(64, 48, roughness=0.5, **STATIC), 1, want=("noisy", "gt"))
    ok = (half["gt"] > 0.01) & (full["noisy"] < 19.0)
    # factor 1 + r (e - 1) against e: half the deviation from the noise-free value
    assert np.allclose((half["noisy"] - half["gt"])[ok], 0.5 * (full["noisy"] - full["gt"])[ok], rtol=1e-5, atol=1e-6)


def test_moving_light_changes_shading_only():
    sc = scene.SceneConfig(64, 48, moving_light=True, **STATIC)
    a, b = scene.render_frame(sc, 0), scene.render_frame(sc, 10)
    assert np.array_equal(a["gbuf_nz"], b["gbuf_nz"]) and np.abs(b["motion"]).max() < 1e-9
    assert not np.array_equal(a["gt"], b["gt"])
    still = scene.SceneConfig(64, 48, **STATIC)
    assert np.array_equal(scene.render_frame(still, 0)["gt"], scene.render_frame(still, 10)["gt"])


def test_shadow_channel_statistics():
    sc = scene.SceneConfig(64, 48, **STATIC)
    s = scene.render_frame(sc, 0, want=("shadow_noisy", "shadow_gt", "shadow_angle"))
    assert set(np.unique(s["shadow_noisy"])) <= {0.0, 1.0}
    assert np.all((s["shadow_gt"] >= 0) & (s["shadow_gt"] <= 1))
    assert np.allclose(s["shadow_gt"] * 64, np.round(s["shadow_gt"] * 64), atol=1e-4)   # 8 x 8 samples
    assert 0.0 < s["shadow_angle"].min() and s["shadow_angle"].max() < 180.0
    pen = (s["shadow_gt"] > 0) & (s["shadow_gt"] < 1)
    assert pen.mean() > 0.005                   # the spherical light casts penumbrae
    acc = np.zeros(s["shadow_gt"].shape)
    n = 300
    for t in range(n):
        acc += scene.render_frame(sc, t, want=("shadow_noisy",))["shadow_noisy"]
    # the 1-sample estimate is unbiased for the disk's visible fraction (the 64-sample
    # stratified value stands in for it): 5 binomial sigmas plus the stratification error
    p = s["shadow_gt"]
    assert np.all(np.abs(acc / n - p) <= 5 * np.sqrt(p * (1 - p) / n) + 0.05)
    big = scene.render_frame(scene.SceneConfig(64, 48, light_radius=1.5, **STATIC), 0, want=("shadow_angle",))
    assert np.all(big["shadow_angle"] > s["shadow_angle"])


def test_shadow_channel_rejects_point_light():
    with pytest.raises(ValueError):
        scene.render_frame(scene.SceneConfig(16, 16, light_radius=0.0), 0, want=("shadow_gt",))
