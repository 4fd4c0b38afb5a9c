"""Pins of the ablation's metric (SSIM of Wang et al. 2004 with a Gaussian window, PSNR, the
display luma) by closed forms and a brute-force window loop; a small GPU run of the ablation."""
import math

import numpy as np
import pytest

from paper_2312_06827_gb300 import ablation

RNG = np.random.default_rng(12)


def test_ssim_identity_symmetry_and_constant_closed_form():
    a = RNG.random((20, 24))
    b = np.clip(a + 0.1 * RNG.standard_normal(a.shape), 0, 1)
    assert ablation.ssim(a, a) == pytest.approx(1.0, abs=1e-12)
    assert ablation.ssim(a, b) == pytest.approx(ablation.ssim(b, a), abs=1e-12)
    assert ablation.ssim(a, b) < 1.0
    c1, c2 = 0.3, 0.7
    C1 = 0.01 ** 2
    want = (2 * c1 * c2 + C1) / (c1 * c1 + c2 * c2 + C1)     # variances and covariance are 0
    assert ablation.ssim(np.full((9, 9), c1), np.full((9, 9), c2)) == pytest.approx(want, rel=1e-12)


def test_ssim_equals_brute_force_window_loop():
    """Every pixel's local moments from an explicit 11x11 Gaussian (sigma 1.5, truncated at 3.5
    sigma -> radius 5) with half-sample mirrored borders, then the SSIM formula, averaged."""
    H, W = 13, 11
    a, b = RNG.random((H, W)), RNG.random((H, W))
    sig, rad = 1.5, 5
    g = np.exp(-0.5 * (np.arange(-rad, rad + 1) / sig) ** 2)
    g /= g.sum()

    def refl(i, n):
        while i < 0 or i >= n:
            i = -i - 1 if i < 0 else 2 * n - 1 - i
        return i

    C1, C2 = 0.01 ** 2, 0.03 ** 2
    vals = []
    for y in range(H):
        for x in range(W):
            m = {k: 0.0 for k in ("a", "b", "aa", "bb", "ab")}
            for dy in range(-rad, rad + 1):
                for dx in range(-rad, rad + 1):
                    w = g[dy + rad] * g[dx + rad]
                    p, q = a[refl(y + dy, H), refl(x + dx, W)], b[refl(y + dy, H), refl(x + dx, W)]
                    m["a"] += w * p; m["b"] += w * q
                    m["aa"] += w * p * p; m["bb"] += w * q * q; m["ab"] += w * p * q
            sa, sb = m["aa"] - m["a"] ** 2, m["bb"] - m["b"] ** 2
            sab = m["ab"] - m["a"] * m["b"]
            vals.append((2 * m["a"] * m["b"] + C1) * (2 * sab + C2) /
                        ((m["a"] ** 2 + m["b"] ** 2 + C1) * (sa + sb + C2)))
    assert ablation.ssim(a, b) == pytest.approx(float(np.mean(vals)), rel=1e-10)


def test_psnr_and_display_luma_closed_forms():
    a = np.zeros((4, 4))
    assert ablation.psnr(a, a + 0.1) == pytest.approx(20.0, rel=1e-12)
    assert ablation.psnr(a, a) == float("inf")
    c = np.array([[[2.0, 2.0, 2.0], [0.0, 0.0, 0.0]]])
    assert np.allclose(ablation.display_luma(c), [[2.0 / 3.0, 0.0]], atol=1e-15)


@pytest.mark.gpu
def test_small_ablation_runs_and_denoising_helps():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    rows = ablation.specular_ablation(torch, dev, 96, 64, 8, 5, roughness=(0.0, 1.0),
                                      movements=("static", "moving objects and light"))
    by = {(r["movement"], r["roughness"], r["variant"]): r for r in rows}
    assert all(-1.0 <= r["ssim"] <= 1.0 for r in rows)
    for mv in ("static", "moving objects and light"):
        assert by[(mv, 0.0, "noisy input")]["ssim"] == 1.0          # a smooth surface is noise-free
        for v, _ in ablation.SPECULAR_VARIANTS:
            assert by[(mv, 1.0, v)]["ssim"] > by[(mv, 1.0, "noisy input")]["ssim"] + 0.05, (mv, v)
    shad = ablation.shadow_ablation(torch, dev, 96, 64, 8, 5, radii=(1.0,), movements=("static",))
    assert {r["variant"] for r in shad} == {v for v, _ in ablation.SHADOW_VARIANTS} | {"noisy input"}
    assert all(-1.0 <= r["ssim"] <= 1.0 and math.isfinite(r["psnr_db"]) for r in shad)
    assert next(r for r in shad if r["variant"] == "noisy input")["ssim"] < 1.0   # penumbrae are noisy
    print(ablation.table(rows, "roughness"))
