"""Pin of the oracle's whole-frame composition (``Sequence`` / ``ora_denoise_frame``).

With the edge functions off, a static scene and zero motion, every stage of the denoiser is a
linear map that scipy writes out directly, so a frame sequence has a closed form:
  - the forward Reinhard map of Sec. 3.4 on the noisy frame: c_n = c / (1 + luma(c));
  - temporal accumulation (Sec. 2, Sec. 3 step 4) against the history reprojected by a pure
    copy: x_n = (1 - a_n) hist_{n-1} + a_n c_n, a_n = max(alpha, 1/n);
  - the colour history is the output of a-trous pass 0 (SVGF's convention; the paper is
    silent): hist_n = B_1(x_n), B_i the dilated B3 correlation at step 2^(i-1), renormalised over
    in-image taps;
  - the output is the inverse map of B_5(...B_1(x_n)), with the variance carried through the
    squared, renormalised kernels: var' = sum h^2 var / (sum h)^2;
  - the variance entering the passes is mu2 - mu1^2 of the moment averages (a_m = max(alpha_m,
    1/n)) once n >= 4, else the 7x7 window variance of those moments (equal weights here).
A routing mistake (the history taken from another pass or from the accumulated colour, the
inverse map skipped or replaced, the variance not propagated) breaks the equality; the
mutations below are planted in the oracle through its configuration and must be caught."""
import numpy as np
import pytest
from scipy import ndimage

import oracle

B3 = np.array([1, 4, 6, 4, 1], np.float64) / 16.0
LUMA = np.array([0.2126, 0.7152, 0.0722])
H, W = 37, 41          # larger than the largest dilated footprint (2 * 16 + 1) in both axes
T = 8                  # frames: the plain mean (n <= 5), then the exponential average; n >= 4 too


def _kernel(step):
    K = np.zeros((4 * step + 1,) * 2)
    for a in range(5):
        for b in range(5):
            K[a * step, b * step] = B3[a] * B3[b]
    return K


def _pass(cv, step):
    """One edges-off a-trous pass by scipy: colour by the renormalised kernel, variance by the
    squared kernel over the squared in-image mass."""
    K = _kernel(step)
    den = ndimage.correlate(np.ones((H, W)), K, mode="constant", cval=0.0)
    out = np.empty_like(cv)
    for c in range(3):
        out[..., c] = ndimage.correlate(cv[..., c], K, mode="constant", cval=0.0) / den
    out[..., 3] = ndimage.correlate(cv[..., 3], K * K, mode="constant", cval=0.0) / den ** 2
    return out


def _box_mean(img, R=3):
    k = np.ones((2 * R + 1, 2 * R + 1))
    den = ndimage.correlate(np.ones((H, W)), k, mode="constant", cval=0.0)
    return ndimage.correlate(img, k, mode="constant", cval=0.0) / den


def closed_form(noisy, alpha=0.2, alpha_m=0.2, iters=5):
    outs, hists = [], []
    hist = None
    mu1 = mu2 = None
    for n, c_lin in enumerate(noisy, start=1):
        c = c_lin / (1.0 + c_lin @ LUMA)[..., None]
        l = c @ LUMA
        a = max(alpha, 1.0 / n)
        am = max(alpha_m, 1.0 / n)
        x = c if hist is None else (1 - a) * hist + a * c
        mu1 = l if mu1 is None else (1 - am) * mu1 + am * l
        mu2 = l * l if mu2 is None else (1 - am) * mu2 + am * l * l
        if n >= 4:
            var = np.maximum(mu2 - mu1 ** 2, 0.0)
        else:
            var = np.maximum(_box_mean(mu2) - _box_mean(mu1) ** 2, 0.0)
        cv = np.concatenate([x, var[..., None]], -1)
        for i in range(iters):
            cv = _pass(cv, 1 << i)
            if i == 0:
                hist = cv[..., :3].copy()
        rgb = cv[..., :3] / (1.0 - cv[..., :3] @ LUMA)[..., None]
        outs.append(np.concatenate([rgb, cv[..., 3:]], -1))
        hists.append(hist)
    return outs, hists


def _inputs(seed=20):
    rng = np.random.default_rng(seed)
    # HDR radiance with per-pixel spread (noise) around a smooth field, up to ~6
    base = 0.5 + 2.0 * rng.random((1, H, W, 3))
    noisy = base * rng.exponential(1.0, (T, H, W, 3))
    return np.minimum(noisy, 6.0)


def _run_oracle(noisy, **kw):
    cfg = oracle.OracleConfig(sigma_l=1e300, sigma_z=1e300, adaptive_start=False, clamp_enable=False,
                              **kw)
    g = np.zeros((H, W, 4))
    g[..., 2] = -1.0
    g[..., 3] = 5.0
    mv = np.zeros((H, W, 2))
    rough = np.full((H, W), 0.5)
    seq = oracle.Sequence(W, H, cfg)
    outs, hists = [], []
    for fr in noisy:
        outs.append(seq.step(fr, g, mv, rough))
        hists.append(seq.hist_rgb.copy())
    return outs, hists


def test_whole_frame_composition_closed_form():
    noisy = _inputs()
    want, want_h = closed_form(noisy)
    got, got_h = _run_oracle(noisy)
    for n in range(T):
        assert np.allclose(got_h[n], want_h[n], rtol=1e-12, atol=0), n
        assert np.allclose(got[n][..., :3], want[n][..., :3], rtol=1e-11, atol=0), n
        assert np.allclose(got[n][..., 3], want[n][..., 3], rtol=1e-9, atol=1e-18), n
    # the frames really pass through both accumulation regimes and both variance estimates
    assert T > 5 and not np.allclose(want[0][..., 3], want[T - 1][..., 3])


@pytest.mark.parametrize("mutation", [dict(history_from_pass=1), dict(history_from_pass=-1),
                                      dict(history_from_pass=4), dict(inverse_mode=1),
                                      dict(atrous_iters=4)])
def test_composition_pin_catches_routing_mistakes(mutation):
    """Each planted routing change (history from pass 1, from the accumulated colour, from the
    last pass; the printed inverse in place of the exact one; a pass dropped) moves the oracle's
    frames off the closed form."""
    noisy = _inputs()
    want, want_h = closed_form(noisy)
    got, got_h = _run_oracle(noisy, **mutation)
    worst = max(float(np.max(np.abs(got[n][..., :3] - want[n][..., :3]) / np.abs(want[n][..., :3])))
                for n in range(T))
    assert worst > 1e-6, (mutation, worst)
