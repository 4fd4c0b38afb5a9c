"""Pins of two oracle options: variance colour clipping as the history rectification (Sec. 3.1,
Fig. 3: the history is moved toward the centre of the 3x3 variance box until it lies inside it)
and the per-pixel a-trous pass budget adapted to the roughness (Sec. 3.5: roughness <= 0 -> 0
passes, <= 0.05 -> 1, otherwise all).

Each pin is fixed by something other than the oracle's own formula: hand-worked values, a
bisection search over the segment from the box centre to the history value, geometric
invariants of the clip, and exact pass-through identities of the budget."""
import math

import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(77)
CLIP = oracle.OracleConfig(rectify_mode=1)


def three_by_three(m, e):
    """3x3 current image whose centre window has per-channel mean m and population std e:
    values m + d u with u = +1 (4 pixels), -1 (4 pixels), 0 (centre); std = d sqrt(8/9)."""
    m, e = np.asarray(m, float), np.asarray(e, float)
    d = e / math.sqrt(8.0 / 9.0)
    u = np.array([[1, -1, 1], [-1, 0, -1], [1, -1, 1]], float)
    return m[None, None, :] + u[:, :, None] * d[None, None, :]


def rectify_centre(cur, h, cfg):
    hist = np.zeros(cur.shape)
    hist[1, 1] = h
    return oracle.clamp(cur, hist, cfg)[1, 1]


@pytest.mark.parametrize("dh,expect", [
    ((3.0, 1.0, 1.0), (1.0, 1.0 / 3.0, 1.0 / 3.0)),     # x leaves by 3 half-extents: scale by 1/3
    ((0.5, -1.0, 2.0), (0.5, -1.0, 2.0)),               # inside (0.5, 0.5, 0.5 of the extents)
    ((0.0, 0.0, -8.0), (0.0, 0.0, -4.0)),               # one channel: clip = clamp
    ((-2.0, 4.0, 0.0), (-1.0, 2.0, 0.0)),               # two channels at twice their extents
])
def test_clip_worked_examples(dh, expect):
    m, e = np.array([0.5, 0.5, 0.5]), np.array([1.0, 2.0, 4.0])
    cur = three_by_three(m, e)
    got = rectify_centre(cur, m + np.array(dh), CLIP)
    assert np.allclose(got, m + np.array(expect), atol=1e-12)


def test_clip_differs_from_clamp_off_axis():
    m, e = np.array([0.2, 0.4, 0.6]), np.array([1.0, 2.0, 4.0])
    cur = three_by_three(m, e)
    h = m + np.array([3.0, 1.0, 1.0])
    clamped = rectify_centre(cur, h, oracle.OracleConfig(rectify_mode=0))
    clipped = rectify_centre(cur, h, CLIP)
    assert np.allclose(clamped, m + np.array([1.0, 1.0, 1.0]), atol=1e-12)
    assert np.allclose(clipped, m + np.array([1.0, 1.0 / 3.0, 1.0 / 3.0]), atol=1e-12)


def _bisect_clip(m, e, h):
    """Largest lam in [0, 1] with m + lam (h - m) inside [m - e, m + e], by bisection."""
    d = h - m
    inside = lambda lam: np.all(np.abs(lam * d) <= e * (1 + 1e-15) + 1e-300)
    if inside(1.0):
        return h
    lo, hi = 0.0, 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if inside(mid) else (lo, mid)
    return m + lo * d


@pytest.mark.parametrize("gamma", [1.0, 0.5, 2.5])
def test_clip_matches_bisection_and_geometry(gamma):
    H, W = 13, 17
    cur = RNG.random((H, W, 3))
    hist = RNG.random((H, W, 3)) * 2.0 - 0.5
    cfg = oracle.OracleConfig(rectify_mode=1, clamp_gamma=gamma)
    out = oracle.clamp(cur, hist, cfg)
    n_clipped = 0
    for y in range(H):
        for x in range(W):
            win = cur[max(0, y - 1):y + 2, max(0, x - 1):x + 2].reshape(-1, 3)
            m, e = win.mean(0), gamma * win.std(0)
            want = _bisect_clip(m, e, hist[y, x])
            assert np.allclose(out[y, x], want, atol=1e-12), (y, x)
            # inside the box, on the segment from m to the history value
            assert np.all(np.abs(out[y, x] - m) <= e + 1e-12)
            d, o = hist[y, x] - m, out[y, x] - m
            lam = float(o @ d / (d @ d))
            assert 0.0 <= lam <= 1.0 + 1e-12 and np.allclose(o, lam * d, atol=1e-12)
            n_clipped += lam < 1.0 - 1e-12
    assert n_clipped > H * W // 4          # the case is not trivially inside
    again = oracle.clamp(cur, out, cfg)
    assert np.allclose(again, out, atol=1e-14)


def test_clip_degenerate_box():
    """A flat neighbourhood (s = 0) leaves no room: any history != m clips to m exactly; a
    channel with zero extent but no offset does not constrain the others."""
    cur = np.full((5, 5, 3), 0.3)
    hist = RNG.random((5, 5, 3))
    out = oracle.clamp(cur, hist, CLIP)
    assert np.array_equal(out, np.full((5, 5, 3), 0.3))
    m, e = np.array([0.5, 0.5, 0.5]), np.array([1.0, 2.0, 0.0])
    cur = three_by_three(m, e)
    got = rectify_centre(cur, m + np.array([2.0, 1.0, 0.0]), CLIP)
    assert np.allclose(got, m + np.array([1.0, 0.5, 0.0]), atol=1e-12)
    got = rectify_centre(cur, m + np.array([0.5, 0.5, 1e-9]), CLIP)
    assert np.allclose(got, m, atol=1e-15)


def test_temporal_with_history_inside_box_same_for_clip_and_clamp():
    """When every reprojected history value lies in its box, neither rectification moves it."""
    H, W = 12, 14
    cur = 0.5 + 0.01 * RNG.standard_normal((H, W, 3))
    noisy = oracle.inverse_tonemap(cur.reshape(-1, 3)).reshape(H, W, 3)
    g = np.zeros((H, W, 4)); g[..., 2] = 1.0; g[..., 3] = 3.0
    mv = np.zeros((H, W, 2))
    hist = np.full((H, W, 3), 0.5)      # the box centres are ~0.5 with std ~0.01 > |0.5 - m|?
    mom = np.zeros((H, W, 3)); mom[..., 2] = 10.0
    a = oracle.temporal(noisy, g, g, mv, hist, mom, True, oracle.OracleConfig(rectify_mode=0))[0]
    b = oracle.temporal(noisy, g, g, mv, hist, mom, True, oracle.OracleConfig(rectify_mode=1))[0]
    off = oracle.temporal(noisy, g, g, mv, hist, mom, True, oracle.OracleConfig(clamp_enable=False))[0]
    inside = np.all(np.isclose(a, off, atol=0, rtol=0), axis=-1)
    assert inside.mean() > 0.3
    assert np.array_equal(a[inside], b[inside])


# ------------------------------------------------------------------ Sec. 3.5 pass budget

def budget_cfg(**kw):
    return oracle.OracleConfig(iter_by_roughness=True, **kw)


def scene_like(H=24, W=28, seed=3):
    rng = np.random.default_rng(seed)
    cv = np.concatenate([rng.random((H, W, 3)), 0.01 * rng.random((H, W, 1))], -1)
    g = np.zeros((H, W, 4))
    g[..., 2] = 1.0
    g[..., 3] = 2.0 + 0.05 * np.arange(W)[None, :]
    return cv, g


@pytest.mark.parametrize("mode", ["5x5", "separable"])
def test_budget_zero_is_identity(mode):
    cv, g = scene_like()
    rough = np.full(cv.shape[:2], 0.7)
    cfg = budget_cfg(iter_rough_t0=2.0, separable=mode == "separable")
    for it in range(5):
        out = oracle.atrous(cv, g, rough, it, cfg, mode)
        assert np.array_equal(out, cv)


@pytest.mark.parametrize("mode", ["5x5", "separable"])
def test_budget_full_equals_no_budget(mode):
    cv, g = scene_like()
    rough = RNG.random(cv.shape[:2])
    sep = mode == "separable"
    for it in range(3):
        a = oracle.atrous(cv, g, rough, it, oracle.OracleConfig(separable=sep), mode)
        b = oracle.atrous(cv, g, rough, it, budget_cfg(iter_count0=5, iter_count1=5, separable=sep), mode)
        assert np.array_equal(a, b)


def test_budget_thresholds_are_inclusive_and_fp32():
    """roughness 0 -> 0 passes, exactly 0.05 (as FP32) -> 1 pass, the next FP32 above -> all."""
    cv, g = scene_like(8, 8)
    r05 = float(np.float32(0.05))
    above = float(np.nextafter(np.float32(0.05), np.float32(1)))
    for r, n_passes in [(0.0, 0), (-0.1, 0), (r05, 1), (above, 5), (0.6, 5)]:
        rough = np.full((8, 8), r)
        moved = [not np.array_equal(oracle.atrous(cv, g, rough, it, budget_cfg(adaptive_start=False)), cv)
                 for it in range(5)]
        assert moved == [it < n_passes for it in range(5)], (r, moved)


@pytest.mark.parametrize("mode", ["5x5", "separable"])
def test_budget_freezes_pixels_after_their_passes(mode):
    """Over a chain of passes, a pixel with budget b keeps, bit for bit, its value after pass
    b - 1; pixels with the full budget keep changing."""
    H, W = 32, 36
    cv, g = scene_like(H, W, seed=5)
    rough = np.full((H, W), 0.8)
    rough[:, :12] = 0.0           # budget 0
    rough[:, 12:24] = 0.03        # budget 2 (iter_count1 = 2)
    cfg = budget_cfg(iter_count1=2, separable=mode == "separable")
    cur, hist = cv, [cv]
    for it in range(5):
        cur = oracle.atrous(cur, g, rough, it, cfg, mode)
        hist.append(cur)
    assert np.array_equal(hist[5][:, :12], cv[:, :12])
    assert not np.array_equal(hist[2][:, 12:24], cv[:, 12:24])
    for k in (3, 4, 5):
        assert np.array_equal(hist[k][:, 12:24], hist[2][:, 12:24])
    assert not np.array_equal(hist[5][:, 24:], hist[4][:, 24:])


def test_budget_in_whole_frame_leaves_temporal_colour():
    """Budget 0 on every pixel: the frame's output is the inverse tone map of the accumulated
    colour, and the colour history is that colour too."""
    H, W = 16, 20
    rng = np.random.default_rng(9)
    noisy = rng.random((H, W, 3)) * 3
    g = np.zeros((H, W, 4)); g[..., 2] = 1.0; g[..., 3] = 4.0
    mv = np.zeros((H, W, 2))
    rough = np.zeros((H, W))
    cfg = budget_cfg()
    seq = oracle.Sequence(W, H, cfg)
    out = seq.step(noisy, g, mv, rough)
    cv, _, _ = oracle.temporal(noisy, g, None, mv, None, None, False, cfg)
    want = oracle.inverse_tonemap(cv[..., :3].reshape(-1, 3), cfg).reshape(H, W, 3)
    assert np.array_equal(out[..., :3], want)
    assert np.array_equal(seq.hist_rgb, cv[..., :3])
