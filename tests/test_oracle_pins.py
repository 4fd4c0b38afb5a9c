"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test fixes one oracle function by something other than the oracle itself: values the
paper prints (tests/golden/paper_constants.json), closed forms, brute-force convolution by a
library routine (scipy.ndimage), invariances, and special cases that reduce to a textbook
quantity.  A dropped term, a wrong sign or index, a swapped axis or operand in the oracle
fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import ndimage

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")
B3 = np.array([1, 4, 6, 4, 1], np.float64) / 16.0
RNG = np.random.default_rng(1234)


def flat_gbuf(H, W, depth=5.0, normal=(0.0, 0.0, -1.0)):
    g = np.zeros((H, W, 4))
    g[..., 0], g[..., 1], g[..., 2] = normal
    g[..., 3] = depth
    return g


def edges_off(**kw):
    """Edge functions switched off: sigma_l huge (with positive variance), sigma_z huge with a
    constant depth, equal normals."""
    base = dict(sigma_l=1e300, sigma_z=1e300, sigma_n=128.0, adaptive_start=False)
    base.update(kw)
    return oracle.OracleConfig(**base)


def norm_correlate(img, K):
    """Zero-padded correlation renormalised by the in-image kernel mass (per channel)."""
    mask = np.ones(img.shape[:2])
    den = ndimage.correlate(mask, K, mode="constant", cval=0.0)
    out = np.empty_like(img)
    for c in range(img.shape[2]):
        out[..., c] = ndimage.correlate(img[..., c], K, mode="constant", cval=0.0) / den
    return out, den


def dilated(k1, step):
    K = np.zeros(((len(k1) - 1) * step + 1,) * 2)
    for a, ka in enumerate(k1):
        for b, kb in enumerate(k1):
            K[a * step, b * step] = ka * kb
    return K


# --------------------------------------------------------------------------- paper values

def test_golden_paper_constants():
    g = json.load(open(GOLDEN))
    cfg = oracle.OracleConfig()
    assert cfg.roughness_threshold == g["adaptive_start_roughness_threshold"]["value"]
    assert oracle.atrous_taps(False) == g["atrous_taps_5x5"]["value"]
    assert oracle.atrous_taps(True) == g["atrous_taps_separable"]["value"]
    ex = g["reinhard_forward_example"]
    assert np.allclose(oracle.tonemap(np.array([ex["input"]])), [ex["output"]], rtol=0, atol=1e-15)
    ex = g["reinhard_paper_inverse_example"]
    got = oracle.inverse_tonemap(np.array([ex["input"]]), oracle.OracleConfig(inverse_mode=1))
    assert np.allclose(got, [ex["output"]], rtol=0, atol=1e-15)
    ex = g["reinhard_exact_inverse_example"]
    got = oracle.inverse_tonemap(np.array([ex["input"]]), oracle.OracleConfig(inverse_mode=0))
    assert np.allclose(got, [ex["output"]], rtol=0, atol=1e-15)


def test_clamp_window_is_3x3():
    """A history value is clamped by its 3x3 box only: an outlier 2 pixels away (outside the
    window of g['clamp_window']=3) leaves the box of the centre pixel untouched."""
    g = json.load(open(GOLDEN))
    assert g["clamp_window"]["value"] == 3
    H = W = 7
    cur = np.full((H, W, 3), 0.3)
    cur[3, 5] = 5.0              # 2 px right of the centre: outside the 3x3 window
    hist = np.full((H, W, 3), 0.9)
    out = oracle.clamp(cur, hist)
    assert np.allclose(out[3, 3], 0.3)    # box of the centre is the single value 0.3
    assert out[3, 4, 0] > 0.3             # neighbour's window contains the outlier


# --------------------------------------------------------------------------- Reinhard

def test_luma_is_linear_with_unit_white():
    assert oracle.luma(np.ones(3)) == pytest.approx(1.0, abs=1e-15)
    a, b = RNG.random(3), RNG.random(3)
    assert oracle.luma(2 * a - 3 * b) == pytest.approx(2 * oracle.luma(a) - 3 * oracle.luma(b), abs=1e-14)
    assert oracle.luma(np.array([0.0, 1.0, 0.0])) > oracle.luma(np.array([1.0, 0.0, 0.0])) > \
        oracle.luma(np.array([0.0, 0.0, 1.0]))


@pytest.mark.parametrize("k", [1.0, 0.5, 2.0])
def test_reinhard_round_trip_and_luma_closed_form(k):
    cfg = oracle.OracleConfig(luma_k=k)
    c = RNG.random((1000, 3)) * 20.0
    t = oracle.tonemap(c, cfg)
    L = np.array([oracle.luma(x) for x in c])
    Lt = np.array([oracle.luma(x) for x in t])
    assert np.allclose(Lt, L / (1 + k * L), rtol=1e-14, atol=0)
    back = oracle.inverse_tonemap(t, cfg)
    assert np.allclose(back, c, rtol=1e-13, atol=1e-15)


def test_paper_literal_inverse_differs_from_exact():
    """The printed inverse multiplies by (1 + luma(c')) * w: at luma 0.5 that is 1.5x where the
    exact inverse is 2x."""
    c = np.array([[0.5, 0.5, 0.5], [0.2, 0.4, 0.1]])
    lit = oracle.inverse_tonemap(c, oracle.OracleConfig(inverse_mode=1, inv_weight=2.0))
    L = 0.2126 * 0.2 + 0.7152 * 0.4 + 0.0722 * 0.1
    assert np.allclose(lit[0], 1.5), lit
    assert np.allclose(lit[1], c[1] * (1 + L) * 2.0)


# --------------------------------------------------------------------------- depth gradient

def test_depth_gradient_exact_on_planes_and_degenerate_axes():
    H, W = 9, 13
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    g = flat_gbuf(H, W)
    g[..., 3] = 3.0 + 0.25 * x - 0.125 * y
    d = oracle.depth_gradient(g)
    assert np.allclose(d[..., 0], 0.25, atol=1e-14) and np.allclose(d[..., 1], -0.125, atol=1e-14)
    d1 = oracle.depth_gradient(g[:1])
    assert np.allclose(d1[..., 1], 0.0) and np.allclose(d1[..., 0], 0.25)
    dq = oracle.depth_gradient(np.concatenate([g[..., :3], (x ** 2)[..., None]], -1))
    assert np.allclose(dq[:, 1:-1, 0], 2 * x[:, 1:-1])   # central difference exact for x^2


# --------------------------------------------------------------------------- a-trous

@pytest.mark.parametrize("it", [0, 1, 2])
@pytest.mark.parametrize("shape", [(23, 37), (16, 16), (5, 40)])
def test_atrous_5x5_edges_off_is_dilated_b3_convolution(it, shape):
    H, W = shape
    cv = RNG.random((H, W, 4))
    cv[..., 3] += 0.5
    g = flat_gbuf(H, W)
    out = oracle.atrous(cv, g, None, it, edges_off(), mode="5x5")
    K = dilated(B3, 1 << it)
    ref, den = norm_correlate(cv[..., :3], K)
    assert np.allclose(out[..., :3], ref, rtol=1e-12, atol=1e-14)
    var_ref = ndimage.correlate(cv[..., 3], K * K, mode="constant") / den ** 2
    assert np.allclose(out[..., 3], var_ref, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("it", [0, 2])
def test_atrous_separable_edges_off_is_h_then_v_convolution(it):
    H, W = 21, 34
    cv = RNG.random((H, W, 4))
    cv[..., 3] += 0.5
    g = flat_gbuf(H, W)
    out = oracle.atrous(cv, g, None, it, edges_off(), mode="separable")
    s = 1 << it
    h = np.zeros(4 * s + 1)
    h[::s] = B3
    ones = np.ones((H, W))
    dx = ndimage.correlate1d(ones, h, axis=1, mode="constant")
    dy = ndimage.correlate1d(ones, h, axis=0, mode="constant")
    mid = np.stack([ndimage.correlate1d(cv[..., c], h, axis=1, mode="constant") / dx for c in range(3)], -1)
    ref = np.stack([ndimage.correlate1d(mid[..., c], h, axis=0, mode="constant") / dy for c in range(3)], -1)
    assert np.allclose(out[..., :3], ref, rtol=1e-12, atol=1e-14)
    # the colour of H-then-V equals the 5x5 kernel (rectangular clipping factorises)
    full = oracle.atrous(cv, g, None, it, edges_off(), mode="5x5")
    assert np.allclose(out[..., :3], full[..., :3], rtol=1e-12, atol=1e-14)
    # variance: only the vertical pass updates it
    var_ref = ndimage.correlate1d(cv[..., 3], h * h, axis=0, mode="constant") / dy ** 2
    assert np.allclose(out[..., 3], var_ref, rtol=1e-12, atol=1e-14)


def test_separable_variance_only_vertical():
    """Variance constant along y and varying along x: the vertical-only update keeps it a
    function of x (times sum h^2 / (sum h)^2 = 70/256 inside)."""
    H, W = 16, 20
    cv = RNG.random((H, W, 4))
    cv[..., 3] = (1.0 + np.arange(W) % 3)[None, :]
    out = oracle.atrous(cv, flat_gbuf(H, W), None, 0, edges_off(), mode="separable")
    assert np.allclose(out[2:-2, :, 3], (70.0 / 256.0) * cv[2:-2, :, 3], rtol=1e-12)


def test_variance_propagation_closed_form():
    H, W = 12, 12
    cv = np.concatenate([RNG.random((H, W, 3)), np.full((H, W, 1), 2.0)], -1)
    out = oracle.atrous(cv, flat_gbuf(H, W), None, 0, edges_off(), mode="5x5")
    assert np.allclose(out[2:-2, 2:-2, 3], (70.0 / 256.0) ** 2 * 2.0, rtol=1e-12)


@pytest.mark.parametrize("mode", ["5x5", "separable"])
def test_atrous_constant_image_unchanged_with_edges_on(mode):
    from paper_2312_06827_gb300 import scene
    fr = scene.render_frame(scene.C0_128, 0)
    H, W = fr["roughness"].shape
    cv = np.zeros((H, W, 4))
    cv[..., :3] = [0.3, 0.5, 0.7]
    cv[..., 3] = 0.01
    for it in range(3):
        out = oracle.atrous(cv, fr["gbuf_nz"], fr["roughness"], it, mode=mode)
        assert np.allclose(out[..., :3], cv[..., :3], rtol=1e-13)


@pytest.mark.parametrize("mode", ["5x5", "separable"])
def test_atrous_linear_image_unchanged_inside(mode):
    """Symmetric weights on a linear signal return the centre value: linear colour, planar
    depth, constant normal, constant variance, edge functions on."""
    H, W, it = 40, 44, 1
    s = 1 << it
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    cv = np.zeros((H, W, 4))
    cv[..., 0] = 0.01 * x + 0.02 * y
    cv[..., 1] = 0.5 - 0.003 * x
    cv[..., 2] = 0.2 + 0.004 * y
    cv[..., 3] = 0.05
    g = flat_gbuf(H, W)
    g[..., 3] = 4.0 + 0.01 * x + 0.0137 * y   # no tap offset with grad . offset = 0
    out = oracle.atrous(cv, g, None, it, oracle.OracleConfig(adaptive_start=False), mode=mode)
    m = 2 * s
    assert np.allclose(out[m:-m, m:-m, :3], cv[m:-m, m:-m, :3], rtol=1e-12, atol=1e-14)


def test_depth_weight_on_a_plane():
    """Depth z = a x: for taps off the centre column |dz| equals |grad z . offset|, so the depth
    weight is exp(-1/sigma_z) there and 1 on the centre column."""
    H, W, sz = 14, 30, 2.0
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    cv = RNG.random((H, W, 4))
    cv[..., 3] = 1.0
    g = flat_gbuf(H, W)
    g[..., 3] = 2.0 + 0.3 * x
    out = oracle.atrous(cv, g, None, 0, edges_off(sigma_z=sz), mode="5x5")
    K = np.outer(B3, B3)
    K[:, [0, 1, 3, 4]] *= math.exp(-1.0 / sz)
    ref, _ = norm_correlate(cv[..., :3], K)
    assert np.allclose(out[..., :3], ref, rtol=1e-9)


@pytest.mark.parametrize("sn", [3.0, 32.0, 64.0, 128.0])
def test_normal_weight_on_two_normals(sn):
    """Columns alternate between unit normals na and nb: the normal weight of odd-column taps
    is (na . nb)^sigma_n (also at the sharp weights the CUDA path takes by the series alone)."""
    H, W = 10, 24
    na, nb = np.array([0.0, 0.0, 1.0]), np.array([0.6, 0.0, 0.8])
    cv = RNG.random((H, W, 4))
    cv[..., 3] = 1.0
    g = flat_gbuf(H, W)
    g[:, 0::2, :3] = na
    g[:, 1::2, :3] = nb
    out = oracle.atrous(cv, g, None, 0, edges_off(sigma_n=sn), mode="5x5")
    K = np.outer(B3, B3)
    K[:, [1, 3]] *= float(na @ nb) ** sn
    ref, _ = norm_correlate(cv[..., :3], K)
    assert np.allclose(out[..., :3], ref, rtol=1e-9)
    opposite = g.copy()
    opposite[:, 1::2, :3] = -na                       # anti-parallel normals never mix
    out2 = oracle.atrous(cv, opposite, None, 0, edges_off(sigma_n=sn), mode="5x5")
    K2 = np.outer(B3, B3)
    K2[:, [1, 3]] = 0.0
    ref2, _ = norm_correlate(cv[..., :3], K2)
    assert np.allclose(out2[..., :3], ref2, rtol=1e-9)


def test_luminance_weight_on_two_levels():
    """Columns alternate between grey levels la, lb with constant variance V: odd-column taps
    weigh exp(-|la - lb| / (sigma_l sqrt(V)))."""
    H, W, sl, V = 10, 24, 4.0, 0.09
    cv = np.zeros((H, W, 4))
    cv[:, 0::2, :3] = 0.3
    cv[:, 1::2, :3] = 0.7
    cv[..., 3] = V
    out = oracle.atrous(cv, flat_gbuf(H, W), None, 0,
                        oracle.OracleConfig(sigma_l=sl, sigma_z=1e300, adaptive_start=False), mode="5x5")
    K = np.outer(B3, B3)
    K[:, [1, 3]] *= math.exp(-0.4 / (sl * math.sqrt(V)))
    ref, _ = norm_correlate(cv[..., :3], K)
    assert np.allclose(out[..., :3], ref, rtol=1e-9)


def test_atrous_scale_invariance():
    """Colour x s, variance x s^2: the luminance weight is invariant, so colour scales by s and
    the propagated variance by s^2."""
    from paper_2312_06827_gb300 import scene
    fr = scene.render_frame(scene.C0_128, 1)
    H, W = fr["roughness"].shape
    cv = np.concatenate([scene_tm(fr["noisy"]), RNG.random((H, W, 1)) * 0.05 + 1e-3], -1)
    a = oracle.atrous(cv, fr["gbuf_nz"], fr["roughness"], 1)
    s = 3.7
    cv2 = cv.copy()
    cv2[..., :3] *= s
    cv2[..., 3] *= s * s
    b = oracle.atrous(cv2, fr["gbuf_nz"], fr["roughness"], 1)
    assert np.allclose(b[..., :3], s * a[..., :3], rtol=1e-9)
    assert np.allclose(b[..., 3], s * s * a[..., 3], rtol=1e-9)


def scene_tm(rgb):
    return oracle.tonemap(rgb)


def test_atrous_outputs_are_convex_combinations():
    from paper_2312_06827_gb300 import scene
    fr = scene.render_frame(scene.C0_128, 2)
    H, W = fr["roughness"].shape
    cv = np.concatenate([scene_tm(fr["noisy"]), RNG.random((H, W, 1)) * 0.05], -1)
    for mode in ("5x5", "separable"):
        out = oracle.atrous(cv, fr["gbuf_nz"], fr["roughness"], 0, mode=mode)
        for c in range(3):
            assert out[..., c].min() >= cv[..., c].min() - 1e-15
            assert out[..., c].max() <= cv[..., c].max() + 1e-15
        assert (out[..., 3] >= 0).all()


def test_adaptive_start_is_one_scale_higher():
    """Sec. 3.2: above the roughness threshold iteration i uses the step of iteration i+1."""
    from paper_2312_06827_gb300 import scene
    fr = scene.render_frame(scene.C0_128, 1)
    H, W = fr["roughness"].shape
    cv = np.concatenate([scene_tm(fr["noisy"]), RNG.random((H, W, 1)) * 0.05], -1)
    rough = np.where(np.arange(W)[None, :] < W // 2, 0.1, 0.7) * np.ones((H, W))
    on = oracle.atrous(cv, fr["gbuf_nz"], rough, 1, oracle.OracleConfig(adaptive_start=True))
    off1 = oracle.atrous(cv, fr["gbuf_nz"], rough, 1, oracle.OracleConfig(adaptive_start=False))
    off2 = oracle.atrous(cv, fr["gbuf_nz"], rough, 2, oracle.OracleConfig(adaptive_start=False))
    left, right = rough < 0.2, rough > 0.2
    assert np.array_equal(on[left], off1[left])
    assert np.array_equal(on[right], off2[right])


def test_atrous_single_pixel_and_thin_images():
    for H, W in [(1, 1), (1, 9), (9, 1), (2, 3)]:
        cv = RNG.random((H, W, 4))
        out = oracle.atrous(cv, flat_gbuf(H, W), None, 0, edges_off())
        if H * W == 1:
            assert np.allclose(out[..., :3], cv[..., :3]) and np.allclose(out[..., 3], (36 / 256) ** 2 * cv[..., 3] / (36 / 256) ** 2)
        assert np.isfinite(out).all()


# --------------------------------------------------------------------------- clamp

def test_clamp_bounds_and_idempotence():
    H, W, gamma = 17, 19, 1.0
    cur = RNG.random((H, W, 3))
    hist = RNG.random((H, W, 3)) * 1.5 - 0.25
    out = oracle.clamp(cur, hist, oracle.OracleConfig(clamp_gamma=gamma))
    for y in range(H):
        for x in range(W):
            win = cur[max(0, y - 1):y + 2, max(0, x - 1):x + 2].reshape(-1, 3)
            m, s = win.mean(0), win.std(0)      # population std (ddof=0)
            lo, hi = m - gamma * s, m + gamma * s
            assert np.all(out[y, x] >= lo - 1e-14) and np.all(out[y, x] <= hi + 1e-14)
            expect = np.minimum(np.maximum(hist[y, x], lo), hi)
            assert np.allclose(out[y, x], expect, atol=1e-14)
    again = oracle.clamp(cur, out)
    assert np.allclose(again, out, atol=1e-15)
    mean_only = oracle.clamp(cur, hist, oracle.OracleConfig(clamp_gamma=0.0))
    assert np.allclose(mean_only[5, 5], cur[4:7, 4:7].reshape(-1, 3).mean(0))


def test_clamp_linear_window_sigma():
    """Ramp a*x: the 3x3 window holds c-a, c, c+a three times each, sigma = |a| sqrt(2/3)."""
    H, W, a = 6, 8, 0.1
    x = np.arange(W, dtype=np.float64)[None, :, None] * np.ones((H, 1, 3))
    cur = 0.2 + a * x
    hist = cur + 1.0
    out = oracle.clamp(cur, hist)
    assert np.allclose(out[1:-1, 1:-1], cur[1:-1, 1:-1] + a * math.sqrt(2.0 / 3.0), rtol=1e-12)


# --------------------------------------------------------------------------- reprojection

def test_reproject_integer_motion_is_a_shift():
    H, W = 12, 15
    g = flat_gbuf(H, W)
    mv = np.zeros((H, W, 2))
    mv[..., 0], mv[..., 1] = 2.0, -1.0
    hist = RNG.random((H, W, 3))
    mom = np.concatenate([RNG.random((H, W, 2)), RNG.integers(1, 9, (H, W, 1)).astype(float)], -1)
    rgb, m, valid, _ = oracle.reproject(g, g, mv, hist, mom)
    for y in range(H):
        for x in range(W):
            sx, sy = x - 2, y + 1          # previous position = p - mv
            inside = 0 <= sx < W and 0 <= sy < H
            assert valid[y, x] == inside
            if inside:
                assert np.allclose(rgb[y, x], hist[sy, sx]) and np.allclose(m[y, x], mom[sy, sx])


def test_reproject_fractional_motion_reproduces_linear_history():
    H, W = 12, 14
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    g = flat_gbuf(H, W)
    mv = np.zeros((H, W, 2))
    mv[..., 0], mv[..., 1] = 0.3, -0.7
    hist = np.stack([0.1 * x + 0.05 * y, 0.5 + 0.02 * x, 0.3 - 0.01 * y], -1)
    mom = np.concatenate([hist[..., :2], np.ones((H, W, 1))], -1)
    rgb, _, valid, _ = oracle.reproject(g, g, mv, hist, mom)
    px, py = x - 0.3, y + 0.7
    ref = np.stack([0.1 * px + 0.05 * py, 0.5 + 0.02 * px, 0.3 - 0.01 * py], -1)
    inner = valid & (x >= 1) & (x <= W - 2) & (y <= H - 3)
    assert inner.sum() > 50
    assert np.allclose(rgb[inner], ref[inner], rtol=1e-12)


def test_reproject_rejects_depth_and_normal_changes():
    H, W = 8, 8
    g = flat_gbuf(H, W)
    mv = np.zeros((H, W, 2))
    hist, mom = RNG.random((H, W, 3)), np.ones((H, W, 3))
    prev = g.copy()
    prev[:, :4, 3] *= 1.5                       # depth jump
    prev[:4, 4:, :3] = [0.0, 1.0, 0.0]          # normal turned 90 degrees
    _, _, valid, _ = oracle.reproject(g, prev, mv, hist, mom)
    assert not valid[:, :4].any() and not valid[:4, 4:].any() and valid[4:, 4:].all()
    _, _, v0, _ = oracle.reproject(g, None, mv, hist, mom, has_history=False)
    assert not v0.any()


# --------------------------------------------------------------------------- temporal

def _temporal_seq(frames, clamp=False, tonemap=False, H=6, W=7):
    cfg = oracle.OracleConfig(clamp_enable=clamp, tonemap=tonemap, atrous_iters=0,
                              sigma_z=1e300)
    g = flat_gbuf(H, W)
    mv = np.zeros((H, W, 2))
    hist, mom, have = None, None, False
    outs = []
    for c in frames:
        cv, mom, _ = oracle.temporal(c, g, g if have else None, mv, hist, mom, have, cfg)
        hist, have = cv[..., :3], True
        outs.append((cv, mom))
    return outs


def test_static_sequence_closed_form():
    """Zero motion, constant geometry, clamp off: the accumulated colour is the plain mean of
    the first n frames while 1/n >= alpha (n <= 5), then an exponential moving average."""
    T, alpha = 12, 0.2
    vals = RNG.random((T, 3)) * 2.0
    frames = [np.broadcast_to(v, (6, 7, 3)).copy() for v in vals]
    outs = _temporal_seq(frames)
    for n in range(1, T + 1):
        if n <= 5:
            expect = vals[:n].mean(0)
        else:
            x5 = vals[:5].mean(0)
            expect = (1 - alpha) ** (n - 5) * x5 + sum(alpha * (1 - alpha) ** (n - k) * vals[k - 1]
                                                       for k in range(6, n + 1))
        assert np.allclose(outs[n - 1][0][3, 3, :3], expect, rtol=1e-12), n
        assert outs[n - 1][1][3, 3, 2] == n


def test_variance_zero_on_constant_sequence_and_nonnegative():
    frames = [np.full((6, 7, 3), 0.4) for _ in range(8)]
    for cv, _ in _temporal_seq(frames):
        assert np.allclose(cv[..., 3], 0.0, atol=1e-15)
    rnd = [RNG.random((6, 7, 3)) for _ in range(8)]
    for cv, _ in _temporal_seq(rnd, clamp=True, tonemap=True):
        assert (cv[..., 3] >= 0).all()


def test_temporal_variance_is_moment_difference_after_four_frames():
    """For n >= 4 the variance is mu2 - mu1^2 of the exponentially weighted luminance moments;
    with zero motion and clamp off those are the sample moments of the first n frames for
    n <= 5."""
    vals = RNG.random((5, 3))
    frames = [np.broadcast_to(v, (6, 7, 3)).copy() for v in vals]
    outs = _temporal_seq(frames)
    L = vals @ np.array([0.2126, 0.7152, 0.0722])
    for n in (4, 5):
        assert outs[n - 1][0][3, 3, 3] == pytest.approx(np.var(L[:n]), rel=1e-10)


@pytest.mark.parametrize("R", [3, 0, 1, 5, 7])
def test_spatial_variance_for_short_history_is_window_variance(R):
    """First frame, edge weights off: the (2R+1)^2 spatial estimate (7x7 by default) is the
    population variance of the luminance over the in-image window; radius 0 gives 0."""
    H, W = 11, 13
    c = RNG.random((H, W, 3))
    cfg = oracle.OracleConfig(clamp_enable=False, tonemap=False, sigma_z=1e300, spatial_var_radius=R)
    g = flat_gbuf(H, W)
    cv, mom, _ = oracle.temporal(c, g, None, np.zeros((H, W, 2)), None, None, False, cfg)
    L = c @ np.array([0.2126, 0.7152, 0.0722])
    for y in range(H):
        for x in range(W):
            win = L[max(0, y - R):y + R + 1, max(0, x - R):x + R + 1]
            assert cv[y, x, 3] == pytest.approx(win.var(), rel=1e-10, abs=1e-15)
    assert np.allclose(mom[..., 2], 1.0)
    if R == 0:
        assert np.all(cv[..., 3] == 0.0)


def test_history_length_saturates():
    frames = [np.full((2, 2, 3), 0.5) for _ in range(260)]
    outs = _temporal_seq(frames, H=2, W=2)
    assert outs[-1][1][0, 0, 2] == 255 and outs[254][1][0, 0, 2] == 255 and outs[253][1][0, 0, 2] == 254


def test_disocclusion_restarts_history():
    H, W = 6, 7
    cfg = oracle.OracleConfig(atrous_iters=0)
    g = flat_gbuf(H, W)
    prev = g.copy()
    prev[..., 3] = 50.0
    c = RNG.random((H, W, 3))
    hist, mom = RNG.random((H, W, 3)), np.concatenate([RNG.random((H, W, 2)), np.full((H, W, 1), 9.0)], -1)
    cv, m, _ = oracle.temporal(c, g, prev, np.zeros((H, W, 2)), hist, mom, True, cfg)
    assert np.allclose(m[..., 2], 1.0)
    assert np.allclose(cv[..., :3], oracle.tonemap(c))


# --------------------------------------------------------------------------- whole frame

def test_single_pixel_frame_round_trips_input():
    """1x1 frame: no neighbours, so accumulation on the first frame returns the tone-mapped
    input, every a-trous pass is the identity and the exact inverse restores the input."""
    seq = oracle.Sequence(1, 1)
    c = np.array([[[3.0, 0.5, 7.0]]])
    out = seq.step(c, flat_gbuf(1, 1), np.zeros((1, 1, 2)), np.full((1, 1), 0.5))
    assert np.allclose(out[..., :3], c, rtol=1e-13)
    assert out[0, 0, 3] == 0.0


def test_luminance_guide_uses_prefiltered_centre_variance():
    """Columns alternate between two grey levels, variance varies per pixel.  Inside, the even
    and odd columns of the B3 kernel each hold half the mass, so the output is
    (c_p + e c_other) / (1 + e) with e = exp(-|la - lb| / (sigma_l sqrt(gV_p))), gV the
    [1 2 1]x[1 2 1]/16 blur of the variance at the centre pixel."""
    H, W, sl = 12, 16, 4.0
    cv = np.zeros((H, W, 4))
    cv[:, 0::2, :3] = 0.3
    cv[:, 1::2, :3] = 0.7
    cv[..., 3] = RNG.random((H, W)) * 0.2 + 0.01
    out = oracle.atrous(cv, flat_gbuf(H, W), None, 0,
                        oracle.OracleConfig(sigma_l=sl, sigma_z=1e300, adaptive_start=False), mode="5x5")
    k = np.array([1.0, 2.0, 1.0]) / 4.0
    gV = ndimage.correlate(cv[..., 3], np.outer(k, k), mode="constant")
    e = np.exp(-0.4 / (sl * np.sqrt(gV)))
    other = np.where(np.arange(W)[None, :] % 2 == 0, 0.7, 0.3) * np.ones((H, W))
    expect = (cv[..., 0] + e * other) / (1.0 + e)
    assert np.allclose(out[2:-2, 2:-2, 0], expect[2:-2, 2:-2], rtol=1e-12)


def test_previous_history_length_is_longest_valid_tap():
    """Fractional motion blends four taps; the history length carried over is the largest
    among the valid taps with non-zero weight (a reading: SVGF filters it bilinearly)."""
    H, W = 6, 6
    g = flat_gbuf(H, W)
    mv = np.zeros((H, W, 2))
    mv[..., 0] = 0.5                       # taps x-1 and x (weights 1/2, 1/2)
    mom = np.zeros((H, W, 3))
    mom[..., 2] = np.where(np.arange(W)[None, :] % 2 == 0, 3.0, 7.0)
    _, m, valid, _ = oracle.reproject(g, g, mv, np.zeros((H, W, 3)), mom)
    assert valid[:, 1:].all()
    assert np.all(m[:, 1:, 2] == 7.0)
    assert np.all(m[:, 0, 2] == 3.0)       # only tap x = 0 is inside


def test_moment_factor_is_separate_from_colour_factor():
    """alpha_moments = 0.1: the luminance moments are plain means up to n = 10 while the
    colour switches to its EMA after n = 5."""
    T = 10
    vals = RNG.random((T, 3))
    frames = [np.broadcast_to(v, (4, 4, 3)).copy() for v in vals]
    cfg = oracle.OracleConfig(clamp_enable=False, tonemap=False, atrous_iters=0,
                              sigma_z=1e300, alpha_moments=0.1)
    g = flat_gbuf(4, 4)
    hist, mom, have = None, None, False
    L = vals @ np.array([0.2126, 0.7152, 0.0722])
    for n, c in enumerate(frames, 1):
        cv, mom, _ = oracle.temporal(c, g, g if have else None, np.zeros((4, 4, 2)), hist, mom, have, cfg)
        hist, have = cv[..., :3], True
        assert mom[1, 1, 0] == pytest.approx(L[:n].mean(), rel=1e-12)
        assert mom[1, 1, 1] == pytest.approx((L[:n] ** 2).mean(), rel=1e-12)


@pytest.mark.parametrize("z", [0.5, 2.0, 50.0])
def test_reprojection_depth_test_is_relative(z):
    """The previous depth is accepted within depth_rel_tol * z of the current depth, at every
    depth scale: 9% off is kept, 11% off is dropped (tolerance 0.1)."""
    H, W = 4, 4
    g = flat_gbuf(H, W, depth=z)
    mv = np.zeros((H, W, 2))
    hist, mom = RNG.random((H, W, 3)), np.ones((H, W, 3))
    for f, keep in ((1.09, True), (0.91, True), (1.11, False), (0.89, False)):
        prev = g.copy()
        prev[..., 3] = z * f
        _, _, valid, _ = oracle.reproject(g, prev, mv, hist, mom)
        assert valid.all() == keep and valid.any() == keep
