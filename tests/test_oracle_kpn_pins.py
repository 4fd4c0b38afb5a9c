"""Pins of the oracle's learned part (network, kernel application, loss gradient, features)
against finite differences, library convolution (scipy), closed forms and special cases."""
import numpy as np
import pytest
from scipy import ndimage

import oracle

RNG = np.random.default_rng(77)


def rand_case(B=2, H=9, W=11, scale=0.1):
    f = RNG.standard_normal((B, H, W, 10))
    c0 = RNG.random((B, H, W, 3))
    T = RNG.random((B, H, W, 3))
    prm = RNG.standard_normal(oracle.kpn_param_count()) * scale
    return f, c0, T, prm


def test_param_count_matches_layer_shapes():
    n = sum(co * 9 * ci + co for ci, co in zip(oracle.KPN_CIN, oracle.KPN_COUT))
    assert oracle.kpn_param_count() == n == 28633


def test_gradient_matches_finite_differences_in_every_layer():
    f, c0, T, prm = rand_case()
    loss, g = oracle.kpn_grad(f, c0, T, prm)
    assert loss == pytest.approx(oracle.kpn_loss(f, c0, T, prm), rel=1e-14)
    offs = np.cumsum([0] + [co * 9 * ci + co for ci, co in zip(oracle.KPN_CIN, oracle.KPN_COUT)])
    for l in range(4):
        wn = oracle.KPN_COUT[l] * 9 * oracle.KPN_CIN[l]
        picks = list(RNG.choice(wn, 4, replace=False) + offs[l]) + [offs[l] + wn + 1]   # weights and a bias
        for k in picks:
            h = 1e-5
            p1, p2 = prm.copy(), prm.copy()
            p1[k] += h
            p2[k] -= h
            fd = (oracle.kpn_loss(f, c0, T, p1) - oracle.kpn_loss(f, c0, T, p2)) / (2 * h)
            assert abs(g[k] - fd) <= 1e-6 * abs(fd) + 1e-11, (l, k, g[k], fd)


def test_one_hot_centre_kernel_is_identity():
    f, c0, T, prm = rand_case()
    w3, b3 = oracle.kpn_unflatten(prm)[3]
    w3[:] = 0.0
    b3[:] = 0.0
    b3[12] = 60.0                      # centre tap (ky, kx) = (0, 0)
    K, c1, c2 = oracle.kpn_forward(f, c0, prm)
    assert np.allclose(K[..., 12], 1.0, atol=1e-20) and np.allclose(c1, c0, atol=1e-20)
    assert np.allclose(c2, c0, atol=1e-20)


def test_uniform_kernel_is_renormalised_box_filter():
    f, c0, T, prm = rand_case(B=1, H=14, W=17)
    w3, b3 = oracle.kpn_unflatten(prm)[3]
    w3[:] = 0.0
    b3[:] = 0.0
    K, c1, c2 = oracle.kpn_forward(f, c0, prm)
    assert np.allclose(K, 1.0 / 25.0, rtol=1e-14)

    def box(img, d):
        k = np.zeros((4 * d + 1, 4 * d + 1))
        k[::d, ::d] = 1.0
        den = ndimage.correlate(np.ones(img.shape[:2]), k, mode="constant")
        return np.stack([ndimage.correlate(img[..., c], k, mode="constant") / den for c in range(3)], -1)
    e1 = box(c0[0], 1)
    assert np.allclose(c1[0], e1, rtol=1e-12)
    assert np.allclose(c2[0], box(e1, 4), rtol=1e-12)


def test_conv_layer_is_library_correlation():
    x = RNG.standard_normal((2, 7, 9, 5))
    w = RNG.standard_normal((3, 9, 5))
    b = RNG.standard_normal(3)
    z = oracle.kpn_conv(x, w, b)
    for n in range(2):
        for co in range(3):
            ref = np.full((7, 9), b[co])
            for ci in range(5):
                k = w[co, :, ci].reshape(3, 3)          # tap = (dy + 1) * 3 + (dx + 1)
                ref += ndimage.correlate(x[n, ..., ci], k, mode="constant")
            assert np.allclose(z[n, ..., co], ref, rtol=1e-12, atol=1e-12)


def test_features_closed_form_and_octahedral_round_trip():
    H, W = 5, 6
    cv = RNG.random((H, W, 4))
    n = RNG.standard_normal((H, W, 3))
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    z = RNG.random((H, W)) * 20 + 0.5
    g = np.concatenate([n, z[..., None]], -1)
    alb = RNG.random((H, W, 3))
    f = oracle.kpn_features(cv, g, alb)
    assert np.allclose(f[..., :3], cv[..., :3]) and np.allclose(f[..., 3], np.sqrt(cv[..., 3]))
    assert np.allclose(f[..., 4], np.log2(z)) and np.allclose(f[..., 7:], alb)
    # decode the octahedral pair (textbook inverse) and recover the normal
    ox, oy = f[..., 5], f[..., 6]
    nz = 1.0 - np.abs(ox) - np.abs(oy)
    t = np.clip(-nz, 0.0, None)
    dx = ox - np.where(ox >= 0, t, -t)
    dy = oy - np.where(oy >= 0, t, -t)
    d = np.stack([dx, dy, nz], -1)
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    assert np.allclose(d, n, atol=1e-12)


# ------------------------------------------------------------ BF16 rounding mode (quant = 1)

def _bf16_brute(v):
    """Nearest BF16 to float32(v) by comparing the two BF16 neighbours (ties to the even one)."""
    f = np.float32(v)
    u = int(np.array(f).view(np.uint32))
    lo = u & 0xFFFF0000
    hi = lo + 0x10000
    a = np.array(lo, np.uint32).view(np.float32).astype(np.float64)
    b = np.array(hi, np.uint32).view(np.float32).astype(np.float64)
    x = float(f)
    da, db = abs(x - a), abs(b - x)
    if da < db or (da == db and ((lo >> 16) & 1) == 0):
        return a
    return b


def test_bf16_round_is_nearest_even():
    vals = np.concatenate([RNG.standard_normal(2000) * 10.0 ** RNG.integers(-6, 6, 2000),
                           [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 1.0 + 2 ** -9, -(1.0 + 3 * 2 ** -9)]])
    got = oracle.bf16_round(vals)
    want = np.array([_bf16_brute(v) for v in vals])
    assert np.array_equal(got, want)
    # ties: 1 + 2^-8 (halfway between 1 and 1 + 2^-7) goes to 1, 1 + 3 2^-8 to 1 + 2^-6
    assert oracle.bf16_round([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8]).tolist() == [1.0, 1.0 + 2 ** -6]


def _shift(img, dy, dx):
    """out[y, x] = img[y + dy, x + dx], zero outside (img [H, W, C])."""
    H, W = img.shape[:2]
    out = np.zeros_like(img)
    if abs(dy) >= H or abs(dx) >= W:
        return out
    ys, yd = slice(max(0, -dy), min(H, H - dy)), slice(max(0, dy), min(H, H + dy))
    xs, xd = slice(max(0, -dx), min(W, W - dx)), slice(max(0, dx), min(W, W + dx))
    out[ys, xs] = img[yd, xd]
    return out


def _softmax_apply(logits, c0):
    """The kernel softmax and its two renormalised applications (dilation 1, then 4), by numpy
    on shifted images (c0 [B, H, W, 3])."""
    z = logits - logits.max(-1, keepdims=True)
    K = np.exp(z) / np.exp(z).sum(-1, keepdims=True)
    offs = [(i // 5 - 2, i % 5 - 2) for i in range(25)]

    def apply(src, d):
        out, S = [], []
        for n in range(src.shape[0]):
            one = np.ones(src.shape[1:3] + (1,))
            out.append(sum(K[n, ..., i:i + 1] * _shift(src[n], d * ky, d * kx) for i, (ky, kx) in enumerate(offs)))
            S.append(sum(K[n, ..., i:i + 1] * _shift(one, d * ky, d * kx) for i, (ky, kx) in enumerate(offs)))
        return np.stack(out) / np.stack(S)
    c1 = apply(c0, 1)
    return K, c1, apply(c1, 4)


def test_rounding_mode_forward_is_the_rounded_composition():
    """quant = 1 equals the network composed layer by layer from the pinned convolution with the
    BF16 rounding applied to the weights and to each activation after its ReLU, then the softmax
    and both applications (written here with numpy); and it differs from the FP64 network."""
    f, c0, T, prm = rand_case(B=2, H=10, W=13, scale=0.3)
    f = oracle.bf16_round(f)                 # the features come in as BF16 values
    x = f
    for l, (w, b) in enumerate(oracle.kpn_unflatten(prm)):
        z = oracle.kpn_conv(x, oracle.bf16_round(w), b)
        x = oracle.bf16_round(np.maximum(z, 0.0)) if l < 3 else z
    K_want, c1_want, c2_want = _softmax_apply(x, c0)
    K, c1, c2 = oracle.kpn_forward(f, c0, prm, quant=True)
    assert np.allclose(K, K_want, rtol=1e-12, atol=1e-15)
    assert np.allclose(c2, c2_want, rtol=1e-12, atol=1e-15)
    _, _, c2_64 = oracle.kpn_forward(f, c0, prm)
    assert np.abs(c2_64 - c2).max() > 1e-6


def test_rounding_mode_gradient_of_the_logits_layer_matches_finite_differences():
    """In the rounding mode the loss is smooth in the logits layer's bias (nothing is rounded
    after it) and, with steps of one BF16 unit in the last place, in its weights; central
    differences there match the gradient within the rounding of the logits' gradient to BF16
    (relative 2^-8 per summand)."""
    f, c0, T, prm = rand_case(B=1, H=8, W=9, scale=0.3)
    f = oracle.bf16_round(f)
    prm = prm.copy()
    offs = np.cumsum([0] + [co * 9 * ci + co for ci, co in zip(oracle.KPN_CIN, oracle.KPN_COUT)])
    w3n = 25 * 9 * 32
    prm[offs[3]:offs[3] + w3n] = oracle.bf16_round(prm[offs[3]:offs[3] + w3n])
    loss, g = oracle.kpn_grad(f, c0, T, prm, quant=True)

    def L(p):
        _, _, c2 = oracle.kpn_forward(f, c0, p, quant=True)
        return float(np.mean((c2 - T) ** 2))
    assert loss == pytest.approx(L(prm), rel=1e-12)
    picks = [offs[3] + w3n + i for i in (0, 7, 12, 24)]          # biases of the logits layer
    picks += list(offs[3] + RNG.choice(w3n, 6, replace=False))    # its weights
    for k in picks:
        if k >= offs[3] + w3n:
            h = 1e-5
        else:                                                      # one BF16 ulp of the weight
            e = np.floor(np.log2(abs(prm[k]))) if prm[k] != 0 else -30
            h = 2.0 ** (e - 7)
        p1, p2 = prm.copy(), prm.copy()
        p1[k] += h
        p2[k] -= h
        fd = (L(p1) - L(p2)) / (2 * h)
        assert abs(g[k] - fd) <= 2 ** -7 * np.abs(fd) + 1e-9, (k, g[k], fd)


def _grad_by_chain_rule(f, c0, T, prm, rnd):
    """Loss gradient of the network on one image, written out from the chain rule with numpy:
    rnd() is applied where the rounding mode rounds (weights, activations after the ReLU, the
    logits' gradient, each data gradient after the ReLU mask)."""
    H, W = c0.shape[:2]
    layers = [(rnd(w), b) for w, b in oracle.kpn_unflatten(prm)]
    taps = [(t // 3 - 1, t % 3 - 1) for t in range(9)]
    xs, zs, x = [], [], f
    for l, (w, b) in enumerate(layers):
        z = b + sum(_shift(x, dy, dx) @ w[:, t, :].T for t, (dy, dx) in enumerate(taps))
        xs.append(x)
        zs.append(z)
        if l < 3:
            x = rnd(np.maximum(z, 0.0))
    zl = zs[3]
    K = np.exp(zl - zl.max(-1, keepdims=True))
    K /= K.sum(-1, keepdims=True)
    offs = [(i // 5 - 2, i % 5 - 2) for i in range(25)]
    inside = lambda d: np.stack([_shift(np.ones((H, W, 1)), d * ky, d * kx)[..., 0] for ky, kx in offs], -1)
    m1, m4 = inside(1), inside(4)
    S1, S4 = (K * m1).sum(-1), (K * m4).sum(-1)
    c1 = sum(K[..., i:i + 1] * _shift(c0, ky, kx) for i, (ky, kx) in enumerate(offs)) / S1[..., None]
    c2 = sum(K[..., i:i + 1] * _shift(c1, 4 * ky, 4 * kx) for i, (ky, kx) in enumerate(offs)) / S4[..., None]
    g2 = 2.0 * (c2 - T) / c2.size
    gK = np.zeros_like(K)
    g1 = np.zeros_like(c1)
    for i, (ky, kx) in enumerate(offs):
        gK[..., i] += m4[..., i] * ((g2 * (_shift(c1, 4 * ky, 4 * kx) - c2)).sum(-1) / S4)
        # c1(q) receives from p = q - 4 o_i
        g1 += _shift(m4[..., i:i + 1] * g2 * K[..., i:i + 1] / S4[..., None], -4 * ky, -4 * kx)
    for i, (ky, kx) in enumerate(offs):
        gK[..., i] += m1[..., i] * ((g1 * (_shift(c0, ky, kx) - c1)).sum(-1) / S1)
    dz = rnd(K * (gK - (K * gK).sum(-1, keepdims=True)))
    grads = [None] * 4
    for l in range(3, -1, -1):
        w, _ = layers[l]
        gw = np.stack([np.einsum("yxo,yxi->oi", dz, _shift(xs[l], dy, dx)) for dy, dx in taps], 1)
        grads[l] = (gw, dz.sum((0, 1)))
        if l == 0:
            break
        dx_ = sum(_shift(dz, -dy, -dx) @ w[:, t, :] for t, (dy, dx) in enumerate(taps))
        dz = rnd(np.where(zs[l - 1] > 0.0, dx_, 0.0))
    return np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads])


@pytest.mark.parametrize("quant", [False, True])
def test_gradient_equals_the_chain_rule_written_out(quant):
    """The oracle's gradient (FP64, and the rounding mode with its BF16 weights, activations and
    data gradients) equals the chain rule written out independently with numpy on a small image."""
    f, c0, T, prm = rand_case(B=1, H=7, W=9, scale=0.3)
    f = oracle.bf16_round(f)
    rnd = oracle.bf16_round if quant else (lambda a: np.asarray(a, np.float64))
    want = _grad_by_chain_rule(f[0], c0[0], T[0], prm, rnd)
    _, got = oracle.kpn_grad(f, c0, T, prm, quant=quant)
    scale = np.abs(want).max()
    assert np.allclose(got, want, rtol=1e-9, atol=1e-12 * scale)
