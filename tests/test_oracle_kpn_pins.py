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
