"""The four-layer network kernel (k_kpn_net, svgf_kpn_predict form 0) against the layer-by-layer
convolutions and against the oracle.

The kernel keeps the activations in shared memory, computes each layer on 128 lanes of which it
keeps the exact 122, recomputes the rows a chunk's neighbours also compute, and writes zeros for
the next layer wherever a layer's output lies outside the image.  Its accumulation order is the
per-layer kernels' (input rows, then horizontal taps, then 16-channel steps, in one FP32
accumulator), and its epilogues are theirs, so the per-pixel kernels must equal those of the
per-layer path bit for bit: one segment and several, ragged widths, one-row images, batches, a
grid whose blocks walk two chunks, and the full 1920 x 1080 frame the learned form runs.  The
oracle's rounding mode (BF16 weights and activations, FP64 sums) checks the kernels element-wise
within FP16 rounding plus the rare one-unit BF16 flip of an activation."""
import numpy as np
import pytest

import oracle
from paper_2312_06827_gb300 import svgf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
RNG = np.random.default_rng(77)


def bf16_bits(a):
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return (((u + 0x7FFF + ((u >> 16) & 1)) >> 16) & 0xFFFF).astype(np.uint16).view(np.int16)


def features(B, H, W):
    f10 = RNG.standard_normal((B, H, W, 10)).astype(np.float32)
    feats = np.zeros((B, H, W, 16), np.int16)
    feats[..., :10] = bf16_bits(f10)
    f10 = (feats[..., :10].astype(np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return f10, torch.from_numpy(feats).cuda()


def predict(k, feats, form):
    B, H, W = feats.shape[:3]
    out = torch.full((B, H, W, 32), -1, dtype=torch.int16, device="cuda")
    k.predict(feats, out, form=form)
    return out


@pytest.mark.parametrize("B,H,W", [(1, 1, 5), (1, 7, 130), (2, 17, 250), (1, 120, 200), (1, 37, 371),
                                   (3, 9, 122), (1, 64, 123), (20, 24, 1000), (1, 1080, 1920)])
def test_fused_network_equals_per_layer_bitwise(B, H, W):
    k = svgf.KPN(B * H * W, train=False)
    k.init_params(5, last_scale=1.0)
    _, feats = features(B, H, W)
    a = predict(k, feats, 0)
    b = predict(k, feats, 1)
    torch.cuda.synchronize()
    assert k.check_device() == 0
    same = (a == b).all(dim=-1)
    assert bool(same.all()), f"{int((~same).sum())} of {B * H * W} pixels differ, first at {torch.nonzero(~same)[0].tolist()}"
    assert bool((a[..., 25:] == 0).all())               # the 7 unused weights are zero


@pytest.mark.parametrize("B,H,W", [(1, 1, 5), (1, 7, 130), (2, 17, 250), (1, 37, 371), (3, 9, 126),
                                   (1, 64, 127), (20, 24, 1000), (1, 1080, 1920)])
def test_two_layer_kernels_equal_per_layer_bitwise(B, H, W):
    """Form 2 (layers 0-1, then 2-3, each pair in one kernel with 126 exact lanes a segment)
    against the per-layer path, bit for bit."""
    k = svgf.KPN(B * H * W, train=False)
    k.init_params(6, last_scale=1.0)
    _, feats = features(B, H, W)
    a = predict(k, feats, 2)
    b = predict(k, feats, 1)
    torch.cuda.synchronize()
    assert k.check_device() == 0
    same = (a == b).all(dim=-1)
    assert bool(same.all()), f"{int((~same).sum())} of {B * H * W} pixels differ, first at {torch.nonzero(~same)[0].tolist()}"


def test_fused_network_kernels_match_rounding_oracle():
    """Element-wise against the oracle's rounding mode at three column segments (121 .. 366
    px), both image edges and a ragged last segment: within FP16 rounding of the weights (half a
    unit, 2^-12 below 1) at 99 % of the values, 2e-3 at every one (an activation next to a BF16
    rounding boundary can round the other way and move a logit by up to ~2e-3)."""
    B, H, W = 1, 40, 300
    k = svgf.KPN(B * H * W, train=False)
    k.init_params(9, last_scale=1.0)
    f10, feats = features(B, H, W)
    got = predict(k, feats, 0)
    torch.cuda.synchronize()
    g = got.cpu().numpy()[..., :25].view(np.float16).astype(np.float64)
    prm = k.params.cpu().numpy().astype(np.float64)
    K, _, _ = oracle.kpn_forward(f10, np.zeros((B, H, W, 3)), prm, quant=True)
    err = np.abs(g - K)
    p99 = float(np.quantile(err, 0.99))
    print(f"[kpn-net] kernels vs rounding oracle: max abs {err.max():.2e}, p99 {p99:.2e}, mean {err.mean():.2e}")
    assert err.max() <= 2e-3 and p99 <= 2.5e-4 and err.mean() <= 1e-5
    assert np.allclose(g.sum(-1), 1.0, atol=25 * 2.5e-4)
    assert k.check_device() == 0


def test_predict_rejects_bad_arguments():
    k = svgf.KPN(64, train=False)
    k.init_params(1)
    _, feats = features(1, 8, 8)
    out = torch.empty(1, 8, 8, 32, dtype=torch.int16, device="cuda")
    with pytest.raises(svgf.SvgfError):
        k.predict(feats, out, form=3)
    _, big = features(1, 9, 8)
    with pytest.raises(svgf.SvgfError):
        k.predict(big, torch.empty(1, 9, 8, 32, dtype=torch.int16, device="cuda"))


@pytest.mark.parametrize("W,H", [(200, 120), (333, 77), (31, 9), (1920, 1080)])
def test_learned_frame_equals_its_stages(W, H):
    """The learned frame equals its stages called one by one (temporal stage, pass 0, features,
    the network by each of its three forms, the two applications with the inverse tone map), bit
    for bit."""
    from paper_2312_06827_gb300 import scene
    sc = scene.SceneConfig(W, H, n_spheres=12, moving_sphere=True, seed=41)
    cfg = svgf.default_config(W, H)
    k = svgf.KPN(W * H, train=False)
    k.init_params(3, last_scale=1.0)
    fr = scene.render_frame(sc, 0)
    dv = {n: torch.from_numpy(fr[n]).cuda() for n in ("noisy", "gbuf_nz", "motion", "roughness", "albedo")}
    f = svgf.make_frame(dv["noisy"], dv["gbuf_nz"], dv["motion"], dv["roughness"])
    frame_out = torch.empty(H, W, 4, device="cuda")
    assert k.denoise_frame(svgf.Denoiser(cfg), f, dv["albedo"], frame_out) == 0
    d = svgf.Denoiser(cfg)
    cv, cv0 = torch.empty(H, W, 4, device="cuda"), torch.empty(H, W, 4, device="cuda")
    d.reproject_accumulate(f, cv)
    d.atrous(0, f, cv, cv0)
    feats = torch.empty(1, H, W, 16, dtype=torch.int16, device="cuda")
    c0 = torch.empty(1, H, W, 4, device="cuda")
    k.features(d, cv0, f, dv["albedo"], feats[0], c0[0])
    for form in (1, 0, 2):
        kern = predict(k, feats, form)
        out = torch.full((H, W, 4), -1.0, device="cuda")
        k.apply(d, kern[0], c0[0], out)
        torch.cuda.synchronize()
        assert torch.equal(out, frame_out), form
    assert k.check_device() == 0
