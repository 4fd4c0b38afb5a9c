"""Learned part on the GPU against the FP64 oracle: features, network forward (BF16 tensor-core
convolutions, FP32 accumulation), loss and per-layer gradients; training on pairs the plain
pipeline generates lowers the loss and gains PSNR against the plain output over the untrained
network; the fallback reproduces the plain pipeline on flagged tiles bit for bit.

The primary comparisons are element-wise against the oracle's rounding mode, which rounds to
BF16 exactly where the tensor-core path does (weights, activations, data gradients) and sums in
FP64: the forward output within 2e-3 of it at every pixel (the rare one-unit BF16 rounding flips)
and within 1e-4 at 99 % of them, each layer's gradient within 1 % relative L2.  Against the FP64 network (secondary) tolerances follow BF16 operands (8-bit
mantissa, unit roundoff u = 2^-9): the forward output must be within 40 dB PSNR of it.  Gradients: every layer between a weight and the loss
adds a BF16-rounded activation and a BF16-rounded data gradient, and the weight gradient is a
sum with cancellation over all pixels, so the bound grows with the depth below the loss:
relative L2 error <= 3 % x (layers between the weight and the loss + 1), cosine >= 0.999 at the
logits layer down to 0.995 at the first layer.  A wrong tap, transpose or mask moves the cosine
far below these bounds."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2312_06827_gb300 import kpn_train, scene, svgf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
RNG = np.random.default_rng(2024)


def bf16_round(a):
    """Round float32 values to BF16 (nearest even) and return them as float64."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_bits(a):
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return (((u + 0x7FFF + ((u >> 16) & 1)) >> 16) & 0xFFFF).astype(np.uint16).view(np.int16)


def random_batch(B, H, W):
    f10 = RNG.standard_normal((B, H, W, 10)).astype(np.float32)
    f10 = bf16_round(f10)                       # the network's input precision, both sides
    feats = np.zeros((B, H, W, 16), np.int16)
    feats[..., :10] = bf16_bits(f10)
    c0 = RNG.random((B, H, W, 4)).astype(np.float32)
    target = RNG.random((B, H, W, 4)).astype(np.float32)
    return f10, feats, c0, target


def make_kpn(max_px, seed=1):
    k = svgf.KPN(max_px)
    k.init_params(seed, last_scale=1.0)
    return k


def test_forward_matches_oracle():
    B, H, W = 2, 24, 40
    f10, feats, c0, _ = random_batch(B, H, W)
    k = make_kpn(B * H * W)
    out = torch.empty(B, H, W, 4, device="cuda")
    k.forward(torch.from_numpy(feats).cuda(), torch.from_numpy(c0).cuda(), out)
    torch.cuda.synchronize()
    g = out.cpu().numpy()[..., :3].astype(np.float64)
    _, _, o = oracle.kpn_forward(f10, c0[..., :3], k.params.cpu().numpy().astype(np.float64))
    mse = float(np.mean((g - o) ** 2))
    p = 10 * np.log10(1.0 / mse)
    print(f"[kpn] forward PSNR vs oracle {p:.1f} dB, max abs {np.abs(g - o).max():.2e}")
    assert p >= 40.0
    assert k.check_device() == 0


# Sizes for the element-wise comparisons: a small frame pair, and one with three 128-pixel
# column tiles (the last one pixel wide), two 16-row chunks per image and 51 images, i.e. 306
# tiles for a grid capped at 2 x 152 blocks: the column-tile halo and a block's second tile.
SIZES = [(2, 24, 40), (51, 17, 257)]
# Element-wise bounds on the output colour against the rounding-mode oracle.  Away from rounding
# boundaries the two differ by FP32 against FP64 sums (~1e-6 of the colour).  An activation whose
# FP32 value lies within that distance of a BF16 rounding boundary may round the other way: one
# BF16 unit (at most 2^-7 relative) moves a next-layer sum by |w| 2^-7 |a| (|w| <= 0.3 for these
# Kaiming-initialised weights), i.e. up to ~2e-3 of a logit, and a logit error moves the colour
# (a convex combination of colours in [0, 1]) by at most as much.  Such pixels are few.
FWD_ABS = 2e-3
FWD_MEAN = 1e-5
FWD_P99 = 1e-4
GRAD_REL = 0.01     # relative L2 bound per layer against the rounding-mode oracle


@pytest.mark.parametrize("B,H,W", SIZES)
def test_forward_matches_rounding_oracle_elementwise(B, H, W):
    """The forward output against the oracle in its rounding mode (BF16 weights and activations
    where the tensor-core path keeps them, FP64 sums): every pixel within FWD_ABS.  What remains
    is FP32 accumulation and the rare activation whose FP32 value sits next to a BF16 rounding
    boundary and rounds the other way (one BF16 unit, 2^-8 relative, in one of 288 summands of
    the next layer).  The FP64 network is the secondary check (PSNR >= 40 dB)."""
    f10, feats, c0, _ = random_batch(B, H, W)
    k = make_kpn(B * H * W)
    out = torch.empty(B, H, W, 4, device="cuda")
    k.forward(torch.from_numpy(feats).cuda(), torch.from_numpy(c0).cuda(), out)
    torch.cuda.synchronize()
    g = out.cpu().numpy()[..., :3].astype(np.float64)
    prm = k.params.cpu().numpy().astype(np.float64)
    _, _, oq = oracle.kpn_forward(f10, c0[..., :3], prm, quant=True)
    err = np.abs(g - oq)
    p99 = float(np.quantile(err, 0.99))
    print(f"[kpn] {B}x{H}x{W} forward vs rounding oracle: max abs {err.max():.2e}, p99 {p99:.2e}, "
          f"mean {err.mean():.2e}")
    assert err.max() <= FWD_ABS and p99 <= FWD_P99 and err.mean() <= FWD_MEAN
    _, _, o = oracle.kpn_forward(f10, c0[..., :3], prm)
    assert 10 * np.log10(1.0 / float(np.mean((g - o) ** 2))) >= 40.0
    assert k.check_device() == 0


@pytest.mark.parametrize("B,H,W,seed", [(2, 16, 24, 3), (2, 16, 24, 4), (51, 17, 257, 5)])
def test_gradients_match_rounding_oracle_per_layer(B, H, W, seed):
    """Per-layer loss gradients against the oracle's rounding mode (BF16 weights, activations and
    data gradients as the tensor-core kernels keep them): relative L2 <= GRAD_REL, cosine >=
    0.9999 in every layer, including the size with several column tiles and more tiles than
    blocks."""
    f10, feats, c0, target = random_batch(B, H, W)
    k = make_kpn(B * H * W, seed=seed)
    loss = k.compute_grad(torch.from_numpy(feats).cuda(), torch.from_numpy(c0).cuda(),
                          torch.from_numpy(target).cuda())
    torch.cuda.synchronize()
    g = k.grad.cpu().numpy().astype(np.float64)
    lo, go = oracle.kpn_grad(f10, c0[..., :3], target[..., :3], k.params.cpu().numpy().astype(np.float64),
                             quant=True)
    assert float(loss.item()) == pytest.approx(lo, rel=1e-3)
    off = 0
    for l, (ci, co) in enumerate(zip(oracle.KPN_CIN, oracle.KPN_COUT)):
        for name, n in (("W", co * 9 * ci), ("b", co)):
            a, b = g[off:off + n], go[off:off + n]
            rel = np.linalg.norm(a - b) / np.linalg.norm(b)
            cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))
            print(f"[kpn] {B}x{H}x{W} layer {l} {name} vs rounding oracle: rel L2 {rel:.2e}, cosine {cos:.7f}")
            assert rel <= GRAD_REL and cos >= 0.9999, (l, name, rel, cos)
            off += n
    assert k.check_device() == 0


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    """Failure detection without a fault: the self-test waits, with the convolutions' bounded
    wait, on a barrier phase nothing completes.  The wait gives up, the error word reads 2
    (SVGF_ERR_TIMEOUT from the C call), reading clears it, and the same handle then runs a
    forward pass that matches the oracle with a clean word."""
    B, H, W = 1, 16, 24
    f10, feats, c0, _ = random_batch(B, H, W)
    k = make_kpn(B * H * W)
    for tries in (1, 1000):
        k.wait_selftest(tries)
        assert k.check_device() == 2
        assert k.check_device() == 0            # cleared by the read
    w = ctypes.c_int()
    k.wait_selftest(10)
    assert k._L.svgf_kpn_check_device(k._k, ctypes.byref(w), None) == 4 and w.value == 2
    for bad in (0, -1, (1 << 20) + 1):
        with pytest.raises(svgf.SvgfError):
            k.wait_selftest(bad)
    out = torch.empty(B, H, W, 4, device="cuda")
    k.forward(torch.from_numpy(feats).cuda(), torch.from_numpy(c0).cuda(), out)
    torch.cuda.synchronize()
    _, _, o = oracle.kpn_forward(f10, c0[..., :3], k.params.cpu().numpy().astype(np.float64))
    assert 10 * np.log10(1.0 / float(np.mean((out.cpu().numpy()[..., :3] - o) ** 2))) >= 40.0
    assert k.check_device() == 0


@pytest.mark.parametrize("seed", [3, 4])
def test_gradients_match_oracle_per_layer(seed):
    B, H, W = 2, 16, 24
    f10, feats, c0, target = random_batch(B, H, W)
    k = make_kpn(B * H * W, seed=seed)
    loss = k.compute_grad(torch.from_numpy(feats).cuda(), torch.from_numpy(c0).cuda(),
                          torch.from_numpy(target).cuda())
    torch.cuda.synchronize()
    g = k.grad.cpu().numpy().astype(np.float64)
    lo, go = oracle.kpn_grad(f10, c0[..., :3], target[..., :3], k.params.cpu().numpy().astype(np.float64))
    assert float(loss.item()) == pytest.approx(lo, rel=1e-2)
    off, res = 0, []
    for l, (ci, co) in enumerate(zip(oracle.KPN_CIN, oracle.KPN_COUT)):
        for name, n in (("W", co * 9 * ci), ("b", co)):
            a, b = g[off:off + n], go[off:off + n]
            rel = np.linalg.norm(a - b) / np.linalg.norm(b)
            cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))
            print(f"[kpn] layer {l} {name}: rel L2 {rel:.2e}, cosine {cos:.6f}")
            res.append((l, name, rel, cos))
            off += n
    for l, name, rel, cos in res:
        depth = 3 - l                      # layers between this one and the loss
        assert rel <= 0.03 * (depth + 1), (l, name, rel, cos)
        assert cos >= 0.999 - 0.0013 * depth, (l, name, rel, cos)


def test_features_match_oracle():
    sc = scene.SceneConfig(96, 64, n_spheres=8, moving_sphere=True, seed=12)
    fr = scene.render_frame(sc, 0)
    H, W = 64, 96
    cv = RNG.random((H, W, 4)).astype(np.float32)
    d = svgf.Denoiser(svgf.default_config(W, H))
    k = svgf.KPN(H * W, train=False)
    feats = torch.empty(H, W, 16, dtype=torch.int16, device="cuda")
    c0 = torch.empty(H, W, 4, device="cuda")
    dv = {n: torch.from_numpy(fr[n]).cuda() for n in ("noisy", "gbuf_nz", "motion", "roughness", "albedo")}
    f = svgf.make_frame(dv["noisy"], dv["gbuf_nz"], dv["motion"], dv["roughness"])
    k.features(d, torch.from_numpy(cv).cuda(), f, dv["albedo"], feats, c0)
    torch.cuda.synchronize()
    got = (feats.cpu().numpy().view(np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    want = oracle.kpn_features(cv, fr["gbuf_nz"], fr["albedo"])
    assert np.allclose(got[..., :10], want, rtol=2 ** -8, atol=1e-6)
    assert np.all(got[..., 10:] == 0.0)
    assert np.array_equal(c0.cpu().numpy(), cv)


@pytest.fixture(scope="module")
def small_data():
    scenes = [scene.SceneConfig(192, 128, n_spheres=14, moving_sphere=True, seed=1000 + i) for i in range(4)]
    train = kpn_train.make_examples(scenes[:3], frames_per_scene=3)
    held = kpn_train.make_examples(scenes[3:], frames_per_scene=2)
    return train, held


def test_training_lowers_loss_and_gains_over_untrained(small_data):
    train, held = small_data
    k = svgf.KPN(8 * 64 * 64)
    k.init_params(0)
    untrained, pass0 = kpn_train.evaluate(k, held)
    losses = kpn_train.train(k, train, steps=400, batch=8, crop=64, lr=2e-3, seed=0, log_every=100)
    trained, _ = kpn_train.evaluate(k, held)
    print(f"[kpn] losses {losses}; held-out PSNR vs plain: pass-0 only {pass0:.2f} dB, "
          f"untrained {untrained:.2f} dB, trained {trained:.2f} dB")
    assert losses[-1][1] < 0.5 * losses[0][1]
    assert trained > untrained + 3.0
    assert trained > pass0


def test_fallback_reproduces_plain_pipeline_on_flagged_tiles(small_data):
    sc = scene.SceneConfig(160, 96, n_spheres=10, moving_sphere=True, seed=7)
    W, H = sc.width, sc.height
    cfg = svgf.default_config(W, H)
    k = svgf.KPN(W * H, train=False)
    k.init_params(5)
    a, b = svgf.Denoiser(cfg), svgf.Denoiser(cfg)
    prev = None
    for t in range(3):
        fr = scene.render_frame(sc, t)
        dv = {n: torch.from_numpy(fr[n]).cuda() for n in ("noisy", "gbuf_nz", "motion", "roughness", "albedo")}
        f = svgf.make_frame(dv["noisy"], dv["gbuf_nz"], dv["motion"], dv["roughness"], prev)
        plain = torch.empty(H, W, 4, device="cuda")
        a.denoise_frame(f, plain)
        learned = torch.empty(H, W, 4, device="cuda")
        n = k.denoise_frame(b, f, dv["albedo"], learned, detail_threshold=-1.0)   # every tile falls back
        torch.cuda.synchronize()
        assert n == ((W + 31) // 32) * ((H + 31) // 32)
        assert torch.equal(plain[..., :3], learned[..., :3])
        none = torch.empty(H, W, 4, device="cuda")
        c = svgf.Denoiser(cfg)
        assert k.denoise_frame(c, f, dv["albedo"], none, detail_threshold=1e30) == 0
        prev = dv["gbuf_nz"]


def _tile_detail(c0, T=32):
    """The fallback statistic in FP64: per 32x32 tile, the population standard deviation of the
    luminance of c0's colour (ragged edge tiles over their in-image pixels)."""
    H, W = c0.shape[:2]
    lum = c0[..., :3].astype(np.float64) @ np.array([0.2126, 0.7152, 0.0722])
    out = np.zeros(((H + T - 1) // T, (W + T - 1) // T))
    for ty in range(out.shape[0]):
        for tx in range(out.shape[1]):
            out[ty, tx] = lum[ty * T:(ty + 1) * T, tx * T:(tx + 1) * T].std()
    return out


@pytest.mark.parametrize("mode,prec", [(svgf.ATROUS_5X5, svgf.FP32), (svgf.SEPARABLE, svgf.FP32),
                                       (svgf.ATROUS_5X5, svgf.FP16)])
def test_partial_fallback_is_plain_on_flagged_tiles_and_learned_elsewhere(mode, prec):
    """A threshold that flags a few percent of the tiles: the flagged tiles equal the plain
    pipeline bit for bit (so the plain passes, run only on the tiles the flagged ones depend on,
    covered every pixel they read), the others equal the learned frame without fallback, and the
    reported count is the number of tiles above the threshold."""
    sc = scene.SceneConfig(1280, 704, n_spheres=40, moving_sphere=True, seed=11)
    W, H = sc.width, sc.height
    cfg = svgf.default_config(W, H)
    cfg.spatial_mode, cfg.precision = mode, prec
    k = svgf.KPN(W * H, train=False)
    k.init_params(3)
    plain_d, fb_d, nofb_d, stage_d = (svgf.Denoiser(cfg) for _ in range(4))
    tiles_x, tiles_y = (W + 31) // 32, (H + 31) // 32
    prev = None
    for t in range(3):
        fr = scene.render_frame(sc, t)
        dv = {n: torch.from_numpy(fr[n]).cuda() for n in ("noisy", "gbuf_nz", "motion", "roughness", "albedo")}
        f = svgf.make_frame(dv["noisy"], dv["gbuf_nz"], dv["motion"], dv["roughness"], prev)
        # the pass-0 colour the statistic is taken on, through the stage calls
        cv, cv0 = torch.empty(H, W, 4, device="cuda"), torch.empty(H, W, 4, device="cuda")
        stage_d.reproject_accumulate(f, cv)
        stage_d.atrous(0, f, cv, cv0)
        feats = torch.empty(H, W, 16, dtype=torch.int16, device="cuda")
        c0 = torch.empty(H, W, 4, device="cuda")
        k.features(stage_d, cv0, f, dv["albedo"], feats, c0)
        torch.cuda.synchronize()
        det = _tile_detail(c0.cpu().numpy())
        # a threshold in the widest gap of the sorted statistics between the 93rd and the 97th
        # percentile (3-7 % of the tiles fall back)
        v = np.sort(det.ravel())
        i0, i1 = int(0.93 * v.size), int(0.97 * v.size)
        gaps = [(v[i + 1] - v[i]) / max(v[i + 1], 1e-12) for i in range(i0, i1)]
        i = i0 + int(np.argmax(gaps))
        assert gaps[i - i0] > 1e-3
        tau = 0.5 * (v[i] + v[i + 1])
        flagged = det > tau
        plain = torch.empty(H, W, 4, device="cuda")
        plain_d.denoise_frame(f, plain)
        got = torch.empty(H, W, 4, device="cuda")
        n = k.denoise_frame(fb_d, f, dv["albedo"], got, detail_threshold=float(tau))
        learned = torch.empty(H, W, 4, device="cuda")
        assert k.denoise_frame(nofb_d, f, dv["albedo"], learned) == 0
        torch.cuda.synchronize()
        assert n == int(flagged.sum()) and 0 < n < tiles_x * tiles_y // 10
        px = np.kron(flagged, np.ones((32, 32), bool))[:H, :W]
        g, p_, l_ = got.cpu().numpy(), plain.cpu().numpy(), learned.cpu().numpy()
        assert np.array_equal(g[px], p_[px])
        assert np.array_equal(g[~px], l_[~px])
        print(f"[kpn] frame {t}: {n} of {tiles_x * tiles_y} tiles fall back (tau {tau:.4g})")
        prev = dv["gbuf_nz"]
    assert k.check_device() == 0


def test_inference_with_fp16_kernels_matches_fp32_kernels():
    """The inference call passes the 25 kernel weights per pixel as FP16 (pixel-major); the same
    frame through the stage calls, the FP32-kernel forward and the inverse tone map agrees with
    it to FP16 rounding of the weights (<= 2e-3 absolute in tone-mapped space, channel 3 exact)."""
    sc = scene.SceneConfig(200, 120, n_spheres=12, moving_sphere=True, seed=31)
    W, H = sc.width, sc.height
    cfg = svgf.default_config(W, H)
    k = svgf.KPN(W * H, train=False)
    k.init_params(2, last_scale=1.0)
    fr = scene.render_frame(sc, 0)
    dv = {n: torch.from_numpy(fr[n]).cuda() for n in ("noisy", "gbuf_nz", "motion", "roughness", "albedo")}
    f = svgf.make_frame(dv["noisy"], dv["gbuf_nz"], dv["motion"], dv["roughness"])
    got = torch.empty(H, W, 4, device="cuda")
    assert k.denoise_frame(svgf.Denoiser(cfg), f, dv["albedo"], got, detail_threshold=float("inf")) == 0
    d = svgf.Denoiser(cfg)
    cv, cv0 = torch.empty(H, W, 4, device="cuda"), torch.empty(H, W, 4, device="cuda")
    d.reproject_accumulate(f, cv)
    d.atrous(0, f, cv, cv0)
    feats = torch.empty(1, H, W, 16, dtype=torch.int16, device="cuda")
    c0 = torch.empty(1, H, W, 4, device="cuda")
    k.features(d, cv0, f, dv["albedo"], feats[0], c0[0])
    c2 = torch.empty(1, H, W, 4, device="cuda")
    k.forward(feats, c0, c2)
    ref = torch.empty(H, W, 4, device="cuda")
    d.inverse_tonemap(c2[0], ref)
    torch.cuda.synchronize()
    g, r = got.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)

    def reinhard(c):       # back to the tone-mapped space the network and the applications work in
        return c / (1.0 + c @ np.array([0.2126, 0.7152, 0.0722]))[..., None]

    err = np.abs(reinhard(g[..., :3]) - reinhard(r[..., :3]))
    print(f"[kpn] FP16 against FP32 kernels (tone-mapped): max abs {err.max():.2e}, mean {err.mean():.2e}")
    assert err.max() <= 2e-3
    assert np.array_equal(g[..., 3], cv0.cpu().numpy()[..., 3])
    assert k.check_device() == 0


def test_checkpoint_round_trip_and_resume(small_data):
    """svgf_kpn_save / svgf_kpn_load: the parameters and Adam state come back bit for bit, a
    resumed run follows the original (the weight gradients are reduced with float atomics, so the
    comparison after further steps is to rounding), a damaged header is refused, and an
    inference-only handle loads the parameters alone."""
    train, held = small_data
    a = svgf.KPN(8 * 64 * 64)
    a.init_params(3)
    kpn_train.train(a, train, steps=20, batch=8, crop=64, lr=2e-3, seed=1, log_every=100)
    blob = a.save()
    n = svgf.KPN_PARAM_COUNT
    assert len(blob) == 24 + 4 * 3 * n
    b = svgf.KPN(8 * 64 * 64)
    b.init_params(9)
    b.load(blob)
    torch.cuda.synchronize()
    assert torch.equal(a.params, b.params)
    assert torch.equal(a.adam_m, b.adam_m) and torch.equal(a.adam_v, b.adam_v)
    assert b.save() == blob
    kpn_train.train(a, train, steps=5, batch=8, crop=64, lr=2e-3, seed=2, log_every=100)
    kpn_train.train(b, train, steps=5, batch=8, crop=64, lr=2e-3, seed=2, log_every=100)
    torch.cuda.synchronize()
    assert torch.allclose(a.params, b.params, rtol=1e-4, atol=1e-6)
    bad = bytearray(blob)
    bad[0] ^= 1
    with pytest.raises(svgf.SvgfError):
        b.load(bytes(bad))
    with pytest.raises(svgf.SvgfError):
        b.load(blob[:100])
    c = svgf.KPN(64 * 64, train=False)
    c.load(blob)
    torch.cuda.synchronize()
    assert torch.equal(c.params, torch.from_numpy(
        np.frombuffer(blob, np.float32, count=n, offset=24).copy()).cuda())
    assert len(c.save()) == 24 + 4 * n
