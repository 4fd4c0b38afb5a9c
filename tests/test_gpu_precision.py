"""Reduced-precision storage (FP16 colour with BF16 variance; all-BF16 variant) against the FP64
oracle: PSNR of the tone-mapped output per frame and per stage (temporal, each a-trous pass,
final), at 128x128 and at 4K; the stage-composition rule and the state round trip in 16-bit
storage.  Bar: FP16 storage >= 60 dB PSNR on tone-mapped output; the BF16 variant is reported."""
import numpy as np
import pytest

import oracle
from paper_2312_06827_gb300 import scene, svgf

from parity import LUMA, oracle_config, tm64

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP16_PSNR_DB = 60.0
BF16_PSNR_FLOOR_DB = 40.0     # sanity floor for the variant; its measured value is printed
KEYS = ("noisy", "gbuf_nz", "motion", "roughness")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def decode(t, prec):
    """8-byte records [H, W, 4] of 16-bit fields -> float64 [H, W, 4]."""
    torch.cuda.synchronize()
    u = t.cpu().numpy().view(np.uint16)
    bf = lambda v: (v.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    out = np.empty(u.shape, np.float64)
    out[..., :3] = u[..., :3].view(np.float16).astype(np.float64) if prec == svgf.FP16 else bf(u[..., :3])
    out[..., 3] = bf(u[..., 3])
    return out


def psnr(a, b):
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10.0 * np.log10(1.0 / mse)


def cv_buffer(H, W, prec):
    if prec == svgf.FP32:
        return torch.empty(H, W, 4, device="cuda")
    return torch.empty(H, W, 4, dtype=torch.int16, device="cuda")


@pytest.mark.parametrize("prec", [svgf.FP16, svgf.BF16])
@pytest.mark.parametrize("sc,n", [(scene.C0_128, 4), (scene.SceneConfig(256, 192, n_spheres=12, moving_sphere=True, seed=9), 6)])
def test_sixteen_bit_sequence_psnr(prec, sc, n):
    cfg = svgf.default_config(sc.width, sc.height)
    cfg.precision = prec
    d = svgf.Denoiser(cfg)
    seq = oracle.Sequence(sc.width, sc.height, oracle_config(cfg))
    prev = None
    for t in range(n):
        fr = scene.render_frame(sc, t)
        dv = {k: dev(fr[k]) for k in KEYS}
        out = torch.empty(sc.height, sc.width, 4, device="cuda")
        d.denoise_frame(svgf.make_frame(dv["noisy"], dv["gbuf_nz"], dv["motion"], dv["roughness"], prev), out)
        torch.cuda.synchronize()
        g = out.cpu().numpy().astype(np.float64)
        o = seq.step(fr["noisy"], fr["gbuf_nz"], fr["motion"], fr["roughness"])
        p = psnr(tm64(g[..., :3], cfg), tm64(o[..., :3], cfg))
        print(f"[precision] {'FP16' if prec == svgf.FP16 else 'BF16'} {sc.width}x{sc.height} frame {t}: PSNR {p:.2f} dB")
        assert p >= (FP16_PSNR_DB if prec == svgf.FP16 else BF16_PSNR_FLOOR_DB), (t, p)
        prev = dv["gbuf_nz"]


@pytest.mark.parametrize("prec", [svgf.FP16, svgf.BF16])
def test_4k_error_per_stage(prec):
    """3840x2160, frame 0 through denoise_frame, frame 1 stage by stage on both sides; PSNR of
    each stage's tone-mapped colour (temporal, a-trous 0..4) and of the final output."""
    sc = scene.C2_4K
    W, H = sc.width, sc.height
    cfg = svgf.default_config(W, H)
    cfg.precision = prec
    oc = oracle_config(cfg)
    f0, f1 = scene.render_frame(sc, 0), scene.render_frame(sc, 1)
    d = svgf.Denoiser(cfg)
    d0 = {k: dev(f0[k]) for k in KEYS}
    out = torch.empty(H, W, 4, device="cuda")
    d.denoise_frame(svgf.make_frame(d0["noisy"], d0["gbuf_nz"], d0["motion"], d0["roughness"]), out)
    seq = oracle.Sequence(W, H, oc)
    seq.step(f0["noisy"], f0["gbuf_nz"], f0["motion"], f0["roughness"])

    d1 = {k: dev(f1[k]) for k in KEYS}
    fr = svgf.make_frame(d1["noisy"], d1["gbuf_nz"], d1["motion"], d1["roughness"], d0["gbuf_nz"])
    bufs = [cv_buffer(H, W, prec), cv_buffer(H, W, prec)]
    d.reproject_accumulate(fr, bufs[0])
    o_cv, _, _ = oracle.temporal(f1["noisy"], f1["gbuf_nz"], f0["gbuf_nz"], f1["motion"], seq.hist_rgb,
                                 seq.hist_mom, True, oc)
    name = "FP16" if prec == svgf.FP16 else "BF16"
    stages = [("temporal", psnr(decode(bufs[0], prec)[..., :3], o_cv[..., :3]))]
    cur = o_cv
    for it in range(cfg.atrous_iters):
        d.atrous(it, fr, bufs[it & 1], bufs[(it + 1) & 1])
        cur = oracle.atrous(cur, f1["gbuf_nz"], f1["roughness"], it, oc)
        g = decode(bufs[(it + 1) & 1], prec)
        stages.append((f"atrous {it}", psnr(g[..., :3], cur[..., :3])))
        lg = g[..., :3] @ LUMA
        var_rel = np.abs(g[..., 3] - cur[..., 3]) / np.maximum(np.maximum(np.abs(cur[..., 3]), (cur[..., :3] @ LUMA) ** 2), 1e-12)
        print(f"[precision] {name} 4K atrous {it}: variance rel err p99 {np.percentile(var_rel, 99):.2e}")
        del lg
    final = torch.empty(H, W, 4, device="cuda")
    d.inverse_tonemap(bufs[cfg.atrous_iters & 1], final)
    torch.cuda.synchronize()
    o_final = oracle.inverse_tonemap(cur[..., :3].reshape(-1, 3), oc).reshape(H, W, 3)
    stages.append(("final", psnr(tm64(final.cpu().numpy()[..., :3], cfg), tm64(o_final, cfg))))
    for s_name, p in stages:
        print(f"[precision] {name} 4K frame 1 {s_name}: PSNR {p:.2f} dB")
    floor = FP16_PSNR_DB if prec == svgf.FP16 else BF16_PSNR_FLOOR_DB
    assert all(p >= floor for _, p in stages), stages


@pytest.mark.parametrize("prec", [svgf.FP16, svgf.BF16])
def test_sixteen_bit_composition_and_state(prec):
    sc = scene.SceneConfig(160, 96, n_spheres=8, moving_sphere=True, seed=4)
    W, H = sc.width, sc.height
    for mode in (svgf.ATROUS_5X5, svgf.SEPARABLE):
        cfg = svgf.default_config(W, H)
        cfg.precision, cfg.spatial_mode = prec, mode
        a, b = svgf.Denoiser(cfg), svgf.Denoiser(cfg)
        prev = None
        for t in range(3):
            fr = scene.render_frame(sc, t)
            dv = {k: dev(fr[k]) for k in KEYS}
            f = svgf.make_frame(dv["noisy"], dv["gbuf_nz"], dv["motion"], dv["roughness"], prev)
            whole = torch.empty(H, W, 4, device="cuda")
            a.denoise_frame(f, whole)
            cv = [cv_buffer(H, W, prec), cv_buffer(H, W, prec)]
            b.reproject_accumulate(f, cv[0])
            for it in range(cfg.atrous_iters):
                b.atrous(it, f, cv[it & 1], cv[(it + 1) & 1])
            staged = torch.empty(H, W, 4, device="cuda")
            b.inverse_tonemap(cv[cfg.atrous_iters & 1], staged)
            torch.cuda.synchronize()
            assert torch.equal(whole, staged)
            prev = dv["gbuf_nz"]
        # state export -> import into a fresh handle reproduces the next frame bit for bit
        h, m = torch.empty(H, W, 4, device="cuda"), torch.empty(H, W, 4, device="cuda")
        a.history_export(h, m)
        c = svgf.Denoiser(cfg)
        c.history_import(h, m, True)
        fr = scene.render_frame(sc, 3)
        dv = {k: dev(fr[k]) for k in KEYS}
        f = svgf.make_frame(dv["noisy"], dv["gbuf_nz"], dv["motion"], dv["roughness"], prev)
        oa, oc_ = torch.empty(H, W, 4, device="cuda"), torch.empty(H, W, 4, device="cuda")
        a.denoise_frame(f, oa)
        c.denoise_frame(f, oc_)
        torch.cuda.synchronize()
        assert torch.equal(oa, oc_)
        assert float(m[..., 2].max()) == 3.0
