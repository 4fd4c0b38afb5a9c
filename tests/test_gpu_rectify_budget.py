"""Variance colour clipping (Sec. 3.1) and the roughness-adapted a-trous pass budget (Sec. 3.5)
on the GPU against the FP64 oracle: the stand-alone rectification stage, every a-trous pass
with pixels of every budget, whole sequences in both spatial modes, the stage-composition rule
in FP32 and FP16 storage, and the batched path bit for bit against single streams.  Pixels past
their budget must keep their input exactly."""
import numpy as np
import pytest

import oracle
from paper_2312_06827_gb300 import scene, svgf

from parity import COLOUR_TOL, VAR_TOL, colour_err, oracle_config, var_err
from test_gpu_parity import check_sequence, dev, host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
KEYS = ("noisy", "gbuf_nz", "motion", "roughness")
R05 = float(np.float32(0.05))


def budget_roughness(r):
    """Roughness with every budget class in 12-pixel blocks across the image: 0 (iter_count0
    passes), exactly 0.05 or 0.03 (iter_count1 passes), and the scene's own roughness where it
    is above 0.06 (all passes, both adaptive start levels; 0.5 elsewhere)."""
    r = np.asarray(r, np.float32)
    H, W = r.shape
    yy, xx = np.mgrid[0:H, 0:W]
    cls = (xx // 12 + 2 * (yy // 12)) % 3
    low = np.where((xx // 12) % 2 == 0, np.float32(R05), np.float32(0.03))
    high = np.where(r > 0.06, r, np.float32(0.5))
    return np.where(cls == 0, np.float32(0.0), np.where(cls == 1, low, high)).astype(np.float32)


def frames_of(sc, n, budget=False):
    out = []
    for t in range(n):
        fr = scene.render_frame(sc, t)
        if budget:
            fr["roughness"] = budget_roughness(fr["roughness"])
        out.append(fr)
    return out


def test_clip_stage_matches_oracle():
    sc = scene.SceneConfig(128, 96, n_spheres=8, moving_sphere=True, seed=21)
    fr = scene.render_frame(sc, 1)
    cfg = svgf.default_config(128, 96)
    cfg.rectify_mode = svgf.RECTIFY_CLIP
    rng = np.random.default_rng(8)
    hist = (rng.random((96, 128, 4)) * 1.2).astype(np.float32)
    d = svgf.Denoiser(cfg)
    out = torch.empty(96, 128, 4, device="cuda")
    d.clamp(svgf.make_frame(dev(fr["noisy"]), dev(fr["gbuf_nz"]), dev(fr["motion"]), dev(fr["roughness"])),
            dev(hist), out)
    g = host(out)
    oc = oracle_config(cfg)
    o = oracle.clamp(oracle.tonemap(fr["noisy"].astype(np.float64), oc), hist[..., :3], oc)
    clamp = oracle.clamp(oracle.tonemap(fr["noisy"].astype(np.float64), oc), hist[..., :3],
                         oracle_config(svgf.default_config(128, 96)))
    moved = np.any(np.abs(o - clamp) > 1e-3, axis=-1).mean()
    print(f"[clip] pixels where clipping differs from clamping: {moved:.1%}")
    assert moved > 0.05
    assert colour_err(g[..., :3], o).max() <= COLOUR_TOL
    assert np.array_equal(g[..., 3], hist[..., 3])


@pytest.mark.parametrize("mode", [svgf.ATROUS_5X5, svgf.SEPARABLE])
def test_clip_sequence_matches_oracle(mode):
    cfg = svgf.default_config(128, 128)
    cfg.rectify_mode, cfg.spatial_mode = svgf.RECTIFY_CLIP, mode
    sc = scene.SceneConfig(128, 128, n_spheres=10, moving_sphere=True, seed=6)
    check_sequence(f"clip mode {mode}", cfg, frames_of(sc, 6))


@pytest.mark.parametrize("mode", [svgf.ATROUS_5X5, svgf.SEPARABLE])
def test_budget_each_pass_matches_oracle_and_freezes(mode):
    sc = scene.SceneConfig(160, 112, n_spheres=12, moving_sphere=True, seed=31)
    fr = frames_of(sc, 1, budget=True)[0]
    cfg = svgf.default_config(160, 112)
    cfg.spatial_mode, cfg.iter_by_roughness, cfg.iter_count1 = mode, 1, 2
    oc = oracle_config(cfg)
    rough = fr["roughness"]
    classes = [(rough <= 0).mean(), ((rough > 0) & (rough <= R05)).mean(), (rough > R05).mean()]
    print(f"[budget] pixel share with 0 / 2 / all passes: {classes}")
    assert min(classes) > 0.02
    cv0, _, _ = oracle.temporal(fr["noisy"], fr["gbuf_nz"], None, fr["motion"], None, None, False, oc)
    d = svgf.Denoiser(cfg)
    f = svgf.make_frame(dev(fr["noisy"]), dev(fr["gbuf_nz"]), dev(fr["motion"]), dev(rough))
    d.reproject_accumulate(f, torch.empty(112, 160, 4, device="cuda"))
    cur = cv0.astype(np.float32)
    budget = np.where(rough <= 0, 0, np.where(rough <= R05, 2, 5))
    for it in range(5):
        out = torch.empty(112, 160, 4, device="cuda")
        d.atrous(it, f, dev(cur), out)
        g = host(out)
        frozen = budget <= it
        assert np.array_equal(g[frozen], cur.astype(np.float64)[frozen]), it
        o = oracle.atrous(cur.astype(np.float64), fr["gbuf_nz"], rough, it, oc)
        ce = colour_err(g[..., :3], o[..., :3]).max()
        ve = var_err(g[..., 3], o[..., 3], o[..., :3]).max()
        print(f"[budget] mode {mode} pass {it}: frozen {frozen.mean():.1%} colour {ce:.2e} var {ve:.2e}")
        assert ce <= COLOUR_TOL and ve <= VAR_TOL, (it, ce, ve)
        cur = o.astype(np.float32)


@pytest.mark.parametrize("opts", [dict(spatial_mode=svgf.ATROUS_5X5), dict(spatial_mode=svgf.SEPARABLE),
                                  dict(adaptive_start=0), dict(rectify_mode=svgf.RECTIFY_CLIP, iter_count1=3)])
def test_budget_sequence_matches_oracle(opts):
    cfg = svgf.default_config(128, 128)
    cfg.iter_by_roughness = 1
    for k, v in opts.items():
        setattr(cfg, k, v)
    sc = scene.SceneConfig(128, 128, n_spheres=12, moving_sphere=True, seed=8)
    check_sequence(f"budget {opts}", cfg, frames_of(sc, 5, budget=True))


@pytest.mark.parametrize("prec", [svgf.FP32, svgf.FP16])
@pytest.mark.parametrize("mode", [svgf.ATROUS_5X5, svgf.SEPARABLE])
def test_composition_with_clip_and_budget(prec, mode):
    sc = scene.SceneConfig(144, 80, n_spheres=10, moving_sphere=True, seed=4)
    W, H = sc.width, sc.height
    cfg = svgf.default_config(W, H)
    cfg.precision, cfg.spatial_mode = prec, mode
    cfg.rectify_mode, cfg.iter_by_roughness = svgf.RECTIFY_CLIP, 1
    a, b = svgf.Denoiser(cfg), svgf.Denoiser(cfg)
    prev = None
    buf = (lambda: torch.empty(H, W, 4, device="cuda")) if prec == svgf.FP32 else \
        (lambda: torch.empty(H, W, 4, dtype=torch.int16, device="cuda"))
    for fr in frames_of(sc, 3, budget=True):
        t = {k: dev(fr[k]) for k in KEYS}
        f = svgf.make_frame(t["noisy"], t["gbuf_nz"], t["motion"], t["roughness"], prev)
        whole = torch.empty(H, W, 4, device="cuda")
        a.denoise_frame(f, whole)
        cv = [buf(), buf()]
        b.reproject_accumulate(f, cv[0])
        for it in range(cfg.atrous_iters):
            b.atrous(it, f, cv[it & 1], cv[(it + 1) & 1])
        staged = torch.empty(H, W, 4, device="cuda")
        b.inverse_tonemap(cv[cfg.atrous_iters & 1], staged)
        torch.cuda.synchronize()
        assert torch.equal(whole, staged)
        prev = t["gbuf_nz"]


def test_batch_with_clip_and_budget_equals_single_streams():
    sizes = [(96, 64), (160, 90), (33, 17)]
    streams = [scene.SceneConfig(w, h, n_spheres=8, moving_sphere=True, seed=500 + i, stream=i)
               for i, (w, h) in enumerate(sizes)]

    def cfg_of(sc):
        c = svgf.default_config(sc.width, sc.height)
        c.rectify_mode, c.iter_by_roughness, c.precision = svgf.RECTIFY_CLIP, 1, svgf.FP16
        return c

    def run(batched, shape=None):
        ds = [svgf.Denoiser(cfg_of(sc)) for sc in streams]
        bt = svgf.Batch(ds) if batched else None
        if bt is not None and shape is not None:
            bt.tuning = (shape, 0)
        res, prev = [], [None] * len(streams)
        for t in range(3):
            data = [{k: dev(v) for k, v in fr.items() if k in KEYS}
                    for fr in (frames_of_one(sc, t) for sc in streams)]
            frames = [svgf.make_frame(x["noisy"], x["gbuf_nz"], x["motion"], x["roughness"], prev[i])
                      for i, x in enumerate(data)]
            outs = [torch.empty(sc.height, sc.width, 4, device="cuda") for sc in streams]
            if bt is None:
                for d_, f, o in zip(ds, frames, outs):
                    d_.denoise_frame(f, o)
            else:
                bt.denoise(frames, outs)
            torch.cuda.synchronize()
            res.append([o.cpu() for o in outs])
            prev = [x["gbuf_nz"] for x in data]
        return res

    def frames_of_one(sc, t):
        fr = scene.render_frame(sc, t)
        fr["roughness"] = budget_roughness(fr["roughness"])
        return fr

    ref = run(False)
    for shape in range(len(svgf.ATROUS_SHAPES)):
        got = run(True, shape)
        for t in range(3):
            for i in range(len(streams)):
                assert torch.equal(ref[t][i], got[t][i]), (shape, t, i)
