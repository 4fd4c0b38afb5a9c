"""Batched streams: one persistent launch per stage over frames of uneven sizes.  The batched
result must equal each stream denoised on its own (svgf_denoise_frame) bit for bit -- for every
compiled a-trous tile shape, with the per-frame CUDA graph, after autotuning, in FP32 and 16-bit
storage, 5x5 and separable, and past the 64-streams-per-launch chunk -- and match the oracle."""
import numpy as np
import pytest

import oracle
from paper_2312_06827_gb300 import scene, svgf

from parity import COLOUR_TOL, colour_err, oracle_config

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
KEYS = ("noisy", "gbuf_nz", "motion", "roughness")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def make_streams(sizes, seed0=100):
    return [scene.SceneConfig(w, h, n_spheres=8, moving_sphere=True, seed=seed0 + i, stream=i)
            for i, (w, h) in enumerate(sizes)]


def run(streams, n_frames, cfg_of, batched, shape=None, graph=False, autotune=False):
    ds = [svgf.Denoiser(cfg_of(sc)) for sc in streams]
    b = svgf.Batch(ds) if batched else None
    side = torch.cuda.Stream()
    if b is not None:
        if shape is not None:
            b.tuning = (shape, 6 if shape % 2 else 0)      # persistent and one-block-per-tile grids
        if graph:
            b.use_graph(True)
    outs_all, prev = [], [None] * len(streams)
    with torch.cuda.stream(side):
        for t in range(n_frames):
            data = [{k: dev(v) for k, v in scene.render_frame(sc, t).items() if k in KEYS} for sc in streams]
            frames = [svgf.make_frame(d["noisy"], d["gbuf_nz"], d["motion"], d["roughness"], prev[i])
                      for i, d in enumerate(data)]
            outs = [torch.empty(sc.height, sc.width, 4, device="cuda") for sc in streams]
            if b is None:
                for d_, f, o in zip(ds, frames, outs):
                    d_.denoise_frame(f, o)
            elif autotune and t == 1:
                report = b.autotune(frames, outs)
                assert report.count("ms") == 16, report
            else:
                b.denoise(frames, outs)
            side.synchronize()
            outs_all.append([o.cpu() for o in outs])
            prev = [d["gbuf_nz"] for d in data]
    return outs_all, b


SIZES = [(96, 64), (160, 90), (128, 128), (33, 17)]


def cfg_factory(prec=svgf.FP32, mode=svgf.ATROUS_5X5):
    def f(sc):
        c = svgf.default_config(sc.width, sc.height)
        c.precision, c.spatial_mode = prec, mode
        return c
    return f


@pytest.mark.parametrize("prec", [svgf.FP32, svgf.FP16])
@pytest.mark.parametrize("mode", [svgf.ATROUS_5X5, svgf.SEPARABLE])
def test_batch_equals_single_streams_bitwise(prec, mode):
    streams = make_streams(SIZES)
    ref, _ = run(streams, 3, cfg_factory(prec, mode), batched=False)
    for shape in range(len(svgf.ATROUS_SHAPES)):
        got, _ = run(streams, 3, cfg_factory(prec, mode), batched=True, shape=shape)
        for t in range(3):
            for i in range(len(streams)):
                assert torch.equal(ref[t][i], got[t][i]), (shape, t, i)


def test_batch_graph_and_autotune_equal_single_streams():
    streams = make_streams(SIZES)
    ref, _ = run(streams, 4, cfg_factory(svgf.FP16), batched=False)
    got, b = run(streams, 4, cfg_factory(svgf.FP16), batched=True, graph=True, autotune=True)
    shape, bps = b.tuning
    assert 0 <= shape < len(svgf.ATROUS_SHAPES) and 0 <= bps <= 64
    for t in range(4):
        for i in range(len(streams)):
            assert torch.equal(ref[t][i], got[t][i]), (t, i)


def test_batch_per_stream_variance_radius_equals_single_streams():
    """Streams of one batch with different spatial-variance radii (per-stream parameters of the
    batched spatial-variance launch), through the persistent and the one-block-per-tile grids."""
    streams = make_streams(SIZES, seed0=700)
    radii = [3, 0, 7, 5]

    def cfg_of(sc):
        c = svgf.default_config(sc.width, sc.height)
        c.spatial_var_radius = radii[sc.stream]
        return c

    ref, _ = run(streams, 3, cfg_of, batched=False)
    for shape in (0, 1):
        got, _ = run(streams, 3, cfg_of, batched=True, shape=shape)
        for t in range(3):
            for i in range(len(streams)):
                assert torch.equal(ref[t][i], got[t][i]), (shape, t, i)


def test_batch_per_stream_normal_weight_form_equals_single_streams():
    """Streams whose sigma_n selects different forms of the normal term (the series alone from
    64 up) in one batched 5x5 launch, each bit-identical to its own single-frame launch."""
    streams = make_streams(SIZES, seed0=800)
    sigmas = [128.0, 16.0, 64.0, 63.0]

    def cfg_of(sc):
        c = svgf.default_config(sc.width, sc.height)
        c.sigma_n = sigmas[sc.stream]
        return c

    ref, _ = run(streams, 3, cfg_of, batched=False)
    for shape in (0, 3):
        got, _ = run(streams, 3, cfg_of, batched=True, shape=shape)
        for t in range(3):
            for i in range(len(streams)):
                assert torch.equal(ref[t][i], got[t][i]), (shape, t, i)


def test_batch_uniform_log2_normal_form_equals_single_streams():
    """Every stream at sigma_n = 16 (the series with the log2 fallback, one launch-wide copy of
    the parameters) through the persistent and the one-block-per-tile grids."""
    streams = make_streams(SIZES, seed0=900)

    def cfg_of(sc):
        c = svgf.default_config(sc.width, sc.height)
        c.sigma_n = 16.0
        return c

    ref, _ = run(streams, 3, cfg_of, batched=False)
    for shape in (1, 3):
        got, _ = run(streams, 3, cfg_of, batched=True, shape=shape)
        for t in range(3):
            for i in range(len(streams)):
                assert torch.equal(ref[t][i], got[t][i]), (shape, t, i)


def test_batch_beyond_one_launch_chunk():
    streams = make_streams([(16 + (i % 5) * 8, 8 + (i % 3) * 8) for i in range(70)], seed0=300)
    ref, _ = run(streams, 2, cfg_factory(), batched=False)
    got, _ = run(streams, 2, cfg_factory(), batched=True)
    for t in range(2):
        for i in range(len(streams)):
            assert torch.equal(ref[t][i], got[t][i]), (t, i)


def test_batch_matches_oracle():
    streams = make_streams([(96, 64), (64, 80)], seed0=500)
    got, _ = run(streams, 3, cfg_factory(), batched=True)
    for i, sc in enumerate(streams):
        cfg = cfg_factory()(sc)
        seq = oracle.Sequence(sc.width, sc.height, oracle_config(cfg))
        for t in range(3):
            fr = scene.render_frame(sc, t)
            o = seq.step(fr["noisy"], fr["gbuf_nz"], fr["motion"], fr["roughness"])
            g = got[t][i].numpy().astype(np.float64)
            assert colour_err(g[..., :3], o[..., :3], cfg, mapped=True).max() <= COLOUR_TOL


def test_batch_rejects_mixed_configs_and_default_stream_graph():
    a = svgf.Denoiser(cfg_factory()(scene.SceneConfig(32, 32)))
    c2 = cfg_factory(svgf.FP16)(scene.SceneConfig(32, 32))
    b_ = svgf.Denoiser(c2)
    with pytest.raises(svgf.SvgfError):
        svgf.Batch([a, b_])
    with pytest.raises(svgf.SvgfError):
        svgf.Batch([a, a])
    bt = svgf.Batch([a])
    bt.use_graph(True)
    fr = scene.render_frame(scene.SceneConfig(32, 32), 0)
    d = {k: dev(fr[k]) for k in KEYS}
    with pytest.raises(svgf.SvgfError):     # the legacy default stream cannot be captured
        bt.denoise([svgf.make_frame(d["noisy"], d["gbuf_nz"], d["motion"], d["roughness"])],
                   [torch.empty(32, 32, 4, device="cuda")], stream=torch.cuda.default_stream())
