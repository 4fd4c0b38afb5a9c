"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element by element, on
seeded synthetic scenes.  Per stage (temporal, clamp, every a-trous pass in both modes, inverse),
per frame over sequences (128x128 x 4 frames; odd sizes; 1080p and 4K with the moving sphere in
the launch configuration the benchmark times), plus the stage-composition rule and state I/O."""
import numpy as np
import pytest
from scipy import ndimage

import oracle
from paper_2312_06827_gb300 import scene, svgf

from parity import (COLOUR_TOL, SEQ_VAR_TOL, VAR_TOL, colour_err, excluded_mask, flip_candidates,
                    oracle_config, report, tm64, var_err, var_err_est)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def frames_of(sc, n, start=0):
    return [scene.render_frame(sc, start + t) for t in range(n)]


def run_gpu_sequence(cfg, frames):
    d = svgf.Denoiser(cfg)
    outs, prev = [], None
    for fr in frames:
        t = {k: dev(v) for k, v in fr.items() if k in ("noisy", "gbuf_nz", "motion", "roughness")}
        f = svgf.make_frame(t["noisy"], t["gbuf_nz"], t["motion"], t["roughness"], prev)
        out = torch.empty(cfg.height, cfg.width, 4, device="cuda")
        d.denoise_frame(f, out)
        outs.append(host(out))
        prev = t["gbuf_nz"]
        keep = t  # noqa: F841  (inputs stay alive until the copy above synchronised)
    return outs, d


def run_oracle_sequence(cfg, frames):
    seq = oracle.Sequence(cfg.width, cfg.height, oracle_config(cfg))
    outs, margins = [], []
    for fr in frames:
        outs.append(seq.step(fr["noisy"], fr["gbuf_nz"], fr["motion"], fr["roughness"]))
        margins.append(seq.margin.copy())
    return outs, margins


def check_sequence(name, cfg, frames):
    g, _ = run_gpu_sequence(cfg, frames)
    o, margins = run_oracle_sequence(cfg, frames)
    flags = np.zeros((cfg.height, cfg.width), bool)
    worst = (0.0, 0.0)
    for t in range(len(frames)):
        flags |= flip_candidates(margins[t])
        ce, ve, frac = report(f"{name} frame {t}", colour_err(g[t][..., :3], o[t][..., :3], cfg, mapped=True),
                              var_err(g[t][..., 3], o[t][..., 3], tm64(o[t][..., :3], cfg)), flags,
                              excluded_mask(flags, cfg))
        assert frac <= 1e-4, (t, frac)
        assert ce <= COLOUR_TOL, (t, ce)
        assert ve <= SEQ_VAR_TOL, (t, ve)
        worst = (max(worst[0], ce), max(worst[1], ve))
    return worst


# ------------------------------------------------------------------------- per stage

@pytest.fixture(scope="module")
def c0():
    return frames_of(scene.C0_128, 2)


def test_temporal_first_frame_matches_oracle(c0):
    fr = c0[0]
    cfg = svgf.default_config(128, 128)
    d = svgf.Denoiser(cfg)
    t = {k: dev(v) for k, v in fr.items()}
    cv = torch.empty(128, 128, 4, device="cuda")
    d.reproject_accumulate(svgf.make_frame(t["noisy"], t["gbuf_nz"], t["motion"], t["roughness"]), cv)
    g = host(cv)
    o, mom, _ = oracle.temporal(fr["noisy"], fr["gbuf_nz"], None, fr["motion"], None, None, False,
                                oracle_config(cfg))
    # first frame: colour = tone-mapped input, variance = 7x7 spatial estimate
    assert colour_err(g[..., :3], o[..., :3]).max() <= COLOUR_TOL
    assert var_err_est(g[..., 3], o[..., 3], o[..., :3]).max() <= VAR_TOL
    hist = torch.empty(128, 128, 4, device="cuda")
    moms = torch.empty(128, 128, 4, device="cuda")
    d.history_export(hist, moms)
    m = host(moms)          # exported in central form (mu1, S = mu2 - mu1^2, n)
    assert np.allclose(m[..., 2], 1.0) and colour_err(m[..., 0], mom[..., 0]).max() <= COLOUR_TOL
    assert var_err_est(m[..., 1], mom[..., 1] - mom[..., 0] ** 2, o[..., :3]).max() <= VAR_TOL


@pytest.mark.parametrize("radius", [0, 1, 2, 5, 7])
def test_spatial_variance_radius_matches_oracle(radius):
    """The 7x7 window of Sec. 2 at other radii (the runtime-radius body; radius 3 has its own
    unrolled one), on a ragged 150x70 frame: partial tiles on the right and bottom edges, windows
    cut by every border.  First frame: every pixel takes the spatial estimate."""
    sc = scene.SceneConfig(150, 70, n_spheres=10, moving_sphere=True, seed=61)
    fr = scene.render_frame(sc, 0)
    cfg = svgf.default_config(150, 70)
    cfg.spatial_var_radius = radius
    d = svgf.Denoiser(cfg)
    t = {k: dev(v) for k, v in fr.items()}
    cv = torch.empty(70, 150, 4, device="cuda")
    d.reproject_accumulate(svgf.make_frame(t["noisy"], t["gbuf_nz"], t["motion"], t["roughness"]), cv)
    g = host(cv)
    o, _, _ = oracle.temporal(fr["noisy"], fr["gbuf_nz"], None, fr["motion"], None, None, False,
                              oracle_config(cfg))
    assert colour_err(g[..., :3], o[..., :3]).max() <= COLOUR_TOL
    assert var_err_est(g[..., 3], o[..., 3], o[..., :3]).max() <= VAR_TOL
    if radius == 0:
        assert np.all(g[..., 3] == 0.0)       # a one-pixel window: no spread of the first moment


@pytest.mark.parametrize("clamp", [1, 0])
def test_temporal_with_history_matches_oracle(c0, clamp):
    """History imported into the GPU handle from the oracle's state (rounded to FP32), so the
    temporal stage alone is compared."""
    cfg = svgf.default_config(128, 128)
    cfg.clamp_enable = clamp
    oc = oracle_config(cfg)
    f0, f1 = c0
    cv0, mom0, _ = oracle.temporal(f0["noisy"], f0["gbuf_nz"], None, f0["motion"], None, None, False, oc)
    hist32 = np.concatenate([cv0[..., :3], np.zeros((128, 128, 1))], -1).astype(np.float32)
    # the handle's state holds (mu1, S = mu2 - mu1^2, n); give the oracle the same FP32 state
    central = np.stack([mom0[..., 0], mom0[..., 1] - mom0[..., 0] ** 2, mom0[..., 2]], -1)
    mom32 = np.concatenate([central, np.zeros((128, 128, 1))], -1).astype(np.float32)
    m64 = mom32[..., :3].astype(np.float64)
    ora_mom = np.stack([m64[..., 0], m64[..., 1] + m64[..., 0] ** 2, m64[..., 2]], -1)
    d = svgf.Denoiser(cfg)
    d.history_import(dev(hist32), dev(mom32), True)
    t = {k: dev(v) for k, v in f1.items()}
    prev = dev(f0["gbuf_nz"])
    cv = torch.empty(128, 128, 4, device="cuda")
    d.reproject_accumulate(svgf.make_frame(t["noisy"], t["gbuf_nz"], t["motion"], t["roughness"], prev), cv)
    g = host(cv)
    o, mom1, margin = oracle.temporal(f1["noisy"], f1["gbuf_nz"], f0["gbuf_nz"], f1["motion"],
                                      hist32[..., :3].astype(np.float64), ora_mom, True, oc)
    keep = margin >= 1e-5
    assert keep.mean() > 0.999
    assert colour_err(g[..., :3], o[..., :3])[keep].max() <= COLOUR_TOL
    assert var_err_est(g[..., 3], o[..., 3], o[..., :3])[keep].max() <= VAR_TOL
    assert (mom1[..., 2] == 2).mean() > 0.5       # most pixels kept their history


def test_clamp_stage_matches_oracle(c0):
    fr = c0[1]
    cfg = svgf.default_config(128, 128)
    rng = np.random.default_rng(7)
    hist = rng.random((128, 128, 4)).astype(np.float32)
    d = svgf.Denoiser(cfg)
    out = torch.empty(128, 128, 4, device="cuda")
    d.clamp(svgf.make_frame(dev(fr["noisy"]), dev(fr["gbuf_nz"]), dev(fr["motion"]), dev(fr["roughness"])),
            dev(hist), out)
    g = host(out)
    oc = oracle_config(cfg)
    cur = oracle.tonemap(fr["noisy"].astype(np.float64), oc)
    o = oracle.clamp(cur, hist[..., :3], oc)
    # an active clamp returns m -/+ gamma sigma of the 3x3 window, an addition whose FP32 rounding
    # is a few u (|m| + gamma sigma) however small the result: the bar adds that term to the
    # colour bar (u = 2^-24)
    ones = np.ones((128, 128))
    k = np.ones((3, 3))
    cnt = ndimage.correlate(ones, k, mode="constant")
    m = np.stack([ndimage.correlate(cur[..., c], k, mode="constant") / cnt for c in range(3)], -1)
    sq = np.stack([ndimage.correlate(cur[..., c] ** 2, k, mode="constant") / cnt for c in range(3)], -1)
    scale = np.abs(m) + cfg.clamp_gamma * np.sqrt(np.maximum(sq - m * m, 0.0))
    err = np.abs(g[..., :3] - o)
    tol = COLOUR_TOL * np.maximum(np.abs(o), 1e-3) + 16 * 2.0 ** -24 * scale
    print(f"[parity] clamp stage: max err/tol {float((err / tol).max()):.3f}, "
          f"max rel {float(colour_err(g[..., :3], o).max()):.3e}")
    assert (err <= tol).all()
    assert np.array_equal(g[..., 3], hist[..., 3])


def check_each_atrous_pass(c0, mode, sigma_n=None):
    fr = c0[0]
    cfg = svgf.default_config(128, 128)
    cfg.spatial_mode = mode
    if sigma_n is not None:
        cfg.sigma_n = sigma_n
    oc = oracle_config(cfg)
    cv0, _, _ = oracle.temporal(fr["noisy"], fr["gbuf_nz"], None, fr["motion"], None, None, False, oc)
    rough = fr["roughness"].copy()
    rough[:, ::3] = 0.1                          # both start levels present
    d = svgf.Denoiser(cfg)
    f = svgf.make_frame(dev(fr["noisy"]), dev(fr["gbuf_nz"]), dev(fr["motion"]), dev(rough))
    d.reproject_accumulate(f, torch.empty(128, 128, 4, device="cuda"))
    cur = cv0.astype(np.float32)
    for it in range(5):
        out = torch.empty(128, 128, 4, device="cuda")
        d.atrous(it, f, dev(cur), out)
        g = host(out)
        o = oracle.atrous(cur.astype(np.float64), fr["gbuf_nz"], rough, it, oc)
        ce = colour_err(g[..., :3], o[..., :3]).max()
        ve = var_err(g[..., 3], o[..., 3], o[..., :3]).max()
        print(f"[parity] atrous mode {mode} sigma_n {cfg.sigma_n} iter {it}: colour {ce:.3e} var {ve:.3e}")
        assert ce <= COLOUR_TOL and ve <= VAR_TOL, (it, ce, ve)
        cur = o.astype(np.float32)


@pytest.mark.parametrize("mode", [svgf.ATROUS_5X5, svgf.SEPARABLE])
def test_each_atrous_pass_matches_oracle(c0, mode):
    check_each_atrous_pass(c0, mode)


@pytest.mark.parametrize("sigma_n,mode", [(4.0, svgf.ATROUS_5X5), (32.0, svgf.ATROUS_5X5),
                                          (63.5, svgf.ATROUS_5X5), (64.0, svgf.ATROUS_5X5),
                                          (512.0, svgf.ATROUS_5X5), (16.0, svgf.SEPARABLE)])
def test_atrous_pass_normal_weight_forms_match_oracle(c0, sigma_n, mode):
    """Both forms of the normal term in the 5x5 pass: below sigma_n = 64 the series near t2 = 0 and
    the lg2 form beyond t2 = 1/8; from 64 up the series alone (error bound 2.2e-7 at 64)."""
    check_each_atrous_pass(c0, mode, sigma_n)


@pytest.mark.parametrize("mode", [svgf.INVERSE_EXACT, svgf.INVERSE_PAPER])
def test_inverse_stage_matches_oracle(mode):
    rng = np.random.default_rng(3)
    c = rng.random((64, 64, 4)).astype(np.float32)
    c[..., :3] *= 0.9                                     # luma < 1/k
    cfg = svgf.default_config(64, 64)
    cfg.inverse_mode = mode
    d = svgf.Denoiser(cfg)
    out = torch.empty(64, 64, 4, device="cuda")
    d.inverse_tonemap(dev(c), out)
    g = host(out)
    o = oracle.inverse_tonemap(c[..., :3].astype(np.float64), oracle_config(cfg))
    assert colour_err(g[..., :3], o).max() <= 2e-6
    assert np.array_equal(g[..., 3], c[..., 3])


# ------------------------------------------------------------------------- sequences

@pytest.mark.parametrize("mode", [svgf.ATROUS_5X5, svgf.SEPARABLE])
def test_c0_sequence_matches_oracle(mode):
    cfg = svgf.default_config(128, 128)
    cfg.spatial_mode = mode
    check_sequence(f"C0 128x128 mode {mode}", cfg, frames_of(scene.C0_128, 4))


@pytest.mark.parametrize("opts", [dict(clamp_enable=0), dict(adaptive_start=0), dict(tonemap=0),
                                  dict(history_from_pass=-1), dict(inverse_mode=1), dict(atrous_iters=0),
                                  dict(atrous_iters=3, spatial_mode=1)])
def test_c0_sequence_options_match_oracle(opts):
    cfg = svgf.default_config(128, 128)
    for k, v in opts.items():
        setattr(cfg, k, v)
    sc = scene.SceneConfig(128, 128, n_spheres=8, moving_sphere=True, seed=5)
    check_sequence(f"C0 {opts}", cfg, frames_of(sc, 5))


@pytest.mark.parametrize("hw", [(1, 1), (5, 7), (17, 33), (40, 1), (1, 40), (61, 97)])
def test_odd_sizes_match_oracle(hw):
    H, W = hw
    sc = scene.SceneConfig(W, H, n_spheres=6, moving_sphere=True, seed=11)
    for mode in (svgf.ATROUS_5X5, svgf.SEPARABLE):
        cfg = svgf.default_config(W, H)
        cfg.spatial_mode = mode
        check_sequence(f"{W}x{H} mode {mode}", cfg, frames_of(sc, 5))


def test_stage_composition_is_bit_identical():
    """reproject_accumulate -> atrous(0..4) -> inverse_tonemap equals denoise_frame bit for bit."""
    fr = frames_of(scene.C0_128, 3)
    for mode in (svgf.ATROUS_5X5, svgf.SEPARABLE):
        cfg = svgf.default_config(128, 128)
        cfg.spatial_mode = mode
        a, b = svgf.Denoiser(cfg), svgf.Denoiser(cfg)
        prev = None
        for x in fr:
            t = {k: dev(v) for k, v in x.items()}
            f = svgf.make_frame(t["noisy"], t["gbuf_nz"], t["motion"], t["roughness"], prev)
            whole = torch.empty(128, 128, 4, device="cuda")
            a.denoise_frame(f, whole)
            cv = [torch.empty(128, 128, 4, device="cuda") for _ in range(2)]
            b.reproject_accumulate(f, cv[0])
            for it in range(cfg.atrous_iters):
                b.atrous(it, f, cv[it & 1], cv[(it + 1) & 1])
            staged = torch.empty(128, 128, 4, device="cuda")
            b.inverse_tonemap(cv[cfg.atrous_iters & 1], staged)
            torch.cuda.synchronize()
            assert torch.equal(whole, staged)
            prev = t["gbuf_nz"]


def test_history_export_import_round_trip():
    fr = frames_of(scene.C0_128, 3)
    cfg = svgf.default_config(128, 128)
    a = svgf.Denoiser(cfg)
    t = [{k: dev(v) for k, v in x.items()} for x in fr]
    out = torch.empty(128, 128, 4, device="cuda")
    for i in range(2):
        a.denoise_frame(svgf.make_frame(t[i]["noisy"], t[i]["gbuf_nz"], t[i]["motion"], t[i]["roughness"],
                                        t[i - 1]["gbuf_nz"] if i else None), out)
    h, m = torch.empty(128, 128, 4, device="cuda"), torch.empty(128, 128, 4, device="cuda")
    a.history_export(h, m)
    b = svgf.Denoiser(cfg)
    b.history_import(h, m, True)
    f2 = svgf.make_frame(t[2]["noisy"], t[2]["gbuf_nz"], t[2]["motion"], t[2]["roughness"], t[1]["gbuf_nz"])
    oa, ob = torch.empty_like(out), torch.empty_like(out)
    a.denoise_frame(f2, oa)
    b.denoise_frame(f2, ob)
    torch.cuda.synchronize()
    assert torch.equal(oa, ob)


def test_launch_count():
    cfg = svgf.default_config(64, 64)
    for mode, per_iter in ((svgf.ATROUS_5X5, 1), (svgf.SEPARABLE, 2)):
        cfg.spatial_mode = mode
        d = svgf.Denoiser(cfg)
        fr = scene.render_frame(scene.SceneConfig(64, 64), 0)
        t = {k: dev(v) for k, v in fr.items()}
        d.denoise_frame(svgf.make_frame(t["noisy"], t["gbuf_nz"], t["motion"], t["roughness"]),
                        torch.empty(64, 64, 4, device="cuda"))
        torch.cuda.synchronize()
        assert d.launch_count == 2 + per_iter * cfg.atrous_iters


# ------------------------------------------------------------------------- full size

def test_1080p_sequence_matches_oracle():
    """Full 1080p frames with the moving sphere (disocclusions), the benchmark's launch
    configuration (denoise_frame, default config), 8 frames: the spatial estimate (n < 4), the
    temporal variance (n >= 4) and the exponential average (n > 5), every pixel compared."""
    cfg = svgf.default_config(1920, 1080)
    check_sequence("1080p", cfg, frames_of(scene.C1_1080P, 8))


def test_1080p_separable_matches_oracle():
    cfg = svgf.default_config(1920, 1080)
    cfg.spatial_mode = svgf.SEPARABLE
    check_sequence("1080p separable", cfg, frames_of(scene.C1_1080P, 8))


def test_4k_sequence_matches_oracle():
    cfg = svgf.default_config(3840, 2160)
    check_sequence("4K", cfg, frames_of(scene.C2_4K, 6))


def steady_state_stages(W, H, sc, mode, n_hist):
    """The oracle runs n_hist frames; its state (colour history, moments, previous G-buffer) is
    imported into a GPU handle, and frame n_hist is then compared stage by stage, each stage
    given the oracle's input rounded to FP32: the temporal stage (mostly the n >= 4 temporal
    variance and the exponential average by then) and every a-trous pass, every pixel, colour
    and variance to 1e-5 relative to the value itself."""
    cfg = svgf.default_config(W, H)
    cfg.spatial_mode = mode
    oc = oracle_config(cfg)
    frames = frames_of(sc, n_hist + 1)
    seq = oracle.Sequence(W, H, oc)
    for fr in frames[:n_hist]:
        seq.step(fr["noisy"], fr["gbuf_nz"], fr["motion"], fr["roughness"])
    f0, f1 = frames[n_hist - 1], frames[n_hist]
    hist32 = np.concatenate([seq.hist_rgb, np.zeros((H, W, 1))], -1).astype(np.float32)
    m = seq.hist_mom
    central = np.stack([m[..., 0], m[..., 1] - m[..., 0] ** 2, m[..., 2]], -1)
    mom32 = np.concatenate([central, np.zeros((H, W, 1))], -1).astype(np.float32)
    m64 = mom32[..., :3].astype(np.float64)
    ora_mom = np.stack([m64[..., 0], m64[..., 1] + m64[..., 0] ** 2, m64[..., 2]], -1)
    d = svgf.Denoiser(cfg)
    d.history_import(dev(hist32), dev(mom32), True)
    t = {k: dev(v) for k, v in f1.items() if k in ("noisy", "gbuf_nz", "motion", "roughness")}
    f = svgf.make_frame(t["noisy"], t["gbuf_nz"], t["motion"], t["roughness"], dev(f0["gbuf_nz"]))
    cv = torch.empty(H, W, 4, device="cuda")
    d.reproject_accumulate(f, cv)
    g = host(cv)
    o, mom1, margin = oracle.temporal(f1["noisy"], f1["gbuf_nz"], f0["gbuf_nz"], f1["motion"],
                                      hist32[..., :3].astype(np.float64), ora_mom, True, oc)
    keep = margin >= 1e-5
    assert keep.mean() > 0.9999
    assert (mom1[..., 2] >= 4).mean() > 0.99 and (mom1[..., 2] > 5).mean() > 0.9
    ce = colour_err(g[..., :3], o[..., :3])[keep].max()
    ve = var_err_est(g[..., 3], o[..., 3], o[..., :3])[keep].max()
    print(f"[parity] steady {W}x{H} mode {mode} temporal: colour {ce:.3e} var {ve:.3e}")
    assert ce <= COLOUR_TOL and ve <= VAR_TOL
    cur = o.astype(np.float32)
    for it in range(cfg.atrous_iters):
        out = torch.empty(H, W, 4, device="cuda")
        d.atrous(it, f, dev(cur), out)
        g = host(out)
        oo = oracle.atrous(cur.astype(np.float64), f1["gbuf_nz"], f1["roughness"], it, oc)
        ce = colour_err(g[..., :3], oo[..., :3]).max()
        ve = var_err(g[..., 3], oo[..., 3], oo[..., :3]).max()
        print(f"[parity] steady {W}x{H} mode {mode} pass {it}: colour {ce:.3e} var {ve:.3e}")
        assert ce <= COLOUR_TOL and ve <= VAR_TOL, (it, ce, ve)
        cur = oo.astype(np.float32)


@pytest.mark.parametrize("mode", [svgf.ATROUS_5X5, svgf.SEPARABLE])
def test_1080p_steady_state_stages_match_oracle(mode):
    steady_state_stages(1920, 1080, scene.C1_1080P, mode, 8)


def test_4k_steady_state_stages_match_oracle():
    steady_state_stages(3840, 2160, scene.C2_4K, svgf.ATROUS_5X5, 6)


def test_host_buffer_entry_point_equals_device_path():
    """svgf_denoise_frame_host (pageable or pinned host buffers, copies inside the call) gives
    the device path's result bit for bit, frame after frame."""
    sc = scene.SceneConfig(96, 80, n_spheres=8, moving_sphere=True, seed=31)
    cfg = svgf.default_config(sc.width, sc.height)
    a, b = svgf.Denoiser(cfg), svgf.Denoiser(cfg)
    b.enable_host_staging()
    prev = None
    for t in range(4):
        fr = scene.render_frame(sc, t)
        dv = {k: dev(fr[k]) for k in ("noisy", "gbuf_nz", "motion", "roughness")}
        out_d = torch.empty(sc.height, sc.width, 4, device="cuda")
        a.denoise_frame(svgf.make_frame(dv["noisy"], dv["gbuf_nz"], dv["motion"], dv["roughness"], prev), out_d)
        hv = {k: torch.from_numpy(fr[k]) for k in ("noisy", "gbuf_nz", "motion", "roughness")}
        if t % 2:
            hv = {k: v.pin_memory() for k, v in hv.items()}
        out_h = torch.empty(sc.height, sc.width, 4)
        b.denoise_frame_host(hv["noisy"], hv["gbuf_nz"], hv["motion"], hv["roughness"], out_h)
        torch.cuda.synchronize()
        assert torch.equal(out_d.cpu(), out_h)
        prev = dv["gbuf_nz"]


def test_pipelined_host_submit_equals_device_path():
    """svgf_host_submit / svgf_host_wait: frames enqueued back to back from pinned buffers (two in
    flight, uploads and downloads on the handle's copy streams) give the device path's results
    bit for bit, also when a synchronous call and a history reset come in between."""
    sc = scene.SceneConfig(128, 72, n_spheres=9, moving_sphere=True, seed=33)
    cfg = svgf.default_config(sc.width, sc.height)
    a, b = svgf.Denoiser(cfg), svgf.Denoiser(cfg)
    b.enable_host_staging()
    keys = ("noisy", "gbuf_nz", "motion", "roughness")
    n = 9
    frames = [scene.render_frame(sc, t) for t in range(n)]
    host = [{k: torch.from_numpy(f[k]).pin_memory() for k in keys} for f in frames]
    outs = [torch.empty(sc.height, sc.width, 4).pin_memory() for _ in range(n)]
    ref, prev = [], None
    for t, fr in enumerate(frames):
        if t == 6:
            a.reset_history()
            prev = None
        dv = {k: dev(fr[k]) for k in keys}
        o = torch.empty(sc.height, sc.width, 4, device="cuda")
        a.denoise_frame(svgf.make_frame(dv["noisy"], dv["gbuf_nz"], dv["motion"], dv["roughness"], prev), o)
        ref.append(o.cpu())
        prev = dv["gbuf_nz"]
    for t in range(n):
        h = host[t]
        if t == 6:
            b.wait_host()
            b.reset_history()
        if t == 4:
            b.denoise_frame_host(h["noisy"], h["gbuf_nz"], h["motion"], h["roughness"], outs[t])
        else:
            b.submit_host(h["noisy"], h["gbuf_nz"], h["motion"], h["roughness"], outs[t])
    b.wait_host()
    for t in range(n):
        assert torch.equal(ref[t], outs[t]), t


def test_profiling_counts_every_kernel():
    cfg = svgf.default_config(64, 48)
    for mode, kinds in ((svgf.ATROUS_5X5, {"temporal": 1, "spatial_var": 1, "atrous_5x5": 5}),
                        (svgf.SEPARABLE, {"temporal": 1, "spatial_var": 1, "atrous_h": 5, "atrous_v": 5})):
        cfg.spatial_mode = mode
        d = svgf.Denoiser(cfg)
        d.profile_enable(True)
        fr = scene.render_frame(scene.SceneConfig(64, 48), 0)
        t = {k: dev(fr[k]) for k in ("noisy", "gbuf_nz", "motion", "roughness")}
        for _ in range(3):
            d.denoise_frame(svgf.make_frame(t["noisy"], t["gbuf_nz"], t["motion"], t["roughness"]),
                            torch.empty(48, 64, 4, device="cuda"))
        torch.cuda.synchronize()
        prof = d.profile_read()
        for k, v in prof.items():
            assert v[1] == 3 * kinds.get(k, 0), (k, v)
            assert (v[0] > 0) == (k in kinds)
        assert all(v == (0.0, 0) for v in d.profile_read().values())     # read clears
