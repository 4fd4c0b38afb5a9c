"""Synthetic ablation of the paper's cumulative techniques (Sec. 4, Fig. 5-11, Fig. 12-17).

The paper measures SSIM against the ground truth per surface roughness (indirect specular) or
shadow angle (shadows), for three kinds of movement, as techniques are added one on top of the
other: its SVGF, history rectification (the clamp), the blur adapted to the roughness / shadow
angle (the adaptive start), the separable blur, and Reinhard tone mapping (indirect specular
only); it also times each technique.  Here the scenes are the seeded generator's
(``paper_2312_06827_gb300.scene``) with every surface at one roughness and the noise amplitude
scaled by it (``rough_noise``), and the denoiser is this library's CUDA path; the metric is
computed here on the host from the outputs.

    python -m paper_2312_06827_gb300.ablation [--width 640 --height 360 --frames 16] [--time]

Metric (the paper names SSIM without its parameters): SSIM of Wang et al. (2004) with an
isotropic Gaussian window (sigma 1.5, truncated at 3.5 sigma), K1 = 0.01, K2 = 0.03, dynamic
range 1, on the Rec. 709 luma of the display-mapped colour c / (1 + c) per channel, averaged
over the image and over the frames from ``eval_from`` on (after the history has built up).
PSNR on the same luma is reported beside it.  For the shadow channel both are taken on the
visibility itself."""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
from scipy import ndimage

from . import scene, svgf

LUMA = np.array([0.2126, 0.7152, 0.0722])

SPECULAR_VARIANTS = (
    ("svgf", dict(clamp_enable=0, adaptive_start=0, spatial_mode=svgf.ATROUS_5X5, tonemap=0)),
    ("+clamp", dict(clamp_enable=1, adaptive_start=0, spatial_mode=svgf.ATROUS_5X5, tonemap=0)),
    ("+adaptive", dict(clamp_enable=1, adaptive_start=1, spatial_mode=svgf.ATROUS_5X5, tonemap=0)),
    ("+separable", dict(clamp_enable=1, adaptive_start=1, spatial_mode=svgf.SEPARABLE, tonemap=0)),
    ("+reinhard", dict(clamp_enable=1, adaptive_start=1, spatial_mode=svgf.SEPARABLE, tonemap=1)),
)
SHADOW_VARIANTS = SPECULAR_VARIANTS[:4]
MOVEMENTS = {
    "static": dict(pan_px_per_frame=0.0, moving_sphere=False, moving_light=False),
    "moving camera": dict(pan_px_per_frame=0.5, moving_sphere=False, moving_light=False),
    "moving objects and light": dict(pan_px_per_frame=0.0, moving_sphere=True, moving_light=True),
}
ROUGHNESS = (0.0, 0.1, 0.2, 0.3, 0.4, 0.6, 1.0)
LIGHT_RADII = (0.25, 0.5, 0.75, 1.0, 1.5)


def ssim(a, b, sigma=1.5, k1=0.01, k2=0.03, data_range=1.0):
    """Mean SSIM of two 2-D images with a Gaussian window (Wang, Bovik, Sheikh & Simoncelli,
    IEEE TIP 2004): l c s = ((2 mu_a mu_b + C1)(2 s_ab + C2)) / ((mu_a^2 + mu_b^2 + C1)(s_a^2 +
    s_b^2 + C2)), C1 = (k1 L)^2, C2 = (k2 L)^2, local moments by Gaussian filtering (borders
    mirrored)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    f = lambda x: ndimage.gaussian_filter(x, sigma, mode="reflect", truncate=3.5)
    mu_a, mu_b = f(a), f(b)
    s_aa = f(a * a) - mu_a * mu_a
    s_bb = f(b * b) - mu_b * mu_b
    s_ab = f(a * b) - mu_a * mu_b
    c1, c2 = (k1 * data_range) ** 2, (k2 * data_range) ** 2
    m = ((2 * mu_a * mu_b + c1) * (2 * s_ab + c2)) / ((mu_a ** 2 + mu_b ** 2 + c1) * (s_aa + s_bb + c2))
    return float(m.mean())


def psnr(a, b, data_range=1.0):
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10.0 * math.log10(data_range ** 2 / mse)


def display_luma(rgb):
    """Rec. 709 luma of the per-channel display map c / (1 + c): an image in [0, 1)."""
    c = np.maximum(np.asarray(rgb, np.float64), 0.0)
    return (c / (1.0 + c)) @ LUMA


def _run_sequences(torch, device, sc, n_frames, inputs_at, configs, eval_from, metric_of):
    """Denoise one sequence with every configuration; returns per configuration the mean
    (ssim, psnr) over frames >= eval_from, plus the same for the noisy input."""
    ds = [svgf.Denoiser(c, device=device) for c in configs]
    outs = [torch.empty(sc.height, sc.width, 4, device=device) for _ in configs]
    sums = np.zeros((len(configs) + 1, 2))
    n_eval, prev = 0, None
    for t in range(n_frames):
        x, ref, noisy_img = inputs_at(t)
        d = {k: torch.from_numpy(np.ascontiguousarray(v)).to(device) for k, v in x.items()}
        f = svgf.make_frame(d["noisy"], d["gbuf_nz"], d["motion"], d["roughness"], prev)
        for den, o in zip(ds, outs):
            den.denoise_frame(f, o)
        torch.cuda.synchronize(device)
        if t >= eval_from:
            for i, o in enumerate(outs):
                sums[i] += metric_of(o.cpu().numpy()[..., :3], ref)
            sums[-1] += metric_of(noisy_img, ref)
            n_eval += 1
        prev = d["gbuf_nz"]
    return sums / max(n_eval, 1)


def specular_ablation(torch, device, width, height, n_frames, eval_from, roughness=ROUGHNESS,
                      movements=tuple(MOVEMENTS), seed=7):
    rows = []

    def metric(img, ref):
        a, b = display_luma(img), display_luma(ref)
        return np.array([ssim(a, b), psnr(a, b)])

    for mv in movements:
        for r in roughness:
            sc = scene.SceneConfig(width, height, n_spheres=24, seed=seed, roughness=r, rough_noise=True,
                                   **MOVEMENTS[mv])

            def inputs_at(t, sc=sc):
                fr = scene.render_frame(sc, t, want=("noisy", "gt", "gbuf_nz", "motion", "roughness"))
                return fr, fr["gt"], fr["noisy"]

            cfgs = []
            for _, opts in SPECULAR_VARIANTS:
                c = svgf.default_config(width, height)
                for k, v in opts.items():
                    setattr(c, k, v)
                cfgs.append(c)
            res = _run_sequences(torch, device, sc, n_frames, inputs_at, cfgs, eval_from, metric)
            for (name, _), (s, p) in zip(SPECULAR_VARIANTS, res[:-1]):
                rows.append(dict(channel="indirect specular", movement=mv, roughness=r, variant=name,
                                 ssim=round(s, 4), psnr_db=round(p, 2)))
            rows.append(dict(channel="indirect specular", movement=mv, roughness=r, variant="noisy input",
                             ssim=round(res[-1][0], 4), psnr_db=round(res[-1][1], 2)))
    return rows


def shadow_ablation(torch, device, width, height, n_frames, eval_from, radii=LIGHT_RADII,
                    movements=("static", "moving objects and light"), seed=7):
    rows = []

    def metric(img, ref):
        a = np.clip(np.asarray(img, np.float64) @ LUMA, 0.0, 1.0)
        return np.array([ssim(a, ref), psnr(a, ref)])

    for mv in movements:
        for R in radii:
            sc = scene.SceneConfig(width, height, n_spheres=24, seed=seed, light_radius=R, **MOVEMENTS[mv])
            angles = []

            def inputs_at(t, sc=sc, angles=angles):
                # the 64-sample visibility is only rendered for the evaluated frames
                want = ("gbuf_nz", "motion", "shadow_noisy", "shadow_angle") + \
                    (("shadow_gt",) if t >= eval_from else ())
                fr = scene.render_frame(sc, t, want=want)
                angles.append(float(np.median(fr["shadow_angle"])))
                rgb = np.repeat(fr["shadow_noisy"][..., None], 3, axis=-1)
                x = {"noisy": rgb, "gbuf_nz": fr["gbuf_nz"], "motion": fr["motion"],
                     "roughness": fr["shadow_angle"]}
                gt = fr["shadow_gt"].astype(np.float64) if "shadow_gt" in fr else None
                return x, gt, rgb

            cfgs = []
            for _, opts in SHADOW_VARIANTS:
                c = svgf.channel_config(svgf.CHANNEL_SHADOW, width, height)
                for k, v in opts.items():
                    setattr(c, k, v)
                cfgs.append(c)
            res = _run_sequences(torch, device, sc, n_frames, inputs_at, cfgs, eval_from, metric)
            ang = round(float(np.median(angles)), 2)
            for (name, _), (s, p) in zip(SHADOW_VARIANTS, res[:-1]):
                rows.append(dict(channel="shadow", movement=mv, light_radius=R, shadow_angle_deg=ang,
                                 variant=name, ssim=round(s, 4), psnr_db=round(p, 2)))
            rows.append(dict(channel="shadow", movement=mv, light_radius=R, shadow_angle_deg=ang,
                             variant="noisy input", ssim=round(res[-1][0], 4), psnr_db=round(res[-1][1], 2)))
    return rows


def time_variants(torch, device, width=1920, height=1080, steps=30, warmup=5):
    """ms per frame of each cumulative variant on the default 1080p scene (CUDA events on the
    launching stream, L2 flushed between timed frames), as in the paper's per-technique timings."""
    sc = scene.SceneConfig(width, height, n_spheres=40, moving_sphere=True, seed=0)
    n = warmup + steps
    frames = [{k: torch.from_numpy(v).to(device) for k, v in
               scene.render_frame(sc, t, want=("noisy", "gbuf_nz", "motion", "roughness")).items()}
              for t in range(n)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    out = torch.empty(height, width, 4, device=device)
    res = {}
    for name, opts in SPECULAR_VARIANTS:
        c = svgf.default_config(width, height)
        for k, v in opts.items():
            setattr(c, k, v)
        d = svgf.Denoiser(c, device=device)
        total = 0.0
        for t in range(n):
            f = frames[t]
            fr = svgf.make_frame(f["noisy"], f["gbuf_nz"], f["motion"], f["roughness"],
                                 frames[t - 1]["gbuf_nz"] if t else None)
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            d.denoise_frame(fr, out)
            b.record()
            b.synchronize()
            if t >= warmup:
                total += a.elapsed_time(b)
        res[name] = round(total / steps, 4)
    return res


def table(rows, key):
    """Markdown table: one row per (movement, x), one column per variant, SSIM values."""
    variants = list(dict.fromkeys(r["variant"] for r in rows))
    groups = {}
    for r in rows:
        groups.setdefault((r["movement"], r[key]), {})[r["variant"]] = r["ssim"]
    head = f"| movement | {key} | " + " | ".join(variants) + " |"
    lines = [head, "|" + "---|" * (len(variants) + 2)]
    for (mv, x), v in groups.items():
        lines.append(f"| {mv} | {x} | " + " | ".join(f"{v.get(n, float('nan')):.4f}" for n in variants) + " |")
    return "\n".join(lines)


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--width", type=int, default=640)
    ap.add_argument("--height", type=int, default=360)
    ap.add_argument("--frames", type=int, default=16)
    ap.add_argument("--eval-from", type=int, default=8)
    ap.add_argument("--time", action="store_true", help="also time every variant at 1080p")
    ap.add_argument("--json", default=None, help="write the rows to this file")
    a = ap.parse_args(argv)
    dev = torch.device("cuda", 0)
    t0 = time.perf_counter()
    spec = specular_ablation(torch, dev, a.width, a.height, a.frames, a.eval_from)
    shad = shadow_ablation(torch, dev, a.width, a.height, a.frames, a.eval_from)
    out = {"specular": spec, "shadow": shad, "seconds": round(time.perf_counter() - t0, 1)}
    if a.time:
        out["ms_per_frame_1080p"] = time_variants(torch, dev)
    print("indirect specular, SSIM vs noise-free radiance\n" + table(spec, "roughness"))
    print("\nshadow, SSIM vs 64-sample visibility\n" + table(shad, "light_radius"))
    if a.time:
        print("\nms per frame at 1080p:", out["ms_per_frame_1080p"])
    if a.json:
        with open(a.json, "w") as fh:
            json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
