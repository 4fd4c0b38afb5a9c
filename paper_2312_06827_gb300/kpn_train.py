"""Training of the kernel-predicting network on pairs the denoiser itself generates.

``make_examples`` runs the plain pipeline through the C ABI (temporal stage, a-trous pass 0,
features of the pass-0 output, a-trous passes 1..4) on seeded synthetic sequences and keeps, per
frame, the network input (features, pass-0 colour) and the target (the plain pipeline's
tone-mapped output).  ``train`` takes random crops and runs the library's train step (forward,
backward and Adam all in the library's kernels).  ``calibrate_threshold`` picks the fallback
threshold on held-out frames: the largest 32x32-tile standard deviation of the pass-0 luminance
such that at least 99 % of the tiles at or below it meet the PSNR bound against the plain output.  PyTorch only holds memory and gathers crops.
"""
from __future__ import annotations

import math

import numpy as np

from . import scene, svgf

KEYS = ("noisy", "gbuf_nz", "motion", "roughness", "albedo")


def make_examples(scenes, frames_per_scene: int, skip: int = 3, device=None, stream=None):
    """Returns dict of tensors: feats [N, H, W, 16] (BF16 bits as int16), c0 and target
    [N, H, W, 4] float32, plus the pass-0 variance in c0[..., 3].  All scenes share one size."""
    import torch
    dev = device or torch.device("cuda")
    W, H = scenes[0].width, scenes[0].height
    feats, c0s, targets = [], [], []
    kpn_feat = KPN_FEATURES_ONLY(W * H, dev)
    for sc in scenes:
        cfg = svgf.default_config(W, H)
        d = svgf.Denoiser(cfg, device=dev)
        prev = None
        cv = [torch.empty(H, W, 4, device=dev) for _ in range(2)]
        for t in range(skip + frames_per_scene):
            fr = scene.render_frame(sc, t, want=KEYS)
            dv = {k: torch.from_numpy(fr[k]).to(dev) for k in KEYS}
            f = svgf.make_frame(dv["noisy"], dv["gbuf_nz"], dv["motion"], dv["roughness"], prev)
            d.reproject_accumulate(f, cv[0], stream)
            d.atrous(0, f, cv[0], cv[1], stream)
            if t >= skip:
                ft = torch.empty(H, W, 16, dtype=torch.int16, device=dev)
                c0 = torch.empty(H, W, 4, device=dev)
                kpn_feat.features(d, cv[1], f, dv["albedo"], ft, c0, stream)
            for it in range(1, cfg.atrous_iters):          # pass i reads cv[i & 1], writes the other
                d.atrous(it, f, cv[it & 1], cv[(it + 1) & 1], stream)
            if t >= skip:
                feats.append(ft)
                c0s.append(c0)
                targets.append(cv[cfg.atrous_iters & 1].clone())
            prev = dv["gbuf_nz"]
            keep = dv  # noqa: F841
    torch.cuda.synchronize(dev)
    return {"feats": torch.stack(feats), "c0": torch.stack(c0s), "target": torch.stack(targets)}


def KPN_FEATURES_ONLY(max_pixels, device):
    """A KPN handle used only for its feature kernel (no optimiser state)."""
    return svgf.KPN(max_pixels, train=False, device=device)


def crops(data, rng, batch: int, size: int):
    """Random size x size crops of random frames (gathered with torch indexing)."""
    import torch
    N, H, W = data["c0"].shape[:3]
    n = rng.integers(0, N, batch)
    y = rng.integers(0, H - size + 1, batch)
    x = rng.integers(0, W - size + 1, batch)
    dev = data["c0"].device
    iy = torch.as_tensor(y, device=dev)[:, None] + torch.arange(size, device=dev)[None, :]
    ix = torch.as_tensor(x, device=dev)[:, None] + torch.arange(size, device=dev)[None, :]
    nn_ = torch.as_tensor(n, device=dev)[:, None, None]
    out = {}
    for k in ("feats", "c0", "target"):
        out[k] = data[k][nn_, iy[:, :, None], ix[:, None, :]].contiguous()
    return out


def train(kpn, data, steps: int, batch: int = 16, crop: int = 256, lr: float = 1e-3, seed: int = 0,
          log_every: int = 0):
    """Adam steps on random crops; returns the per-step losses (read back every log_every steps
    and at the end, so that the loop does not wait on the GPU each step)."""
    import torch
    rng = np.random.default_rng(seed)
    losses = []
    for s in range(steps):
        b = crops(data, rng, batch, crop)
        loss = kpn.train_step(b["feats"], b["c0"], b["target"], lr)
        if (log_every and s % log_every == 0) or s == steps - 1:
            losses.append((s, float(loss.item())))
    torch.cuda.synchronize()
    return losses


def psnr(a, b) -> float:
    mse = float(((a[..., :3].double() - b[..., :3].double()) ** 2).mean())
    return float("inf") if mse == 0 else 10.0 * math.log10(1.0 / mse)


def evaluate(kpn, data):
    """Mean PSNR over frames of the network output (tone-mapped) against the plain target, and of
    the pass-0 output (the method without iterations 2..) against it."""
    import torch
    out = torch.empty_like(data["c0"][:1])
    p_net, p_pass0 = [], []
    for i in range(data["c0"].shape[0]):
        kpn.forward(data["feats"][i:i + 1], data["c0"][i:i + 1], out)
        torch.cuda.synchronize()
        p_net.append(psnr(out[0], data["target"][i]))
        p_pass0.append(psnr(data["c0"][i], data["target"][i]))
    return float(np.mean(p_net)), float(np.mean(p_pass0))


def tile_stats(kpn, data, tile: int = 32):
    """Per 32x32 tile of every frame: the fallback rule's statistic (the population standard
    deviation of the pass-0 luminance, tone-mapped) and the tile PSNR of the network output
    against the plain output.  Returns two flat arrays."""
    import torch
    out = torch.empty_like(data["c0"][:1])
    lw = torch.tensor([0.2126, 0.7152, 0.0722], device=out.device, dtype=torch.float64)
    ds, ps = [], []
    for i in range(data["c0"].shape[0]):
        kpn.forward(data["feats"][i:i + 1], data["c0"][i:i + 1], out)
        torch.cuda.synchronize()
        H, W = out.shape[1:3]
        Ht, Wt = H // tile * tile, W // tile * tile
        err = ((out[0, :Ht, :Wt, :3].double() - data["target"][i, :Ht, :Wt, :3].double()) ** 2).mean(-1)
        mse = err.reshape(Ht // tile, tile, Wt // tile, tile).mean((1, 3))
        lum = data["c0"][i, :Ht, :Wt, :3].double() @ lw
        lum = lum.reshape(Ht // tile, tile, Wt // tile, tile)
        dev = (lum - lum.mean((1, 3), keepdim=True)).pow(2).mean((1, 3)).sqrt()
        ds.append(dev.flatten().cpu().numpy())
        ps.append((10.0 * torch.log10(1.0 / mse.clamp_min(1e-30))).flatten().cpu().numpy())
    return np.concatenate(ds), np.concatenate(ps)


def calibrate_threshold(kpn, data, psnr_bound: float = 40.0, coverage: float = 0.99, tile: int = 32):
    """Fallback threshold on the tile statistic of tile_stats (the pass-0 luminance standard
    deviation): the largest tau such that, of the held-out tiles at or below tau, at least
    `coverage` meet the PSNR bound against the plain output (the tiles above tau take the plain
    passes).  Returns (tau, stats) with the share of tiles that fall back and the share of kept
    tiles that meet the bound; tau = +inf when every tile meets it, -1 (always fall back) when no
    prefix does."""
    v, p = tile_stats(kpn, data, tile)
    order = np.argsort(v, kind="stable")
    v, ok = v[order], p[order] >= psnr_bound
    n = len(v)
    good = np.cumsum(ok)
    k = np.arange(1, n + 1)
    # a threshold must keep whole groups of equal statistics together
    last_of_value = np.r_[v[1:] != v[:-1], True]
    valid = (good >= coverage * k) & last_of_value
    if valid.all() or ok.all():
        tau, kept = float("inf"), n
    elif not valid.any():
        tau, kept = -1.0, 0
    else:
        kept = int(np.nonzero(valid)[0].max()) + 1
        tau = float(v[kept - 1])
    stats = {"tiles": n, "fallback_share": 1.0 - kept / n,
             "kept_meeting_bound": float(good[kept - 1] / kept) if kept else 1.0,
             "all_meeting_bound": float(ok.mean()), "psnr_bound": psnr_bound, "coverage": coverage,
             "statistic": "32x32-tile standard deviation of the pass-0 luminance"}
    return tau, stats


def infer_sequence(width: int = 1920, height: int = 1080, frames: int = 4, seed: int = 1200,
                   init_seed: int = 0, detail_threshold: float = float("inf"), device=None):
    """Denoise `frames` consecutive frames of a seeded 40-sphere scene with the learned form
    (a network initialised from `init_seed`; fallback off by default); returns the last output and
    the device error word of the tensor-core convolutions (0 when every wait completed)."""
    import torch
    dev = device or torch.device("cuda", 0)
    sc = scene.SceneConfig(width, height, n_spheres=40, moving_sphere=True, seed=seed)
    keys = ("noisy", "gbuf_nz", "motion", "roughness", "albedo")
    d = svgf.Denoiser(svgf.default_config(width, height), device=dev)
    k = svgf.KPN(width * height, train=False, device=dev)
    k.init_params(init_seed)
    out = torch.empty(height, width, 4, device=dev)
    prev = None
    for t in range(frames):
        f = {n: torch.from_numpy(v).to(dev) for n, v in scene.render_frame(sc, t, want=keys).items()}
        fr = svgf.make_frame(f["noisy"], f["gbuf_nz"], f["motion"], f["roughness"], prev)
        k.denoise_frame(d, fr, f["albedo"], out, detail_threshold=detail_threshold)
        prev = f["gbuf_nz"]
    torch.cuda.synchronize(dev)
    return out, k.check_device()


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser(description="learned-form inference on synthetic frames")
    ap.add_argument("--width", type=int, default=1920)
    ap.add_argument("--height", type=int, default=1080)
    ap.add_argument("--frames", type=int, default=4)
    a = ap.parse_args()
    _, err = infer_sequence(a.width, a.height, a.frames)
    print(f"denoised {a.frames} frames of {a.width}x{a.height}; device error word {err}")
    raise SystemExit(0 if err == 0 else 1)
