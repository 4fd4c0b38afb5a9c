"""The helpers behind the bench line's reported numbers (no GPU): algorithmic bytes per pixel,
the a-trous FP32 operation count and its peak, the share of pixels a pass budget leaves
filtering, and the rule that recorded DRAM traffic is reported only for the kernel sources it
was taken on."""
import json

import numpy as np
import pytest

import bench


def test_bytes_per_pixel():
    # temporal: noisy 12, G 16, G_prev 16, mv 8 + history, moments in, cv, moments out
    assert bench.bytes_per_px("temporal", 0) == 12 + 16 + 16 + 8 + 4 * 16
    assert bench.bytes_per_px("temporal", 1) == 12 + 16 + 16 + 8 + 4 * 8
    # 5x5 pass: cv in, G, roughness, cv out; the last pass writes FP32 rgb (16 B) instead
    assert bench.bytes_per_px("atrous_5x5", 0) == 16 + 16 + 4 + 16
    assert bench.bytes_per_px("atrous_5x5", 1, last_pass_share=1.0) == 8 + 16 + 4 + 16
    assert bench.bytes_per_px("atrous_5x5", 1, last_pass_share=0.2) == pytest.approx(8 + 16 + 4 + 8 + 0.2 * 8)
    assert bench.bytes_per_px("nonsense", 0) is None


def test_atrous_operation_count_and_peak():
    assert bench.FP32_PEAK_OPS == pytest.approx(152 * 128 * 2.07e9)
    npx, t = 1920 * 1080, 86e-6                      # one 1080p pass of 86 us
    r = bench.atrous_alu("atrous_5x5", npx, t)
    assert r["fp32_ops_per_px"] == 24 * 24 + 36
    assert r["achieved"] == pytest.approx(612 * npx / t / 1e12, abs=0.006)
    assert r["frac"] == pytest.approx(612 * npx / t / bench.FP32_PEAK_OPS, abs=1e-4)
    assert bench.atrous_alu("atrous_h", 1000, 1e-6)["fp32_ops_per_px"] == 4 * 24 + 36
    assert bench.atrous_alu("temporal", 1000, 1e-6) is None
    assert bench.atrous_alu("atrous_5x5", 1000, 0.0) is None


class Cfg:
    iter_by_roughness = 1
    atrous_iters = 5
    iter_rough_t0, iter_rough_t1 = 0.0, 0.05
    iter_count0, iter_count1 = 0, 1


def test_pass_activity():
    frames = [{"roughness": np.array([0.0, 0.03, 0.5, 1.0], np.float32)}]
    # budgets 0, 1, 5, 5: pass 0 filters 3 of 4 pixels, passes 1-4 two of 4
    assert bench.pass_activity(Cfg, frames) == pytest.approx((0.75 + 4 * 0.5) / 5)
    # the threshold compares in FP32: 0.05 itself takes the one-pass budget
    edge = [{"roughness": np.array([0.05], np.float32)}]
    assert bench.pass_activity(Cfg, edge) == pytest.approx(1 / 5)
    off = type("Off", (Cfg,), {"iter_by_roughness": 0})
    assert bench.pass_activity(off, frames) is None


def test_recorded_traffic_only_for_the_same_sources(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    rec = {"k_atrous<0>": {"1080p": {"kernel_source_sha256": "abc", "dram_bytes_per_launch": 9.0e7}}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_sha256", lambda: "abc")
    assert bench.recorded_traffic("k_atrous<0>", "1080p") == 9.0e7
    assert bench.recorded_traffic("k_atrous<0>", "4k") is None
    monkeypatch.setattr(bench, "kernel_source_sha256", lambda: "changed")
    assert bench.recorded_traffic("k_atrous<0>", "1080p") is None


def test_frame_bytes_per_pixel():
    """The plain FP32 frame: temporal 116 B/px (noisy 12, G-buffers 32, motion 8, history and
    moments read and written as float4) + five 5x5 passes of 52 B/px + the pass-0 history write
    (16) = 392 B/px (the scope's ~400); the separable mode reads and writes its intermediate
    image once more per iteration; 16-bit storage halves the image records."""
    from paper_2312_06827_gb300 import svgf
    c = svgf.default_config(64, 64)
    assert bench.frame_bytes_per_px(c) == 116 + 5 * 52 + 16 == 392
    c.spatial_mode = svgf.SEPARABLE
    assert bench.frame_bytes_per_px(c) == 116 + 5 * (52 + 52) + 16
    c.spatial_mode, c.precision = svgf.ATROUS_5X5, svgf.FP16
    assert bench.frame_bytes_per_px(c) == (12 + 16 + 16 + 8 + 4 * 8) + 5 * (8 + 16 + 4 + 8) + 8 + 8


def test_binding_roof_leads_with_the_roof_that_binds():
    """Above the ridge point (FP32 lane peak / measured HBM bandwidth) the arithmetic roof leads
    and the HBM figures move to a sub-block; below it the HBM figures lead."""
    npx = 1920 * 1080
    hbm = {"bound": "hbm", "achieved": 1330.0, "peak": 6685.8, "unit": "GB/s", "frac": 0.1989, "traffic": 1.0e8,
           "kernel": "k_atrous<0>", "algorithmic_bytes_per_launch": 52 * npx, "avg_launch_us": 86.06,
           "alu": bench.atrous_alu("atrous_5x5", npx, 86.06e-6)}
    r = bench.binding_roof(dict(hbm))
    assert r["bound"] == "alu" and r["hbm"]["bound"] == "hbm" and r["traffic"] == 1.0e8
    assert r["ops_per_algorithmic_byte"] > r["ridge_ops_per_byte"]
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-3
    low = dict(hbm, algorithmic_bytes_per_launch=1000 * npx)     # 0.6 operations a byte
    assert bench.binding_roof(low)["bound"] == "hbm"
    assert bench.binding_roof({k: v for k, v in hbm.items() if k != "alu"})["bound"] == "hbm"
