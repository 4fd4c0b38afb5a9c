"""The C-ABI library loads and exports every symbol include/svgf.h declares; the binding's
struct layout matches the header; argument errors come back as status codes before any CUDA
call (these run without a GPU)."""
import ctypes
import json
import os
import re
import subprocess

import pytest

import oracle
from paper_2312_06827_gb300 import svgf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "svgf.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(svgf_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    L = svgf.lib()
    names = declared_functions()
    assert len(names) >= 16
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(svgf.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", svgf.lib_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (svgf_\w+)", out))
    assert set(names) <= exported


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "layout.c"
    fields = [n for n, _ in svgf._Config._fields_]
    body = "".join(f'printf("%s %zu\\n", "{f}", offsetof(svgf_config, {f}));' for f in fields)
    ffields = [n for n, _ in svgf._Frame._fields_]
    body += "".join(f'printf("F%s %zu\\n", "{f}", offsetof(svgf_frame, {f}));' for f in ffields)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "svgf.h"\nint main(void){'
                   + body + 'printf("size %zu %zu\\n", sizeof(svgf_config), sizeof(svgf_frame));return 0;}')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    lines = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines()
                 if not l.startswith("size"))
    for f in fields:
        assert int(lines[f]) == getattr(svgf._Config, f).offset, f
    for f in ffields:
        assert int(lines["F" + f]) == getattr(svgf._Frame, f).offset, f
    size_line = subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines()[-1].split()
    assert int(size_line[1]) == ctypes.sizeof(svgf._Config) and int(size_line[2]) == ctypes.sizeof(svgf._Frame)


def test_defaults_match_paper_and_oracle():
    c = svgf.default_config(64, 32)
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")))
    assert c.roughness_threshold == pytest.approx(g["adaptive_start_roughness_threshold"]["value"])
    o = oracle.OracleConfig()
    for f in ("alpha", "alpha_moments", "clamp_gamma", "atrous_iters", "sigma_z", "sigma_n", "sigma_l",
              "roughness_threshold", "luma_k", "inv_weight", "inverse_mode", "history_from_pass",
              "depth_rel_tol", "normal_cos_tol", "disocclusion_weight", "max_history",
              "min_temporal_frames", "spatial_var_radius", "eps"):
        assert getattr(c, f) == pytest.approx(getattr(o, f), rel=1e-6), f
    assert bool(c.clamp_enable) == o.clamp_enable and bool(c.adaptive_start) == o.adaptive_start
    assert bool(c.tonemap) == o.tonemap and (c.spatial_mode == svgf.SEPARABLE) == o.separable


def _create(**kw):
    L = svgf.lib()
    cfg = svgf.default_config(16, 16)
    for k, v in kw.items():
        setattr(cfg, k, v)
    h = ctypes.c_void_p()
    st = L.svgf_create(ctypes.byref(cfg._c()), ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("kw,expect", [
    (dict(width=0), 1), (dict(height=-3), 1), (dict(width=40000), 1), (dict(alpha=0.0), 1),
    (dict(alpha=1.5), 1), (dict(atrous_iters=9), 1), (dict(spatial_mode=7), 1), (dict(eps=0.0), 1),
    (dict(sigma_n=float("inf")), 1), (dict(precision=9), 1), (dict(precision=-1), 1),
    (dict(max_history=0), 1), (dict(spatial_var_radius=8), 1), (dict(history_from_pass=-2), 1),
    (dict(rectify_mode=2), 1), (dict(iter_by_roughness=3), 1), (dict(iter_rough_t0=0.1), 1),
    (dict(iter_rough_t1=float("nan")), 1), (dict(iter_count0=9), 1), (dict(iter_count1=-1), 1),
    (dict(atrous_iters=0), 0), (dict(iter_count0=8, atrous_iters=3), 0),
    (dict(rectify_mode=1, iter_by_roughness=1), 0),
])
def test_invalid_config_is_rejected(kw, expect):
    st, h = _create(**kw)
    assert st == expect and bool(h.value) == (expect == 0)
    svgf.lib().svgf_destroy(h)


def test_invalid_calls_return_codes_without_touching_the_gpu():
    L = svgf.lib()
    st, h = _create()
    assert st == 0 and h.value
    try:
        fr = svgf._Frame()
        # no workspace bound yet
        assert L.svgf_denoise_frame(h, ctypes.byref(fr), ctypes.c_void_p(256), None) == 6
        n = ctypes.c_size_t()
        assert L.svgf_workspace_size(h, ctypes.byref(n)) == 0 and n.value >= 7 * 16 * 16 * 16
        assert L.svgf_bind_workspace(h, ctypes.c_void_p(0x1001), n.value) == 1     # misaligned
        assert L.svgf_bind_workspace(h, ctypes.c_void_p(0x100000), n.value - 1) == 6  # too small
        # a fake (never dereferenced) aligned address: binding only records pointers
        assert L.svgf_bind_workspace(h, ctypes.c_void_p(0x100000), n.value) == 0
        assert L.svgf_denoise_frame(h, None, ctypes.c_void_p(256), None) == 1
        assert L.svgf_denoise_frame(h, ctypes.byref(fr), ctypes.c_void_p(256), None) == 1  # NULL inputs
        fr2 = svgf._Frame(0x1000, 0x1008, 0, 0x2000, 0x3000)      # misaligned G-buffer
        assert L.svgf_denoise_frame(h, ctypes.byref(fr2), ctypes.c_void_p(256), None) == 1
        fr3 = svgf._Frame(0x1000, 0x1010, 0, 0x2000, 0)            # adaptive start needs roughness
        assert L.svgf_denoise_frame(h, ctypes.byref(fr3), ctypes.c_void_p(256), None) == 1
        fr4 = svgf._Frame(0x1000, 0x1010, 0, 0x2000, 0x3000)
        assert L.svgf_atrous(h, -1, ctypes.byref(fr4), ctypes.c_void_p(256), ctypes.c_void_p(512), None) == 1
        assert L.svgf_atrous(h, 0, ctypes.byref(fr4), ctypes.c_void_p(256), ctypes.c_void_p(256), None) == 1
        assert L.svgf_history_import(h, None, None, 1, None) == 1
        assert L.svgf_reset_history(h) == 0
        assert L.svgf_status_string(3) == b"CUDA error"
        assert L.svgf_launch_count(h) == 0
    finally:
        L.svgf_destroy(h)
    assert L.svgf_destroy(None) == 0


def test_sixteen_bit_storage_halves_the_image_workspace():
    L = svgf.lib()
    sizes = {}
    for prec in (svgf.FP32, svgf.FP16, svgf.BF16):
        st, h = _create(precision=prec)
        assert st == 0
        n = ctypes.c_size_t()
        assert L.svgf_workspace_size(h, ctypes.byref(n)) == 0
        sizes[prec] = n.value
        L.svgf_destroy(h)
    images = 7 * 16 * 16   # seven images of 16x16 pixels
    assert sizes[svgf.FP32] - sizes[svgf.FP16] == images * 8
    assert sizes[svgf.FP16] == sizes[svgf.BF16]


def test_pass_budget_needs_roughness_and_defaults():
    c = svgf.default_config(8, 8)
    o = oracle.OracleConfig()
    assert c.rectify_mode == svgf.RECTIFY_CLAMP == o.rectify_mode
    assert (c.iter_by_roughness, c.iter_count0, c.iter_count1) == (0, o.iter_count0, o.iter_count1)
    assert c.iter_rough_t0 == pytest.approx(o.iter_rough_t0) and c.iter_rough_t1 == pytest.approx(o.iter_rough_t1)
    L = svgf.lib()
    st, h = _create(adaptive_start=0, iter_by_roughness=1)
    assert st == 0 and h.value
    try:
        n = ctypes.c_size_t()
        assert L.svgf_workspace_size(h, ctypes.byref(n)) == 0
        assert L.svgf_bind_workspace(h, ctypes.c_void_p(0x100000), n.value) == 0
        fr = svgf._Frame(0x1000, 0x1010, 0, 0x2000, 0)             # no roughness image
        assert L.svgf_denoise_frame(h, ctypes.byref(fr), ctypes.c_void_p(256), None) == 1
    finally:
        L.svgf_destroy(h)


def test_channel_configs_on_the_host():
    spec = svgf.channel_config(svgf.CHANNEL_INDIRECT_SPECULAR, 64, 48)
    shadow = svgf.channel_config(svgf.CHANNEL_SHADOW, 64, 48)
    assert spec == svgf.default_config(64, 48)
    assert (shadow.tonemap, shadow.roughness_threshold) == (0, 6.0)
    L = svgf.lib()
    c = svgf._Config()
    assert L.svgf_channel_config(2, 8, 8, ctypes.byref(c)) == 1
    assert L.svgf_channel_config(svgf.CHANNEL_SHADOW, 0, 8, ctypes.byref(c)) == 1
    assert L.svgf_channel_config(svgf.CHANNEL_SHADOW, 8, 8, None) == 1
