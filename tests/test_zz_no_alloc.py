"""svgf_atrous_separable_noalloc, the separable a-trous iteration that allocates nothing,
against the workspace path (svgf_atrous with spatial_mode = SVGF_SEPARABLE), through the C ABI.

Some callers cannot allocate device memory at all -- code on a host callback or a real-time
thread with a no-allocation rule, or an embedding that hands out only its own buffers -- so they
cannot bind a workspace.  This entry point keeps the horizontal pass's intermediate in a fixed
device array inside the library instead.  The file name makes pytest collect it last, so a
failure here comes after every other test has run; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2312_06827_gb300 import scene, svgf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5          # the parity tests' colour tolerance (the two paths share their kernels)
KEYS = ("noisy", "gbuf_nz", "motion", "roughness")


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


CASES = [
    # (storage precision, the no-allocation handle's own spatial mode, option overrides)
    (svgf.FP32, svgf.SEPARABLE, {}),
    (svgf.FP32, svgf.ATROUS_5X5, {}),
    (svgf.FP16, svgf.SEPARABLE, {}),
    (svgf.FP16, svgf.ATROUS_5X5, {}),
    (svgf.BF16, svgf.SEPARABLE, {}),
    (svgf.BF16, svgf.ATROUS_5X5, {}),
    (svgf.FP32, svgf.ATROUS_5X5, dict(adaptive_start=0)),
    (svgf.FP32, svgf.SEPARABLE, dict(iter_by_roughness=1)),
    (svgf.FP16, svgf.SEPARABLE, dict(iter_by_roughness=1, adaptive_start=0)),
]


def _buf(prec, H, W):
    """A colour+variance image in the handle's storage layout, filled with a pattern no kernel
    writes (NaN in FP32, 0xffff in the 16-bit records), so a pixel left unwritten shows."""
    if prec == svgf.FP32:
        return torch.full((H, W, 4), float("nan"), device="cuda")
    return torch.full((H, W, 4), -1, dtype=torch.int16, device="cuda")


@pytest.mark.parametrize("prec,mode,opts", CASES)
def test_noalloc_matches_the_workspace_path_on_two_calls_in_a_row(prec, mode, opts):
    """Two calls in a row (iterations 0 and 1 of consecutive frames) equal the workspace path's
    separable iteration bit for bit, in every storage precision, whatever the handle's own spatial
    mode, with the adaptive start off and with the roughness-adapted pass budget on."""
    W, H = 640, 360
    sc = scene.SceneConfig(W, H, n_spheres=12, moving_sphere=True, seed=21)
    cfg = svgf.default_config(W, H)
    cfg.precision = prec
    for k, v in opts.items():
        setattr(cfg, k, v)
    cfg.spatial_mode = svgf.SEPARABLE
    ref = svgf.Denoiser(cfg)                       # workspace-backed handle, separable
    cfg.spatial_mode = mode
    L = svgf.lib()
    h = ctypes.c_void_p()
    assert L.svgf_create(ctypes.byref(cfg._c()), ctypes.byref(h)) == 0   # no workspace bound
    try:
        prev = None
        for call in range(2):
            fr = scene.render_frame(sc, call)
            dv = {k: torch.from_numpy(fr[k]).cuda() for k in KEYS}
            f = svgf.make_frame(dv["noisy"], dv["gbuf_nz"], dv["motion"], dv["roughness"], prev)
            cv = _buf(prec, H, W)
            ref.reproject_accumulate(f, cv)
            expect = _buf(prec, H, W)
            ref.atrous(call, f, cv, expect)
            got = _buf(prec, H, W)
            st = L.svgf_atrous_separable_noalloc(h, call, ctypes.byref(f), ctypes.c_void_p(cv.data_ptr()),
                                                 ctypes.c_void_p(got.data_ptr()), _stream())
            assert st == 0, (st, L.svgf_last_error(h))
            torch.cuda.synchronize()
            if prec == svgf.FP32:
                e, g = expect.cpu().numpy().astype(np.float64), got.cpu().numpy().astype(np.float64)
                assert np.isfinite(g).all() and np.isfinite(e).all()
                rel = np.abs(g - e) / np.maximum(np.abs(e), 1e-3)
                assert rel.max() <= TOL, (call, rel.max())
            # the same kernels on the same input: every record equal bit for bit
            assert torch.equal(got, expect), call
            prev = dv["gbuf_nz"]
    finally:
        L.svgf_destroy(h)


def test_noalloc_rejects_frames_beyond_its_scratch():
    L = svgf.lib()
    W, H = 2049, 1024                              # 2,098,176 pixels > 2^21
    cfg = svgf.default_config(W, H)
    h = ctypes.c_void_p()
    assert L.svgf_create(ctypes.byref(cfg._c()), ctypes.byref(h)) == 0
    try:
        # full-size buffers, so nothing could go out of bounds even if the size check were missing
        z = lambda *s: torch.zeros(*s, device="cuda")
        f = svgf.make_frame(z(H, W, 3), z(H, W, 4), z(H, W, 2), z(H, W))
        cv_in, cv_out = z(H, W, 4), z(H, W, 4)
        st = L.svgf_atrous_separable_noalloc(h, 0, ctypes.byref(f), ctypes.c_void_p(cv_in.data_ptr()),
                                             ctypes.c_void_p(cv_out.data_ptr()), _stream())
        torch.cuda.synchronize()
        assert st == 1                              # SVGF_ERR_INVALID_ARG
        assert b"exceeds the no-allocation scratch" in L.svgf_last_error(h)
        assert svgf.NOALLOC_MAX_PIXELS == 1 << 21 and W * H > svgf.NOALLOC_MAX_PIXELS
    finally:
        L.svgf_destroy(h)
