"""Thin Python binding of the C ABI in ``include/svgf.h`` (``lib/libsvgf.so``).

Argument marshalling only: every step of the denoiser runs in the library's CUDA kernels.
PyTorch supplies device memory (``torch.Tensor`` on CUDA) and the current stream.  The binding
fails loudly when the library is missing or cannot load: there is no CPU fallback.

Function names follow the C entry points (``svgf_`` prefix dropped on ``Denoiser`` methods).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading

from . import _build

SVGF_OK = 0
STATUS = {0: "SVGF_OK", 1: "SVGF_ERR_INVALID_ARG", 2: "SVGF_ERR_UNSUPPORTED", 3: "SVGF_ERR_CUDA",
          4: "SVGF_ERR_TIMEOUT", 5: "SVGF_ERR_DEVICE_CHECK", 6: "SVGF_ERR_NO_WORKSPACE"}
ATROUS_5X5, SEPARABLE = 0, 1
INVERSE_EXACT, INVERSE_PAPER = 0, 1
FP32, FP16, BF16 = 0, 1, 2
RECTIFY_CLAMP, RECTIFY_CLIP = 0, 1
CHANNEL_INDIRECT_SPECULAR, CHANNEL_SHADOW = 0, 1


class SvgfError(RuntimeError):
    def __init__(self, fn, status, detail=""):
        self.status = status
        super().__init__(f"{fn} -> {STATUS.get(status, status)}" + (f": {detail}" if detail else ""))


class _Config(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_int), ("height", ctypes.c_int),
        ("alpha", ctypes.c_float), ("alpha_moments", ctypes.c_float), ("clamp_gamma", ctypes.c_float),
        ("atrous_iters", ctypes.c_int),
        ("sigma_z", ctypes.c_float), ("sigma_n", ctypes.c_float), ("sigma_l", ctypes.c_float),
        ("spatial_mode", ctypes.c_int), ("clamp_enable", ctypes.c_int), ("adaptive_start", ctypes.c_int),
        ("roughness_threshold", ctypes.c_float), ("tonemap", ctypes.c_int),
        ("luma_k", ctypes.c_float), ("inv_weight", ctypes.c_float), ("inverse_mode", ctypes.c_int),
        ("history_from_pass", ctypes.c_int),
        ("depth_rel_tol", ctypes.c_float), ("normal_cos_tol", ctypes.c_float),
        ("disocclusion_weight", ctypes.c_float),
        ("max_history", ctypes.c_int), ("min_temporal_frames", ctypes.c_int),
        ("spatial_var_radius", ctypes.c_int), ("eps", ctypes.c_float), ("precision", ctypes.c_int),
        ("rectify_mode", ctypes.c_int), ("iter_by_roughness", ctypes.c_int),
        ("iter_rough_t0", ctypes.c_float), ("iter_rough_t1", ctypes.c_float),
        ("iter_count0", ctypes.c_int), ("iter_count1", ctypes.c_int),
    ]


class _Frame(ctypes.Structure):
    _fields_ = [("noisy_rgb", ctypes.c_void_p), ("gbuf_nz", ctypes.c_void_p),
                ("prev_gbuf_nz", ctypes.c_void_p), ("motion", ctypes.c_void_p),
                ("roughness", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()
EXPORTS = ("svgf_default_config", "svgf_channel_config", "svgf_create", "svgf_destroy", "svgf_workspace_size",
           "svgf_bind_workspace", "svgf_reset_history", "svgf_reproject_accumulate", "svgf_clamp",
           "svgf_atrous", "svgf_inverse_tonemap", "svgf_denoise_frame", "svgf_history_export",
           "svgf_history_import", "svgf_status_string", "svgf_last_error", "svgf_launch_count",
           "svgf_staging_size", "svgf_bind_staging", "svgf_denoise_frame_host", "svgf_profile_enable",
           "svgf_profile_read", "svgf_atrous_separable_noalloc", "svgf_host_submit", "svgf_host_wait", "svgf_kpn_check_device", "svgf_kpn_wait_selftest", "svgf_kpn_save", "svgf_kpn_load", "svgf_batch_create", "svgf_batch_destroy",
           "svgf_batch_denoise", "svgf_batch_use_graph", "svgf_batch_autotune", "svgf_batch_get_tuning",
           "svgf_batch_set_tuning", "svgf_kpn_workspace_size", "svgf_kpn_create", "svgf_kpn_destroy",
           "svgf_kpn_params_changed", "svgf_kpn_forward", "svgf_kpn_grad", "svgf_kpn_train_step",
           "svgf_kpn_features", "svgf_kpn_denoise_frame", "svgf_kpn_predict", "svgf_kpn_apply")
KPN_PARAM_COUNT = 28633
KPN_CIN, KPN_COUT = (10, 32, 32, 32), (32, 32, 32, 25)
ATROUS_SHAPES = ((32, 8), (32, 4), (16, 16), (64, 4))
NOALLOC_MAX_PIXELS = 1 << 21
KERNEL_KINDS = ("temporal", "spatial_var", "atrous_5x5", "atrous_h", "atrous_v", "inverse", "clamp")


def lib_path():
    return str(_build.SVGF_LIB)


def lib(build_if_missing: bool = True):
    """Load the CUDA library (building it with nvcc if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing:
                _build.build_svgf()
            if not os.path.exists(lib_path()):
                raise RuntimeError(f"CUDA library {lib_path()} is missing; run __graft_entry__.build()")
            L = ctypes.CDLL(lib_path())
            V, P, I = ctypes.c_void_p, ctypes.POINTER, ctypes.c_int
            L.svgf_default_config.argtypes = [I, I, P(_Config)]
            L.svgf_channel_config.argtypes = [I, I, I, P(_Config)]
            L.svgf_create.argtypes = [P(_Config), P(V)]
            L.svgf_destroy.argtypes = [V]
            L.svgf_workspace_size.argtypes = [V, P(ctypes.c_size_t)]
            L.svgf_bind_workspace.argtypes = [V, V, ctypes.c_size_t]
            L.svgf_reset_history.argtypes = [V]
            L.svgf_reproject_accumulate.argtypes = [V, P(_Frame), V, V]
            L.svgf_clamp.argtypes = [V, P(_Frame), V, V, V]
            L.svgf_atrous.argtypes = [V, I, P(_Frame), V, V, V]
            L.svgf_inverse_tonemap.argtypes = [V, V, V, V]
            L.svgf_denoise_frame.argtypes = [V, P(_Frame), V, V]
            L.svgf_history_export.argtypes = [V, V, V, V]
            L.svgf_history_import.argtypes = [V, V, V, I, V]
            L.svgf_status_string.argtypes = [I]
            L.svgf_status_string.restype = ctypes.c_char_p
            L.svgf_last_error.argtypes = [V]
            L.svgf_last_error.restype = ctypes.c_char_p
            L.svgf_launch_count.argtypes = [V]
            L.svgf_launch_count.restype = ctypes.c_ulonglong
            L.svgf_staging_size.argtypes = [V, P(ctypes.c_size_t)]
            L.svgf_bind_staging.argtypes = [V, V, ctypes.c_size_t]
            L.svgf_denoise_frame_host.argtypes = [V, P(_Frame), V, V]
            L.svgf_host_submit.argtypes = [V, P(_Frame), V, V]
            L.svgf_host_wait.argtypes = [V]
            L.svgf_profile_enable.argtypes = [V, I]
            L.svgf_profile_read.argtypes = [V, P(ctypes.c_double), P(ctypes.c_ulonglong), I]
            L.svgf_atrous_separable_noalloc.argtypes = [V, I, P(_Frame), V, V, V]
            L.svgf_batch_create.argtypes = [P(V), I, P(V)]
            L.svgf_batch_destroy.argtypes = [V]
            L.svgf_batch_denoise.argtypes = [V, P(_Frame), P(V), V]
            L.svgf_batch_use_graph.argtypes = [V, I]
            L.svgf_batch_autotune.argtypes = [V, P(_Frame), P(V), V, ctypes.c_char_p, ctypes.c_size_t]
            L.svgf_batch_get_tuning.argtypes = [V, P(I), P(I)]
            L.svgf_batch_set_tuning.argtypes = [V, I, I]
            L.svgf_kpn_workspace_size.argtypes = [I, P(ctypes.c_size_t)]
            L.svgf_kpn_create.argtypes = [V, V, V, V, V, ctypes.c_size_t, I, P(V)]
            L.svgf_kpn_destroy.argtypes = [V]
            L.svgf_kpn_check_device.argtypes = [V, P(I), V]
            L.svgf_kpn_wait_selftest.argtypes = [V, I, V]
            L.svgf_kpn_save.argtypes = [V, V, P(ctypes.c_size_t), V]
            L.svgf_kpn_load.argtypes = [V, V, ctypes.c_size_t, V]
            L.svgf_kpn_params_changed.argtypes = [V, I, V]
            L.svgf_kpn_forward.argtypes = [V, V, V, I, I, I, V, V]
            L.svgf_kpn_grad.argtypes = [V, V, V, V, I, I, I, V, V]
            L.svgf_kpn_train_step.argtypes = [V, V, V, V, I, I, I, ctypes.c_float, V, V]
            L.svgf_kpn_features.argtypes = [V, V, P(_Frame), V, V, V, V]
            L.svgf_kpn_predict.argtypes = [V, V, I, I, I, V, I, V]
            L.svgf_kpn_apply.argtypes = [V, V, V, V, V, V]
            L.svgf_kpn_denoise_frame.argtypes = [V, V, P(_Frame), V, V, ctypes.c_float, P(I), V]
            for name in EXPORTS:
                if name not in ("svgf_status_string", "svgf_last_error", "svgf_launch_count"):
                    getattr(L, name).restype = ctypes.c_int
            _lib = L
    return _lib


@dataclasses.dataclass
class Config:
    width: int
    height: int
    alpha: float = 0.2
    alpha_moments: float = 0.2
    clamp_gamma: float = 1.0
    atrous_iters: int = 5
    sigma_z: float = 1.0
    sigma_n: float = 128.0
    sigma_l: float = 4.0
    spatial_mode: int = ATROUS_5X5
    clamp_enable: int = 1
    adaptive_start: int = 1
    roughness_threshold: float = 0.2
    tonemap: int = 1
    luma_k: float = 1.0
    inv_weight: float = 1.0
    inverse_mode: int = INVERSE_EXACT
    history_from_pass: int = 0
    depth_rel_tol: float = 0.1
    normal_cos_tol: float = 0.9
    disocclusion_weight: float = 1e-4
    max_history: int = 255
    min_temporal_frames: int = 4
    spatial_var_radius: int = 3
    eps: float = 1e-10
    precision: int = FP32
    rectify_mode: int = RECTIFY_CLAMP
    iter_by_roughness: int = 0
    iter_rough_t0: float = 0.0
    iter_rough_t1: float = 0.05
    iter_count0: int = 0
    iter_count1: int = 1

    def _c(self) -> _Config:
        return _Config(*[getattr(self, n) for n, _ in _Config._fields_])


def default_config(width: int, height: int) -> Config:
    c = _Config()
    st = lib().svgf_default_config(width, height, ctypes.byref(c))
    if st != SVGF_OK:
        raise SvgfError("svgf_default_config", st)
    return Config(**{n: getattr(c, n) for n, _ in _Config._fields_})


def channel_config(channel: int, width: int, height: int) -> Config:
    """Defaults of one denoised channel (CHANNEL_INDIRECT_SPECULAR or CHANNEL_SHADOW)."""
    c = _Config()
    st = lib().svgf_channel_config(int(channel), width, height, ctypes.byref(c))
    if st != SVGF_OK:
        raise SvgfError("svgf_channel_config", st)
    return Config(**{n: getattr(c, n) for n, _ in _Config._fields_})


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device (CUDA) tensors are required")
    if not t.is_contiguous():
        raise ValueError("contiguous tensors are required")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def make_frame(noisy, gbuf_nz, motion, roughness=None, prev_gbuf_nz=None) -> _Frame:
    """Pack device tensors (float32: [H,W,3], [H,W,4], [H,W,2], [H,W], [H,W,4]) into an svgf_frame."""
    def v(t):
        return None if t is None else t.data_ptr()
    for t in (noisy, gbuf_nz, motion, roughness, prev_gbuf_nz):
        if t is not None and (not t.is_cuda or not t.is_contiguous()):
            raise ValueError("frame tensors must be contiguous CUDA tensors")
    fr = _Frame(v(noisy), v(gbuf_nz), v(prev_gbuf_nz), v(motion), v(roughness))
    fr._keep = (noisy, gbuf_nz, motion, roughness, prev_gbuf_nz)   # the frame owns its tensors
    return fr


class Denoiser:
    """One denoiser handle with a torch-allocated, caller-owned workspace."""

    def __init__(self, cfg: Config, device=None):
        import torch
        self.cfg = cfg
        self._L = lib()
        h = ctypes.c_void_p()
        self._check("svgf_create", self._L.svgf_create(ctypes.byref(cfg._c()), ctypes.byref(h)))
        self._h = h
        n = ctypes.c_size_t()
        self._check("svgf_workspace_size", self._L.svgf_workspace_size(self._h, ctypes.byref(n)))
        self.workspace_bytes = n.value
        self.workspace = torch.empty(n.value + 256, dtype=torch.uint8,
                                     device=device or torch.device("cuda"))
        base = self.workspace.data_ptr()
        off = (-base) % 256
        self._check("svgf_bind_workspace",
                    self._L.svgf_bind_workspace(self._h, ctypes.c_void_p(base + off), n.value))

    def _check(self, fn, st):
        if st != SVGF_OK:
            detail = ""
            if getattr(self, "_h", None) is not None:
                detail = (self._L.svgf_last_error(self._h) or b"").decode()
            raise SvgfError(fn, st, detail)

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._L.svgf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def launch_count(self) -> int:
        return int(self._L.svgf_launch_count(self._h))

    def reset_history(self):
        self._check("svgf_reset_history", self._L.svgf_reset_history(self._h))

    def reproject_accumulate(self, frame: _Frame, cv_out, stream=None):
        self._check("svgf_reproject_accumulate",
                    self._L.svgf_reproject_accumulate(self._h, ctypes.byref(frame), _ptr(cv_out), _stream(stream)))

    def clamp(self, frame: _Frame, hist_in, hist_out, stream=None):
        self._check("svgf_clamp", self._L.svgf_clamp(self._h, ctypes.byref(frame), _ptr(hist_in),
                                                      _ptr(hist_out), _stream(stream)))

    def atrous(self, it: int, frame: _Frame, cv_in, cv_out, stream=None):
        self._check("svgf_atrous", self._L.svgf_atrous(self._h, int(it), ctypes.byref(frame), _ptr(cv_in),
                                                        _ptr(cv_out), _stream(stream)))

    def inverse_tonemap(self, cv_in, rgb_out, stream=None):
        self._check("svgf_inverse_tonemap",
                    self._L.svgf_inverse_tonemap(self._h, _ptr(cv_in), _ptr(rgb_out), _stream(stream)))

    def denoise_frame(self, frame: _Frame, rgb_out, stream=None):
        self._check("svgf_denoise_frame",
                    self._L.svgf_denoise_frame(self._h, ctypes.byref(frame), _ptr(rgb_out), _stream(stream)))

    def history_export(self, hist_rgb, moments, stream=None):
        self._check("svgf_history_export",
                    self._L.svgf_history_export(self._h, _ptr(hist_rgb), _ptr(moments), _stream(stream)))

    def enable_host_staging(self):
        """Bind a torch-allocated staging area so denoise_frame_host can take host buffers."""
        import torch
        n = ctypes.c_size_t()
        self._check("svgf_staging_size", self._L.svgf_staging_size(self._h, ctypes.byref(n)))
        self.staging = torch.empty(n.value + 256, dtype=torch.uint8, device=self.workspace.device)
        base = self.staging.data_ptr()
        self._check("svgf_bind_staging",
                    self._L.svgf_bind_staging(self._h, ctypes.c_void_p(base + (-base) % 256), n.value))

    def denoise_frame_host(self, noisy, gbuf_nz, motion, roughness, rgb_out, stream=None):
        """Host (CPU, ideally pinned) tensors in, host tensor out; returns when rgb_out is ready."""
        for t in (noisy, gbuf_nz, motion, roughness, rgb_out):
            if t is not None and (t.is_cuda or not t.is_contiguous()):
                raise ValueError("host (CPU) contiguous tensors are required")
        fr = _Frame(noisy.data_ptr(), gbuf_nz.data_ptr(), None, motion.data_ptr(),
                    None if roughness is None else roughness.data_ptr())
        self._check("svgf_denoise_frame_host",
                    self._L.svgf_denoise_frame_host(self._h, ctypes.byref(fr), ctypes.c_void_p(rgb_out.data_ptr()),
                                                    _stream(stream)))

    def submit_host(self, noisy, gbuf_nz, motion, roughness, rgb_out, stream=None):
        """Pipelined form: enqueue one frame from host tensors and return at once; rgb_out holds
        the result after wait_host().  The input tensors must stay unchanged until then."""
        for t in (noisy, gbuf_nz, motion, roughness, rgb_out):
            if t is not None and (t.is_cuda or not t.is_contiguous()):
                raise ValueError("host (CPU) contiguous tensors are required")
        fr = _Frame(noisy.data_ptr(), gbuf_nz.data_ptr(), None, motion.data_ptr(),
                    None if roughness is None else roughness.data_ptr())
        self._check("svgf_host_submit",
                    self._L.svgf_host_submit(self._h, ctypes.byref(fr), ctypes.c_void_p(rgb_out.data_ptr()),
                                             _stream(stream)))

    def wait_host(self):
        self._check("svgf_host_wait", self._L.svgf_host_wait(self._h))

    def profile_enable(self, on=True):
        self._check("svgf_profile_enable", self._L.svgf_profile_enable(self._h, int(bool(on))))

    def profile_read(self):
        """{kernel kind: (total ms, launches)} since the last read (the stream must be idle)."""
        n = len(KERNEL_KINDS)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_ulonglong * n)()
        self._check("svgf_profile_read", self._L.svgf_profile_read(self._h, ms, cnt, n))
        return {k: (ms[i], int(cnt[i])) for i, k in enumerate(KERNEL_KINDS)}

    def history_import(self, hist_rgb, moments, has_history=True, stream=None):
        self._check("svgf_history_import",
                    self._L.svgf_history_import(self._h, _ptr(hist_rgb), _ptr(moments), int(bool(has_history)),
                                                _stream(stream)))


class Batch:
    """A batch of denoisers (streams) that share the storage precision, the spatial mode and the
    pass count; the other fields and the frame size may differ (e.g. channels of one frame)."""

    def __init__(self, denoisers):
        self._L = lib()
        self.denoisers = list(denoisers)        # the handles must outlive the batch
        arr = (ctypes.c_void_p * len(self.denoisers))(*[d._h.value for d in self.denoisers])
        b = ctypes.c_void_p()
        st = self._L.svgf_batch_create(arr, len(self.denoisers), ctypes.byref(b))
        if st != SVGF_OK:
            raise SvgfError("svgf_batch_create", st)
        self._b = b

    def close(self):
        if getattr(self, "_b", None) is not None:
            self._L.svgf_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _args(self, frames, outs):
        if len(frames) != len(self.denoisers) or len(outs) != len(self.denoisers):
            raise ValueError("one frame and one output per stream")
        fa = (_Frame * len(frames))(*frames)
        oa = (ctypes.c_void_p * len(outs))(*[_ptr(o).value for o in outs])
        return fa, oa

    def _check(self, fn, st):
        if st != SVGF_OK:
            detail = (self._L.svgf_last_error(self.denoisers[0]._h) or b"").decode()
            raise SvgfError(fn, st, detail)

    def use_graph(self, on=True):
        self._check("svgf_batch_use_graph", self._L.svgf_batch_use_graph(self._b, int(bool(on))))

    def denoise(self, frames, outs, stream=None):
        fa, oa = self._args(frames, outs)
        self._check("svgf_batch_denoise", self._L.svgf_batch_denoise(self._b, fa, oa, _stream(stream)))

    def autotune(self, frames, outs, stream=None) -> str:
        fa, oa = self._args(frames, outs)
        buf = ctypes.create_string_buffer(4096)
        self._check("svgf_batch_autotune",
                    self._L.svgf_batch_autotune(self._b, fa, oa, _stream(stream), buf, len(buf)))
        return buf.value.decode()

    @property
    def tuning(self):
        a, b = ctypes.c_int(), ctypes.c_int()
        self._check("svgf_batch_get_tuning", self._L.svgf_batch_get_tuning(self._b, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    @tuning.setter
    def tuning(self, v):
        self._check("svgf_batch_set_tuning", self._L.svgf_batch_set_tuning(self._b, int(v[0]), int(v[1])))


class KPN:
    """The kernel-predicting network: caller-owned (torch) parameters, optimiser state and
    workspace for batches or frames of up to max_pixels pixels."""

    def __init__(self, max_pixels: int, train: bool = True, device=None):
        import torch
        self._L = lib()
        dev = device or torch.device("cuda")
        f32 = dict(dtype=torch.float32, device=dev)
        self.params = torch.zeros(KPN_PARAM_COUNT, **f32)
        self.grad = torch.zeros(KPN_PARAM_COUNT, **f32) if train else None
        self.adam_m = torch.zeros(KPN_PARAM_COUNT, **f32) if train else None
        self.adam_v = torch.zeros(KPN_PARAM_COUNT, **f32) if train else None
        n = ctypes.c_size_t()
        st = self._L.svgf_kpn_workspace_size(int(max_pixels), ctypes.byref(n))
        if st != SVGF_OK:
            raise SvgfError("svgf_kpn_workspace_size", st)
        self.workspace = torch.empty(n.value + 256, dtype=torch.uint8, device=dev)
        base = self.workspace.data_ptr()
        k = ctypes.c_void_p()
        ptr = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
        st = self._L.svgf_kpn_create(ptr(self.params), ptr(self.grad), ptr(self.adam_m), ptr(self.adam_v),
                                     ctypes.c_void_p(base + (-base) % 256), n.value, int(max_pixels), ctypes.byref(k))
        if st != SVGF_OK:
            raise SvgfError("svgf_kpn_create", st)
        self._k = k
        self.max_pixels = int(max_pixels)
        self.loss = torch.zeros(1, **f32)

    def _check(self, fn, st):
        if st != SVGF_OK:
            raise SvgfError(fn, st)

    def close(self):
        if getattr(self, "_k", None) is not None:
            self._L.svgf_kpn_destroy(self._k)
            self._k = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, flat, reset_adam=True, stream=None):
        self.params.copy_(flat)
        self._check("svgf_kpn_params_changed", self._L.svgf_kpn_params_changed(self._k, int(reset_adam), _stream(stream)))

    def init_params(self, seed: int = 0, last_scale: float = 0.1):
        """Kaiming-normal weights (std sqrt(2 / (9 ci))), zero biases; the logits layer scaled by
        last_scale so that the first kernels are close to uniform."""
        import numpy as np
        import torch
        rng = np.random.default_rng(seed)
        parts = []
        for l, (ci, co) in enumerate(zip(KPN_CIN, KPN_COUT)):
            w = rng.standard_normal(co * 9 * ci) * np.sqrt(2.0 / (9 * ci)) * (last_scale if l == 3 else 1.0)
            parts += [w, np.zeros(co)]
        self.set_params(torch.from_numpy(np.concatenate(parts).astype(np.float32)))

    def save(self, stream=None) -> bytes:
        """Checkpoint (parameters, and the Adam state when training) as bytes."""
        n = ctypes.c_size_t()
        self._check("svgf_kpn_save", self._L.svgf_kpn_save(self._k, None, ctypes.byref(n), _stream(stream)))
        buf = ctypes.create_string_buffer(n.value)
        self._check("svgf_kpn_save", self._L.svgf_kpn_save(self._k, buf, ctypes.byref(n), _stream(stream)))
        return buf.raw[:n.value]

    def load(self, data: bytes, stream=None):
        buf = ctypes.create_string_buffer(bytes(data), len(data))
        self._check("svgf_kpn_load", self._L.svgf_kpn_load(self._k, buf, len(data), _stream(stream)))

    def check_device(self, stream=None):
        """Read and clear the device error word; returns it (0 when no tensor-core wait gave up,
        2 when one did)."""
        w = ctypes.c_int()
        st = self._L.svgf_kpn_check_device(self._k, ctypes.byref(w), _stream(stream))
        if st not in (SVGF_OK, 4, 5):
            raise SvgfError("svgf_kpn_check_device", st)
        return w.value

    def wait_selftest(self, tries=1000, stream=None):
        """Enqueue the bounded-wait self-test (a wait on a barrier phase nothing completes, given
        up after `tries` polls); check_device() then returns 2."""
        self._check("svgf_kpn_wait_selftest", self._L.svgf_kpn_wait_selftest(self._k, int(tries), _stream(stream)))

    def forward(self, feats, c0, c2_out, stream=None):
        B, H, W = c0.shape[:3]
        self._check("svgf_kpn_forward", self._L.svgf_kpn_forward(self._k, _ptr(feats), _ptr(c0), B, H, W,
                                                                 _ptr(c2_out), _stream(stream)))

    def predict(self, feats, kernels_out, form=0, stream=None):
        """The per-pixel kernels for features [B][H][W][16] (BF16 bits) into kernels_out
        [B][H][W][32] (FP16 bits, 25 used): form 0 the four layers in one kernel, 1 layer by layer,
        2 two kernels of two layers."""
        B, H, W = feats.shape[:3]
        self._check("svgf_kpn_predict", self._L.svgf_kpn_predict(self._k, _ptr(feats), B, H, W, _ptr(kernels_out),
                                                                 int(form), _stream(stream)))

    def apply(self, denoiser, kernels, c0, rgb_out, stream=None):
        """Both kernel applications and the inverse tone map: kernels [H][W][32] (FP16 bits), c0
        [H][W][4] -> rgb_out [H][W][4]."""
        self._check("svgf_kpn_apply", self._L.svgf_kpn_apply(self._k, denoiser._h, _ptr(kernels), _ptr(c0),
                                                             _ptr(rgb_out), _stream(stream)))

    def compute_grad(self, feats, c0, target, stream=None):
        B, H, W = c0.shape[:3]
        self._check("svgf_kpn_grad", self._L.svgf_kpn_grad(self._k, _ptr(feats), _ptr(c0), _ptr(target), B, H, W,
                                                           _ptr(self.loss), _stream(stream)))
        return self.loss

    def train_step(self, feats, c0, target, lr=1e-3, stream=None):
        B, H, W = c0.shape[:3]
        self._check("svgf_kpn_train_step",
                    self._L.svgf_kpn_train_step(self._k, _ptr(feats), _ptr(c0), _ptr(target), B, H, W,
                                                ctypes.c_float(lr), _ptr(self.loss), _stream(stream)))
        return self.loss

    def features(self, denoiser, cv, frame, albedo, feats_out, c0_out=None, stream=None):
        self._check("svgf_kpn_features",
                    self._L.svgf_kpn_features(denoiser._h, _ptr(cv), ctypes.byref(frame), _ptr(albedo),
                                              _ptr(feats_out), _ptr(c0_out), _stream(stream)))

    def denoise_frame(self, denoiser, frame, albedo, rgb_out, detail_threshold=float("inf"), stream=None):
        """The learned frame; tiles whose pass-0 luminance standard deviation exceeds
        detail_threshold take the plain passes.  Returns the number of such tiles."""
        n = ctypes.c_int(0)
        self._check("svgf_kpn_denoise_frame",
                    self._L.svgf_kpn_denoise_frame(self._k, denoiser._h, ctypes.byref(frame), _ptr(albedo),
                                                   _ptr(rgb_out), ctypes.c_float(detail_threshold), ctypes.byref(n),
                                                   _stream(stream)))
        return n.value
