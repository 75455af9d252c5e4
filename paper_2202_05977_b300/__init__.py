"""B300-native weight-sharing kernel-prediction Monte Carlo denoiser
(Fan, Wang, Huo, Bao, EGSR 2021).

Thin Python binding over libwskpn.so (include/wskpn.h).  It only marshals
torch tensors (pointers, sizes, the current stream) into C-ABI calls; every
step of the denoiser runs in the library's CUDA kernels.  PyTorch is used
for device memory and streams.
"""
from __future__ import annotations

import ctypes

from . import _lib
from ._lib import BF16, FP8, FP32, WskpnError

__all__ = ["Denoiser", "decode_fuse_fwd", "decode_fuse_bwd", "prep", "default_config", "n_weights", "WskpnError",
           "FP32", "BF16", "FP8", "PRECISIONS"]

PRECISIONS = {"fp32": FP32, "bf16": BF16, "fp8": FP8}
_KEYS = ("radiance", "albedo", "normal", "depth")


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_f32(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def default_config(precision="bf16", widths=(10, 32, 48, 64, 12), conv_ks: int = 5,
                   ksizes=(3, 5, 7, 9, 11, 13), eps: float = 1e-2, gamma: float = 2.2,
                   depth_range=(1.0, 10.0), max_batch: int = 1, max_hw=(1080, 1920)) -> _lib.Config:
    lib = _lib.load()
    c = _lib.Config()
    _lib.check(lib.wskpn_config_default(ctypes.byref(c)))
    c.n_layers = len(widths) - 1
    for i, w in enumerate(widths):
        c.widths[i] = w
    c.conv_ks = conv_ks
    c.n_kernels = len(ksizes)
    for i, k in enumerate(ksizes):
        c.ksizes[i] = k
    c.prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    c.albedo_eps = eps
    c.gamma = gamma
    c.depth_near, c.depth_far = depth_range
    c.max_batch = max_batch
    c.max_h, c.max_w = max_hw
    return c


def n_weights(cfg: _lib.Config) -> int:
    return int(_lib.load().wskpn_n_weights(ctypes.byref(cfg)))


def _frames(radiance, albedo, normal, depth, device=True):
    """Per-frame pointer structs for [B, C, H, W] float32 tensors."""
    B, _, H, W = radiance.shape
    arr = (_lib.Frame * B)()
    for nm, t, c in zip(_KEYS, (radiance, albedo, normal, depth), (3, 3, 3, 1)):
        if device:
            _dev_f32(t, nm)
        elif t.is_cuda or not t.is_contiguous():
            raise TypeError(f"{nm} must be a contiguous host tensor")
        if tuple(t.shape) != (B, c, H, W):
            raise ValueError(f"{nm} must have shape {(B, c, H, W)}, got {tuple(t.shape)}")
        for b in range(B):
            setattr(arr[b], nm, t[b].data_ptr())
    return arr, B, H, W


class Denoiser:
    """A wskpn context: weights resident on the current CUDA device plus
    workspaces for max_batch x max_hw frames."""

    def __init__(self, weights, precision="bf16", **cfg_kw):
        import numpy as np
        self._lib = _lib.load()
        self.cfg = default_config(precision, **cfg_kw)
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.float32).ravel())
        if w.size != n_weights(self.cfg):
            raise ValueError(f"expected {n_weights(self.cfg)} weights, got {w.size}")
        h = ctypes.c_void_p()
        _lib.check(self._lib.wskpn_create(ctypes.byref(self.cfg), w.ctypes.data, w.size, ctypes.byref(h)))
        self._h = h
        self.M = self.cfg.n_kernels
        self.nw = w.size

    def close(self):
        if getattr(self, "_h", None):
            self._lib.wskpn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, s):
        _lib.check(s, self._h)

    def denoise(self, radiance, albedo, normal, depth, out=None, stream=None):
        """D_Theta(r, f) for [B, C, H, W] float32 CUDA tensors -> [B, 3, H, W]."""
        import torch
        fr, B, H, W = _frames(radiance, albedo, normal, depth)
        if out is None:
            out = torch.empty((B, 3, H, W), device=radiance.device, dtype=torch.float32)
        self._check(self._lib.wskpn_denoise(self._h, fr, B, H, W, _dev_f32(out, "out"), _stream(stream)))
        return out

    def denoise_host(self, radiance, albedo, normal, depth, out, stream=None, wait=True):
        """Denoise of HOST float32 tensors [B, C, H, W] (pinned recommended)
        into host tensor `out` [B, 3, H, W]; the library copies the inputs in
        and the result back.  wait=False returns once the work is queued:
        `out` holds the result when `stream` (the current stream if None) has
        reached the point after the call, and the host tensors must be kept
        alive and unmodified until then."""
        fr, B, H, W = _frames(radiance, albedo, normal, depth, device=False)
        if out.is_cuda or not out.is_contiguous() or tuple(out.shape) != (B, 3, H, W):
            raise TypeError("out must be a contiguous host tensor [B, 3, H, W]")
        fn = self._lib.wskpn_denoise_host if wait else self._lib.wskpn_denoise_host_async
        self._check(fn(self._h, fr, B, H, W, ctypes.c_void_p(out.data_ptr()), _stream(stream)))
        return out

    def logits(self, radiance, albedo, normal, depth, out=None, stream=None):
        """ImportanceNet output z [B, 2M, H, W] (importance maps, then fusion logits)."""
        import torch
        fr, B, H, W = _frames(radiance, albedo, normal, depth)
        if out is None:
            out = torch.empty((B, 2 * self.M, H, W), device=radiance.device, dtype=torch.float32)
        self._check(self._lib.wskpn_logits(self._h, fr, B, H, W, _dev_f32(out, "out"), _stream(stream)))
        return out

    def set_weights(self, weights, stream=None):
        import numpy as np
        import torch
        if isinstance(weights, torch.Tensor) and weights.is_cuda:
            self._check(self._lib.wskpn_set_weights(self._h, _dev_f32(weights, "weights"), self.nw, 1,
                                                    _stream(stream)))
        else:
            w = np.ascontiguousarray(np.asarray(weights, dtype=np.float32).ravel())
            self._check(self._lib.wskpn_set_weights(self._h, w.ctypes.data, w.size, 0, _stream(stream)))

    def get_weights(self, stream=None):
        import torch
        out = torch.empty(self.nw, device="cuda", dtype=torch.float32)
        self._check(self._lib.wskpn_get_weights(self._h, _dev_f32(out, "out"), self.nw, _stream(stream)))
        return out

    def calibrate(self, radiance, albedo, normal, depth, margin=2.0, stream=None):
        """FP8 only: set the per-layer activation scales from these frames."""
        fr, B, H, W = _frames(radiance, albedo, normal, depth)
        self._check(self._lib.wskpn_calibrate(self._h, fr, B, H, W, float(margin), _stream(stream)))

    # ------------------------------------------------------------ training
    def forward_train(self, radiance, albedo, normal, depth, out=None, z=None, stream=None):
        """Forward for training: (out [B,3,H,W], z [B,2M,H,W]); z is what backward needs."""
        import torch
        fr, B, H, W = _frames(radiance, albedo, normal, depth)
        if out is None:
            out = torch.empty((B, 3, H, W), device=radiance.device, dtype=torch.float32)
        if z is None:
            z = torch.empty((B, 2 * self.M, H, W), device=radiance.device, dtype=torch.float32)
        self._check(self._lib.wskpn_forward_train(self._h, fr, B, H, W, _dev_f32(out, "out"), _dev_f32(z, "z"),
                                                  _stream(stream)))
        return out, z

    def backward(self, radiance, albedo, normal, depth, z, dout, want_dz=False, stream=None):
        """(dL/dweights [n_weights], dL/dz or None) from dout = dL/d(out)."""
        import torch
        fr, B, H, W = _frames(radiance, albedo, normal, depth)
        dw = torch.empty(self.nw, device=radiance.device, dtype=torch.float32)
        dz = torch.empty((B, 2 * self.M, H, W), device=radiance.device, dtype=torch.float32) if want_dz else None
        self._check(self._lib.wskpn_backward(self._h, fr, B, H, W, _dev_f32(z, "z"), _dev_f32(dout, "dout"),
                                             _dev_f32(dz, "dz") if dz is not None else None, _dev_f32(dw, "dw"),
                                             _stream(stream)))
        return dw, dz

    def l1_loss(self, out, target, want_grad=True, stream=None):
        """(loss [1] device tensor, dL/d(out) or None), L1 mean over all elements."""
        import torch
        loss = torch.empty(1, device=out.device, dtype=torch.float32)
        g = torch.empty_like(out) if want_grad else None
        self._check(self._lib.wskpn_l1_loss(self._h, _dev_f32(out, "out"), _dev_f32(target, "target"), out.numel(),
                                            _dev_f32(loss, "loss"), _dev_f32(g, "dout") if g is not None else None,
                                            _stream(stream)))
        return loss, g

    def adam_step(self, grad, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        self._check(self._lib.wskpn_adam_step(self._h, _dev_f32(grad, "grad"), lr, beta1, beta2, eps, step,
                                              _stream(stream)))

    def profile(self, enable: bool = True):
        """Start/stop recording per-stage CUDA events on each call's stream."""
        self._check(self._lib.wskpn_profile_enable(self._h, int(enable)))

    def profile_read(self):
        """(summed ms per stage [prep, conv1..L, reconstruct], number of calls); clears."""
        ms = (ctypes.c_float * (_lib.MAX_LAYERS + 2))()
        n, calls = ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.wskpn_profile_read(self._h, ms, len(ms), ctypes.byref(n), ctypes.byref(calls)))
        return [ms[i] for i in range(n.value)], calls.value

    def set_tuning(self, key: int, value: int):
        self._check(self._lib.wskpn_set_tuning(self._h, key, value))

    def device_status(self) -> int:
        """Reads and clears the device status word (0 = no bounded wait expired)."""
        v = ctypes.c_uint32()
        s = self._lib.wskpn_device_status(self._h, ctypes.byref(v))
        if s not in (_lib.OK, _lib.ETIMEOUT):
            self._check(s)
        return int(v.value)

    def numeric_fallbacks(self) -> int:
        v = ctypes.c_uint64()
        self._check(self._lib.wskpn_numeric_fallbacks(self._h, ctypes.byref(v)))
        return int(v.value)


def prep(radiance, albedo, normal, depth, gamma=2.2, depth_range=(1.0, 10.0), out=None, stream=None):
    """Sec. 5.1 input assembly -> [B, 10, H, W] float32."""
    import torch
    lib = _lib.load()
    fr, B, H, W = _frames(radiance, albedo, normal, depth)
    if out is None:
        out = torch.empty((B, 10, H, W), device=radiance.device, dtype=torch.float32)
    _lib.check(lib.wskpn_prep(fr, B, H, W, gamma, depth_range[0], depth_range[1], _dev_f32(out, "out"),
                              _stream(stream)))
    return out


def decode_fuse_bwd(z, radiance, albedo, dout, ksizes=(3, 5, 7, 9, 11, 13), eps=1e-2, dz=None, scratch=None,
                    fallbacks=None, stream=None):
    """dL/dz [B, 2M, H, W] from dL/d(out) for the Eq. 3-5 reconstruction."""
    import torch
    lib = _lib.load()
    B, C, H, W = z.shape
    M = len(ksizes)
    if dz is None:
        dz = torch.empty_like(z)
    if scratch is None:
        scratch = torch.empty(int(lib.wskpn_decode_fuse_bwd_scratch_floats(B, H, W, M)), device=z.device,
                              dtype=torch.float32)
    ks = (ctypes.c_int * M)(*ksizes)
    fb = ctypes.c_void_p(fallbacks.data_ptr()) if fallbacks is not None else None
    _lib.check(lib.wskpn_decode_fuse_bwd(_dev_f32(z, "z"), _dev_f32(radiance, "radiance"), _dev_f32(albedo, "albedo"),
                                         _dev_f32(dout, "dout"), B, H, W, M, ks, eps, _dev_f32(dz, "dz"),
                                         _dev_f32(scratch, "scratch"), fb, _stream(stream)))
    return dz


def decode_fuse_fwd(z, radiance, albedo, ksizes=(3, 5, 7, 9, 11, 13), eps=1e-2, out=None,
                    fallbacks=None, stream=None):
    """Eq. 3-5 reconstruction from network outputs z [B, 2M, H, W]."""
    import torch
    lib = _lib.load()
    B, C, H, W = z.shape
    M = len(ksizes)
    if C != 2 * M:
        raise ValueError("z must have 2 * len(ksizes) channels")
    if out is None:
        out = torch.empty((B, 3, H, W), device=z.device, dtype=torch.float32)
    ks = (ctypes.c_int * M)(*ksizes)
    fb = ctypes.c_void_p(fallbacks.data_ptr()) if fallbacks is not None else None
    _lib.check(lib.wskpn_decode_fuse_fwd(_dev_f32(z, "z"), _dev_f32(radiance, "radiance"),
                                         _dev_f32(albedo, "albedo"), B, H, W, M, ks, eps,
                                         _dev_f32(out, "out"), fb, _stream(stream)))
    return out
