"""Temporal accumulation before denoising (Sec. 4.3) through the C ABI
(argument marshalling only; the work runs in csrc/temporal.cu)."""
from __future__ import annotations

import ctypes

from . import _dev_f32, _lib, _stream


class TemporalAccumulator:
    """History of one stream of h x w frames.  `step` takes float32 CUDA
    tensors radiance/position/normal [3,h,w] (or [1,3,h,w]) and motion
    [2,h,w] and returns the accumulated radiance [3,h,w]."""

    def __init__(self, h: int, w: int, alpha_min: float = None, tau_pos: float = None,
                 tau_normal: float = None, min_weight: float = None):
        lib = _lib.load()
        cfg = _lib.TemporalConfig()
        lib.wskpn_temporal_config_default(ctypes.byref(cfg))
        for k, v in (("alpha_min", alpha_min), ("tau_pos", tau_pos), ("tau_normal", tau_normal),
                     ("min_weight", min_weight)):
            if v is not None:
                setattr(cfg, k, float(v))
        self.config = {k: getattr(cfg, k) for k, _ in _lib.TemporalConfig._fields_}
        self.h, self.w = int(h), int(w)
        self._t = ctypes.c_void_p()
        _lib.check(lib.wskpn_temporal_create(ctypes.byref(cfg), self.h, self.w, ctypes.byref(self._t)))

    def _plane(self, t, c, name):
        if tuple(t.shape[-3:]) != (c, self.h, self.w):
            raise ValueError(f"{name} must be [{c},{self.h},{self.w}]")
        return _dev_f32(t.contiguous(), name)

    def _out(self, t):
        if tuple(t.shape[-3:]) != (3, self.h, self.w):
            raise ValueError(f"out must be [3,{self.h},{self.w}]")
        return _dev_f32(t, "out")

    def step(self, radiance, position, normal, motion, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((3, self.h, self.w), device=radiance.device, dtype=torch.float32)
        _lib.check(_lib.load().wskpn_temporal_step(
            self._t, self._plane(radiance, 3, "radiance"), self._plane(position, 3, "position"),
            self._plane(normal, 3, "normal"), self._plane(motion, 2, "motion"), self._out(out),
            _stream(stream)))
        return out

    def history(self, stream=None):
        import torch
        h = torch.empty((self.h, self.w), device="cuda", dtype=torch.float32)
        _lib.check(_lib.load().wskpn_temporal_history(self._t, _dev_f32(h, "history"), _stream(stream)))
        return h

    def reset(self, stream=None):
        _lib.check(_lib.load().wskpn_temporal_reset(self._t, _stream(stream)))

    def close(self):
        if self._t:
            _lib.load().wskpn_temporal_destroy(self._t)
            self._t = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
