"""Multi-resolution variant of the denoiser (Eq. 7) through the C ABI
(argument marshalling only; the work runs in csrc/multires.cu)."""
from __future__ import annotations

import ctypes

from . import _frames, _lib, _stream


def n_weights() -> int:
    return int(_lib.load().wskpn_mr_n_weights())


class MultiResDenoiser:
    """U-Net + 3-level reconstruction with kernels 3 and 5 per level; the
    U-Net in FP32 (SIMT) or BF16 (tensor cores, hi/lo activations)."""

    def __init__(self, weights, max_hw=(1080, 1920), precision="fp32", albedo_eps=1e-2, gamma=2.2, depth_near=1.0,
                 depth_far=10.0):
        import numpy as np
        self._lib = _lib.load()
        cfg = _lib.MrConfig()
        self._lib.wskpn_mr_config_default(ctypes.byref(cfg))
        cfg.max_h, cfg.max_w = int(max_hw[0]), int(max_hw[1])
        cfg.albedo_eps, cfg.gamma, cfg.depth_near, cfg.depth_far = albedo_eps, gamma, depth_near, depth_far
        cfg.prec = {"fp32": _lib.FP32, "bf16": _lib.BF16}[precision]
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.float32).ravel())
        h = ctypes.c_void_p()
        _lib.check(self._lib.wskpn_mr_create(ctypes.byref(cfg), w.ctypes.data, w.size, ctypes.byref(h)))
        self._h = h

    def _check(self, status):
        if status != _lib.OK:
            msg = self._lib.wskpn_mr_last_error(self._h)
            raise _lib.WskpnError(status, msg.decode() if msg else "")

    def denoise(self, radiance, albedo, normal, depth, out=None, stream=None):
        """One frame: [1, C, H, W] (or [C, H, W]) float32 CUDA tensors -> [1, 3, H, W]."""
        import torch
        sq = lambda t: t if t.dim() == 4 else t.unsqueeze(0)
        fr, B, H, W = _frames(sq(radiance), sq(albedo), sq(normal), sq(depth))
        if B != 1:
            raise ValueError("one frame per call")
        if out is None:
            out = torch.empty((1, 3, H, W), device=radiance.device, dtype=torch.float32)
        self._check(self._lib.wskpn_mr_denoise(self._h, fr, H, W, ctypes.c_void_p(out.data_ptr()), _stream(stream)))
        return out

    def logits(self, radiance, albedo, normal, depth, stream=None):
        """The U-Net outputs [z0 [5,H,W], z1 [5,H1,W1], z2 [4,H2,W2]]."""
        import torch
        sq = lambda t: t if t.dim() == 4 else t.unsqueeze(0)
        fr, B, H, W = _frames(sq(radiance), sq(albedo), sq(normal), sq(depth))
        h1, w1 = (H + 1) // 2, (W + 1) // 2
        h2, w2 = (h1 + 1) // 2, (w1 + 1) // 2
        zs = [torch.empty(s, device=radiance.device, dtype=torch.float32)
              for s in ((5, H, W), (5, h1, w1), (4, h2, w2))]
        self._check(self._lib.wskpn_mr_logits(self._h, fr, H, W, *(ctypes.c_void_p(z.data_ptr()) for z in zs),
                                              _stream(stream)))
        return zs

    def close(self):
        if getattr(self, "_h", None):
            self._lib.wskpn_mr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
