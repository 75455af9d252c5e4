"""RepVGG re-parameterisation (Sec. 4.1) through the C ABI (marshalling only)."""
from __future__ import annotations

import ctypes

from . import _dev_f32, _lib, _stream


def fold(w5, b5, w3, b3, w1, b1, identity=False, stream=None):
    """(W [Co,Ci,5,5], b [Co]) of the single 5x5 conv equal to the block."""
    import torch
    co, ci = w5.shape[:2]
    W = torch.empty((co, ci, 5, 5), device=w5.device, dtype=torch.float32)
    b = torch.empty((co,), device=w5.device, dtype=torch.float32)
    _lib.check(_lib.load().wskpn_repvgg_fold(*(_dev_f32(t.contiguous(), "w") for t in (w5, b5, w3, b3, w1, b1)),
                                             ci, co, int(identity), _dev_f32(W, "W"), _dev_f32(b, "b"),
                                             _stream(stream)))
    return W, b


def fold_grad(gW, stream=None):
    """(dL/dw5, dL/dw3, dL/dw1) from dL/dW."""
    import torch
    co, ci = gW.shape[:2]
    g5 = torch.empty((co, ci, 5, 5), device=gW.device, dtype=torch.float32)
    g3 = torch.empty((co, ci, 3, 3), device=gW.device, dtype=torch.float32)
    g1 = torch.empty((co, ci, 1, 1), device=gW.device, dtype=torch.float32)
    _lib.check(_lib.load().wskpn_repvgg_fold_grad(_dev_f32(gW.contiguous(), "gW"), ci, co, _dev_f32(g5, "g5"),
                                                  _dev_f32(g3, "g3"), _dev_f32(g1, "g1"), _stream(stream)))
    return g5, g3, g1
