"""Temporal accumulation before denoising (paper Sec. 4.3, "temporal
accumulation"): the previous frame's accumulated radiance is reprojected to
the current frame with the motion vectors, each reprojected sample is kept
only if its geometry agrees with the current pixel (world position and
shading normal), and the current 1-spp radiance is blended with the kept
history; pixels with no consistent history keep their own 1-spp value.

TEST INFRASTRUCTURE ONLY (part of the oracle; see oracle/__init__.py).

The paper names the steps but not their constants; the readings taken here:

* reprojection: the previous position of pixel p = (x, y) is q = p + m(p)
  (pixel centres at integer coordinates); the history at q is the bilinear
  combination of the 4 pixels around q;
* consistency, per tap: inside the image, a history exists (h > 0),
  |P_prev - P|^2 < tau_pos^2 and n_prev . n > tau_normal;
* the kept taps' bilinear weights are renormalised; a pixel whose kept
  weight sum W is not above min_weight gets no history;
* blend: h = (reprojected history length) + 1, alpha = max(1 / h, alpha_min),
  A = A_prev + alpha (c - A_prev), i.e. a running mean for the first
  1 / alpha_min frames and an exponential moving average after that;
* defaults: alpha_min = 0.2, tau_pos = 0.1 world units, tau_normal = 0.9,
  min_weight = 1e-3.

Everything a branch depends on -- q and its floor, the four bilinear
weights, their kept sum W and the two consistency measures -- is evaluated
in float32 with one rounding per operation in a fixed order (no fused
multiply-add), so a float32 implementation that follows the same order takes
the same decisions.  The blend arithmetic itself is float64.
"""
from __future__ import annotations

import numpy as np

DEFAULTS = dict(alpha_min=0.2, tau_pos=0.1, tau_normal=0.9, min_weight=1e-3)

f32 = np.float32


class TemporalState:
    """History of one stream: accumulated radiance A[3,H,W], world position
    P[3,H,W], normal n[3,H,W] and history length h[H,W] (0 = no history)."""

    def __init__(self, H: int, W: int):
        self.A = np.zeros((3, H, W))
        self.P = np.zeros((3, H, W), dtype=np.float32)
        self.n = np.zeros((3, H, W), dtype=np.float32)
        self.h = np.zeros((H, W))


def _tap_weights(fx, fy):
    """Bilinear weights of the taps (0,0), (1,0), (0,1), (1,1), float32."""
    one = f32(1.0)
    a = (one - fx).astype(f32)
    b = (one - fy).astype(f32)
    return [(a * b).astype(f32), (fx * b).astype(f32), (a * fy).astype(f32), (fx * fy).astype(f32)]


def accumulate(state: TemporalState, radiance, position, normal, motion, alpha_min=DEFAULTS["alpha_min"],
               tau_pos=DEFAULTS["tau_pos"], tau_normal=DEFAULTS["tau_normal"],
               min_weight=DEFAULTS["min_weight"]):
    """One frame of temporal accumulation.  Inputs are float32 planar
    [3,H,W] (radiance, position, normal) and [2,H,W] (motion, (x, y) offset
    to the previous frame).  Returns the accumulated radiance (float64
    [3,H,W]) and updates `state` to this frame."""
    c = np.asarray(radiance, dtype=np.float64)
    P = np.asarray(position, dtype=f32)
    n = np.asarray(normal, dtype=f32)
    m = np.asarray(motion, dtype=f32)
    _, H, W = c.shape
    ys, xs = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")

    # 1. reprojection: q = p + m, its integer corner and fractional offset
    qx = (xs.astype(f32) + m[0]).astype(f32)
    qy = (ys.astype(f32) + m[1]).astype(f32)
    x0 = np.floor(qx).astype(np.int64)
    y0 = np.floor(qy).astype(np.int64)
    fx = (qx - np.floor(qx).astype(f32)).astype(f32)
    fy = (qy - np.floor(qy).astype(f32)).astype(f32)
    wts = _tap_weights(fx, fy)

    # 2. consistency of each tap, 3. kept weights and their sum (float32, in tap order)
    tp2 = f32(tau_pos) * f32(tau_pos)
    Wsum = np.zeros((H, W), dtype=f32)
    Aacc = np.zeros((3, H, W))
    hacc = np.zeros((H, W))
    for t, (dx, dy) in enumerate(((0, 0), (1, 0), (0, 1), (1, 1))):
        tx, ty = x0 + dx, y0 + dy
        inside = (tx >= 0) & (tx < W) & (ty >= 0) & (ty < H)
        cx, cy = np.clip(tx, 0, W - 1), np.clip(ty, 0, H - 1)
        Pp = state.P[:, cy, cx]
        np_ = state.n[:, cy, cx]
        d = [(Pp[i] - P[i]).astype(f32) for i in range(3)]
        dist2 = (((d[0] * d[0]).astype(f32) + (d[1] * d[1]).astype(f32)).astype(f32)
                 + (d[2] * d[2]).astype(f32)).astype(f32)
        dot = (((np_[0] * n[0]).astype(f32) + (np_[1] * n[1]).astype(f32)).astype(f32)
               + (np_[2] * n[2]).astype(f32)).astype(f32)
        keep = inside & (state.h[cy, cx] > 0) & (dist2 < tp2) & (dot > f32(tau_normal))
        w = np.where(keep, wts[t], f32(0.0)).astype(f32)
        Wsum = (Wsum + w).astype(f32)
        Aacc += w.astype(np.float64)[None] * state.A[:, cy, cx]
        hacc += w.astype(np.float64) * state.h[cy, cx]

    # 4. blend with the renormalised history, or restart from the 1-spp value
    has = Wsum > f32(min_weight)
    Wd = np.where(has, Wsum.astype(np.float64), 1.0)
    A_prev = Aacc / Wd[None]
    h_new = np.where(has, hacc / Wd + 1.0, 1.0)
    alpha = np.maximum(1.0 / h_new, alpha_min)
    A = np.where(has[None], A_prev + alpha[None] * (c - A_prev), c)

    state.A, state.P, state.n, state.h = A, P.copy(), n.copy(), h_new
    return A
