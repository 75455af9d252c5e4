"""Multi-resolution variant of the denoiser (the paper's Tungsten
configuration, Sec. 5.3 "Implementation" and Eq. 7): a U-Net predicts, at 3
resolutions, two importance maps (kernel sizes 3 and 5), their two fusion
logits and (except at the coarsest level) a blending logit; each level filters
the demodulated irradiance downsampled to its resolution with its two fused
kernels (Eq. 3-5), and the levels are combined from the coarsest with Eq. 7:

    o_p = i^f_p - alpha_p [U D i^f]_p + alpha_p [U i^c]_p

TEST INFRASTRUCTURE ONLY (part of the oracle; see oracle/__init__.py).  The
convolutions and the per-level decode are the C oracle's pinned routines;
the rest is numpy in float64.

The paper leaves the network to a supplement that is not available; the
readings taken here:

* D is the 2x2 box average (a block cut by the image border averages its
  in-image pixels), U the nearest-neighbour upsampling to the finer size;
* levels 0, 1, 2 have sizes (H, W), ceil halves, ceil quarters;
* U-Net with 3x3 convolutions, zero padding 1, ReLU after every conv but the
  heads; encoder E0 10->32, E0b 32->32 | D | E1 32->48, E1b 48->48 | D |
  E2 48->64, E2b 64->64; head H2 64->4 on E2b; decoder level 1:
  concat(U E2b, E1b) 112->48 (D1), head H1 48->5; level 0: concat(U D1,
  E0b) 80->32 (D0), head H0 32->5;
* head channels: importance maps for k = 3, 5, fusion logits for k = 3, 5,
  then (levels 0 and 1) the blending logit b, alpha = sigmoid(b);
* the irradiance is y = r / (a + eps) and the output (a + eps) o_0.
"""
from __future__ import annotations

import numpy as np

from . import _d, conv2d, decode_boxsum, prep, DEFAULT_EPS, DEFAULT_GAMMA, DEPTH_FAR, DEPTH_NEAR

KSIZES = (3, 5)
LEVELS = 3
CONV_KS = 3
# (name, cin, cout, relu) in weight-blob order; every layer is W[cout][cin][3][3] then b[cout]
LAYERS = (("E0", 10, 32, True), ("E0b", 32, 32, True), ("E1", 32, 48, True), ("E1b", 48, 48, True),
          ("E2", 48, 64, True), ("E2b", 64, 64, True), ("H2", 64, 4, False), ("D1", 112, 48, True),
          ("H1", 48, 5, False), ("D0", 80, 32, True), ("H0", 32, 5, False))


def weight_shapes():
    return [((co, ci, CONV_KS, CONV_KS), (co,)) for _, ci, co, _ in LAYERS]


def n_weights() -> int:
    return sum(co * ci * CONV_KS * CONV_KS + co for _, ci, co, _ in LAYERS)


def split_weights(blob):
    blob = _d(blob)
    out, off = {}, 0
    for name, ci, co, relu in LAYERS:
        nw = co * ci * CONV_KS * CONV_KS
        out[name] = (blob[off:off + nw].reshape(co, ci, CONV_KS, CONV_KS), blob[off + nw:off + nw + co], relu)
        off += nw + co
    assert off == blob.size, (off, blob.size)
    return out


def level_sizes(H: int, W: int):
    sizes = [(H, W)]
    for _ in range(LEVELS - 1):
        h, w = sizes[-1]
        sizes.append(((h + 1) // 2, (w + 1) // 2))
    return sizes


def downsample(x):
    """D: 2x2 box average of [C, H, W] to [C, ceil(H/2), ceil(W/2)]; a block
    cut by the border averages its in-image pixels."""
    x = _d(x)
    C, H, W = x.shape
    h, w = (H + 1) // 2, (W + 1) // 2
    s = np.zeros((C, h, w))
    n = np.zeros((h, w))
    for dy in (0, 1):
        for dx in (0, 1):
            part = x[:, dy::2, dx::2]
            s[:, :part.shape[1], :part.shape[2]] += part
            n[:part.shape[1], :part.shape[2]] += 1.0
    return s / n[None]


def upsample(x, H: int, W: int):
    """U: nearest-neighbour upsampling of [C, h, w] to [C, H, W]: out(y, x) = in(y // 2, x // 2)."""
    x = _d(x)
    return x[:, np.arange(H) // 2][:, :, np.arange(W) // 2]


def logits(frame, weights, gamma=DEFAULT_GAMMA, dnear=DEPTH_NEAR, dfar=DEPTH_FAR):
    """U-Net outputs [z0 [5,H,W], z1 [5,H1,W1], z2 [4,H2,W2]] of one frame."""
    L = split_weights(weights)
    x0 = prep(frame["radiance"], frame["albedo"], frame["normal"], frame["depth"], gamma, dnear, dfar)

    def c(name, x):
        w, b, relu = L[name]
        return conv2d(x, w, b, relu)

    e0 = c("E0b", c("E0", x0))
    e1 = c("E1b", c("E1", downsample(e0)))
    e2 = c("E2b", c("E2", downsample(e1)))
    z2 = c("H2", e2)
    d1 = c("D1", np.concatenate([upsample(e2, *e1.shape[1:]), e1]))
    z1 = c("H1", d1)
    d0 = c("D0", np.concatenate([upsample(d1, *e0.shape[1:]), e0]))
    z0 = c("H0", d0)
    return [z0, z1, z2]


def filter_level(z, y, ksizes=KSIZES):
    """Eq. 3-5 without re-modulation at one level: sum_i softmax_i(z[M+i]) R_i,
    R_i the k_i-window filtering of y [3, h, w] with importance map z[i]."""
    z, y = _d(z), _d(y)
    M = len(ksizes)
    Rs = np.stack([decode_boxsum(z[i], y, k) for i, k in enumerate(ksizes)])
    a = z[M:2 * M]
    e = np.exp(a - a.max(axis=0, keepdims=True))
    alpha = e / e.sum(axis=0, keepdims=True)
    return np.einsum("ihw,ichw->chw", alpha, Rs)


def combine(i_levels, blend_logits):
    """Eq. 7 from the coarsest level: o_{L-1} = i_{L-1};
    o_l = i_l - alpha_l U D i_l + alpha_l U o_{l+1}, alpha_l = sigmoid(b_l)."""
    o = _d(i_levels[-1])
    for l in range(len(i_levels) - 2, -1, -1):
        i_f = _d(i_levels[l])
        _, H, W = i_f.shape
        alpha = 1.0 / (1.0 + np.exp(-_d(blend_logits[l])))
        o = i_f - alpha[None] * upsample(downsample(i_f), H, W) + alpha[None] * upsample(o, H, W)
    return o


def reconstruct(zs, rad, alb, eps=DEFAULT_EPS, ksizes=KSIZES):
    """Multi-resolution reconstruction from the U-Net outputs zs."""
    rad, alb = _d(rad), _d(alb)
    M = len(ksizes)
    y = rad / (alb + eps)
    ys = [y]
    for _ in range(len(zs) - 1):
        ys.append(downsample(ys[-1]))
    i_levels = [filter_level(z[:2 * M], yl, ksizes) for z, yl in zip(zs, ys)]
    o = combine(i_levels, [z[2 * M] for z in zs[:-1]])
    return (alb + eps) * o


def term_scale(zs, rad, alb, eps=DEFAULT_EPS, ksizes=KSIZES):
    """Per-element magnitude of the three terms Eq. 7 sums at the finest level,
    (a + eps)(|i_0| + alpha_0 |U D i_0| + alpha_0 |U o_1|): the scale that the
    rounding error of any evaluation of the combination is proportional to
    (the combination can cancel to values far below its terms)."""
    rad, alb = _d(rad), _d(alb)
    M = len(ksizes)
    y = rad / (alb + eps)
    ys = [y]
    for _ in range(len(zs) - 1):
        ys.append(downsample(ys[-1]))
    i_levels = [filter_level(z[:2 * M], yl, ksizes) for z, yl in zip(zs, ys)]
    o1 = combine(i_levels[1:], [z[2 * M] for z in zs[1:-1]])
    _, H, W = i_levels[0].shape
    alpha = 1.0 / (1.0 + np.exp(-_d(zs[0][2 * M])))
    t = (np.abs(i_levels[0]) + alpha[None] * np.abs(upsample(downsample(i_levels[0]), H, W))
         + alpha[None] * np.abs(upsample(o1, H, W)))
    return (alb + eps) * t


def denoise(frame, weights, eps=DEFAULT_EPS):
    """The whole multi-resolution denoiser on one frame: [3, H, W] float64."""
    return reconstruct(logits(frame, weights), frame["radiance"], frame["albedo"], eps)
