"""Seeded synthetic inputs for the weight-sharing kernel-prediction denoiser.

This module only *generates data*: 1-spp-like frames (noisy radiance, albedo,
shading normal, depth), training targets and random-init network weights.  It
contains none of the denoiser's arithmetic (no tone mapping, convolution,
kernel construction, filtering or fusion), so both the FP64 oracle and the
CUDA path may draw their inputs from it without sharing any method code.

Frames stand in for the BMFR dataset's 1280x720 1-spp frames (paper Sec. 5.1),
which are not available here.  Recipe (all draws from numpy's PCG64 keyed by
the seed):

* scene: pinhole camera at (0, 1, 0) looking down +z with a 60 degree vertical
  field of view; a ground plane y = 0, a back plane z = 12 and six spheres
  resting on the ground (centre x in [-3, 3], z in [3, 9], radius in
  [0.4, 1.2]), ray-cast analytically;
* normal: the unit surface normal of the first hit (3 channels, in [-1, 1]);
* depth: camera-space z of the hit clamped to [1, 10] (1 channel);
* albedo: uniform [0,1]^3 per cell of an image-space Voronoi partition whose
  64 seeds are jittered on an 8x8 grid (ties go to the lowest seed index);
* clean shading: albedo * (0.1 + sum over two directional lights of
  max(n.l, 0));
* noisy radiance: clean * exp(N(0, 1)) drawn independently per pixel and
  channel, and 2 % of the pixels (Bernoulli per pixel) multiplied by 50 on
  all channels (fireflies).

All buffers are float32, planar, shape [C, H, W].
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "Frame", "make_frame", "make_batch", "make_target", "make_weights",
    "weight_shapes", "n_weights", "make_sequence", "make_weights_for", "DEPTH_NEAR", "DEPTH_FAR",
]

DEPTH_NEAR = 1.0
DEPTH_FAR = 10.0

_LIGHTS = np.array([[1.0, 2.0, -1.0], [-1.5, 1.0, -0.5]], dtype=np.float64)
_LIGHTS /= np.linalg.norm(_LIGHTS, axis=1, keepdims=True)


class Frame(dict):
    """Planar float32 buffers: radiance[3,H,W], albedo[3,H,W], normal[3,H,W],
    depth[1,H,W] and the noise-free shading clean[3,H,W]."""

    @property
    def shape(self):
        return self["radiance"].shape[1:]


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed), int(stream)]))


def _geometry(H: int, W: int, seed: int, origin=(0.0, 1.0, 0.0), with_position: bool = False):
    g = _rng(seed, 1)
    n_sph = 6
    cx = g.uniform(-3.0, 3.0, n_sph)
    cz = g.uniform(3.0, 9.0, n_sph)
    rad = g.uniform(0.4, 1.2, n_sph)
    centres = np.stack([cx, rad, cz], axis=1)

    fov = np.deg2rad(60.0)
    th = np.tan(fov / 2)
    ys = (1.0 - 2.0 * (np.arange(H) + 0.5) / H) * th
    xs = (2.0 * (np.arange(W) + 0.5) / W - 1.0) * th * (W / H)
    dx, dy = np.meshgrid(xs, ys)                      # [H, W]
    d = np.stack([dx, dy, np.ones_like(dx)], axis=0)  # [3, H, W]
    d /= np.linalg.norm(d, axis=0, keepdims=True)
    o = np.asarray(origin, dtype=np.float64)

    t_best = np.full((H, W), np.inf)
    nrm = np.zeros((3, H, W))
    # back plane z = 12, normal (0, 0, -1)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(d[2] > 1e-9, (12.0 - o[2]) / d[2], np.inf)
    hit = t < t_best
    t_best = np.where(hit, t, t_best)
    nrm[:, hit] = np.array([0.0, 0.0, -1.0])[:, None]
    # ground y = 0, normal (0, 1, 0)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(d[1] < -1e-9, (0.0 - o[1]) / d[1], np.inf)
    hit = (t > 1e-6) & (t < t_best)
    t_best = np.where(hit, t, t_best)
    nrm[:, hit] = np.array([0.0, 1.0, 0.0])[:, None]
    # spheres
    for c, r in zip(centres, rad):
        oc = (o - c)[:, None, None]
        b = np.sum(d * oc, axis=0)
        cc = float(np.sum((o - c) ** 2) - r * r)
        disc = b * b - cc
        sq = np.sqrt(np.maximum(disc, 0.0))
        t = np.where(disc > 0, -b - sq, np.inf)
        hit = (t > 1e-6) & (t < t_best)
        t_best = np.where(hit, t, t_best)
        p = o[:, None, None] + d * t_best[None]
        n = (p - c[:, None, None]) / r
        nrm = np.where(hit[None], n, nrm)
    zcam = np.where(np.isfinite(t_best), t_best * d[2], DEPTH_FAR)
    depth = np.clip(zcam, DEPTH_NEAR, DEPTH_FAR)[None]
    nrm /= np.maximum(np.linalg.norm(nrm, axis=0, keepdims=True), 1e-12)
    if with_position:
        pos = o[:, None, None] + d * np.where(np.isfinite(t_best), t_best, 0.0)[None]
        return nrm, depth, pos
    return nrm, depth


def _albedo(H: int, W: int, seed: int) -> np.ndarray:
    g = _rng(seed, 2)
    gy, gx = np.meshgrid(np.arange(8), np.arange(8), indexing="ij")
    sy = ((gy + g.uniform(0, 1, (8, 8))) / 8.0 * H).ravel()
    sx = ((gx + g.uniform(0, 1, (8, 8))) / 8.0 * W).ravel()
    colours = g.uniform(0.0, 1.0, (64, 3))
    yy = np.arange(H, dtype=np.float64)[:, None] + 0.5
    xx = np.arange(W, dtype=np.float64)[None, :] + 0.5
    best = np.full((H, W), np.inf)
    idx = np.zeros((H, W), dtype=np.int64)
    for s in range(64):  # strict '<' keeps the lowest index on ties
        dist = (yy - sy[s]) ** 2 + (xx - sx[s]) ** 2
        closer = dist < best
        best = np.where(closer, dist, best)
        idx = np.where(closer, s, idx)
    return np.transpose(colours[idx], (2, 0, 1))  # [3, H, W]


def make_frame(H: int, W: int, seed: int) -> Frame:
    """One synthetic 1-spp frame of size H x W from `seed` (recipe above)."""
    nrm, depth = _geometry(H, W, seed)
    alb = _albedo(H, W, seed)
    shade = 0.1 + sum(np.maximum(np.einsum("chw,c->hw", nrm, l), 0.0) for l in _LIGHTS)
    clean = alb * shade[None]
    g = _rng(seed, 3)
    noise = np.exp(g.standard_normal((3, H, W)))
    fire = g.uniform(0.0, 1.0, (H, W)) < 0.02
    rad = clean * noise * np.where(fire, 50.0, 1.0)[None]
    f = Frame(
        radiance=rad.astype(np.float32),
        albedo=alb.astype(np.float32),
        normal=nrm.astype(np.float32),
        depth=depth.astype(np.float32),
        clean=clean.astype(np.float32),
    )
    return f


def make_batch(B: int, H: int, W: int, seed: int) -> dict:
    """B frames stacked along a leading batch axis ([B, C, H, W] float32).
    Frame b uses seed `seed * 1000 + b`."""
    frames = [make_frame(H, W, seed * 1000 + b) for b in range(B)]
    return {k: np.stack([f[k] for f in frames]) for k in frames[0]}


def make_target(clean: np.ndarray, seed: int, draws: int = 256) -> np.ndarray:
    """Training target: the mean of `draws` independent noisy renderings of
    `clean` ([..., 3, H, W]) with the same noise model as make_frame."""
    g = _rng(seed, 4)
    acc = np.zeros(clean.shape, dtype=np.float64)
    spatial = clean.shape[:-3] + clean.shape[-2:]
    for _ in range(draws):
        noise = np.exp(g.standard_normal(clean.shape))
        fire = g.uniform(0.0, 1.0, spatial) < 0.02
        acc += clean * noise * np.expand_dims(np.where(fire, 50.0, 1.0), -3)
    return (acc / draws).astype(np.float32)


def weight_shapes(widths=(10, 32, 48, 64, 12), ks: int = 5):
    """[(W_shape, b_shape)] per conv layer; W is [Cout, Cin, ks, ks]."""
    return [((widths[i + 1], widths[i], ks, ks), (widths[i + 1],))
            for i in range(len(widths) - 1)]


def n_weights(widths=(10, 32, 48, 64, 12), ks: int = 5) -> int:
    return sum(int(np.prod(w)) + int(np.prod(b)) for w, b in weight_shapes(widths, ks))


def make_weights_for(shapes, seed: int = 0) -> np.ndarray:
    """Random-init weights for an arbitrary list of conv layers given as
    [((Cout, Cin, k, k), (Cout,)), ...], one flat float32 blob in that order,
    with the same He-normal / uniform recipe as make_weights."""
    g = _rng(seed, 8)
    parts = []
    for ws, bs in shapes:
        fan_in = ws[1] * ws[2] * ws[3]
        parts.append(g.standard_normal(ws).ravel() * np.sqrt(2.0 / fan_in))
        parts.append(g.uniform(-1.0, 1.0, bs) / np.sqrt(fan_in))
    return np.concatenate(parts).astype(np.float32)


def make_weights(widths=(10, 32, 48, 64, 12), ks: int = 5, seed: int = 0) -> np.ndarray:
    """Random-init weights as one flat float32 blob: for each layer in order,
    W[Cout, Cin, ks, ks] then b[Cout].  W ~ He-normal N(0, 2 / (Cin ks^2)),
    b ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in))."""
    g = _rng(seed, 5)
    parts = []
    for (ws, bs) in weight_shapes(widths, ks):
        fan_in = ws[1] * ks * ks
        parts.append(g.standard_normal(ws).ravel() * np.sqrt(2.0 / fan_in))
        parts.append(g.uniform(-1.0, 1.0, bs) / np.sqrt(fan_in))
    return np.concatenate(parts).astype(np.float32)


def _project(pos: np.ndarray, origin, H: int, W: int) -> np.ndarray:
    """Continuous pixel coordinates (x, y) of world points [3, H, W] in the
    camera at `origin` (same orientation and field of view as make_frame;
    pixel centres at integer coordinates)."""
    th = np.tan(np.deg2rad(60.0) / 2)
    d = pos - np.asarray(origin, dtype=np.float64)[:, None, None]
    z = np.maximum(d[2], 1e-9)
    xn = d[0] / (z * th * (W / H))
    yn = d[1] / (z * th)
    return np.stack([(xn + 1.0) * 0.5 * W - 0.5, (1.0 - yn) * 0.5 * H - 0.5])


def make_sequence(H: int, W: int, T: int, seed: int, velocity=(0.04, 0.0, 0.03)) -> list:
    """T consecutive 1-spp frames of one static scene seen from a camera that
    moves by `velocity` (world units) per frame.  Besides the make_frame
    buffers every frame has the world position of the first hit
    position[3,H,W] and the motion vector motion[2,H,W] = (x, y) offset from
    the pixel to where the same surface point projects in the previous
    frame's camera (0 for the first frame).  Albedo is attached to the
    surfaces (uniform [0,1]^3 per cell of a 0.5-unit world grid, hashed into
    a seeded table), so the noise-free radiance of a point is the same in
    every frame; radiance noise is drawn per frame as in make_frame."""
    table = _rng(seed, 6).uniform(0.0, 1.0, (4096, 3))
    frames = []
    for t in range(T):
        origin = (velocity[0] * t, 1.0 + velocity[1] * t, velocity[2] * t)
        nrm, depth, pos = _geometry(H, W, seed, origin, with_position=True)
        cell = np.floor(pos / 0.5).astype(np.int64)
        h = (cell[0] * 73856093) ^ (cell[1] * 19349663) ^ (cell[2] * 83492791)
        alb = np.transpose(table[np.mod(h, 4096)], (2, 0, 1))
        shade = 0.1 + sum(np.maximum(np.einsum("chw,c->hw", nrm, l), 0.0) for l in _LIGHTS)
        clean = alb * shade[None]
        g = _rng(seed * 1000 + t, 7)
        noise = np.exp(g.standard_normal((3, H, W)))
        fire = g.uniform(0.0, 1.0, (H, W)) < 0.02
        rad = clean * noise * np.where(fire, 50.0, 1.0)[None]
        if t == 0:
            motion = np.zeros((2, H, W))
        else:
            prev = (velocity[0] * (t - 1), 1.0 + velocity[1] * (t - 1), velocity[2] * (t - 1))
            q = _project(pos, prev, H, W)
            px = np.arange(W, dtype=np.float64)[None, :]
            py = np.arange(H, dtype=np.float64)[:, None]
            motion = np.stack([q[0] - px, q[1] - py])
        frames.append(Frame(
            radiance=rad.astype(np.float32), albedo=alb.astype(np.float32), normal=nrm.astype(np.float32),
            depth=depth.astype(np.float32), clean=clean.astype(np.float32), position=pos.astype(np.float32),
            motion=motion.astype(np.float32)))
    return frames
