"""Helpers shared by the tests (no method arithmetic)."""
import numpy as np

KSIZES = (3, 5, 7, 9, 11, 13)
KEYS = ("radiance", "albedo", "normal", "depth")


def rel_err(gpu, ref, floor=1e-6):
    """Per-element |gpu - ref| / max(|ref|, floor): (max, mean)."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    e = np.abs(gpu - ref) / np.maximum(np.abs(ref), floor)
    return float(e.max()), float(e.mean())


def to_dev(batch):
    """numpy [B, C, H, W] dict -> dict of float32 CUDA tensors."""
    import torch
    return {k: torch.from_numpy(np.ascontiguousarray(batch[k], dtype=np.float32)).cuda() for k in KEYS}


def stack_frames(frames):
    return {k: np.stack([f[k] for f in frames]) for k in frames[0]}


def args(dev):
    return tuple(dev[k] for k in KEYS)


def sample_pixels(H, W, n, seed):
    """Corners, edge midpoints, tile-boundary pixels and n random pixels (x, y)."""
    g = np.random.default_rng(seed)
    pts = [(0, 0), (W - 1, 0), (0, H - 1), (W - 1, H - 1), (W // 2, 0), (0, H // 2), (W - 1, H // 2),
           (W // 2, H - 1), (63, 15), (64, 16), (127, 8), (128, 9), (W - 7, H - 3)]
    pts += [(int(x), int(y)) for x, y in zip(g.integers(0, W, n), g.integers(0, H, n))]
    return [(min(x, W - 1), min(y, H - 1)) for x, y in pts]
