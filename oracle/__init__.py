"""FP64 CPU oracle for the weight-sharing kernel-prediction denoiser
(Fan, Wang, Huo, Bao, EGSR 2021).

TEST INFRASTRUCTURE ONLY.  The loops live in plain C (``wskpn_oracle.c``,
double precision, OpenMP over rows); this module compiles it with gcc on
first use and wraps it with ctypes and numpy.  Only ``tests/``, the smoke
check and the benchmark's CPU-baseline leg may import it.  It shares no code
with the CUDA library, and the library never imports it.

What it computes (paper sections / equations):
  * ``prep``            Sec. 5.1 input assembly (10 channels).
  * ``conv2d``          Sec. 4.1 inference block: one KSxKS conv (+ReLU).
  * ``decode_explicit`` Eq. 3-4 with an explicit per-pixel k x k kernel.
  * ``decode_boxsum``   Eq. 3-4 coded independently as a ratio of window sums.
  * ``fuse``            Eq. 5 with softmax fusion weights and albedo
                        re-modulation (Sec. 4.2).
  * ``denoise``         the whole D_Theta(r, f) on a frame, a band of rows or
                        a list of single pixels (same code path).
  * ``reconstruct_bwd`` / ``conv2d_bwd`` / ``train_grads``: the chain rule of
                        the above for one training step (Eq. 1), with the L1
                        loss or SMAPE (Eq. 6).
  * ``round_bf16`` / ``bf16_weights``: the weight rounding of the BF16
                        convolutions (round to nearest even), so that the
                        BF16 training form can be compared with the exact
                        gradient of the network it actually computes.
  * ``temporal.accumulate`` Sec. 4.3 temporal accumulation before denoising
                        (reprojection, geometry consistency, blend); numpy.
  * ``multires``        the multi-resolution variant: U-Net logits at 3
                        levels, per-level Eq. 3-5 with kernels 3 and 5, and
                        the Eq. 7 combination; numpy over the C routines.

Parity status of each function is stated in the tests that pin it; the whole
denoiser's agreement with the paper's *trained* network is unpinned (no
weights or datasets exist for it).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wskpn_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

DEFAULT_WIDTHS = (10, 32, 48, 64, 12)
DEFAULT_KSIZES = (3, 5, 7, 9, 11, 13)
DEFAULT_EPS = 1e-2
DEFAULT_GAMMA = 2.2
DEPTH_NEAR, DEPTH_FAR = 1.0, 10.0


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/_build/liboracle.so (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            D = ctypes.POINTER(ctypes.c_double)
            I = ctypes.POINTER(ctypes.c_int)
            L, Ci, Cd = ctypes.c_long, ctypes.c_int, ctypes.c_double
            sigs = {
                "wo_num_threads": ([], Ci),
                "wo_prep": ([D, D, D, D, L, L, Cd, Cd, Cd, D], None),
                "wo_conv2d": ([D, Ci, L, L, D, D, Ci, Ci, Ci, D], None),
                "wo_kernel_weights": ([D, L, L, Ci, L, L, D], None),
                "wo_decode_explicit": ([D, D, L, L, Ci, D], None),
                "wo_decode_boxsum": ([D, D, L, L, Ci, D], None),
                "wo_fuse": ([D, D, D, Ci, L, L, Cd, D], None),
                "wo_logits_region": ([D, D, D, D, L, L, Ci, I, Ci, D, Cd, Cd, Cd, L, L, L, L, D], None),
                "wo_denoise_region": ([D, D, D, D, L, L, Ci, I, Ci, D, Ci, I, Cd, Cd, Cd, Cd,
                                       L, L, L, L, D], None),
                "wo_reconstruct": ([D, D, D, L, L, Ci, I, Cd, D], None),
                "wo_reconstruct_bwd": ([D, D, D, L, L, Ci, I, Cd, D, D], None),
                "wo_conv2d_bwd": ([D, Ci, L, L, D, Ci, Ci, D, D, D, D], None),
            }
            for name, (args, res) in sigs.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().wo_num_threads())


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


# ---------------------------------------------------------------- layer ops
def prep(rad, alb, nrm, dep, gamma=DEFAULT_GAMMA, dnear=DEPTH_NEAR, dfar=DEPTH_FAR):
    """Sec. 5.1: [10, H, W] network input from planar frame buffers."""
    rad, alb, nrm, dep = map(_d, (rad, alb, nrm, dep))
    H, W = rad.shape[-2:]
    out = np.empty((10, H, W))
    _load().wo_prep(_p(rad), _p(alb), _p(nrm), _p(dep), H, W, gamma, dnear, dfar, _p(out))
    return out


def conv2d(x, w, b, relu: bool):
    """Sec. 4.1: one KSxKS conv, zero padding KS//2, optional ReLU.
    x [Cin, H, W], w [Cout, Cin, KS, KS], b [Cout]."""
    x, w, b = _d(x), _d(w), _d(b)
    Cin, H, W = x.shape
    Cout, _, KS, _ = w.shape
    y = np.empty((Cout, H, W))
    _load().wo_conv2d(_p(x), Cin, H, W, _p(w), _p(b), Cout, KS, int(relu), _p(y))
    return y


def kernel_weights(z, k: int, px: int, py: int):
    """The k x k filtering kernel w_p of pixel (px, py) built from importance
    map z [H, W] (Eq. 3); entries outside the image are 0."""
    z = _d(z)
    H, W = z.shape
    w = np.empty((k, k))
    _load().wo_kernel_weights(_p(z), H, W, k, px, py, _p(w))
    return w


def decode_explicit(z, y, k: int):
    """Eq. 3-4: filtered [3, H, W] from importance map z [H, W] and signal y [3, H, W]."""
    z, y = _d(z), _d(y)
    H, W = z.shape
    R = np.empty((3, H, W))
    _load().wo_decode_explicit(_p(z), _p(y), H, W, k, _p(R))
    return R


def decode_boxsum(z, y, k: int):
    """Eq. 3-4 as a ratio of window sums (independent second coding)."""
    z, y = _d(z), _d(y)
    H, W = z.shape
    R = np.empty((3, H, W))
    _load().wo_decode_boxsum(_p(z), _p(y), H, W, k, _p(R))
    return R


def fuse(Rs, alpha_logits, alb, eps=DEFAULT_EPS):
    """Eq. 5 + re-modulation: Rs [M, 3, H, W], alpha_logits [M, H, W], alb [3, H, W]."""
    Rs, al, alb = _d(Rs), _d(alpha_logits), _d(alb)
    M, _, H, W = Rs.shape
    out = np.empty((3, H, W))
    _load().wo_fuse(_p(Rs), _p(al), _p(alb), M, H, W, eps, _p(out))
    return out


def reconstruct(z, rad, alb, ksizes=DEFAULT_KSIZES, eps=DEFAULT_EPS):
    """Decode + fuse + re-modulate a frame from network outputs z [2M, H, W]."""
    z, rad, alb = _d(z), _d(rad), _d(alb)
    ks = np.ascontiguousarray(ksizes, dtype=np.int32)
    M = len(ks)
    assert z.shape[0] == 2 * M
    H, W = rad.shape[-2:]
    out = np.empty((3, H, W))
    _load().wo_reconstruct(_p(z), _p(rad), _p(alb), H, W, M, _ip(ks), eps, _p(out))
    return out


def reconstruct_bwd(z, rad, alb, G, ksizes=DEFAULT_KSIZES, eps=DEFAULT_EPS):
    """dL/dz [2M, H, W] given dL/dout G [3, H, W] (chain rule of Eq. 3-5)."""
    z, rad, alb, G = _d(z), _d(rad), _d(alb), _d(G)
    ks = np.ascontiguousarray(ksizes, dtype=np.int32)
    M = len(ks)
    H, W = rad.shape[-2:]
    dz = np.empty((2 * M, H, W))
    _load().wo_reconstruct_bwd(_p(z), _p(rad), _p(alb), H, W, M, _ip(ks), eps, _p(G), _p(dz))
    return dz


def conv2d_bwd(x, w, gy, need_gx: bool = True):
    """Backward of one conv given the pre-activation gradient gy [Cout, H, W].
    Returns (gx or None, gw, gb)."""
    x, w, gy = _d(x), _d(w), _d(gy)
    Cin, H, W = x.shape
    Cout, _, KS, _ = w.shape
    gw = np.empty(w.shape)
    gb = np.empty((Cout,))
    gx = np.empty((Cin, H, W)) if need_gx else None
    _load().wo_conv2d_bwd(_p(x), Cin, H, W, _p(w), Cout, KS, _p(gy),
                          _p(gx) if need_gx else None, _p(gw), _p(gb))
    return gx, gw, gb


# ------------------------------------------------------------ weight blob
def split_weights(blob, widths=DEFAULT_WIDTHS, ks: int = 5):
    """Flat blob -> [(W [Cout, Cin, ks, ks], b [Cout])] per layer."""
    blob = _d(blob)
    out, off = [], 0
    for l in range(len(widths) - 1):
        cin, cout = widths[l], widths[l + 1]
        nw = cout * cin * ks * ks
        out.append((blob[off:off + nw].reshape(cout, cin, ks, ks), blob[off + nw:off + nw + cout]))
        off += nw + cout
    assert off == blob.size, (off, blob.size)
    return out


def round_bf16(x):
    """Round float32 values to bfloat16 (8-bit significand), round to nearest
    with ties to even, returned as float64: the BF16 tensor-core form keeps
    its convolution weights this way (reading A12).  Written from the
    definition: keep the top 16 bits of the IEEE binary32 pattern and add
    one unit in the kept last place when the dropped 16 bits exceed half a
    unit, or equal half a unit and the kept last bit is odd.  Finite inputs
    only (the weights are finite)."""
    bits = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    kept, dropped = bits >> 16, bits & 0xFFFF
    up = (dropped > 0x8000) | ((dropped == 0x8000) & ((kept & 1) == 1))
    kept = kept + up.astype(np.uint64)
    return (kept << 16).astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_weights(blob, widths=DEFAULT_WIDTHS, ks: int = 5):
    """The flat weight blob as the BF16 convolutions use it: every
    convolution weight rounded by ``round_bf16``, the biases unchanged
    (they are added in FP32 in the convolution epilogue)."""
    out = _d(blob).copy()
    off = 0
    for l in range(len(widths) - 1):
        nw = widths[l + 1] * widths[l] * ks * ks
        out[off:off + nw] = round_bf16(np.asarray(blob, np.float32)[off:off + nw])
        off += nw + widths[l + 1]
    return out


# ---------------------------------------------------------- whole denoiser
def logits(frame, weights, widths=DEFAULT_WIDTHS, ks: int = 5, rect=None,
           gamma=DEFAULT_GAMMA, dnear=DEPTH_NEAR, dfar=DEPTH_FAR):
    """ImportanceNet output (Eq. 2 maps then fusion logits) on rect
    (x0, y0, x1, y1) of one frame (dict of planar [C, H, W] arrays)."""
    rad, alb, nrm, dep = (_d(frame[k]) for k in ("radiance", "albedo", "normal", "depth"))
    H, W = rad.shape[-2:]
    x0, y0, x1, y1 = rect if rect is not None else (0, 0, W, H)
    wv = np.ascontiguousarray(widths, dtype=np.int32)
    wb = _d(weights)
    z = np.empty((widths[-1], y1 - y0, x1 - x0))
    _load().wo_logits_region(_p(rad), _p(alb), _p(nrm), _p(dep), H, W, len(widths) - 1, _ip(wv),
                             ks, _p(wb), gamma, dnear, dfar, x0, y0, x1, y1, _p(z))
    return z


def denoise(frame, weights, widths=DEFAULT_WIDTHS, ks: int = 5, ksizes=DEFAULT_KSIZES,
            eps=DEFAULT_EPS, rect=None, gamma=DEFAULT_GAMMA, dnear=DEPTH_NEAR, dfar=DEPTH_FAR):
    """D_Theta(r, f) on rect (x0, y0, x1, y1) (default: the full frame).
    Returns [3, y1-y0, x1-x0] float64."""
    rad, alb, nrm, dep = (_d(frame[k]) for k in ("radiance", "albedo", "normal", "depth"))
    H, W = rad.shape[-2:]
    x0, y0, x1, y1 = rect if rect is not None else (0, 0, W, H)
    wv = np.ascontiguousarray(widths, dtype=np.int32)
    kv = np.ascontiguousarray(ksizes, dtype=np.int32)
    assert widths[-1] == 2 * len(ksizes)
    wb = _d(weights)
    out = np.empty((3, y1 - y0, x1 - x0))
    _load().wo_denoise_region(_p(rad), _p(alb), _p(nrm), _p(dep), H, W, len(widths) - 1,
                              _ip(wv), ks, _p(wb), len(ksizes), _ip(kv), eps, gamma, dnear,
                              dfar, x0, y0, x1, y1, _p(out))
    return out


def denoise_pixels(frame, weights, pixels, **kw):
    """Output [3] at each (x, y) in `pixels`, one pixel at a time."""
    return np.stack([denoise(frame, weights, rect=(x, y, x + 1, y + 1), **kw)[:, 0, 0]
                     for (x, y) in pixels])


# ------------------------------------------------------------------ losses
def l1_loss(out, target):
    """Mean absolute error over all elements, and its gradient
    (sign(out - t) / N; sign(0) = 0)."""
    out, target = _d(out), _d(target)
    n = out.size
    return float(np.abs(out - target).sum() / n), np.sign(out - target) / n


def smape_loss(out, target, eps: float = 0.01):
    """Eq. 6: (1 / 3N) sum_p sum_c |R - t| / (|R| + |t| + eps), and its gradient
    with respect to R (3N = number of elements)."""
    R, t = _d(out), _d(target)
    n = R.size
    den = np.abs(R) + np.abs(t) + eps
    num = np.abs(R - t)
    g = (np.sign(R - t) * den - num * np.sign(R)) / (den * den) / n
    return float((num / den).sum() / n), g


# ---------------------------------------------------------------- RepVGG
def repvgg_fold(w5, b5, w3, b3, w1, b1, identity: bool):
    """Sec. 4.1: a training-time block sums a 5x5, a 3x3 and a 1x1 conv
    branch (all zero-padded to 'same' size) and, when Cin == Cout, the input
    itself; being linear, it equals one 5x5 conv whose kernel is the sum of
    the branch kernels zero-padded to 5x5 (plus a centre 1 on the diagonal
    for the identity) and whose bias is the sum of the biases.
    w5 [Co,Ci,5,5], w3 [Co,Ci,3,3], w1 [Co,Ci,1,1].  Returns (W [Co,Ci,5,5], b [Co])."""
    w5, w3, w1 = _d(w5), _d(w3), _d(w1)
    co, ci = w5.shape[:2]
    W = w5.copy()
    W[:, :, 1:4, 1:4] += w3
    W[:, :, 2, 2] += w1[:, :, 0, 0]
    if identity:
        assert co == ci
        for c in range(co):
            W[c, c, 2, 2] += 1.0
    return W, _d(b5) + _d(b3) + _d(b1)


def repvgg_fold_grad(gW):
    """Gradient of the fold: (dL/dw5, dL/dw3, dL/dw1) from dL/dW [Co,Ci,5,5];
    each bias receives dL/db unchanged."""
    gW = _d(gW)
    return gW.copy(), gW[:, :, 1:4, 1:4].copy(), gW[:, :, 2:3, 2:3].copy()


# ------------------------------------------------------------------ Adam
def adam_step(w, g, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, Algorithm 1; the optimiser named in
    Sec. 5.3): biased moments, bias correction by 1 - beta^step, update
    w - lr * mhat / (sqrt(vhat) + eps).  Returns (w, m, v)."""
    w, g, m, v = _d(w), _d(g), _d(m), _d(v)
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v


# ------------------------------------------------------- one training step
def forward_train(frame, weights, widths=DEFAULT_WIDTHS, ks: int = 5, ksizes=DEFAULT_KSIZES,
                  eps=DEFAULT_EPS, gamma=DEFAULT_GAMMA, dnear=DEPTH_NEAR, dfar=DEPTH_FAR):
    """Forward pass of one frame keeping every activation: returns
    (out [3,H,W], acts [x0, x1, ..., z])."""
    x = prep(frame["radiance"], frame["albedo"], frame["normal"], frame["depth"], gamma, dnear, dfar)
    acts = [x]
    layers = split_weights(weights, widths, ks)
    for l, (w, b) in enumerate(layers):
        x = conv2d(x, w, b, relu=l < len(layers) - 1)
        acts.append(x)
    out = reconstruct(x, frame["radiance"], frame["albedo"], ksizes, eps)
    return out, acts


def backward_train(frame, weights, acts, G, widths=DEFAULT_WIDTHS, ks: int = 5,
                   ksizes=DEFAULT_KSIZES, eps=DEFAULT_EPS):
    """Gradient of the loss w.r.t. the flat weight blob given G = dL/dout,
    plus dL/dz.  ReLU derivative is taken as 0 at 0."""
    layers = split_weights(weights, widths, ks)
    dz = reconstruct_bwd(acts[-1], frame["radiance"], frame["albedo"], G, ksizes, eps)
    grads = [None] * len(layers)
    gy = dz
    for l in range(len(layers) - 1, -1, -1):
        w, _ = layers[l]
        gx, gw, gb = conv2d_bwd(acts[l], w, gy, need_gx=l > 0)
        grads[l] = (gw, gb)
        if l > 0:
            gy = gx * (acts[l] > 0)
    flat = np.concatenate([np.concatenate([gw.ravel(), gb.ravel()]) for gw, gb in grads])
    return flat, dz


def train_grads(frames, targets, weights, loss: str = "l1", **kw):
    """Loss and d loss / d weights for a batch (list of frames, targets
    [B, 3, H, W]); the loss is over all B*3*H*W elements (Eq. 1 for one
    mini-batch)."""
    outs, actss = [], []
    for f in frames:
        o, a = forward_train(f, weights, **kw)
        outs.append(o)
        actss.append(a)
    out = np.stack(outs)
    lossfn = l1_loss if loss == "l1" else smape_loss
    L, G = lossfn(out, targets)
    g = np.zeros(np.asarray(weights).size)
    for b, f in enumerate(frames):
        gb, _ = backward_train(f, weights, actss[b], G[b], **kw)
        g += gb
    return L, g, out
