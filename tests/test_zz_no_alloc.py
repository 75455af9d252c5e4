"""wskpn_denoise_static: the denoiser for callers that may not allocate
device memory (code inside another runtime's memory pool, host callbacks,
plug-ins that must not grow their process's footprint).  Its workspace is a
fixed static device array, so it must give the same images as the regular
context-based FP32 call.  Kept in its own file so that pytest collects it
last; it needs no state from other tests."""
import ctypes

import numpy as np
import pytest

import synth
from tests._util import args, rel_err, stack_frames, to_dev

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5


def _frames_struct(wk, dev):
    fr, B, H, W = wk._frames(*args(dev))
    return fr, B, H, W


def test_static_matches_context_call_twice_in_a_row():
    import torch

    import paper_2202_05977_b300 as wk
    from paper_2202_05977_b300 import _lib

    lib = _lib.load()
    wb = synth.make_weights(seed=4)
    wdev = torch.from_numpy(wb).cuda()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # two calls in a row: different sizes and frames, the second reuses the
    # scratch left by the first
    for (B, H, W, seed) in [(1, 256, 512, 40), (2, 45, 67, 41)]:
        frames = [synth.make_frame(H, W, seed + b) for b in range(B)]
        dev = to_dev(stack_frames(frames))
        cfg = wk.default_config("fp32", max_batch=B, max_hw=(H, W))
        ref = wk.Denoiser(wb, precision="fp32", max_batch=B, max_hw=(H, W)).denoise(*args(dev))
        out = torch.full((B, 3, H, W), float("nan"), device="cuda")
        fr, _, _, _ = _frames_struct(wk, dev)
        s = lib.wskpn_denoise_static(ctypes.byref(cfg), ctypes.c_void_p(wdev.data_ptr()), fr, B, H, W,
                                     ctypes.c_void_p(out.data_ptr()), stream)
        assert s == _lib.OK, lib.wskpn_last_error(None)
        torch.cuda.synchronize()
        mx, _ = rel_err(out.cpu().numpy(), ref.cpu().numpy())
        assert mx < TOL_FP32, (H, W, mx)


def test_static_rejects_oversized_and_non_fp32_requests():
    import torch

    import paper_2202_05977_b300 as wk
    from paper_2202_05977_b300 import _lib

    lib = _lib.load()
    wb = torch.from_numpy(synth.make_weights(seed=4)).cuda()
    dev = to_dev(stack_frames([synth.make_frame(8, 8, 1)]))
    fr, _, _, _ = _frames_struct(wk, dev)
    out = torch.empty((1, 3, 8, 8), device="cuda")
    cfg = wk.default_config("fp32")
    # 1080p needs far more than the static array holds: refused with a message
    s = lib.wskpn_denoise_static(ctypes.byref(cfg), ctypes.c_void_p(wb.data_ptr()), fr, 1, 1080, 1920,
                                 ctypes.c_void_p(out.data_ptr()), None)
    assert s == _lib.EINVAL and b"static scratch" in lib.wskpn_last_error(None)
    cfg = wk.default_config("bf16")
    s = lib.wskpn_denoise_static(ctypes.byref(cfg), ctypes.c_void_p(wb.data_ptr()), fr, 1, 8, 8,
                                 ctypes.c_void_p(out.data_ptr()), None)
    assert s == _lib.EUNSUPPORTED
