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


def test_static_call_allocates_nothing_and_chunks_large_batches():
    """After a first call (which may load the module and commit the static
    array), further calls leave the device's free memory and torch's
    allocator untouched.  A batch above the per-launch frame limit (16) is
    split into launches over pointers into the shared array; it must still
    equal the context call."""
    import torch

    import paper_2202_05977_b300 as wk
    from paper_2202_05977_b300 import _lib

    lib = _lib.load()
    wb = synth.make_weights(seed=5)
    wdev = torch.from_numpy(wb).cuda()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    B, H, W = 19, 16, 16
    frames = [synth.make_frame(H, W, 60 + b) for b in range(B)]
    dev = to_dev(stack_frames(frames))
    cfg = wk.default_config("fp32", max_batch=B, max_hw=(H, W))
    ref = wk.Denoiser(wb, precision="fp32", max_batch=B, max_hw=(H, W)).denoise(*args(dev))
    out = torch.full((B, 3, H, W), float("nan"), device="cuda")
    fr, _, _, _ = _frames_struct(wk, dev)

    def call():
        s = lib.wskpn_denoise_static(ctypes.byref(cfg), ctypes.c_void_p(wdev.data_ptr()), fr, B, H, W,
                                     ctypes.c_void_p(out.data_ptr()), stream)
        assert s == _lib.OK, lib.wskpn_last_error(None)
        torch.cuda.synchronize()

    call()  # warm-up: module load and first symbol lookup happen here
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    out.fill_(float("nan"))
    call()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert torch.cuda.memory_allocated() == alloc0
    mx, _ = rel_err(out.cpu().numpy(), ref.cpu().numpy())
    assert mx < TOL_FP32, mx


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
