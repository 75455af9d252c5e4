"""The paper's quality variant of ImportanceNet: six blocks (Sec. 4.1, the
6-block network of the timing table), widths 10-32-48-64-64-64-64 and the
output conv to 12, in every precision.  The 64->64 layers' BF16 weight image
(205 KB) runs as two output-channel groups on the tensor cores."""
import numpy as np
import pytest

import oracle
import synth
from _util import args, rel_err, sample_pixels, stack_frames, to_dev

pytestmark = pytest.mark.gpu

WIDTHS6 = (10, 32, 48, 64, 64, 64, 64, 12)


@pytest.fixture(scope="module")
def wk():
    import paper_2202_05977_b300 as wk
    return wk


@pytest.mark.parametrize("H,W", [(64, 64), (37, 141)])
def test_six_blocks_fp32_matches_oracle(wk, H, W):
    f = synth.make_frame(H, W, 70)
    wb = synth.make_weights(WIDTHS6, seed=70)
    out = wk.Denoiser(wb, "fp32", widths=WIDTHS6, max_hw=(H, W)).denoise(*args(to_dev(stack_frames([f]))))
    mx, mean = rel_err(out.cpu().numpy()[0], oracle.denoise(f, wb, widths=WIDTHS6))
    print(f"6-block fp32 {H}x{W}: max rel {mx:.3e} mean {mean:.3e}")
    assert mx < 1e-5


@pytest.mark.parametrize("B,H,W", [(1, 64, 64), (2, 45, 200)])
def test_six_blocks_bf16_matches_oracle(wk, B, H, W):
    frames = [synth.make_frame(H, W, 71 + b) for b in range(B)]
    wb = synth.make_weights(WIDTHS6, seed=71)
    d = wk.Denoiser(wb, "bf16", widths=WIDTHS6, max_hw=(H, W), max_batch=B)
    out = d.denoise(*args(to_dev(stack_frames(frames)))).cpu().numpy()
    assert d.device_status() == 0
    for b in range(B):
        mx, mean = rel_err(out[b], oracle.denoise(frames[b], wb, widths=WIDTHS6))
        print(f"6-block bf16 {H}x{W}[{b}]: max rel {mx:.3e} mean {mean:.3e}")
        assert mx < 1e-2


def test_six_blocks_bf16_logits_match_fp32(wk):
    # the grouped 64->64 layers against the FP32 path on a tile-spanning frame
    f = synth.make_frame(200, 300, 72)
    wb = synth.make_weights(WIDTHS6, seed=72)
    dev = to_dev(stack_frames([f]))
    zb = wk.Denoiser(wb, "bf16", widths=WIDTHS6, max_hw=(200, 300)).logits(*args(dev)).cpu().numpy()
    zf = wk.Denoiser(wb, "fp32", widths=WIDTHS6, max_hw=(200, 300)).logits(*args(dev)).cpu().numpy()
    assert np.abs(zb - zf).max() < 1e-2 * max(1.0, np.abs(zf).max())


def test_six_blocks_1080p_bf16_sampled(wk):
    H, W = 1080, 1920
    f = synth.make_frame(H, W, 2)
    wb = synth.make_weights(WIDTHS6, seed=2)
    dev = to_dev(stack_frames([f]))
    out = wk.Denoiser(wb, "bf16", widths=WIDTHS6, max_hw=(H, W)).denoise(*args(dev)).cpu().numpy()[0]
    pix = sample_pixels(H, W, 24, seed=3)
    ref = oracle.denoise_pixels(f, wb, pix, widths=WIDTHS6)
    mx, mean = rel_err(np.stack([out[:, y, x] for x, y in pix]), ref)
    print(f"6-block bf16 1080p sampled: max rel {mx:.3e} mean {mean:.3e}")
    assert mx < 1e-2


def test_six_blocks_fp8_matches_oracle(wk):
    """FP8 form of the 6-block network: e4m3 hi/lo operands, every pixel
    held to the 3e-2 per-pixel bar of the FP8 form."""
    f = synth.make_frame(64, 96, 73)
    wb = synth.make_weights(WIDTHS6, seed=73)
    dev = to_dev(stack_frames([f]))
    d = wk.Denoiser(wb, "fp8", widths=WIDTHS6, max_hw=(64, 96))
    d.calibrate(*args(to_dev(stack_frames([synth.make_frame(64, 96, 74)]))))
    out = d.denoise(*args(dev)).cpu().numpy()[0]
    assert np.all(np.isfinite(out)) and d.device_status() == 0
    mx, mean = rel_err(out, oracle.denoise(f, wb, widths=WIDTHS6))
    print(f"6-block fp8 64x96: max rel {mx:.3e} mean {mean:.3e}")
    assert mx < 3e-2
