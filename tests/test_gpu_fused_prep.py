"""GPU: the first BF16 / FP8 convolution assembling its own input tiles (Sec. 5.1
tone map and scalings inside the kernel's producer, WSKPN_TUNE_FUSED_PREP =
1, the default) against the separate assembly kernel followed by the
convolution reading the stored input (= 0).  Both run the same per-pixel
assembly functions and feed the MMAs the same BF16 hi/lo operands, so the
network outputs must be bit-identical; oracle parity of the default path is
covered by the BF16 parity tests, which run it."""
import numpy as np
import pytest

import oracle
import synth
from tests._util import args, rel_err, stack_frames, to_dev

pytestmark = pytest.mark.gpu

FUSED_PREP = 12  # wskpn_set_tuning key WSKPN_TUNE_FUSED_PREP


@pytest.fixture(scope="module")
def wk():
    import paper_2202_05977_b300 as wk
    return wk


def _logits_both(wk, wb, frames, precision="bf16", **kw):
    H, W = frames[0]["radiance"].shape[-2:]
    dev = to_dev(stack_frames(frames))
    outs = []
    for fused in (1, 0):
        d = wk.Denoiser(wb, precision=precision, max_hw=(H, W), max_batch=len(frames), **kw)
        if precision == "fp8":  # static activation scales from another frame
            cal = to_dev(stack_frames([synth.make_frame(H, W, 999)]))
            d.calibrate(*args(cal))
        d.set_tuning(FUSED_PREP, fused)
        outs.append(d.logits(*args(dev)).cpu().numpy())
        assert d.device_status() == 0
        d.close()
    return outs


@pytest.mark.parametrize("B,H,W", [(1, 64, 64), (2, 45, 67), (1, 1, 1), (1, 14, 200), (1, 130, 257),
                                   (3, 19, 33), (1, 9, 131)])
def test_fused_prep_bit_identical(wk, B, H, W):
    frames = [synth.make_frame(H, W, 70 + b) for b in range(B)]
    wb = synth.make_weights(seed=7)
    fused, plain = _logits_both(wk, wb, frames)
    assert np.array_equal(fused, plain)


@pytest.mark.parametrize("B,H,W", [(1, 64, 64), (2, 45, 67), (1, 14, 200), (1, 130, 257)])
def test_fused_prep_fp8_bit_identical(wk, B, H, W):
    # e4m3 hi/lo input assembled inside the first layer ([hi | hi | lo | 0])
    frames = [synth.make_frame(H, W, 80 + b) for b in range(B)]
    wb = synth.make_weights(seed=11)
    fused, plain = _logits_both(wk, wb, frames, precision="fp8")
    assert np.array_equal(fused, plain)


def test_fused_prep_batch_over_launch_table(wk):
    # 17 frames: the input-assembling kernel takes at most 16 frame
    # pointers per launch, so the batch runs as two launches
    frames = [synth.make_frame(16, 24, 100 + b) for b in range(17)]
    wb = synth.make_weights(seed=8)
    fused, plain = _logits_both(wk, wb, frames)
    assert np.array_equal(fused, plain)


def test_fused_prep_3x3_network(wk):
    frames = [synth.make_frame(40, 140, 9)]
    wb = synth.make_weights(ks=3, seed=9)
    fused, plain = _logits_both(wk, wb, frames, conv_ks=3)
    assert np.array_equal(fused, plain)


def test_fused_prep_1080p_bit_identical_and_oracle_pixels(wk):
    f = synth.make_frame(1080, 1920, 2)
    wb = synth.make_weights(seed=2)
    fused, plain = _logits_both(wk, wb, [f])
    assert np.array_equal(fused, plain)
    # a few logit pixels against the oracle's (the BF16 logits bar: 1e-2 of
    # the largest logit magnitude, at least 1)
    pts = [(0, 0), (1919, 1079), (127, 7), (128, 8), (960, 540)]
    ref = np.stack([oracle.logits(f, wb, rect=(x, y, x + 1, y + 1))[:, 0, 0] for x, y in pts], axis=1)
    got = np.stack([fused[0][:, y, x] for x, y in pts], axis=1)
    assert np.abs(got - ref).max() < 1e-2 * max(1.0, np.abs(ref).max())
