"""Temporal accumulation (Sec. 4.3) on the GPU against the oracle."""
import numpy as np
import pytest

import oracle
from oracle import temporal as ot
import synth
from _util import rel_err

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _run(seq, **cfg):
    from paper_2202_05977_b300.temporal import TemporalAccumulator
    H, W = seq[0]["radiance"].shape[1:]
    ta = TemporalAccumulator(H, W, **cfg)
    st = ot.TemporalState(H, W)
    kw = {k: v for k, v in cfg.items() if v is not None}
    res = []
    for f in seq:
        got = ta.step(*(_dev(f[k]) for k in ("radiance", "position", "normal", "motion"))).cpu().numpy()
        hist = ta.history().cpu().numpy()
        ref = ot.accumulate(st, f["radiance"], f["position"], f["normal"], f["motion"], **kw)
        res.append((got, hist, ref, st.h.copy()))
    ta.close()
    return res


@pytest.mark.parametrize("hw,seed", [((72, 100), 4), ((33, 47), 5)])
def test_sequence_matches_oracle(hw, seed):
    seq = synth.make_sequence(*hw, 6, seed=seed)
    for t, (got, hist, ref, href) in enumerate(_run(seq)):
        # the same pixels restart (decisions are taken in float32 by both sides)
        np.testing.assert_array_equal(hist == 1.0, href == 1.0)
        assert np.max(np.abs(hist - href) / href) < 1e-5
        e_max, e_mean = rel_err(got, ref)
        assert e_max < 1e-5, (t, e_max)


def test_sequence_1080p_matches_oracle():
    seq = synth.make_sequence(1080, 1920, 3, seed=6, velocity=(0.02, 0.0, 0.01))
    for t, (got, hist, ref, href) in enumerate(_run(seq)):
        np.testing.assert_array_equal(hist == 1.0, href == 1.0)
        e_max, _ = rel_err(got, ref)
        assert e_max < 1e-5, (t, e_max)
        if t > 0:
            assert np.mean(hist > 1.0) > 0.9  # most pixels keep their history


def test_custom_thresholds_match_oracle():
    seq = synth.make_sequence(40, 64, 4, seed=7)
    cfg = dict(alpha_min=0.1, tau_pos=0.05, tau_normal=0.95, min_weight=0.01)
    for got, hist, ref, href in _run(seq, **cfg):
        np.testing.assert_array_equal(hist == 1.0, href == 1.0)
        assert rel_err(got, ref)[0] < 1e-5


def test_reset_restarts_every_pixel():
    import torch
    from paper_2202_05977_b300.temporal import TemporalAccumulator
    seq = synth.make_sequence(24, 32, 3, seed=8)
    ta = TemporalAccumulator(24, 32)
    for f in seq[:2]:
        ta.step(*(_dev(f[k]) for k in ("radiance", "position", "normal", "motion")))
    assert float(ta.history().mean()) > 1.5
    ta.reset()
    f = seq[2]
    out = ta.step(*(_dev(f[k]) for k in ("radiance", "position", "normal", "motion")))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), f["radiance"])
    np.testing.assert_array_equal(ta.history().cpu().numpy(), 1.0)


def test_accumulated_frame_feeds_the_denoiser():
    # the pre-pass composes with the FP32 denoiser exactly as with the oracle chain
    import paper_2202_05977_b300 as wk
    from paper_2202_05977_b300.temporal import TemporalAccumulator
    seq = synth.make_sequence(40, 56, 3, seed=9)
    wb = synth.make_weights(seed=9)
    ta = TemporalAccumulator(40, 56)
    st = ot.TemporalState(40, 56)
    d = wk.Denoiser(wb, precision="fp32", max_hw=(40, 56))
    for f in seq:
        acc = ta.step(*(_dev(f[k]) for k in ("radiance", "position", "normal", "motion")))
        out = d.denoise(acc[None], _dev(f["albedo"][None]), _dev(f["normal"][None]),
                        _dev(f["depth"][None])).cpu().numpy()[0]
        A = ot.accumulate(st, f["radiance"], f["position"], f["normal"], f["motion"])
        fr = dict(f)
        fr["radiance"] = A.astype(np.float32)
        ref = oracle.denoise(fr, wb)
        assert rel_err(out, ref)[0] < 1e-4
