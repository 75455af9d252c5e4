"""Multi-resolution variant (U-Net, 3 levels, Eq. 7) on the GPU against the
FP64 oracle: the U-Net outputs at every level and the denoised frame."""
import numpy as np
import pytest

from oracle import multires as omr
import synth
from _util import args, rel_err, stack_frames, to_dev

pytestmark = pytest.mark.gpu


def _setup(H, W, seed):
    from paper_2202_05977_b300.multires import MultiResDenoiser
    f = synth.make_frame(H, W, seed)
    wb = synth.make_weights_for(omr.weight_shapes(), seed=seed)
    return f, wb, MultiResDenoiser(wb, max_hw=(H, W)), args(to_dev(stack_frames([f])))


@pytest.mark.parametrize("H,W,seed", [(64, 96, 80), (37, 53, 81), (5, 3, 82)])
def test_unet_levels_match_oracle(H, W, seed):
    f, wb, d, a = _setup(H, W, seed)
    zs = [z.cpu().numpy() for z in d.logits(*a)]
    refs = omr.logits(f, wb)
    for l, (z, ref) in enumerate(zip(zs, refs)):
        assert z.shape == ref.shape
        assert np.abs(z - ref).max() < 1e-5 * max(1.0, np.abs(ref).max()), l


def _err(out, f, wb):
    """|gpu - ref| relative to max(|ref|, the magnitude of Eq. 7's terms):
    the combination can cancel to values far below its terms, where any
    float32 evaluation has an error of ~1e-7 of the terms."""
    zs = omr.logits(f, wb)
    ref = omr.reconstruct(zs, f["radiance"], f["albedo"])
    scale = np.maximum(np.abs(ref), omr.term_scale(zs, f["radiance"], f["albedo"]))
    e = np.abs(out - ref) / scale
    return float(e.max()), float(e.mean()), rel_err(out, ref)[1]


@pytest.mark.parametrize("H,W,seed", [(64, 96, 80), (37, 53, 81), (130, 257, 83), (5, 3, 82)])
def test_multires_denoise_matches_oracle(H, W, seed):
    f, wb, d, a = _setup(H, W, seed)
    out = d.denoise(*a).cpu().numpy()[0]
    mx, mean, mean_rel = _err(out, f, wb)
    print(f"multires {H}x{W}: max err / term scale {mx:.3e}, mean {mean:.3e}; mean rel {mean_rel:.3e}")
    assert mx < 1e-5 and mean_rel < 1e-5


def test_multires_constant_irradiance_passes_through():
    import torch
    f, wb, d, _ = _setup(48, 72, 84)
    c = np.array([0.4, 0.9, 1.3], np.float32)[:, None, None]
    f["radiance"] = ((f["albedo"] + np.float32(0.01)) * c).astype(np.float32)
    out = d.denoise(*args(to_dev(stack_frames([f])))).cpu().numpy()[0]
    assert rel_err(out, f["radiance"])[0] < 1e-5


def test_multires_256x384_matches_oracle():
    f, wb, d, a = _setup(256, 384, 85)
    out = d.denoise(*a).cpu().numpy()[0]
    mx, mean, mean_rel = _err(out, f, wb)
    print(f"multires 256x384: max err / term scale {mx:.3e}, mean {mean:.3e}; mean rel {mean_rel:.3e}")
    assert mx < 1e-5 and mean_rel < 1e-5


def _setup_bf16(H, W, seed):
    from paper_2202_05977_b300.multires import MultiResDenoiser
    f = synth.make_frame(H, W, seed)
    wb = synth.make_weights_for(omr.weight_shapes(), seed=seed)
    return f, wb, MultiResDenoiser(wb, max_hw=(H, W), precision="bf16"), args(to_dev(stack_frames([f])))


@pytest.mark.parametrize("H,W,seed", [(64, 96, 90), (37, 53, 91), (5, 3, 92)])
def test_multires_bf16_unet_levels_close_to_oracle(H, W, seed):
    f, wb, d, a = _setup_bf16(H, W, seed)
    for l, (z, ref) in enumerate(zip((z.cpu().numpy() for z in d.logits(*a)), omr.logits(f, wb))):
        assert np.abs(z - ref).max() < 1e-2 * max(1.0, np.abs(ref).max()), l


@pytest.mark.parametrize("H,W,seed", [(64, 96, 90), (130, 257, 93), (256, 384, 94)])
def test_multires_bf16_denoise_close_to_oracle(H, W, seed):
    f, wb, d, a = _setup_bf16(H, W, seed)
    out = d.denoise(*a).cpu().numpy()[0]
    mx, mean, mean_rel = _err(out, f, wb)
    print(f"multires bf16 {H}x{W}: max err / term scale {mx:.3e}, mean {mean:.3e}; mean rel {mean_rel:.3e}")
    assert mx < 1e-2 and mean_rel < 1e-3


@pytest.fixture(scope="module")
def mr1080():
    """1920x1080 seed-2 frame, weights and the oracle's output and Eq. 7
    term scale over every pixel (computed once: about 10 s on 16 cores)."""
    f = synth.make_frame(1080, 1920, 2)
    wb = synth.make_weights_for(omr.weight_shapes(), seed=2)
    zs = omr.logits(f, wb)
    ref = omr.reconstruct(zs, f["radiance"], f["albedo"])
    scale = np.maximum(np.abs(ref), omr.term_scale(zs, f["radiance"], f["albedo"]))
    return f, wb, ref, scale


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("bf16", 1e-2)])
def test_multires_1080p_every_pixel_matches_oracle(mr1080, precision, tol):
    from paper_2202_05977_b300.multires import MultiResDenoiser
    f, wb, ref, scale = mr1080
    d = MultiResDenoiser(wb, max_hw=(1080, 1920), precision=precision)
    out = d.denoise(*args(to_dev(stack_frames([f])))).cpu().numpy()[0]
    e = np.abs(out - ref) / scale
    mean_rel = rel_err(out, ref)[1]
    print(f"multires {precision} 1080p: max err / term scale {e.max():.3e}, mean {e.mean():.3e}; "
          f"mean rel {mean_rel:.3e}")
    assert e.max() < tol and mean_rel < (1e-5 if precision == "fp32" else 1e-3)


def test_multires_bf16_1080p_agrees_with_fp32_path():
    from paper_2202_05977_b300.multires import MultiResDenoiser
    f = synth.make_frame(1080, 1920, 2)
    wb = synth.make_weights_for(omr.weight_shapes(), seed=2)
    a = args(to_dev(stack_frames([f])))
    o16 = MultiResDenoiser(wb, max_hw=(1080, 1920), precision="bf16").denoise(*a).cpu().numpy()[0]
    o32 = MultiResDenoiser(wb, max_hw=(1080, 1920), precision="fp32").denoise(*a).cpu().numpy()[0]
    assert np.all(np.isfinite(o16))
    e = np.abs(o16 - o32) / np.maximum(np.abs(o32), 1e-6)
    print(f"multires bf16 vs fp32 1080p: median rel {np.median(e):.3e} mean {e.mean():.3e}")
    assert np.median(e) < 1e-3
