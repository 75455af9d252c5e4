"""GPU parity of the FP32 plain path and the reconstruction kernel against
the FP64 oracle, through the C ABI.  Tolerance: max relative error 1e-5 per
output element for the FP32 path (|gpu - ref| / max(|ref|, 1e-6))."""
import numpy as np
import pytest

import oracle
import synth
from tests._util import KSIZES, args, rel_err, sample_pixels, stack_frames, to_dev

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5
TOL_DECODE = 2e-6


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


@pytest.fixture(scope="module")
def wk():
    import paper_2202_05977_b300 as wk
    return wk


# ------------------------------------------------------------ reconstruction
@pytest.mark.parametrize("B,H,W", [(1, 64, 64), (2, 45, 67), (1, 1, 1), (1, 13, 13), (1, 14, 200),
                                   (1, 130, 17)])
def test_decode_fuse_fwd_matches_oracle(torch, wk, B, H, W):
    g = np.random.default_rng(H * 1000 + W)
    frames = [synth.make_frame(H, W, 100 + b) for b in range(B)]
    z = (g.standard_normal((B, 12, H, W)) * 1.5).astype(np.float32)
    dev = to_dev(stack_frames(frames))
    fb = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = wk.decode_fuse_fwd(torch.from_numpy(z).cuda(), dev["radiance"], dev["albedo"], KSIZES, 1e-2,
                             fallbacks=fb).cpu().numpy()
    for b in range(B):
        ref = oracle.reconstruct(z[b], frames[b]["radiance"], frames[b]["albedo"])
        mx, _ = rel_err(out[b], ref)
        assert mx < TOL_DECODE, (b, mx)
    assert int(fb.item()) == 0


def test_decode_fuse_fwd_wide_logit_range_takes_exact_path(torch, wk):
    # Logit range > 69 inside a tile: the shifted window sums underflow for
    # some pixels, which must take the exact per-window path and be counted.
    H, W = 40, 70
    f = synth.make_frame(H, W, 7)
    g = np.random.default_rng(7)
    z = (g.standard_normal((1, 12, H, W))).astype(np.float32)
    z[0, :6, 20, 30] = 95.0
    z[0, :6, :, :10] -= 40.0
    dev = to_dev(stack_frames([f]))
    fb = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = wk.decode_fuse_fwd(torch.from_numpy(z).cuda(), dev["radiance"], dev["albedo"], KSIZES, 1e-2,
                             fallbacks=fb).cpu().numpy()
    ref = oracle.reconstruct(z[0], f["radiance"], f["albedo"])
    assert rel_err(out[0], ref)[0] < TOL_DECODE
    assert int(fb.item()) > 0


def test_decode_fuse_fwd_single_and_custom_sizes(torch, wk):
    H, W = 33, 90
    f = synth.make_frame(H, W, 8)
    dev = to_dev(stack_frames([f]))
    g = np.random.default_rng(8)
    for ks in [(1,), (13,), (5, 9), (3, 3, 13)]:
        z = g.standard_normal((1, 2 * len(ks), H, W)).astype(np.float32)
        out = wk.decode_fuse_fwd(torch.from_numpy(z).cuda(), dev["radiance"], dev["albedo"], ks, 1e-2)
        ref = oracle.reconstruct(z[0], f["radiance"], f["albedo"], ksizes=ks)
        assert rel_err(out.cpu().numpy()[0], ref)[0] < TOL_DECODE, ks


def test_constant_irradiance_is_preserved(torch, wk):
    H, W = 50, 77
    f = synth.make_frame(H, W, 9)
    c = np.array([0.5, 3.0, 0.02], np.float32)[:, None, None]
    f["radiance"] = ((f["albedo"] + np.float32(1e-2)) * c).astype(np.float32)
    dev = to_dev(stack_frames([f]))
    z = np.random.default_rng(9).standard_normal((1, 12, H, W)).astype(np.float32) * 3
    out = wk.decode_fuse_fwd(torch.from_numpy(z).cuda(), dev["radiance"], dev["albedo"]).cpu().numpy()
    assert rel_err(out[0], f["radiance"])[0] < TOL_DECODE


# -------------------------------------------------------------------- prep
def test_prep_matches_oracle(torch, wk):
    frames = [synth.make_frame(37, 53, 11), synth.make_frame(37, 53, 12)]
    dev = to_dev(stack_frames(frames))
    x = wk.prep(*args(dev)).cpu().numpy()
    for b, f in enumerate(frames):
        ref = oracle.prep(f["radiance"], f["albedo"], f["normal"], f["depth"])
        np.testing.assert_allclose(x[b], ref, rtol=3e-7, atol=1e-7)


# ------------------------------------------------------------ FP32 network
def _den(wk, wb, **kw):
    return wk.Denoiser(wb, precision="fp32", **kw)


def test_fp32_logits_match_oracle(torch, wk):
    f = synth.make_frame(64, 64, 0)
    wb = synth.make_weights(seed=0)
    d = _den(wk, wb, max_hw=(64, 64))
    z = d.logits(*args(to_dev(stack_frames([f])))).cpu().numpy()[0]
    ref = oracle.logits(f, wb)
    assert np.abs(z - ref).max() < 2e-5 * max(1.0, np.abs(ref).max())


def test_fp32_denoise_64_matches_oracle(torch, wk):
    """Plain method, FP32, single 64x64 frame, seed 0: every pixel."""
    f = synth.make_frame(64, 64, 0)
    wb = synth.make_weights(seed=0)
    d = _den(wk, wb, max_hw=(64, 64))
    out = d.denoise(*args(to_dev(stack_frames([f])))).cpu().numpy()[0]
    mx, mean = rel_err(out, oracle.denoise(f, wb))
    print(f"fp32 64x64: max rel {mx:.3e} mean {mean:.3e}")
    assert mx < TOL_FP32


@pytest.mark.parametrize("B,H,W", [(2, 45, 67), (1, 1, 1), (1, 13, 13), (1, 14, 200), (3, 19, 33)])
def test_fp32_denoise_ragged_matches_oracle(torch, wk, B, H, W):
    frames = [synth.make_frame(H, W, 20 + b) for b in range(B)]
    wb = synth.make_weights(seed=1)
    d = _den(wk, wb, max_hw=(H, W), max_batch=B)
    out = d.denoise(*args(to_dev(stack_frames(frames)))).cpu().numpy()
    for b in range(B):
        mx, _ = rel_err(out[b], oracle.denoise(frames[b], wb))
        assert mx < TOL_FP32, (b, mx)


def test_fp32_denoise_720p_sampled_matches_oracle(torch, wk):
    """Plain method, FP32, 1280x720, seed 1: sampled pixels, each computed by
    the oracle on its own receptive field."""
    H, W = 720, 1280
    f = synth.make_frame(H, W, 1)
    wb = synth.make_weights(seed=1)
    d = _den(wk, wb, max_hw=(H, W))
    out = d.denoise(*args(to_dev(stack_frames([f])))).cpu().numpy()[0]
    pix = sample_pixels(H, W, 40, seed=1)
    ref = oracle.denoise_pixels(f, wb, pix)
    got = np.stack([out[:, y, x] for x, y in pix])
    mx, mean = rel_err(got, ref)
    print(f"fp32 720p sampled: max rel {mx:.3e} mean {mean:.3e}")
    assert mx < TOL_FP32
    assert np.isfinite(out).all() and (out > 0).all()


def test_fp32_batch_invariance(torch, wk):
    frames = [synth.make_frame(48, 80, 30 + b) for b in range(3)]
    wb = synth.make_weights(seed=2)
    d = _den(wk, wb, max_hw=(48, 80), max_batch=3)
    dev = to_dev(stack_frames(frames))
    both = d.denoise(*args(dev)).cpu().numpy()
    for b in range(3):
        one = d.denoise(*(dev[k][b:b + 1].contiguous() for k in ("radiance", "albedo", "normal", "depth")))
        np.testing.assert_array_equal(one.cpu().numpy()[0], both[b])


def test_denoise_host_matches_device_call(torch, wk):
    f = synth.make_frame(40, 72, 31)
    wb = synth.make_weights(seed=3)
    d = _den(wk, wb, max_hw=(40, 72))
    st = stack_frames([f])
    dev = to_dev(st)
    ref = d.denoise(*args(dev)).cpu()
    host = [torch.from_numpy(np.ascontiguousarray(st[k])).pin_memory() for k in ("radiance", "albedo", "normal", "depth")]
    out = torch.empty((1, 3, 40, 72), dtype=torch.float32).pin_memory()
    d.denoise_host(*host, out)
    assert torch.equal(out, ref)


@pytest.mark.parametrize("prec,B,H,W", [("fp32", 2, 600, 200), ("bf16", 1, 1080, 256), ("fp32", 1, 517, 130)])
def test_banded_host_call_matches_device_call(torch, wk, prec, B, H, W):
    """Frames of 432+ rows go through the banded host pipeline (halo rows
    recomputed per band, copies overlapped with compute); the kept rows equal
    the whole-frame device call up to the per-tile exponent shift of the
    reconstruction (FP32 rounding)."""
    frames = [synth.make_frame(H, W, 40 + b) for b in range(B)]
    wb = synth.make_weights(seed=4)
    d = wk.Denoiser(wb, precision=prec, max_hw=(H, W), max_batch=B)
    st = stack_frames(frames)
    ref = d.denoise(*args(to_dev(st))).cpu().numpy()
    host = [torch.from_numpy(np.ascontiguousarray(st[k])).pin_memory() for k in ("radiance", "albedo", "normal", "depth")]
    out = torch.full((B, 3, H, W), float("nan"), dtype=torch.float32).pin_memory()
    d.denoise_host(*host, out)
    mx, _ = rel_err(out.numpy(), ref)
    assert mx < 1e-5, mx


@pytest.mark.parametrize("bands,first", [(3, 40), (7, 100), (2, 70)])
def test_banded_host_call_with_tuned_bands(torch, wk, bands, first):
    """WSKPN_TUNE_HOST_BANDS / WSKPN_TUNE_HOST_FIRST_BAND change only how the
    host pipeline splits the frame, not its result."""
    from paper_2202_05977_b300 import _lib
    H, W = 530, 160
    f = synth.make_frame(H, W, 44)
    wb = synth.make_weights(seed=4)
    d = wk.Denoiser(wb, precision="fp32", max_hw=(H, W))
    st = stack_frames([f])
    ref = d.denoise(*args(to_dev(st))).cpu().numpy()
    d.set_tuning(_lib.TUNE_HOST_BANDS, bands)
    d.set_tuning(_lib.TUNE_HOST_FIRST_BAND, first)
    host = [torch.from_numpy(np.ascontiguousarray(st[k])).pin_memory() for k in ("radiance", "albedo", "normal", "depth")]
    out = torch.full((1, 3, H, W), float("nan"), dtype=torch.float32).pin_memory()
    d.denoise_host(*host, out)
    mx, _ = rel_err(out.numpy(), ref)
    assert mx < 1e-5, mx
    with pytest.raises(wk.WskpnError):
        d.set_tuning(_lib.TUNE_HOST_FIRST_BAND, 5)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_async_host_calls_overlap_and_match_sync_calls(torch, wk, prec):
    """wskpn_denoise_host_async: several frames of different sizes queued
    back to back on one context (banded and unbanded, each into its own host
    buffer), one synchronisation at the end; every result equals the
    synchronous call's, bit for bit (same bands, same kernels)."""
    sizes = [(600, 200), (460, 130), (600, 200), (40, 72), (1080, 256)]
    wb = synth.make_weights(seed=5)
    d = wk.Denoiser(wb, precision=prec, max_hw=(1080, 256))
    hosts, outs, refs = [], [], []
    for i, (H, W) in enumerate(sizes):
        st = stack_frames([synth.make_frame(H, W, 50 + i)])
        host = [torch.from_numpy(np.ascontiguousarray(st[k])).pin_memory() for k in ("radiance", "albedo", "normal", "depth")]
        ref = torch.empty((1, 3, H, W), dtype=torch.float32).pin_memory()
        d.denoise_host(*host, ref)
        hosts.append(host)
        refs.append(ref)
        outs.append(torch.full((1, 3, H, W), float("nan"), dtype=torch.float32).pin_memory())
    s = torch.cuda.Stream()
    for _ in range(2):  # twice: the second round reuses band buffers the first still holds in flight
        for host, out in zip(hosts, outs):
            d.denoise_host(*host, out, stream=s, wait=False)
        s.synchronize()
        for out, ref in zip(outs, refs):
            assert torch.equal(out, ref)
        for out in outs:
            out.fill_(float("nan"))
    assert d.device_status() == 0
