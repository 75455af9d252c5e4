"""Pins of the oracle's multi-resolution variant (Eq. 7 and its U-Net)
against library routines, closed forms and invariants (CPU only)."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle
from oracle import multires as mr
import synth


@pytest.mark.parametrize("H,W", [(8, 12), (7, 9), (1, 5), (6, 1)])
def test_downsample_is_avg_pool_over_in_image_pixels(H, W):
    x = np.random.default_rng(0).standard_normal((3, H, W))
    ref = F.avg_pool2d(torch.from_numpy(x)[None], 2, 2, ceil_mode=True, count_include_pad=False)[0].numpy()
    np.testing.assert_allclose(mr.downsample(x), ref, rtol=1e-14)


@pytest.mark.parametrize("H,W", [(8, 12), (7, 9)])
def test_upsample_is_nearest_interpolation(H, W):
    x = np.random.default_rng(1).standard_normal((2, (H + 1) // 2, (W + 1) // 2))
    ref = F.interpolate(torch.from_numpy(x)[None], scale_factor=2, mode="nearest")[0].numpy()[:, :H, :W]
    np.testing.assert_array_equal(mr.upsample(x, H, W), ref)


def test_eq7_zero_blend_keeps_the_fine_level_and_one_swaps_low_frequencies():
    g = np.random.default_rng(2)
    i0, i1, i2 = g.standard_normal((3, 8, 10)), g.standard_normal((3, 4, 5)), g.standard_normal((3, 2, 3))
    big = np.full((8, 10), 60.0)
    np.testing.assert_allclose(mr.combine([i0, i1, i2], [-big, -big[:4, :5]]), i0, atol=1e-24)
    # alpha = 1 at both levels: o_1 = i1 - UD i1 + U i2 ; o_0 = i0 - UD i0 + U o_1
    o1 = i1 - mr.upsample(mr.downsample(i1), 4, 5) + mr.upsample(i2, 4, 5)
    o0 = i0 - mr.upsample(mr.downsample(i0), 8, 10) + mr.upsample(o1, 8, 10)
    np.testing.assert_allclose(mr.combine([i0, i1, i2], [big, big[:4, :5]]), o0, rtol=1e-12)


def test_eq7_two_level_hand_example():
    # fine 2x2 block [[1,2],[3,5]] (mean 2.75), coarse value 10, alpha = sigmoid(0) = 1/2
    i_f = np.array([[[1.0, 2.0], [3.0, 5.0]]])
    i_c = np.array([[[10.0]]])
    o = mr.combine([i_f, i_c], [np.zeros((2, 2))])
    np.testing.assert_allclose(o, i_f - 0.5 * 2.75 + 0.5 * 10.0, rtol=1e-15)


def test_eq7_preserves_a_constant_signal_for_any_blend():
    g = np.random.default_rng(3)
    c = np.array([0.3, 1.7, 4.0])[:, None, None]
    levels = [np.broadcast_to(c, (3, h, w)).copy() for h, w in mr.level_sizes(13, 21)]
    blends = [g.standard_normal(s) * 3 for s in mr.level_sizes(13, 21)[:2]]
    np.testing.assert_allclose(mr.combine(levels, blends), levels[0], rtol=1e-14)


def test_level_filter_with_constant_importance_is_a_box_average():
    g = np.random.default_rng(4)
    y = g.uniform(0.1, 2.0, (3, 9, 11))
    z = np.zeros((4, 9, 11))
    z[2] = g.standard_normal((9, 11))  # fusion logits: any blend of two box averages
    z[3] = g.standard_normal((9, 11))
    R3 = F.avg_pool2d(torch.from_numpy(y)[None], 3, 1, 1, count_include_pad=False)[0].numpy()
    R5 = F.avg_pool2d(torch.from_numpy(y)[None], 5, 1, 2, count_include_pad=False)[0].numpy()
    a = np.exp(z[2:4]) / np.exp(z[2:4]).sum(0)
    np.testing.assert_allclose(mr.filter_level(z, y), a[0] * R3 + a[1] * R5, rtol=1e-12)


def test_unet_matches_an_independent_torch_float64_network():
    f = synth.make_frame(20, 27, 5)
    wb = synth.make_weights_for(mr.weight_shapes(), seed=5)
    zs = mr.logits(f, wb)
    # torch float64 reimplementation of the stated architecture from library ops
    x = torch.from_numpy(oracle.prep(f["radiance"], f["albedo"], f["normal"], f["depth"]))[None]
    Ls, off = {}, 0
    for name, ci, co, relu in mr.LAYERS:
        n = co * ci * 9
        Ls[name] = (torch.from_numpy(wb[off:off + n].astype(np.float64)).view(co, ci, 3, 3),
                    torch.from_numpy(wb[off + n:off + n + co].astype(np.float64)), relu)
        off += n + co

    def c(name, t):
        w, b, relu = Ls[name]
        y = F.conv2d(t, w, b, padding=1)
        return torch.relu(y) if relu else y

    pool = lambda t: F.avg_pool2d(t, 2, 2, ceil_mode=True, count_include_pad=False)
    up = lambda t, ref: F.interpolate(t, scale_factor=2, mode="nearest")[:, :, :ref.shape[2], :ref.shape[3]]
    e0 = c("E0b", c("E0", x))
    e1 = c("E1b", c("E1", pool(e0)))
    e2 = c("E2b", c("E2", pool(e1)))
    d1 = c("D1", torch.cat([up(e2, e1), e1], 1))
    d0 = c("D0", torch.cat([up(d1, e0), e0], 1))
    for got, ref in zip(zs, (c("H0", d0), c("H1", d1), c("H2", e2))):
        np.testing.assert_allclose(got, ref[0].numpy(), rtol=1e-9, atol=1e-11)


def test_multires_denoiser_passes_a_constant_irradiance_through():
    # r = (a + eps) c: every level filters the constant c, Eq. 7 keeps it, out = r
    f = synth.make_frame(19, 26, 6)
    c = np.array([0.4, 0.9, 1.3])[:, None, None]
    f["radiance"] = ((f["albedo"].astype(np.float64) + 0.01) * c).astype(np.float32)
    wb = synth.make_weights_for(mr.weight_shapes(), seed=6)
    out = mr.denoise(f, wb)
    y = f["radiance"].astype(np.float64) / (f["albedo"] + 0.01)
    np.testing.assert_allclose(out, (f["albedo"] + 0.01) * y, rtol=1e-6)


def test_n_weights_matches_the_layer_list():
    assert mr.n_weights() == synth.make_weights_for(mr.weight_shapes()).size == 188_878  # 2912+9248+13872+20784+27712+36928+2308+48432+2165+23072+1445


def test_term_scale_bounds_the_output():
    f = synth.make_frame(21, 30, 7)
    wb = synth.make_weights_for(mr.weight_shapes(), seed=7)
    zs = mr.logits(f, wb)
    out = mr.reconstruct(zs, f["radiance"], f["albedo"])
    sc = mr.term_scale(zs, f["radiance"], f["albedo"])
    assert np.all(np.abs(out) <= sc * (1 + 1e-12))
