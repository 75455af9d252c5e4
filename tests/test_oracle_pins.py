"""Pins of the FP64 oracle to things other than itself: library routines
(torch float64 conv2d / avg_pool2d), closed forms, invariants the paper
states, brute force on tiny inputs and finite differences.  CPU only."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle
import synth

KS_ALL = (3, 5, 7, 9, 11, 13)


def _rng(seed):
    return np.random.default_rng(seed)


# --------------------------------------------------------------- Sec. 4.1 conv
@pytest.mark.parametrize("KS,Cin,Cout,H,W,relu", [(5, 3, 4, 7, 9, False), (5, 10, 6, 13, 11, True),
                                                  (3, 4, 5, 8, 6, True), (5, 2, 3, 1, 1, False),
                                                  (5, 2, 2, 3, 17, True)])
def test_conv_matches_torch_conv2d_float64(KS, Cin, Cout, H, W, relu):
    g = _rng(KS * 100 + Cin)
    x = g.standard_normal((Cin, H, W))
    w = g.standard_normal((Cout, Cin, KS, KS))
    b = g.standard_normal(Cout)
    ref = F.conv2d(torch.from_numpy(x)[None], torch.from_numpy(w), torch.from_numpy(b), padding=KS // 2)[0]
    if relu:
        ref = torch.relu(ref)
    np.testing.assert_allclose(oracle.conv2d(x, w, b, relu), ref.numpy(), rtol=1e-12, atol=1e-12)


def test_conv_one_hot_tap_is_a_shift():
    # W[0, 1, dy=0, dx=4] = 1: y[0, r, c] = x[1, r - 2, c + 2] (zero outside) —
    # cross-correlation orientation and zero padding, by hand.
    x = np.arange(2 * 6 * 7, dtype=np.float64).reshape(2, 6, 7) + 1.0
    w = np.zeros((1, 2, 5, 5))
    w[0, 1, 0, 4] = 1.0
    y = oracle.conv2d(x, w, np.zeros(1), relu=False)
    exp = np.zeros((6, 7))
    exp[2:, :5] = x[1, :4, 2:]
    np.testing.assert_array_equal(y[0], exp)


# --------------------------------------------------------------- Sec. 5.1 prep
def test_prep_special_values():
    H, W = 2, 3
    rad = np.array([[-0.5, 0.0, 1.0], [2.0, 0.3, 0.9]])[None].repeat(3, 0)
    alb = _rng(1).uniform(0, 1, (3, H, W))
    nrm = np.array([[-1.0, 0.0, 1.0], [0.5, -0.5, 0.25]])[None].repeat(3, 0)
    dep = np.array([[1.0, 10.0, 5.5], [2.0, 3.0, 9.0]])[None]
    x = oracle.prep(rad, alb, nrm, dep)
    assert x.shape == (10, H, W)
    # tone map: clamps to [0,1]; LDR value raised back to gamma gives the radiance
    np.testing.assert_array_equal(x[0, 0, :3], [0.0, 0.0, 1.0])
    assert x[0, 1, 0] == 1.0
    np.testing.assert_allclose(x[0, 1, 1:] ** 2.2, rad[0, 1, 1:], rtol=1e-14)
    np.testing.assert_array_equal(x[3:6], alb)                      # albedo as is
    np.testing.assert_array_equal(x[6:9, 0], [[0.0, 0.5, 1.0]] * 3)  # [-1,1] -> [0,1]
    np.testing.assert_allclose(x[9, 0, :2], [0.0, 1.0])              # [near,far] -> [0,1]
    np.testing.assert_allclose(x[9, 0, 2], 0.5)


# ------------------------------------------------------- Eq. 3-4 kernel decode
@pytest.mark.parametrize("H,W", [(7, 9), (16, 16), (1, 1), (3, 20)])
@pytest.mark.parametrize("k", [1, 3, 5, 7, 9, 11, 13])
def test_decode_two_codings_agree(H, W, k):
    g = _rng(H * 31 + W + k)
    z = g.standard_normal((H, W)) * 2.0
    y = g.lognormal(0.0, 1.0, (3, H, W))
    a = oracle.decode_explicit(z, y, k)
    b = oracle.decode_boxsum(z, y, k)
    np.testing.assert_allclose(a, b, rtol=1e-13, atol=0)


def test_decode_two_codings_agree_64():
    g = _rng(5)
    z = g.standard_normal((64, 64)) * 3.0
    y = g.lognormal(0.0, 1.0, (3, 64, 64))
    for k in KS_ALL:
        np.testing.assert_allclose(oracle.decode_explicit(z, y, k), oracle.decode_boxsum(z, y, k),
                                   rtol=1e-13)


@pytest.mark.parametrize("k", KS_ALL)
def test_decode_constant_importance_is_clipped_box_mean(k):
    # I == const: every weight in the clipped window is equal, so R is the mean
    # of y over the window's in-image part (library routine, float64).
    g = _rng(k)
    y = g.uniform(0.1, 3.0, (3, 11, 14))
    R = oracle.decode_explicit(np.full((11, 14), 0.37), y, k)
    ref = F.avg_pool2d(torch.from_numpy(y)[None], k, stride=1, padding=k // 2,
                       count_include_pad=False)[0].numpy()
    np.testing.assert_allclose(R, ref, rtol=1e-13)


def test_decode_invariants():
    g = _rng(9)
    H, W = 12, 10
    z = g.standard_normal((H, W))
    y = g.lognormal(0, 1, (3, H, W))
    for k in (3, 7, 13):
        # normalised kernels: a constant signal passes unchanged (Sec. 4.2 energy conservation)
        c = np.stack([np.full((H, W), v) for v in (0.3, 1.0, 7.0)])
        np.testing.assert_allclose(oracle.decode_explicit(z, c, k), c, rtol=1e-14)
        # softmax is shift invariant
        np.testing.assert_allclose(oracle.decode_explicit(z + 7.3, y, k), oracle.decode_explicit(z, y, k),
                                   rtol=1e-13)
        # mirror symmetry of the window
        np.testing.assert_allclose(oracle.decode_explicit(z[:, ::-1], y[:, :, ::-1], k),
                                   oracle.decode_explicit(z, y, k)[:, :, ::-1], rtol=1e-13)
        np.testing.assert_allclose(oracle.decode_explicit(z[::-1], y[:, ::-1], k),
                                   oracle.decode_explicit(z, y, k)[:, ::-1], rtol=1e-13)
    # k = 1 is the identity
    np.testing.assert_allclose(oracle.decode_explicit(z, y, 1), y, rtol=0, atol=0)


def test_kernel_weights_properties():
    g = _rng(3)
    H, W = 9, 8
    z = g.standard_normal((H, W))
    for k in (3, 5, 13):
        h = k // 2
        for (px, py) in [(0, 0), (4, 4), (7, 8), (2, 6)]:
            w = oracle.kernel_weights(z, k, px, py)
            assert w.shape == (k, k)
            assert abs(w.sum() - 1.0) < 1e-14 and (w >= 0).all() and (w <= 1).all()
            for dy in range(-h, h + 1):
                for dx in range(-h, h + 1):
                    inside = 0 <= px + dx < W and 0 <= py + dy < H
                    assert (w[dy + h, dx + h] > 0) == inside
    # a dominant spike takes the whole kernel of every window that contains it
    z2 = np.zeros((H, W))
    z2[4, 3] = 60.0
    w = oracle.kernel_weights(z2, 5, 2, 5)
    assert abs(w[4 - 5 + 2, 3 - 2 + 2] - 1.0) < 1e-20 + 169 * np.exp(-60)


def test_decode_spike_copies_the_spike_pixel():
    g = _rng(4)
    H, W = 15, 15
    y = g.lognormal(0, 1, (3, H, W))
    z = g.standard_normal((H, W))
    z[7, 7] = 80.0
    R = oracle.decode_explicit(z, y, 5)
    for py in range(5, 10):
        for px in range(5, 10):
            np.testing.assert_allclose(R[:, py, px], y[:, 7, 7], rtol=1e-12)


# ------------------------------------------------------------ Eq. 5 fusion
def test_fuse_special_cases():
    g = _rng(11)
    M, H, W = 6, 5, 4
    Rs = g.lognormal(0, 1, (M, 3, H, W))
    alb = g.uniform(0, 1, (3, H, W))
    eps = 1e-2
    # equal logits: arithmetic mean of the M filtered images
    np.testing.assert_allclose(oracle.fuse(Rs, np.zeros((M, H, W)), alb, eps),
                               (alb + eps) * Rs.mean(axis=0), rtol=1e-14)
    # one dominant logit selects that size
    for j in range(M):
        lg = np.zeros((M, H, W))
        lg[j] = 800.0
        np.testing.assert_allclose(oracle.fuse(Rs, lg, alb, eps), (alb + eps) * Rs[j], rtol=1e-14)
    # a single size (M = 1) is plain re-modulation
    np.testing.assert_allclose(oracle.fuse(Rs[:1], g.standard_normal((1, H, W)), alb, eps),
                               (alb + eps) * Rs[0], rtol=1e-15)
    # convex weights: the result lies between the per-size extremes
    lg = g.standard_normal((M, H, W)) * 3
    o = oracle.fuse(Rs, lg, alb, eps) / (alb + eps)
    assert (o <= Rs.max(axis=0) * (1 + 1e-14)).all() and (o >= Rs.min(axis=0) * (1 - 1e-14)).all()


# ------------------------------------------------------------- whole denoiser
def test_network_matches_torch_chain():
    # ImportanceNet wiring: ReLU after every block but the last, blob order
    # [W, b] per layer, zero padding — against torch float64 conv2d.
    f = synth.make_frame(21, 26, 3)
    wb = synth.make_weights(seed=3)
    x = torch.from_numpy(oracle.prep(f["radiance"], f["albedo"], f["normal"], f["depth"]))[None]
    layers = oracle.split_weights(wb)
    for l, (w, b) in enumerate(layers):
        x = F.conv2d(x, torch.from_numpy(w), torch.from_numpy(b), padding=2)
        if l < len(layers) - 1:
            x = torch.relu(x)
    np.testing.assert_allclose(oracle.logits(f, wb), x[0].numpy(), rtol=1e-11, atol=1e-11)


def test_constant_irradiance_passes_through_whole_denoiser():
    # r = (a + eps) * c with c constant per channel: every kernel is
    # normalised and the fusion weights sum to 1, so the output is r for any
    # network weights (Eq. 3-5 with demodulation / re-modulation).
    f = synth.make_frame(24, 19, 5)
    c = np.array([0.7, 2.0, 0.05])[:, None, None]
    f["radiance"] = ((f["albedo"].astype(np.float64) + 1e-2) * c).astype(np.float64)
    out = oracle.denoise(f, synth.make_weights(seed=5))
    np.testing.assert_allclose(out, f["radiance"], rtol=1e-13)


def test_region_evaluation_matches_full_frame():
    f = synth.make_frame(33, 40, 6)
    wb = synth.make_weights(seed=6)
    full = oracle.denoise(f, wb)
    band = oracle.denoise(f, wb, rect=(0, 10, 40, 14))
    np.testing.assert_allclose(band, full[:, 10:14], rtol=1e-13)
    pix = [(0, 0), (39, 32), (20, 16), (5, 31), (39, 0)]
    po = oracle.denoise_pixels(f, wb, pix)
    np.testing.assert_allclose(po, np.stack([full[:, y, x] for x, y in pix]), rtol=1e-13)


def test_whole_denoiser_mirror_symmetry():
    f = synth.make_frame(18, 23, 7)
    wb = synth.make_weights(seed=7)
    mirrored = {k: np.ascontiguousarray(v[..., ::-1]) for k, v in f.items()}
    layers = oracle.split_weights(wb)
    flipped = np.concatenate([np.concatenate([w[..., ::-1].ravel(), b]) for w, b in layers])
    np.testing.assert_allclose(oracle.denoise(mirrored, flipped), oracle.denoise(f, wb)[..., ::-1],
                               rtol=1e-12)


def test_composition_from_layer_ops():
    f = synth.make_frame(17, 20, 8)
    wb = synth.make_weights(seed=8)
    out, acts = oracle.forward_train(f, wb)
    np.testing.assert_allclose(out, oracle.denoise(f, wb), rtol=1e-13)
    # reconstruct = explicit decode per size + fuse
    z = acts[-1]
    y = f["radiance"].astype(np.float64) / (f["albedo"].astype(np.float64) + 1e-2)
    Rs = np.stack([oracle.decode_boxsum(z[i], y, k) for i, k in enumerate(KS_ALL)])
    np.testing.assert_allclose(oracle.fuse(Rs, z[6:], f["albedo"]), out, rtol=1e-12)


# -------------------------------------------------------------- backward
def _fd(fun, x, idx, h=1e-6):
    xp, xm = x.copy(), x.copy()
    xp.flat[idx] += h
    xm.flat[idx] -= h
    return (fun(xp) - fun(xm)) / (2 * h)


def test_reconstruct_bwd_matches_finite_differences():
    g = _rng(21)
    H, W = 14, 11
    f = synth.make_frame(H, W, 21)
    z = g.standard_normal((12, H, W))
    G = g.standard_normal((3, H, W))
    dz = oracle.reconstruct_bwd(z, f["radiance"], f["albedo"], G)
    fun = lambda zz: float((oracle.reconstruct(zz, f["radiance"], f["albedo"]) * G).sum())
    for idx in g.choice(z.size, 60, replace=False).tolist() + [0, z.size - 1]:
        np.testing.assert_allclose(dz.flat[idx], _fd(fun, z, idx), rtol=2e-6, atol=1e-8)


def test_conv_bwd_matches_torch_autograd():
    g = _rng(22)
    x = g.standard_normal((3, 9, 7))
    w = g.standard_normal((4, 3, 5, 5))
    gy = g.standard_normal((4, 9, 7))
    gx, gw, gb = oracle.conv2d_bwd(x, w, gy)
    xt = torch.from_numpy(x)[None].requires_grad_()
    wt = torch.from_numpy(w).requires_grad_()
    bt = torch.zeros(4, dtype=torch.float64, requires_grad=True)
    (F.conv2d(xt, wt, bt, padding=2) * torch.from_numpy(gy)[None]).sum().backward()
    np.testing.assert_allclose(gx, xt.grad[0].numpy(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(gw, wt.grad.numpy(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(gb, bt.grad.numpy(), rtol=1e-12, atol=1e-12)


def test_training_gradient_matches_finite_differences():
    # small network (KS 3, widths 10-4-6-4, M = 2 sizes {3,5}) so FD is cheap;
    # random-cotangent VJP keeps the objective smooth.
    widths, ks, ksizes = (10, 4, 6, 4), 3, (3, 5)
    g = _rng(23)
    f = synth.make_frame(10, 12, 23)
    wb = synth.make_weights(widths, ks, seed=23).astype(np.float64)
    G = g.standard_normal((3, 10, 12))
    kw = dict(widths=widths, ks=ks, ksizes=ksizes)
    out, acts = oracle.forward_train(f, wb, **kw)
    grad, _ = oracle.backward_train(f, wb, acts, G, **kw)
    fun = lambda ww: float((oracle.forward_train(f, ww, **kw)[0] * G).sum())
    for idx in g.choice(wb.size, 40, replace=False).tolist() + [0, wb.size - 1]:
        np.testing.assert_allclose(grad[idx], _fd(fun, wb, idx), rtol=5e-5, atol=1e-7)


def test_round_bf16_definition():
    """Hand values of round-to-nearest-even at 8 significand bits, and the
    library conversion (torch's float32 -> bfloat16) on random values."""
    u = 2.0 ** -7  # one unit in the last place of bfloat16 at [1, 2)
    cases = [(1.0, 1.0), (1.0 + u / 2, 1.0),                 # tie, kept last bit even: down
             (1.0 + 3 * u / 2, 1.0 + 2 * u),                   # tie, kept last bit odd: up
             (1.0 + u / 2 + 2.0 ** -20, 1.0 + u),              # above the tie: up
             (1.0 + u / 2 - 2.0 ** -20, 1.0),                  # below the tie: down
             (-(1.0 + 3 * u / 2), -(1.0 + 2 * u)),            # sign symmetric
             (2.0 - u / 4, 2.0), (0.0, 0.0), (3.0e-3, 0.0030059814453125)]
    for x, want in cases:
        assert oracle.round_bf16(np.float32(x)) == want, (x, oracle.round_bf16(np.float32(x)), want)
    x = _rng(31).standard_normal(10000).astype(np.float32) * 0.3
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(oracle.round_bf16(x), ref)
    wb = synth.make_weights(seed=31)
    r = oracle.bf16_weights(wb)
    for (ws, bs), (wr, br), (w0, b0) in zip(synth.weight_shapes(), oracle.split_weights(r), oracle.split_weights(wb)):
        np.testing.assert_array_equal(br, b0)  # biases stay FP32
        np.testing.assert_array_equal(wr, oracle.round_bf16(w0.astype(np.float32)))


def test_training_gradient_matches_fd_at_training_crop_size():
    """Config-5 size pin: a 32 x 32 crop through the default network
    (widths 10-32-48-64-12, 5 x 5 convs, sizes 3..13); central differences
    on weights sampled from every layer (kernel entries and biases) against
    the oracle gradient of a random-cotangent objective."""
    g = _rng(32)
    f = synth.make_frame(32, 32, 32)
    wb = synth.make_weights(seed=32).astype(np.float64)
    G = g.standard_normal((3, 32, 32))
    out, acts = oracle.forward_train(f, wb)
    grad, _ = oracle.backward_train(f, wb, acts, G)
    fun = lambda ww: float((oracle.forward_train(f, ww)[0] * G).sum())
    idx, off = [], 0
    for (ws, bs) in synth.weight_shapes():
        nw = int(np.prod(ws))
        idx += [off + int(i) for i in g.choice(nw, 3, replace=False)] + [off + nw + int(g.integers(bs[0]))]
        off += nw + bs[0]
    scale = np.abs(grad).max()
    for i in idx:
        np.testing.assert_allclose(grad[i], _fd(fun, wb, i, h=1e-5), rtol=1e-4, atol=1e-7 * scale)


def test_losses_and_gradients():
    g = _rng(24)
    out = g.lognormal(0, 1, (2, 3, 4, 5))
    t = g.lognormal(0, 1, (2, 3, 4, 5))
    L, G = oracle.l1_loss(out, t)
    assert abs(L - np.mean(np.abs(out - t))) < 1e-15
    for idx in range(0, out.size, 7):  # away from the kink |out - t| = 0
        np.testing.assert_allclose(G.flat[idx], _fd(lambda o: oracle.l1_loss(o, t)[0], out, idx),
                                   rtol=1e-6)
    L, G = oracle.smape_loss(out, t)
    # Eq. 6 value on a hand case: R = 1, t = 3, eps = 0.01 -> 2 / 4.01
    assert abs(oracle.smape_loss(np.ones((3, 1, 1)), np.full((3, 1, 1), 3.0))[0] - 2 / 4.01) < 1e-15
    for idx in range(0, out.size, 7):
        np.testing.assert_allclose(G.flat[idx], _fd(lambda o: oracle.smape_loss(o, t)[0], out, idx),
                                   rtol=1e-5)


def test_golden_tiny_frame():
    """Regression fixture written by tests/golden/make_golden.py (oracle only)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "tiny_denoise_8x6_seed42.txt")
    ref = np.loadtxt(path).reshape(3, 6, 8)
    f = synth.make_frame(6, 8, 42)
    out = oracle.denoise(f, synth.make_weights(seed=42))
    np.testing.assert_allclose(out, ref, rtol=1e-12)


def test_adam_first_step_is_signed_lr_and_matches_torch():
    # First step: mhat = g, vhat = g^2, so every weight moves by lr * g / (|g| + eps).
    g = _rng(30).standard_normal(50)
    w0 = _rng(31).standard_normal(50)
    w1, m, v = oracle.adam_step(w0, g, np.zeros(50), np.zeros(50), 1, lr=1e-3, eps=1e-8)
    np.testing.assert_allclose(w0 - w1, 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    # several steps against torch.optim.Adam (library routine, float64)
    wt = torch.tensor(w0, requires_grad=True)
    opt = torch.optim.Adam([wt], lr=1e-2, betas=(0.9, 0.99), eps=1e-8)
    w, m, v = w0.copy(), np.zeros(50), np.zeros(50)
    for step in range(1, 6):
        gs = _rng(40 + step).standard_normal(50)
        wt.grad = torch.tensor(gs)
        opt.step()
        w, m, v = oracle.adam_step(w, gs, m, v, step, lr=1e-2, beta1=0.9, beta2=0.99, eps=1e-8)
    np.testing.assert_allclose(w, wt.detach().numpy(), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("ci,co,identity", [(6, 5, False), (4, 4, True)])
def test_repvgg_fold_equals_multi_branch_block(ci, co, identity):
    # Sec. 4.1: the converted single 5x5 conv computes the same as the sum of
    # the 5x5, 3x3, 1x1 branches (+ identity) -- torch float64 convs per branch.
    g = _rng(50 + ci)
    w5, w3, w1 = g.standard_normal((co, ci, 5, 5)), g.standard_normal((co, ci, 3, 3)), g.standard_normal((co, ci, 1, 1))
    b5, b3, b1 = g.standard_normal(co), g.standard_normal(co), g.standard_normal(co)
    x = torch.from_numpy(g.standard_normal((1, ci, 9, 11)))
    ref = (F.conv2d(x, torch.from_numpy(w5), torch.from_numpy(b5), padding=2)
           + F.conv2d(x, torch.from_numpy(w3), torch.from_numpy(b3), padding=1)
           + F.conv2d(x, torch.from_numpy(w1), torch.from_numpy(b1)))
    if identity:
        ref = ref + x
    W, b = oracle.repvgg_fold(w5, b5, w3, b3, w1, b1, identity)
    np.testing.assert_allclose(oracle.conv2d(x[0].numpy(), W, b, relu=False), ref[0].numpy(), rtol=1e-12, atol=1e-12)
    # the fold's gradient maps dL/dW back to the branches (torch autograd through the block)
    w5t, w3t, w1t = (torch.from_numpy(t).requires_grad_() for t in (w5, w3, w1))
    gy = torch.from_numpy(g.standard_normal(ref.shape))
    (F.conv2d(x, w5t, padding=2) + F.conv2d(x, w3t, padding=1) + F.conv2d(x, w1t)).mul(gy).sum().backward()
    Wt = torch.from_numpy(W).requires_grad_()
    F.conv2d(x, Wt, padding=2).mul(gy).sum().backward()
    g5, g3, g1 = oracle.repvgg_fold_grad(Wt.grad.numpy())
    np.testing.assert_allclose(g5, w5t.grad.numpy(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(g3, w3t.grad.numpy(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(g1, w1t.grad.numpy(), rtol=1e-12, atol=1e-12)
