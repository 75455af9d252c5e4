"""Differentiation form on the GPU through the C ABI: the reconstruction
backward kernel, the full training backward, the L1 loss and Adam, against
the FP64 oracle (whose gradients are pinned to finite differences).
Tolerance for FP32 gradients: per tensor max |gpu - ref| <= 2e-4 max |ref|."""
import numpy as np
import pytest

import oracle
import synth
from tests._util import KSIZES, args, stack_frames, to_dev

pytestmark = pytest.mark.gpu

TOL_GRAD = 2e-4
TOL_BF16_TRAIN = 2e-2  # measured 2.7e-3 .. 1.03e-2 per layer on the case below


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


@pytest.fixture(scope="module")
def wk():
    import paper_2202_05977_b300 as wk
    return wk


def _close(gpu, ref, tol=TOL_GRAD, scale=None):
    """max |gpu - ref| <= tol * max(max |ref|, scale); `scale` is the size of
    the whole gradient, so channels whose exact gradient vanishes (rounding
    noise only) are judged against it."""
    gpu, ref = np.asarray(gpu, np.float64), np.asarray(ref, np.float64)
    den = max(np.abs(ref).max(), scale or 0.0, 1e-30)
    return float(np.abs(gpu - ref).max() / den) < tol


@pytest.mark.parametrize("B,H,W", [(1, 45, 67), (2, 33, 90), (1, 1, 1), (1, 14, 200), (1, 70, 20),
                                   (2, 100, 196), (1, 97, 131)])
def test_decode_fuse_bwd_matches_oracle(torch, wk, B, H, W):
    g = np.random.default_rng(B * 100 + H)
    frames = [synth.make_frame(H, W, 200 + b) for b in range(B)]
    dev = to_dev(stack_frames(frames))
    z = (g.standard_normal((B, 12, H, W)) * 1.5).astype(np.float32)
    G = g.standard_normal((B, 3, H, W)).astype(np.float32)
    fb = torch.zeros(1, dtype=torch.int32, device="cuda")
    dz = wk.decode_fuse_bwd(torch.from_numpy(z).cuda(), dev["radiance"], dev["albedo"], torch.from_numpy(G).cuda(),
                            KSIZES, 1e-2, fallbacks=fb).cpu().numpy()
    for b in range(B):
        ref = oracle.reconstruct_bwd(z[b], frames[b]["radiance"], frames[b]["albedo"], G[b])
        # floor: the size of the gradient's terms (|g| |y|); on a 1x1 image
        # every exact gradient is 0 and both sides hold rounding noise only
        y = frames[b]["radiance"] / (frames[b]["albedo"] + np.float32(1e-2))
        scale = max(1e-3 * np.abs(ref).max(), 1e-3 * np.abs(G[b]).max() * np.abs(y).max())
        for c in range(12):
            assert _close(dz[b, c], ref[c], scale=scale), (b, c)
    assert int(fb.item()) == 0


def test_decode_fuse_bwd_wide_range_takes_exact_path(torch, wk):
    H, W = 40, 70
    f = synth.make_frame(H, W, 77)
    g = np.random.default_rng(77)
    z = g.standard_normal((1, 12, H, W)).astype(np.float32)
    z[0, :6, 20, 30] = 95.0
    z[0, :6, :, :10] -= 40.0
    G = g.standard_normal((1, 3, H, W)).astype(np.float32)
    dev = to_dev(stack_frames([f]))
    fb = torch.zeros(1, dtype=torch.int32, device="cuda")
    dz = wk.decode_fuse_bwd(torch.from_numpy(z).cuda(), dev["radiance"], dev["albedo"], torch.from_numpy(G).cuda(),
                            KSIZES, 1e-2, fallbacks=fb).cpu().numpy()
    ref = oracle.reconstruct_bwd(z[0], f["radiance"], f["albedo"], G[0])
    for c in range(12):
        assert _close(dz[0, c], ref[c], 1e-3), c
    assert int(fb.item()) > 0


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_training_backward_matches_oracle(torch, wk, prec):
    """dL/dTheta for a random cotangent dL/dout, B = 2 frames of 24 x 40
    (BF16: activations recomputed in FP32, TUNE_TRAIN_RECOMPUTE = 0)."""
    B, H, W = 2, 24, 40
    frames = [synth.make_frame(H, W, 300 + b) for b in range(B)]
    wb = synth.make_weights(seed=9)
    d = wk.Denoiser(wb, precision=prec, max_batch=B, max_hw=(H, W))
    if prec == "bf16":
        from paper_2202_05977_b300 import _lib
        d.set_tuning(_lib.TUNE_TRAIN_RECOMPUTE, 0)
    dev = to_dev(stack_frames(frames))
    out, z = d.forward_train(*args(dev))
    G = np.random.default_rng(9).standard_normal((B, 3, H, W)).astype(np.float32)
    dw, dz = d.backward(*args(dev), z, torch.from_numpy(G).cuda(), want_dz=True)
    ref = np.zeros(wb.size)
    for b in range(B):
        o, acts = oracle.forward_train(frames[b], wb)
        gb, _ = oracle.backward_train(frames[b], wb, acts, G[b])
        ref += gb
    dw = dw.cpu().numpy()
    tol = TOL_GRAD if prec == "fp32" else 2e-2  # bf16: the saved z (hence dz) carries BF16 rounding
    off = 0
    for (ws, bs) in synth.weight_shapes():
        n = int(np.prod(ws)) + bs[0]
        assert _close(dw[off:off + n], ref[off:off + n], tol), (ws, off)
        off += n
    assert np.isfinite(dz.cpu().numpy()).all()


def test_training_backward_bf16_tensor_core_recompute(torch, wk):
    """The default BF16 training form (convolutions on the tensor cores,
    activations recomputed) against the oracle gradient of the network it
    computes: the same weights rounded to bfloat16 (oracle.bf16_weights,
    biases unchanged).  Per layer, every gradient element is within
    TOL_BF16_TRAIN of that layer's largest oracle gradient; the remaining
    error is the BF16 operands of the gradient GEMMs (one rounding of the
    activation and of the pre-activation gradient per product, 2^-9
    relative each; the gradient is carried between layers as BF16) and
    ReLU masks flipped by the activations' hi/lo rounding (measured per
    layer, 10-32 / 32-48 / 48-64 / 64-12: 6.3e-3, 5.9e-3, 8.6e-3, 1.03e-2 of
    the layer maximum; 0.55-0.75 % in L2)."""
    B, H, W = 2, 64, 96
    frames = [synth.make_frame(H, W, 310 + b) for b in range(B)]
    wb = synth.make_weights(seed=10)
    d = wk.Denoiser(wb, precision="bf16", max_batch=B, max_hw=(H, W))
    dev = to_dev(stack_frames(frames))
    out, z = d.forward_train(*args(dev))
    G = np.random.default_rng(10).standard_normal((B, 3, H, W)).astype(np.float32)
    dw, _ = d.backward(*args(dev), z, torch.from_numpy(G).cuda())
    wr = oracle.bf16_weights(wb)
    ref = np.zeros(wb.size)
    for b in range(B):
        o, acts = oracle.forward_train(frames[b], wr)
        gb, _ = oracle.backward_train(frames[b], wr, acts, G[b])
        ref += gb
    dw = dw.cpu().numpy().astype(np.float64)
    off = 0
    for (ws, bs) in synth.weight_shapes():
        n = int(np.prod(ws)) + bs[0]
        a, r = dw[off:off + n], ref[off:off + n]
        mx = np.abs(a - r).max() / np.abs(r).max()
        rel = np.linalg.norm(a - r) / np.linalg.norm(r)
        print(f"bf16 tc recompute {ws}: max rel (of layer max) {mx:.3e}, L2 rel {rel:.3e}")
        assert mx < TOL_BF16_TRAIN, (ws, mx)
        off += n
    assert d.device_status() == 0


def test_backward_reuses_kept_activations_only_for_the_same_frames(torch, wk):
    """wskpn_forward_train keeps the layer inputs of the BF16 tensor-core
    path; wskpn_backward reuses them for the same frame buffers and
    recomputes otherwise (WSKPN_TUNE_TRAIN_KEEP = 1).  The two give
    bit-identical gradients (the same kernels on the same values), the kept
    forward's z equals wskpn_logits', and a backward over other frames does
    not see the kept activations."""
    from paper_2202_05977_b300 import _lib
    B, H, W = 2, 48, 80
    wb = synth.make_weights(seed=13)
    d = wk.Denoiser(wb, precision="bf16", max_batch=B, max_hw=(H, W))
    d.set_tuning(_lib.TUNE_TRAIN_KEEP, 1)
    devA = to_dev(stack_frames([synth.make_frame(H, W, 340 + b) for b in range(B)]))
    devB = to_dev(stack_frames([synth.make_frame(H, W, 350 + b) for b in range(B)]))
    clone = lambda dev: {k: v.clone() for k, v in dev.items()}
    G = torch.from_numpy(np.random.default_rng(13).standard_normal((B, 3, H, W)).astype(np.float32)).cuda()
    out, z = d.forward_train(*args(devA))
    assert torch.equal(z, d.logits(*args(devA)))
    dw_kept, dz_kept = d.backward(*args(devA), z, G, want_dz=True)     # kept activations
    dw_re, dz_re = d.backward(*args(clone(devA)), z, G, want_dz=True)  # other pointers: recomputed
    assert torch.equal(dw_kept, dw_re) and torch.equal(dz_kept, dz_re)
    d.forward_train(*args(devA))
    dw_b = d.backward(*args(devB), z, G)[0]  # other frames: recomputed from B
    dw_b2 = d.backward(*args(clone(devB)), z, G)[0]
    assert torch.equal(dw_b, dw_b2) and not torch.equal(dw_b, dw_kept)
    assert d.device_status() == 0


@pytest.mark.parametrize("KS,six", [(5, False), (3, False), (5, True)])
def test_tensor_core_gradients_match_fp32(torch, wk, KS, six):
    """Input and weight gradients on the tensor cores (default) against the
    same backward with FP32 SIMT gradient kernels (TUNE_TRAIN_RECOMPUTE = 2):
    both recompute the same BF16 activations, so the ReLU masks agree and
    only BF16 rounding separates them (the gradients carried as BF16 and
    the transposed weights in the input gradients; layer inputs and
    gradients in the weight gradients; FP32 sums).  Every layer's weight
    gradient stays within 1e-2 in L2 and 2e-2 of its largest element
    (measured 2.3-7.5e-3 in L2, at most 9.2e-3 of the maximum); so do the
    inner layers' bias gradients, sums over the pixels of the same BF16-
    carried gradient (measured 2.1-8.0e-3 in L2, at most 1.02e-2 of the
    maximum, for the first layer of the 6-block network); the last layer's
    bias gradient (FP32 sums of the FP32 dL/dz) within 1e-4 (2 frames of 40
    x 200: two tile columns, ragged rows)."""
    from paper_2202_05977_b300 import _lib
    B, H, W = 2, 40, 200
    frames = [synth.make_frame(H, W, 320 + b) for b in range(B)]
    widths = (10, 32, 48, 64, 64, 64, 64, 12) if six else (10, 32, 48, 64, 12)
    wb = synth.make_weights(widths, KS, seed=11)
    d = wk.Denoiser(wb, precision="bf16", widths=widths, conv_ks=KS, max_batch=B, max_hw=(H, W))
    dev = to_dev(stack_frames(frames))
    out, z = d.forward_train(*args(dev))
    G = torch.from_numpy(np.random.default_rng(11).standard_normal((B, 3, H, W)).astype(np.float32)).cuda()
    dw_tc, _ = d.backward(*args(dev), z, G)
    d.set_tuning(_lib.TUNE_TRAIN_RECOMPUTE, 2)
    dw_fp, _ = d.backward(*args(dev), z, G)
    dw_tc = dw_tc.cpu().numpy().astype(np.float64)
    dw_fp = dw_fp.cpu().numpy().astype(np.float64)
    shapes = synth.weight_shapes(widths, KS)
    off = 0
    for i, (ws, bs) in enumerate(shapes):
        nw = int(np.prod(ws))
        a, r = dw_tc[off:off + nw], dw_fp[off:off + nw]
        rel = np.linalg.norm(a - r) / np.linalg.norm(r)
        mx = np.abs(a - r).max() / np.abs(r).max()
        print(f"tc gradients KS={KS} {ws}: L2 rel {rel:.3e}, max {mx:.3e}")
        assert rel < 1e-2 and mx < 2e-2, ws
        ab, rb = dw_tc[off + nw:off + nw + bs[0]], dw_fp[off + nw:off + nw + bs[0]]
        if i < len(shapes) - 1:
            brel = np.linalg.norm(ab - rb) / np.linalg.norm(rb)
            assert brel < 1e-2 and _close(ab, rb, 2e-2), (ws, "bias", brel)
        else:
            assert _close(ab, rb, 1e-4), (ws, "bias")
        off += nw + bs[0]
    assert d.device_status() == 0


@pytest.mark.parametrize("B,H,W", [(3, 1, 1), (1, 7, 3), (2, 33, 129)])
def test_tensor_core_gradients_edge_sizes(torch, wk, B, H, W):
    """The tensor-core input and weight gradients on degenerate and ragged
    sizes (every window and tap partly outside the image; a one-pixel last
    tile column) against the FP32 SIMT gradient kernels on the same
    recomputed activations: within 1e-2 in L2 and 2e-2 of the largest
    element per layer, as the inner layers' bias gradients; the last
    layer's (FP32 sums of the FP32 dL/dz) within 1e-4."""
    from paper_2202_05977_b300 import _lib
    frames = [synth.make_frame(H, W, 330 + b) for b in range(B)]
    wb = synth.make_weights(seed=12)
    d = wk.Denoiser(wb, precision="bf16", max_batch=B, max_hw=(H, W))
    dev = to_dev(stack_frames(frames))
    out, z = d.forward_train(*args(dev))
    G = torch.from_numpy(np.random.default_rng(12).standard_normal((B, 3, H, W)).astype(np.float32)).cuda()
    dw_tc, _ = d.backward(*args(dev), z, G)
    d.set_tuning(_lib.TUNE_TRAIN_RECOMPUTE, 2)
    dw_fp, _ = d.backward(*args(dev), z, G)
    dw_tc = dw_tc.cpu().numpy().astype(np.float64)
    dw_fp = dw_fp.cpu().numpy().astype(np.float64)
    off = 0
    shapes = synth.weight_shapes()
    for i, (ws, bs) in enumerate(shapes):
        nw = int(np.prod(ws))
        a, r = dw_tc[off:off + nw], dw_fp[off:off + nw]
        rel = np.linalg.norm(a - r) / max(np.linalg.norm(r), 1e-30)
        print(f"tc gradients {B}x{H}x{W} {ws}: L2 rel {rel:.3e}")
        assert rel < 1e-2 and _close(a, r, 2e-2), ws
        ab, rb = dw_tc[off + nw:off + nw + bs[0]], dw_fp[off + nw:off + nw + bs[0]]
        assert _close(ab, rb, 2e-2 if i < len(shapes) - 1 else 1e-4), (ws, "bias")
        off += nw + bs[0]
    assert np.isfinite(dw_tc).all()
    assert d.device_status() == 0


def test_l1_loss_and_gradient(torch, wk):
    g = np.random.default_rng(5)
    o = g.lognormal(0, 1, (2, 3, 17, 29)).astype(np.float32)
    t = g.lognormal(0, 1, (2, 3, 17, 29)).astype(np.float32)
    d = wk.Denoiser(synth.make_weights(seed=0), precision="fp32", max_hw=(8, 8))
    loss, grad = d.l1_loss(torch.from_numpy(o).cuda(), torch.from_numpy(t).cuda())
    L, G = oracle.l1_loss(o, t)
    assert abs(loss.item() - L) <= 1e-6 * L
    np.testing.assert_allclose(grad.cpu().numpy(), G, rtol=1e-6)


def test_adam_steps_match_oracle(torch, wk):
    wb = synth.make_weights(seed=3)
    d = wk.Denoiser(wb, precision="fp32", max_hw=(8, 8))
    w, m, v = wb.astype(np.float64), np.zeros(wb.size), np.zeros(wb.size)
    for step in range(1, 4):
        g = np.random.default_rng(step).standard_normal(wb.size).astype(np.float32) * 1e-2
        d.adam_step(torch.from_numpy(g).cuda(), step, lr=1e-3)
        w, m, v = oracle.adam_step(w, g, m, v, step, lr=1e-3)
    got = d.get_weights().cpu().numpy()
    assert np.abs(got - w).max() < 1e-6


def test_autograd_decode_fuse_matches_kernel_and_fd(torch, wk):
    from paper_2202_05977_b300.autograd import decode_fuse
    H, W = 30, 50
    f = synth.make_frame(H, W, 8)
    dev = to_dev(stack_frames([f]))
    g = np.random.default_rng(8)
    z = torch.from_numpy(g.standard_normal((1, 12, H, W)).astype(np.float32)).cuda().requires_grad_()
    G = torch.from_numpy(g.standard_normal((1, 3, H, W)).astype(np.float32)).cuda()
    (decode_fuse(z, dev["radiance"], dev["albedo"]) * G).sum().backward()
    ref = wk.decode_fuse_bwd(z.detach(), dev["radiance"], dev["albedo"], G)
    assert torch.equal(z.grad, ref)
    # directional derivative, central difference in FP32
    v = torch.from_numpy(g.standard_normal((1, 12, H, W)).astype(np.float32)).cuda()
    h = 1e-2
    fp = (wk.decode_fuse_fwd(z.detach() + h * v, dev["radiance"], dev["albedo"]) * G).sum().item()
    fm = (wk.decode_fuse_fwd(z.detach() - h * v, dev["radiance"], dev["albedo"]) * G).sum().item()
    fd = (fp - fm) / (2 * h)
    an = (z.grad * v).sum().item()
    assert abs(fd - an) <= 1e-2 * abs(an) + 1e-3


def test_training_step_256_crops(torch, wk):
    """Differentiation form: 16 crops of 256 x 256, BF16 forward, L1 against
    the mean of 256 noise draws, backward, Adam; the loss is finite and one
    small step along -grad lowers it."""
    B, H, W = 16, 256, 256
    b = synth.make_batch(B, H, W, seed=5)
    target = synth.make_target(b["clean"], seed=5, draws=256)
    wb = synth.make_weights(seed=5)
    d = wk.Denoiser(wb, precision="bf16", max_batch=B, max_hw=(H, W))
    dev = to_dev(b)
    tg = torch.from_numpy(target).cuda()
    out, z = d.forward_train(*args(dev))
    loss0, dout = d.l1_loss(out, tg)
    dw, _ = d.backward(*args(dev), z, dout)
    assert np.isfinite(dw.cpu().numpy()).all() and np.isfinite(loss0.item())
    d.adam_step(dw, 1, lr=1e-4)
    out1, _ = d.forward_train(*args(dev))
    loss1, _ = d.l1_loss(out1, tg, want_grad=False)
    assert loss1.item() < loss0.item()
    assert d.device_status() == 0
