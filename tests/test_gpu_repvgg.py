"""RepVGG fold (Sec. 4.1) on the GPU against the oracle's fold, and the
folded weights running through the denoiser equal to the oracle's
multi-branch network."""
import numpy as np
import pytest

import oracle
import synth
from tests._util import args, rel_err, stack_frames, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("ci,co,identity", [(10, 32, False), (48, 48, True)])
def test_fold_and_grad_match_oracle(ci, co, identity):
    import torch
    from paper_2202_05977_b300 import repvgg
    g = np.random.default_rng(ci + co)
    ws = [g.standard_normal(s).astype(np.float32) for s in ((co, ci, 5, 5), (co,), (co, ci, 3, 3), (co,),
                                                             (co, ci, 1, 1), (co,))]
    W, b = repvgg.fold(*(torch.from_numpy(w).cuda() for w in ws), identity=identity)
    Wr, br = oracle.repvgg_fold(*ws, identity)
    np.testing.assert_allclose(W.cpu().numpy(), Wr, rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(b.cpu().numpy(), br, rtol=1e-6, atol=1e-6)
    gW = g.standard_normal((co, ci, 5, 5)).astype(np.float32)
    for got, ref in zip(repvgg.fold_grad(torch.from_numpy(gW).cuda()), oracle.repvgg_fold_grad(gW)):
        np.testing.assert_array_equal(got.cpu().numpy(), ref.astype(np.float32))


def test_folded_network_denoises_like_the_branch_network():
    import torch
    import paper_2202_05977_b300 as wk
    from paper_2202_05977_b300 import repvgg
    f = synth.make_frame(40, 56, 3)
    widths = (10, 32, 48, 64, 12)
    g = np.random.default_rng(3)
    blob = []
    for l in range(4):
        ci, co = widths[l], widths[l + 1]
        br = [(g.standard_normal(s) * sc).astype(np.float32) for s, sc in
              (((co, ci, 5, 5), 0.3 / np.sqrt(25 * ci)), ((co,), 0.05), ((co, ci, 3, 3), 0.3 / np.sqrt(9 * ci)),
               ((co,), 0.05), ((co, ci, 1, 1), 0.3 / np.sqrt(ci)), ((co,), 0.05))]
        W, b = repvgg.fold(*(torch.from_numpy(x).cuda() for x in br))
        blob += [W.cpu().numpy().ravel(), b.cpu().numpy()]
    wb = np.concatenate(blob)
    out = wk.Denoiser(wb, precision="fp32", max_hw=(40, 56)).denoise(*args(to_dev(stack_frames([f])))).cpu().numpy()[0]
    assert rel_err(out, oracle.denoise(f, wb))[0] < 1e-5
