"""torch.autograd.Function wrappers over the C ABI (marshalling only).

DecodeFuse:  out = reconstruction(z, radiance, albedo)   (Eq. 3-5), with the
             hand-written backward kernel for dL/dz.
DenoiseNet:  out = D_Theta(r, f) as a function of the flat weight blob Theta
             (Eq. 1), backward through the reconstruction and the
             convolutions with activations recomputed.
"""
from __future__ import annotations

import torch

from . import decode_fuse_bwd, decode_fuse_fwd


class DecodeFuse(torch.autograd.Function):
    @staticmethod
    def forward(ctx, z, radiance, albedo, ksizes=(3, 5, 7, 9, 11, 13), eps=1e-2):
        z, radiance, albedo = z.contiguous(), radiance.contiguous(), albedo.contiguous()
        ctx.save_for_backward(z, radiance, albedo)
        ctx.ksizes, ctx.eps = tuple(ksizes), float(eps)
        return decode_fuse_fwd(z, radiance, albedo, ctx.ksizes, ctx.eps)

    @staticmethod
    def backward(ctx, dout):
        z, radiance, albedo = ctx.saved_tensors
        dz = decode_fuse_bwd(z, radiance, albedo, dout.contiguous(), ctx.ksizes, ctx.eps)
        return dz, None, None, None, None


class DenoiseNet(torch.autograd.Function):
    """apply(weights, radiance, albedo, normal, depth, denoiser) -> out.
    `weights` is a float32 CUDA tensor with the blob layout; the denoiser's
    weights are set from it on every forward."""

    @staticmethod
    def forward(ctx, weights, radiance, albedo, normal, depth, den):
        den.set_weights(weights.detach().contiguous())
        xs = [t.contiguous() for t in (radiance, albedo, normal, depth)]
        out, z = den.forward_train(*xs)
        ctx.save_for_backward(z, *xs)
        ctx.den = den
        return out

    @staticmethod
    def backward(ctx, dout):
        z, *xs = ctx.saved_tensors
        dw, _ = ctx.den.backward(*xs, z, dout.contiguous())
        return dw, None, None, None, None, None


def decode_fuse(z, radiance, albedo, ksizes=(3, 5, 7, 9, 11, 13), eps=1e-2):
    return DecodeFuse.apply(z, radiance, albedo, tuple(ksizes), eps)


def denoise_net(weights, radiance, albedo, normal, depth, den):
    return DenoiseNet.apply(weights, radiance, albedo, normal, depth, den)
