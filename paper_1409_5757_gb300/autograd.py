"""Differentiable DFT: forward is the in-place transform on a copy, backward
is the adjoint, i.e. the conjugate-sign unnormalised transform, run by the
same kernels (no separate code path).

For X = F x with F[k, n] = exp(sign*2*pi*i*n*k/N), PyTorch's complex
autograd passes the upstream gradient g = dL/dX* and expects F^H g back;
F is symmetric, so F^H = conj(F), the transform with the opposite sign.
For the loss L = sum_k |w_k X_k|^2 this gives grad_x = 2 F^H (|w|^2 X).
"""
from __future__ import annotations

import torch

from . import EFFT_FLAG_NORMALIZE, fft_, fft_batch_


class _DFT(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, sign: int, normalize: bool):
        ctx.sign = sign
        ctx.normalize = normalize
        y = x.contiguous().clone()
        fft_(y, sign, EFFT_FLAG_NORMALIZE if normalize else 0)
        return y

    @staticmethod
    def backward(ctx, g):
        gx = g.contiguous().clone()
        # adjoint of (1/N) F is (1/N) F^H: same flag, opposite sign
        fft_(gx, -ctx.sign, EFFT_FLAG_NORMALIZE if ctx.normalize else 0)
        return gx, None, None


class _BatchDFT(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sign: int, normalize: bool, *xs):
        ctx.sign = sign
        ctx.normalize = normalize
        ctx.like = [torch.empty(0, dtype=x.dtype, device=x.device) for x in xs]
        ctx.shapes = [x.shape for x in xs]
        ys = [x.contiguous().clone() for x in xs]
        fft_batch_(ys, sign, EFFT_FLAG_NORMALIZE if normalize else 0)
        return tuple(ys)

    @staticmethod
    def backward(ctx, *gs):
        # an output that did not reach the loss has no gradient: zeros
        gx = [g.contiguous().clone() if g is not None else l.new_zeros(sh)
              for g, l, sh in zip(gs, ctx.like, ctx.shapes)]
        fft_batch_(gx, -ctx.sign, EFFT_FLAG_NORMALIZE if ctx.normalize else 0)
        return (None, None, *gx)


def dft(x: torch.Tensor, sign: int = -1, normalize: bool = False) -> torch.Tensor:
    """Out-of-place, differentiable X = F x (1-D contiguous CUDA complex tensor)."""
    return _DFT.apply(x, sign, normalize)


def dft_batch(xs, sign: int = -1, normalize: bool = False) -> list:
    """Differentiable DFTs of a list of 1-D CUDA complex tensors (mixed
    supported lengths, one dtype) by one batch execute forward and one
    (opposite sign) backward."""
    return list(_BatchDFT.apply(sign, normalize, *xs))


__all__ = ["dft", "dft_batch"]
