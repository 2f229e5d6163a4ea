"""Differentiable 3-D transform.

The forward transform Y = F X (unnormalised, exp(-2 pi i jk/n)) is linear; its
adjoint F^H is the unnormalised conjugate-direction transform, so the
backward of a real loss receives dL/dY* and returns F^H (dL/dY*), which is
the library's inverse transform (dir = +1) of the incoming gradient.  Both
directions run through the same C ABI and kernels.
"""
from __future__ import annotations

import torch

from .api import _as_batched, _cached_plan


class ObFFT3(torch.autograd.Function):
    """Y = fft3(X) on the last three axes ([n0,n1,n2] or [batch,n0,n1,n2])."""

    @staticmethod
    def forward(ctx, x: torch.Tensor, mode: str = "fp8") -> torch.Tensor:
        ctx.mode = mode
        xb, squeeze = _as_batched(x.contiguous())
        ctx.squeeze = squeeze
        y = _cached_plan(xb.shape, mode).exec(xb, dir=-1)
        return y[0] if squeeze else y

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        gb, squeeze = _as_batched(g.contiguous())
        gx = _cached_plan(gb.shape, ctx.mode).exec(gb, dir=+1)
        return (gx[0] if squeeze else gx), None


def fft3_autograd(x: torch.Tensor, mode: str = "fp8") -> torch.Tensor:
    return ObFFT3.apply(x, mode)
