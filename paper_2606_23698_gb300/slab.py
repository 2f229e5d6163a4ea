"""Slab decomposition of one 3-D transform over several processes, one GPU each.

The paper describes a single-GPU transform only.  A grid too large for one
GPU is split along n0: rank r holds the slab of planes
[r n0/R, (r + 1) n0/R) in the natural layout [n0/R][n1][n2].

  1. local passes over axes 2 and 1 of the slab (obfft_exec_axes(2, 1)),
     which leave it as [n1][n2][n0/R]: T = n1 n2 lines (t = k1 n2 + k2), each
     holding this rank's n0/R values of axis 0;
  2. one all-to-all: the slab's lines split into R contiguous chunks of T/R
     lines, chunk s goes to rank s (NCCL on the GPU tensors, or staged
     through host memory over any torch.distributed backend);
  3. the received [R][T/R][n0/R] blocks are regrouped into T/R full lines of
     n0 values (obfft_transpose_blocks);
  4. the pass over axis 0 of those lines (obfft_exec_axes(2, 2) of a
     1 x (T/R) x n0 plan), which writes them rotated: [n0][T/R].

Result distribution: rank r holds Y[k0][t] for t in [r T/R, (r + 1) T/R),
t = k1 n2 + k2, as an [n0][T/R] array.  Each line is transformed by the same
kernels, splits and per-column scales as in the single-GPU transform, so the
gathered result is bit-identical to it.

Requirements: n0 and n1 n2 divisible by the number of ranks.
"""
from __future__ import annotations

import torch

from . import _lib
from .api import Plan


def slab_geometry(n0: int, n1: int, n2: int, world: int) -> dict:
    """Sizes of the decomposition: planes per rank, lines T and lines per rank."""
    if world < 1 or n0 % world or (n1 * n2) % world:
        raise ValueError(f"slab decomposition of {n0}x{n1}x{n2} over {world} ranks needs n0 and n1*n2 "
                         f"divisible by {world}")
    return {"n0_local": n0 // world, "lines": n1 * n2, "lines_local": n1 * n2 // world}


def exchange(send: torch.Tensor, world: int, how: str = "nccl", group=None) -> torch.Tensor:
    """All-to-all of `world` equal contiguous chunks of `send` (chunk s to rank s);
    returns the received chunks, chunk s from rank s, on send's device.
    how = "nccl": the device tensors go to the collective directly;
    how = "host": the data are staged through host memory (for backends
    without GPU support, e.g. gloo)."""
    import torch.distributed as dist
    flat = torch.view_as_real(send).reshape(-1) if send.is_complex() else send.reshape(-1)
    if how == "host":
        hs = flat.cpu()
        hr = torch.empty_like(hs)
        dist.all_to_all_single(hr, hs, group=group)
        recv = hr.to(send.device)
    elif how == "nccl":
        recv = torch.empty_like(flat)
        dist.all_to_all_single(recv, flat, group=group)
    else:
        raise ValueError(f"unknown exchange {how!r}")
    if send.is_complex():
        return torch.view_as_complex(recv.reshape(*send.shape, 2))
    return recv.reshape(send.shape)


class SlabPlan:
    """One n0 x n1 x n2 transform split over `world` ranks (this process is
    `rank`, on the current CUDA device).  exec() takes this rank's input slab
    [n0/R][n1][n2] and returns its part [n0][T/R] of the result."""

    def __init__(self, n0: int, n1: int, n2: int, world: int, rank: int, mode="fp8", how: str = "nccl",
                 group=None):
        g = slab_geometry(n0, n1, n2, world)
        self.n = (n0, n1, n2)
        self.world, self.rank, self.how, self.group = world, rank, how, group
        self.n0l, self.T, self.Tl = g["n0_local"], g["lines"], g["lines_local"]
        self.local = Plan(self.n0l, n1, n2, mode=mode)   # passes over axes 2 and 1
        self.lines = Plan(1, self.Tl, n0, mode=mode)     # the pass over axis 0 (its axis 2)
        self.dtype = self.local.dtype

    def exec(self, x: torch.Tensor, dir: int = -1) -> torch.Tensor:
        n0, n1, n2 = self.n
        if x.shape != (self.n0l, n1, n2) or x.dtype != self.dtype or not x.is_cuda or not x.is_contiguous():
            raise ValueError(f"input slab must be a contiguous CUDA {self.dtype} tensor of shape "
                             f"{(self.n0l, n1, n2)}")
        s = torch.cuda.current_stream(x.device).cuda_stream
        a = torch.empty((n1, n2, self.n0l), dtype=self.dtype, device=x.device)
        _lib.obfft_exec_axes(self.local.handle, 2, 1, x.data_ptr(), a.data_ptr(), dir, s)
        recv = exchange(a.reshape(self.world, self.Tl, self.n0l), self.world, self.how, self.group)
        b = torch.empty((self.Tl, n0), dtype=self.dtype, device=x.device)
        _lib.obfft_transpose_blocks(recv.data_ptr(), b.data_ptr(), self.world, self.Tl,
                                    self.n0l * b.element_size(), s)
        y = torch.empty((n0, self.Tl), dtype=self.dtype, device=x.device)
        _lib.obfft_exec_axes(self.lines.handle, 2, 2, b.data_ptr(), y.data_ptr(), dir, s)
        return y

    def close(self):
        self.local.close()
        self.lines.close()
