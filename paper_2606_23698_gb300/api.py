"""torch-tensor layer over the C ABI: plans as objects, tensors as pointers.

Only argument marshalling: the transform itself runs in libobfft.so, on the
GPU.  exec / exec_stage take contiguous CUDA tensors (complex128, or complex64
for the FP32-precision modes "fp32" and "fp32native"); exec_host takes host
tensors, which the library copies to and from the GPU around (and overlapped
with) the same GPU transform.  No CPU compute path exists.
"""
from __future__ import annotations

import torch

from . import _lib


def _mode(mode) -> int:
    if isinstance(mode, str):
        return _lib.MODES[mode]
    return int(mode)


def dtype_of(mode) -> torch.dtype:
    """Element type of a mode's data: complex64 for the FP32-precision modes."""
    return torch.complex64 if _mode(mode) in _lib.COMPLEX64_MODES else torch.complex128


def _check_tensor(t: torch.Tensor, numel: int, name: str, dtype=torch.complex128) -> None:
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (no CPU path)")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, plan needs {numel}")


class Plan:
    """batch x n0 x n1 x n2 transform plan on the current CUDA device (complex128
    data, complex64 for the FP32-precision modes)."""

    def __init__(self, n0: int, n1: int, n2: int, batch: int = 1, mode="fp8"):
        self.shape = (batch, n0, n1, n2)
        self.mode = _mode(mode)
        self.dtype = dtype_of(self.mode)
        self.device = torch.cuda.current_device()
        self.handle = _lib.obfft_plan_create(n0, n1, n2, batch, self.mode)

    @property
    def numel(self) -> int:
        b, n0, n1, n2 = self.shape
        return b * n0 * n1 * n2

    def splits(self, axis: int, grid: int = 0):
        return _lib.obfft_plan_get_splits(self.handle, grid, axis)

    def exec(self, x: torch.Tensor, out: torch.Tensor | None = None, dir: int = -1,
             stream: torch.cuda.Stream | None = None) -> torch.Tensor:
        _check_tensor(x, self.numel, "input", self.dtype)
        if out is None:
            out = torch.empty_like(x)
        _check_tensor(out, self.numel, "output", self.dtype)
        s = stream if stream is not None else torch.cuda.current_stream(x.device)
        _lib.obfft_exec(self.handle, x.data_ptr(), out.data_ptr(), dir, s.cuda_stream)
        return out

    def exec_host(self, x: torch.Tensor, out: torch.Tensor | None = None, dir: int = -1,
                  stream: torch.cuda.Stream | None = None) -> torch.Tensor:
        """Host-to-host transform (obfft_exec_host): x and out are contiguous
        CPU tensors of the plan's dtype, ideally pinned; the copies overlap the
        transform.  The output is complete once `stream` (default: current) is
        synchronised."""
        if x.device.type != "cpu" or x.dtype != self.dtype or not x.is_contiguous() \
                or x.numel() != self.numel:
            raise ValueError(f"input must be a contiguous {self.dtype} CPU tensor of {self.numel} elements")
        if out is None:
            out = torch.empty(x.shape, dtype=x.dtype, pin_memory=x.is_pinned())
        if out.device.type != "cpu" or out.dtype != self.dtype or not out.is_contiguous() \
                or out.numel() != self.numel:
            raise ValueError(f"output must be a contiguous {self.dtype} CPU tensor of {self.numel} elements")
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        _lib.obfft_exec_host(self.handle, x.data_ptr(), out.data_ptr(), dir, s.cuda_stream)
        return out

    def exec_stage(self, axis: int, stage: int, x: torch.Tensor, out: torch.Tensor, dir: int = -1):
        _check_tensor(x, self.numel, "input", self.dtype)
        _check_tensor(out, self.numel, "output", self.dtype)
        s = torch.cuda.current_stream(x.device)
        _lib.obfft_exec_stage(self.handle, axis, stage, x.data_ptr(), out.data_ptr(), dir,
                              s.cuda_stream)
        return out

    def close(self):
        if getattr(self, "handle", None):
            _lib.obfft_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PlanMany:
    """Independent grids of possibly different sizes, transformed together."""

    def __init__(self, dims, mode="fp8"):
        self.dims = [tuple(int(v) for v in d) for d in dims]
        self.mode = _mode(mode)
        self.dtype = dtype_of(self.mode)
        self.handle = _lib.obfft_plan_create_many(self.dims, self.mode)

    def exec(self, xs, outs=None, dir: int = -1, stream=None):
        if outs is None:
            outs = [torch.empty_like(x) for x in xs]
        for x, o, d in zip(xs, outs, self.dims):
            n = d[0] * d[1] * d[2]
            _check_tensor(x, n, "input", self.dtype)
            _check_tensor(o, n, "output", self.dtype)
        s = stream if stream is not None else torch.cuda.current_stream(xs[0].device)
        _lib.obfft_exec_many(self.handle, [x.data_ptr() for x in xs], [o.data_ptr() for o in outs],
                             dir, s.cuda_stream)
        return outs

    def close(self):
        if getattr(self, "handle", None):
            _lib.obfft_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_plan_cache: dict = {}


def _cached_plan(shape, mode) -> Plan:
    key = (tuple(shape), _mode(mode), torch.cuda.current_device())
    p = _plan_cache.get(key)
    if p is None:
        b, n0, n1, n2 = shape
        p = Plan(n0, n1, n2, b, mode)
        _plan_cache[key] = p
    return p


def _as_batched(x: torch.Tensor):
    if x.dim() == 3:
        return x.unsqueeze(0), True
    if x.dim() == 4:
        return x, False
    raise ValueError("expected [n0, n1, n2] or [batch, n0, n1, n2]")


def fft3(x: torch.Tensor, mode="fp8") -> torch.Tensor:
    """Forward 3-D transform of the last three axes (unnormalised)."""
    xb, squeeze = _as_batched(x.contiguous())
    y = _cached_plan(xb.shape, mode).exec(xb, dir=-1)
    return y[0] if squeeze else y


def ifft3(x: torch.Tensor, mode="fp8") -> torch.Tensor:
    """Unnormalised inverse (conjugate-direction) 3-D transform."""
    xb, squeeze = _as_batched(x.contiguous())
    y = _cached_plan(xb.shape, mode).exec(xb, dir=+1)
    return y[0] if squeeze else y
