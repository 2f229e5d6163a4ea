"""Seeded synthetic inputs shared by the tests, the oracle checks and the benchmark.

This module holds no arithmetic of the transform itself: it only turns
(seed, stream, index) triples into numbers.  The generator is counter based
(splitmix64 of a Weyl sequence, S. Vigna's published definition), so any
element can be regenerated independently, on the host or on the device, and
the same call gives the same bits on CPU and CUDA.

Streams: every distinct random quantity (real part, imaginary part, magnitude,
phase, ...) draws from its own stream so that changing one recipe never shifts
another.  The counter of element i in stream s is  s * 2**40 + i.
"""
from __future__ import annotations

import math

import torch

GOLDEN = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1


def _i64(v: int) -> int:
    """Two's complement view of an unsigned 64-bit constant."""
    v &= MASK64
    return v - (1 << 64) if v >= (1 << 63) else v


def _lsr(x: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of int64 tensors (torch's >> is arithmetic)."""
    return (x >> k) & ((1 << (64 - k)) - 1)


def splitmix64(seed: int, counters: torch.Tensor) -> torch.Tensor:
    """splitmix64 output for state seed + (counter + 1) * golden, as int64 bits."""
    z = counters.to(torch.int64) + 1
    z = z * _i64(GOLDEN) + _i64(seed)
    z = (z ^ _lsr(z, 30)) * _i64(MIX1)
    z = (z ^ _lsr(z, 27)) * _i64(MIX2)
    return z ^ _lsr(z, 31)


def splitmix64_scalar(seed: int, counter: int) -> int:
    """Pure-integer reference of one draw (used to pin the tensor version)."""
    z = (seed + (counter + 1) * GOLDEN) & MASK64
    z = ((z ^ (z >> 30)) * MIX1) & MASK64
    z = ((z ^ (z >> 27)) * MIX2) & MASK64
    return z ^ (z >> 31)


def uniform01(seed: int, stream: int, n: int, device="cpu", offset: int = 0) -> torch.Tensor:
    """n doubles in [0, 1): (bits >> 11) * 2**-53."""
    idx = torch.arange(offset, offset + n, dtype=torch.int64, device=device) + stream * (1 << 40)
    bits = _lsr(splitmix64(seed, idx), 11)
    return bits.to(torch.float64) * (2.0 ** -53)


def uniform_pm1(seed: int, stream: int, n: int, device="cpu", offset: int = 0) -> torch.Tensor:
    """n doubles in [-1, 1)."""
    return uniform01(seed, stream, n, device, offset) * 2.0 - 1.0


def complex_uniform(seed: int, shape, device="cpu") -> torch.Tensor:
    """Real and imaginary parts i.i.d. uniform[-1, 1)."""
    n = math.prod(shape)
    re = uniform_pm1(seed, 0, n, device)
    im = uniform_pm1(seed, 1, n, device)
    return torch.complex(re, im).reshape(shape)


def complex_wide_range(seed: int, shape, lo_exp: float = -30.0, hi_exp: float = 30.0,
                       device="cpu") -> torch.Tensor:
    """Magnitude 2**U(lo_exp, hi_exp) (log-uniform), phase uniform[0, 2*pi)."""
    n = math.prod(shape)
    u = uniform01(seed, 0, n, device)
    ph = uniform01(seed, 1, n, device) * (2.0 * math.pi)
    mag = torch.exp2(lo_exp + (hi_exp - lo_exp) * u)
    return torch.polar(mag, ph).reshape(shape)


def complex_gaussian(seed: int, shape, device="cpu") -> torch.Tensor:
    """Real and imaginary parts N(0, 1) by Box-Muller on two uniform streams."""
    n = math.prod(shape)
    u1 = 1.0 - uniform01(seed, 0, n, device)  # (0, 1]
    u2 = uniform01(seed, 1, n, device)
    rad = torch.sqrt(-2.0 * torch.log(u1))
    return torch.polar(rad, 2.0 * math.pi * u2).reshape(shape)


def spectral_mask(seed: int, shape, device="cpu") -> torch.Tensor:
    """Magnitude uniform[0, 1), phase uniform[0, 2*pi) (the autograd loss weights)."""
    n = math.prod(shape)
    mag = uniform01(seed, 2, n, device)
    ph = uniform01(seed, 3, n, device) * (2.0 * math.pi)
    return torch.polar(mag, ph).reshape(shape)


# Seeds of the five workloads (forward 64^3, wide-range 256^3, 1024^3,
# uneven batch, autograd 8 x 128^3).
SEED_64 = 20260001
SEED_256_WIDE = 20260002
SEED_1024 = 20260003
SEED_UNEVEN = 20260004
SEED_GRAD = 20260005

UNEVEN_BATCH = ([(64, 64, 64)] * 16 + [(96, 128, 128)] * 12 + [(192, 192, 192)] * 8
                + [(256, 256, 384)] * 4)
