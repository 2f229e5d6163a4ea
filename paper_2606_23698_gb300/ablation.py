"""Epilogue ablation driver: synthetic inputs and timing of the exact
alternative forms of the Phase-B Kulisch accumulator (word widths 32, 16, 8
against the stage kernels' grouped 64-bit form) and of the deconstruction
residues (pieces + Barrett, dp4a, 64-bit remainder, dp4a + H0 fold-and-add); see
obfft_ablation_phase_b / obfft_ablation_residues in include/obfft.h.

Inputs are built with the library's own CRT constants (obfft_host_crt_constants)
from seeded random offset residues, so that they have the structure of real
Phase-A accumulators.  Everything timed runs in the library's kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib

PHASE_B_VARIANTS = (0, 32, 16, 8)
RESIDUE_VARIANTS = (0, 1, 2, 3)


def crt_constants():
    L = _lib.load()
    mods = (ctypes.c_uint32 * 12)()
    us = (ctypes.c_uint8 * 180)()
    ws = (ctypes.c_uint8 * 72)()
    M4 = (ctypes.c_uint32 * 4)()
    _lib.check(L.obfft_host_crt_constants(mods, us, ws, M4))
    u = np.array(us, np.int64).reshape(12, 15)
    w = np.array(ws, np.int64).reshape(12, 6)
    return np.array(mods, np.int64), u, w


def phase_b_inputs(n: int, seed: int = 1, et: int = -104):
    """Accumulators (uint32 [n][21], FP32 bit patterns 2^23 + P) of n outputs
    with uniformly random offset residues in [2, 2046] below each modulus' range."""
    mods, u, w = crt_constants()
    rng = np.random.default_rng(seed)
    v = 1024 + rng.integers(-(mods // 2), mods // 2 + 1, (n, 12))
    acc = np.concatenate([v @ u, v @ w], axis=1) + 0x4B000000
    return acc.astype(np.uint32), np.full(n, et, np.int32)


def residue_inputs(n: int, seed: int = 2):
    rng = np.random.default_rng(seed)
    return rng.integers(-(2 ** 53) + 1, 2 ** 53, n, dtype=np.int64)


def _time(fn, reps=3):
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def measure(n_unique: int = 1 << 18, n_total: int = 1 << 24, reps: int = 16):
    """ns per item and items per second of every variant: n_total items from
    n_unique L2-resident inputs, each computed `reps` times (perturbed), so the
    launches are bound by the arithmetic."""
    acc, et = phase_b_inputs(n_unique)
    dacc = torch.from_numpy(acc.view(np.int32)).cuda()
    det = torch.from_numpy(et).cuda()
    ck = torch.zeros(1, dtype=torch.int64, device="cuda")
    out = {"n_unique": n_unique, "n_total": n_total, "reps": reps, "phase_b": {}, "residues": {}}
    for v in PHASE_B_VARIANTS:
        ms = _time(lambda: _lib.obfft_ablation_phase_b(v, n_unique, n_total, dacc.data_ptr(), det.data_ptr(),
                                                       None, ck.data_ptr(), reps=reps))
        n = n_total * reps
        out["phase_b"][str(v)] = {"ns_per_output": ms * 1e6 / n, "G_outputs_per_s": n / ms / 1e6}
    xt = torch.from_numpy(residue_inputs(n_unique)).cuda()
    for v in RESIDUE_VARIANTS:
        ms = _time(lambda: _lib.obfft_ablation_residues(v, n_unique, n_total, xt.data_ptr(), None, ck.data_ptr(),
                                                        reps=reps))
        n = n_total * reps
        out["residues"][str(v)] = {"ns_per_element": ms * 1e6 / n, "G_elements_per_s": n / ms / 1e6}
    return out
