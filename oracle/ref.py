"""Python driver of the CPU oracle (ctypes over ozaki_ref.c plus numpy glue).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and
bench.py's CPU-baseline / reference legs, never by the product path.

Index conventions follow the paper's Bailey paragraph: for a line of length
N = p q, input index j = j1 + p j2 and output index k = k2 + q k1.  Stage 1 is
the length-q DFT over j2 (matrix F_q), stage 2 the length-p DFT over j1 with
the twiddle fused into the per-k2 matrices F_p^(k2) (Eq. twiddle-fusion).  A
3-D grid [n0][n1][n2] is transformed axis 2 first, then axis 1, then axis 0.
Forward uses omega = exp(-2 pi i / N); the inverse is the unnormalised
conjugate transform.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from functools import lru_cache

import numpy as np

from . import constants as C

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ozaki_ref.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the C oracle in place (plain gcc, portable: x86-64 and aarch64)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-shared",
               "-fPIC", SRC, "-o", LIB + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(LIB + ".tmp", LIB)
    return LIB


class _Consts(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64 * 12),
                ("us", (ctypes.c_uint8 * 15) * 12),
                ("ws", (ctypes.c_uint8 * 6) * 12),
                ("M", ctypes.c_uint32 * 4)]


class _Consts32(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64 * 6),
                ("us", (ctypes.c_uint8 * 8) * 6),
                ("ws", (ctypes.c_uint8 * 3) * 6),
                ("M", ctypes.c_uint64)]


class _Dump32(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("v", "P", "Q", "zhat", "R", "col_exp", "xt")]


class _Dump(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in
                ("col_exp", "xt", "def_", "v", "P", "Q", "zhat", "Rlimbs")]


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


@lru_cache(maxsize=1)
def lib():
    L = ctypes.CDLL(build())
    L.ob_ref_stage.restype = ctypes.c_int64
    L.ob_ref_stage.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                               ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(_Consts),
                               ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(_Dump)]
    L.ob_ref_stage32.restype = ctypes.c_int64
    L.ob_ref_stage32.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(_Consts32),
                                 ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(_Dump32)]
    L.ob_ref_pack32.restype = ctypes.c_float
    L.ob_ref_pack32.argtypes = [ctypes.c_int64, ctypes.c_int]
    L.ob_ref_pack.restype = ctypes.c_double
    L.ob_ref_pack.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int]
    L.ob_ref_kulisch.restype = None
    L.ob_ref_kulisch.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.POINTER(_Consts), ctypes.c_void_p, ctypes.c_void_p]
    L.ob_ref_dft_dd_axis.restype = None
    L.ob_ref_dft_dd_axis.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p]
    L.ob_ref_fft_lines.restype = None
    L.ob_ref_fft_lines.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p]
    L.ob_ref_dft_dd_point.restype = None
    L.ob_ref_dft_dd_point.argtypes = [ctypes.c_int] * 3 + [ctypes.c_void_p] * 4 + \
        [ctypes.c_int] * 3 + [ctypes.c_void_p]
    return L


def consts(moduli=C.MODULI) -> _Consts:
    c = _Consts()
    Mp = C.modulus_product(moduli)
    us = [C.byte_slices(u, C.S_RAW) for u in C.idempotents(moduli)]
    ws = [C.byte_slices(w, C.S_FRAC) for w in C.lift_weights(moduli)]
    for k, m in enumerate(moduli):
        c.m[k] = m
        for s in range(C.S_RAW):
            c.us[k][s] = us[k][s]
        for t in range(C.S_FRAC):
            c.ws[k][t] = ws[k][t]
    for i in range(4):
        c.M[i] = (Mp >> (32 * i)) & 0xFFFFFFFF
    return c


def consts32() -> _Consts32:
    c = _Consts32()
    for k, m in enumerate(C.MODULI_FP32):
        c.m[k] = m
        for s_ in range(C.S_RAW_FP32):
            c.us[k][s_] = C.U_SLICES_FP32[k][s_]
        for t in range(C.S_FRAC_FP32):
            c.ws[k][t] = C.W_SLICES_FP32[k][t]
    c.M = C.M_FP32
    return c


# Per-precision parameters: numpy complex type and the constants' scale exponent.
PRECISIONS = {"fp64": (np.complex128, C.SIGMA_F_EXP), "fp32": (np.complex64, C.SIGMA_F_EXP_FP32)}


# --------------------------------------------------------------------------
# Tables
# --------------------------------------------------------------------------
@lru_cache(maxsize=None)
def table_q(q: int, sign: int, scale_exp: int = C.SIGMA_F_EXP) -> np.ndarray:
    """F_q as int64 [1][q][q][2] (k2, j2, re/im)."""
    return np.ascontiguousarray(np.array(C.dft_matrix_q(q, sign, scale_exp), dtype=np.int64)[None])


@lru_cache(maxsize=None)
def table_p(p: int, q: int, sign: int, scale_exp: int = C.SIGMA_F_EXP) -> np.ndarray:
    """F_p^(k2) as int64 [q][p][p][2] (k2, k1, j1, re/im)."""
    return np.ascontiguousarray(np.array(C.fused_matrices_p(p, q, sign, scale_exp), dtype=np.int64))


@lru_cache(maxsize=None)
def dd_twiddles(N: int, sign: int) -> np.ndarray:
    return np.ascontiguousarray(np.array([C.dd_twiddle(m, N, sign) for m in range(N)],
                                         dtype=np.float64))


# --------------------------------------------------------------------------
# Stage / line / grid transforms
# --------------------------------------------------------------------------
def stage(cols: np.ndarray, Ftab: np.ndarray, group: np.ndarray | None = None,
          use_crt: bool = True, dump: bool = False, moduli=C.MODULI):
    """One Ozaki-II complex stage on independent columns.

    cols: complex128 [ncols][K]; Ftab: int64 [ngroups][Kout][K][2];
    group: int32 [ncols] (which matrix each column uses) or None.
    Returns (y complex128 [ncols][Kout], mismatches, dump dict or None)."""
    cols = np.ascontiguousarray(cols, dtype=np.complex128)
    ncols, K = cols.shape
    Kout = Ftab.shape[1]
    assert Ftab.shape[2] == K and K <= 64
    y = np.empty((ncols, Kout), dtype=np.complex128)
    g = None if group is None else np.ascontiguousarray(group, dtype=np.int32)
    d = _Dump()
    arrays = None
    if dump:
        arrays = dict(col_exp=np.zeros(ncols, np.int32), xt=np.zeros((ncols, K, 2), np.int64),
                      def_=np.zeros((ncols, Kout, 12, 3), np.uint16),
                      v=np.zeros((ncols, Kout, 2, 12), np.uint16),
                      P=np.zeros((ncols, Kout, 2, 15), np.int64),
                      Q=np.zeros((ncols, Kout, 2, 6), np.int64),
                      zhat=np.zeros((ncols, Kout, 2), np.int64),
                      Rlimbs=np.zeros((ncols, Kout, 2, 2), np.int64))
        for k, a in arrays.items():
            setattr(d, k, a.ctypes.data)
    cst = consts(moduli)
    mism = lib().ob_ref_stage(ncols, K, Kout, _ptr(cols.view(np.float64)),
                              _ptr(np.ascontiguousarray(Ftab)), _ptr(g), ctypes.byref(cst),
                              1 if use_crt else 0, _ptr(y.view(np.float64)), ctypes.byref(d))
    if arrays is not None:
        arrays["def"] = arrays.pop("def_")
    return y, mism, arrays


def stage32(cols: np.ndarray, Ftab: np.ndarray, group: np.ndarray | None = None,
            use_crt: bool = True, dump: bool = False):
    """The FP32-precision variant of `stage`: complex64 columns, constants
    RNE(2^23 omega), six moduli.  Returns (y complex64 [ncols][Kout], mismatches, dump)."""
    cols = np.ascontiguousarray(cols, dtype=np.complex64)
    ncols, K = cols.shape
    Kout = Ftab.shape[1]
    assert Ftab.shape[2] == K and K <= 64
    y = np.empty((ncols, Kout), dtype=np.complex64)
    g = None if group is None else np.ascontiguousarray(group, dtype=np.int32)
    d = _Dump32()
    arrays = None
    if dump:
        arrays = dict(v=np.zeros((ncols, Kout, 2, 6), np.uint16),
                      P=np.zeros((ncols, Kout, 2, 8), np.int64),
                      Q=np.zeros((ncols, Kout, 2, 3), np.int64),
                      zhat=np.zeros((ncols, Kout, 2), np.int64),
                      R=np.zeros((ncols, Kout, 2), np.int64),
                      col_exp=np.zeros(ncols, np.int32), xt=np.zeros((ncols, K, 2), np.int64))
        for k, a in arrays.items():
            setattr(d, k, a.ctypes.data)
    cst = consts32()
    mism = lib().ob_ref_stage32(ncols, K, Kout, _ptr(cols.view(np.float32)),
                                _ptr(np.ascontiguousarray(Ftab)), _ptr(g), ctypes.byref(cst),
                                1 if use_crt else 0, _ptr(y.view(np.float32)), ctypes.byref(d))
    return y, mism, arrays


def _stage_of(prec: str):
    return stage if prec == "fp64" else stage32


def bailey_lines(x: np.ndarray, p: int, q: int, sign: int = -1, use_crt: bool = True,
                 prec: str = "fp64"):
    """Ozaki-Bailey 1-D transform of every row of x ([L][N], N = p q; complex128
    for prec "fp64", complex64 for the FP32 variant "fp32").

    Returns (Y [L][N], mismatches)."""
    ctype, sexp = PRECISIONS[prec]
    x = np.asarray(x, dtype=ctype)
    L, N = x.shape
    assert N == p * q
    if N == 1:
        return x.copy(), 0
    st = _stage_of(prec)
    # stage 1: columns (l, j1) over j2; x[l, j1 + p j2] -> view [L][q][p]
    c1 = x.reshape(L, q, p).transpose(0, 2, 1).reshape(L * p, q)
    y1, m1, _ = st(c1, table_q(q, sign, sexp), None, use_crt)
    y1 = y1.reshape(L, p, q)                        # Y'[l][j1][k2]
    # stage 2: columns (l, k2) over j1, matrix F_p^(k2)
    c2 = y1.transpose(0, 2, 1).reshape(L * q, p)
    grp = np.tile(np.arange(q, dtype=np.int32), L)
    z, m2, _ = st(c2, table_p(p, q, sign, sexp), grp, use_crt)
    z = z.reshape(L, q, p)                          # Z[l][k2][k1]
    Y = z.transpose(0, 2, 1).reshape(L, N)          # Y[k2 + q k1]
    return np.ascontiguousarray(Y), m1 + m2


def obfft3d(x: np.ndarray, splits, sign: int = -1, use_crt: bool = True, prec: str = "fp64"):
    """3-D Ozaki-Bailey transform of x [..., n0, n1, n2]; splits = ((p0,q0),(p1,q1),(p2,q2)).

    Axis 2 first, then 1, then 0.  Returns (Y, total mismatches)."""
    x = np.asarray(x, dtype=PRECISIONS[prec][0])
    y = x
    mism = 0
    for axis in (2, 1, 0):
        ax = x.ndim - 3 + axis
        n = y.shape[ax]
        p, q = splits[axis]
        moved = np.moveaxis(y, ax, -1)
        shp = moved.shape
        Y, m = bailey_lines(np.ascontiguousarray(moved).reshape(-1, n), p, q, sign, use_crt, prec)
        mism += m
        y = np.moveaxis(Y.reshape(shp), -1, ax)
    return np.ascontiguousarray(y), mism


def pack(R: int, e: int) -> float:
    lo = R & ((1 << 64) - 1)
    hi = (R >> 64) & ((1 << 64) - 1)
    if lo >= 1 << 63:
        lo -= 1 << 64
    if hi >= 1 << 63:
        hi -= 1 << 64
    return lib().ob_ref_pack(lo, hi, e)


def pack32(R: int, e: int) -> np.float32:
    """RNE(R 2^e) to binary32 (|R| < 2^63), the FP32 variant's single rounding."""
    return np.float32(lib().ob_ref_pack32(int(R), int(e)))


def kulisch(P: np.ndarray, Q: np.ndarray, moduli=C.MODULI):
    """Algorithm 2 on a batch of (P[15], Q[6]) vectors -> (zhat, R as Python ints)."""
    P = np.ascontiguousarray(P, dtype=np.int64).reshape(-1, 15)
    Q = np.ascontiguousarray(Q, dtype=np.int64).reshape(-1, 6)
    n = P.shape[0]
    z = np.zeros(n, np.int64)
    Rl = np.zeros((n, 2), np.int64)
    cst = consts(moduli)
    lib().ob_ref_kulisch(n, _ptr(P), _ptr(Q), ctypes.byref(cst), _ptr(z), _ptr(Rl))
    Rs = [(int(hi) << 64) + (int(lo) & ((1 << 64) - 1)) for lo, hi in Rl]
    return z, Rs


# --------------------------------------------------------------------------
# Double-double references
# --------------------------------------------------------------------------
def dft_dd_lines(x_dd: np.ndarray, sign: int = -1) -> np.ndarray:
    """Direct DFT of each row in double-double. x_dd: float64 [L][N][4]."""
    L, N, _ = x_dd.shape
    out = np.empty_like(x_dd)
    lib().ob_ref_dft_dd_axis(L, N, _ptr(np.ascontiguousarray(x_dd)), _ptr(dd_twiddles(N, sign)),
                             _ptr(out))
    return out


def to_dd(x: np.ndarray) -> np.ndarray:
    out = np.zeros(x.shape + (4,), np.float64)
    out[..., 0] = x.real
    out[..., 2] = x.imag
    return out


def dft3d_dd(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """Separable direct 3-D DFT in double-double (small grids); returns float64 [...,4]."""
    y = to_dd(np.asarray(x, np.complex128))
    for ax in (x.ndim - 1, x.ndim - 2, x.ndim - 3):
        moved = np.moveaxis(y, ax, -2)
        shp = moved.shape
        r = dft_dd_lines(np.ascontiguousarray(moved).reshape(-1, shp[-2], 4), sign)
        y = np.moveaxis(r.reshape(shp), -2, ax)
    return np.ascontiguousarray(y)


def dft3d_dd_point(x: np.ndarray, k, sign: int = -1) -> np.ndarray:
    """One output of the 3-D DFT of a single grid x [n0][n1][n2], double-double."""
    n0, n1, n2 = x.shape
    xc = np.ascontiguousarray(x, np.complex128)
    res = np.zeros(4, np.float64)
    lib().ob_ref_dft_dd_point(n0, n1, n2, _ptr(xc.view(np.float64)),
                              _ptr(dd_twiddles(n0, sign)), _ptr(dd_twiddles(n1, sign)),
                              _ptr(dd_twiddles(n2, sign)), int(k[0]), int(k[1]), int(k[2]),
                              _ptr(res))
    return res


@lru_cache(maxsize=None)
def fp64_twiddles(N: int, sign: int) -> np.ndarray:
    """exp(sign 2 pi i m / N), m < N, rounded to double (from the fixed-point values)."""
    t = dd_twiddles(N, sign)
    return np.ascontiguousarray(np.stack([t[:, 0], t[:, 2]], axis=1))


def fft_lines(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """Plain FP64 mixed-radix FFT of every row of x (complex128 [L][N])."""
    x = np.ascontiguousarray(x, dtype=np.complex128)
    L, N = x.shape
    y = np.empty_like(x)
    lib().ob_ref_fft_lines(L, N, _ptr(fp64_twiddles(N, sign)), _ptr(x.view(np.float64)), _ptr(y.view(np.float64)))
    return y


def fft3d(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """Plain FP64 3-D FFT of x [..., n0, n1, n2] (axis 2 first, then 1, then 0)."""
    y = np.asarray(x, dtype=np.complex128)
    for ax in (y.ndim - 1, y.ndim - 2, y.ndim - 3):
        moved = np.moveaxis(y, ax, -1)
        shp = moved.shape
        y = np.moveaxis(fft_lines(np.ascontiguousarray(moved).reshape(-1, shp[-1]), sign).reshape(shp), -1, ax)
    return np.ascontiguousarray(y)


def dd_to_complex(y: np.ndarray) -> np.ndarray:
    return (y[..., 0] + y[..., 1]) + 1j * (y[..., 2] + y[..., 3])


def normwise_error(y: np.ndarray, ref_dd: np.ndarray) -> float:
    """||y - ref|| / ||ref|| with the difference taken against the double-double value."""
    dr = (y.real - ref_dd[..., 0]) - ref_dd[..., 1]
    di = (y.imag - ref_dd[..., 2]) - ref_dd[..., 3]
    num = np.sqrt(np.sum(dr * dr + di * di))
    den = np.sqrt(np.sum(ref_dd[..., 0] ** 2 + ref_dd[..., 2] ** 2))
    return float(num / den) if den > 0 else float(num)
