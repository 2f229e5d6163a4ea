"""Pins of the oracle's FP32-precision variant (Sec. "Ozaki-II for FP32").

The variant reconstructs complex64 Bailey stages from r = 6 moduli: 24-bit
significands, S = 8 byte slices, f = 24 fractional lift bits, one rounding to
binary32 at the end.  Each check below ties the oracle to something other
than itself: the paper's printed sizes, number theory, the exact integer
definition of a stage, numpy's own float32 rounding, and closed forms of the
DFT.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import constants as C
from oracle import ref

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


# --------------------------------------------------------------------------
# constants
# --------------------------------------------------------------------------
def test_fp32_modulus_set_is_the_unique_62_6_bit_subset():
    g = GOLD["fp32_log2_M"]
    hits = [c for c in itertools.combinations(C.MODULI, GOLD["fp32_r"]["value"])
            if abs(sum(math.log2(m) for m in c) - g["value"]) < g["tol"]]
    assert hits == [C.MODULI_FP32]
    for i, a in enumerate(C.MODULI_FP32):
        for b in C.MODULI_FP32[i + 1:]:
            assert math.gcd(a, b) == 1


def test_fp32_capacity_and_slices():
    g = GOLD["fp32_capacity_rhs_bits"]
    assert C.capacity_bits(g["K"], g["k"]) == g["value"]
    assert math.log2(C.M_FP32) > g["value"]
    assert C.S_RAW_FP32 == GOLD["fp32_S_raw"]["value"] == math.ceil(C.M_FP32.bit_length() / 8)
    # the real-form complex product of 24-bit significands: |C| <= 2 K 2^23 2^24
    assert 2 * 32 * 2 ** 23 * 2 ** 24 < C.M_FP32 // 2


def test_fp32_idempotents_and_accumulator_width():
    for k, u in enumerate(C.U_FP32):
        assert 0 <= u < C.M_FP32
        for j, m in enumerate(C.MODULI_FP32):
            assert u % m == (1 if j == k else 0)
    # The paper's 77-bit accumulator is the loose envelope of Eq. (accwidth),
    # log2(r 2 max(m) M), taken for the FP32 set; the exact bounds from the
    # idempotents sit below it (canonical and signed residues, as for Rev-34)
    env = math.log2(C.R_FP32 * 2 * max(C.MODULI_FP32) * C.M_FP32)
    assert math.floor(env) == GOLD["fp32_accumulator_bits"]["value"]
    e_can = sum((m - 1) * u for m, u in zip(C.MODULI_FP32, C.U_FP32))
    e_sgn = sum((2 * m - 1) * u for m, u in zip(C.MODULI_FP32, C.U_FP32))
    assert (e_can + 1) % C.M_FP32 == 0 and (e_sgn + 1) % C.M_FP32 == 0
    assert e_can.bit_length() <= e_sgn.bit_length() <= GOLD["fp32_accumulator_bits"]["value"]
    # Phase-A column sums: exact FP32 integers below 2^23 (for offset residues up to 2047 too)
    assert C.R_FP32 * 2047 * 255 < 2 ** 23
    # lift: r max(v) 2^-f < 1/4, the bound the two-sided correction needs
    assert C.R_FP32 * 2047 / 2 ** C.F_BITS_FP32 < 0.25
    for u, w in zip(C.U_FP32, C.W_FP32):
        assert abs(w * C.M_FP32 - (u << C.F_BITS_FP32)) <= C.M_FP32 // 2


def test_fp32_quantised_constants_vs_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 200
    for N in (8, 12, 32, 1024):
        for m in range(0, N, max(1, N // 48)):
            re, im = C.quantised_twiddle(m, N, -1, C.SIGMA_F_EXP_FP32)
            th = 2 * mp.pi * m / N
            for got, val in ((re, mp.cos(th)), (im, -mp.sin(th))):
                x = val * 2 ** 23
                fl = int(mp.floor(x))
                want = fl + 1 if x - fl > 0.5 else fl
                assert got == want
                assert abs(got) <= 2 ** 23


# --------------------------------------------------------------------------
# the single rounding to binary32
# --------------------------------------------------------------------------
def _np_round32(R: int, e: int) -> np.float32:
    """numpy's own binary32 rounding of R 2^e, for |R| <= 2^53 (exact in double)."""
    with np.errstate(over="ignore"):
        return np.float32(math.ldexp(float(R), e))


def test_pack32_matches_numpy_rounding():
    rng = np.random.default_rng(5)
    cases = []
    for _ in range(4000):
        bits = int(rng.integers(1, 54))
        R = int(rng.integers(1, 2 ** bits)) * (1 if rng.random() < 0.5 else -1)
        e = int(rng.integers(-220, 120))
        cases.append((R, e))
    # ties at the 24-bit boundary, in the normal and in the subnormal range
    for k in range(1, 30):
        for base in (2 ** 24 + 1, 2 ** 24 + 3, 2 ** 23 + 5):
            cases += [(base * 2 ** k + 2 ** (k - 1), -k - 10), (base * 2 ** k + 2 ** (k - 1), -170)]
    cases += [(1, -149), (1, -150), (3, -151), (2 ** 24 - 1, 104), (2 ** 24 - 1, 105), (0, 0)]
    for R, e in cases:
        got = ref.pack32(R, e)
        want = _np_round32(R, e)
        assert got.tobytes() == want.tobytes() or (R == 0 and got == 0), (R, e, got, want)


def test_pack32_beyond_53_bits_via_long_double():
    if np.finfo(np.longdouble).nmant < 63:
        pytest.skip("long double narrower than 64 bits here")
    rng = np.random.default_rng(6)
    for _ in range(2000):
        R = int(rng.integers(2 ** 53, 2 ** 62)) * (1 if rng.random() < 0.5 else -1)
        e = int(rng.integers(-200, 60))
        ld = np.longdouble(R) * np.longdouble(2.0) ** e    # exact: R has <= 63 bits
        with np.errstate(over="ignore"):
            want = np.float32(ld)
        assert ref.pack32(R, e).tobytes() == want.tobytes(), (R, e)


# --------------------------------------------------------------------------
# one stage: the CRT chain against the exact integer definition
# --------------------------------------------------------------------------
def _cols(rng, n, K, wide=False):
    re = rng.uniform(-1, 1, (n, K))
    im = rng.uniform(-1, 1, (n, K))
    if wide:
        re *= 2.0 ** rng.integers(-30, 31, (n, K))
        im *= 2.0 ** rng.integers(-30, 31, (n, K))
    return (re + 1j * im).astype(np.complex64)


@pytest.mark.parametrize("K", [1, 2, 5, 8, 16, 32])
def test_stage32_crt_reconstructs_exact_product(K):
    rng = np.random.default_rng(K)
    cols = _cols(rng, 300, K, wide=K % 2 == 0)
    cols[0] = 0
    cols[1] = np.complex64(-1 - 1j)       # DC-like extremes
    cols[2, :] = np.complex64(np.float32(1 - 2 ** -24) * (1 + 1j))
    F = ref.table_q(K, -1, C.SIGMA_F_EXP_FP32)
    _, mism, _ = ref.stage32(cols, F)
    assert mism == 0


def test_stage32_definition_by_brute_force():
    """y = RNE32(2^(e - 46) sum_j F~ x~), x~ = RNE(x 2^(23 - e)), in Python integers."""
    rng = np.random.default_rng(11)
    K = 6
    cols = _cols(rng, 40, K, wide=True)
    F = ref.table_q(K, -1, C.SIGMA_F_EXP_FP32)
    y, mism, d = ref.stage32(cols, F, dump=True)
    assert mism == 0
    for c in range(cols.shape[0]):
        xs = [(float(v.real), float(v.imag)) for v in cols[c]]
        amax = max(max(abs(a), abs(b)) for a, b in xs)
        e = math.frexp(amax)[1] - 1 if amax > 0 else 0
        xt = [(round(math.ldexp(a, 23 - e)), round(math.ldexp(b, 23 - e))) for a, b in xs]  # ties to even
        for k in range(K):
            cr = ci = 0
            for j in range(K):
                fr, fi = int(F[0, k, j, 0]), int(F[0, k, j, 1])
                cr += fr * xt[j][0] - fi * xt[j][1]
                ci += fr * xt[j][1] + fi * xt[j][0]
            assert int(d["R"][c, k, 0]) == cr and int(d["R"][c, k, 1]) == ci
            assert y[c, k].real.tobytes() == _np_round32(cr, e - 46).tobytes()
            assert y[c, k].imag.tobytes() == _np_round32(ci, e - 46).tobytes()


def test_stage32_phase_a_slices_recombine():
    """P_s, Q_t are the byte-slice contractions of the canonical residues."""
    rng = np.random.default_rng(12)
    cols = _cols(rng, 20, 8)
    _, _, d = ref.stage32(cols, ref.table_q(8, -1, C.SIGMA_F_EXP_FP32), dump=True)
    v = d["v"].reshape(-1, 6).astype(np.int64)
    P = d["P"].reshape(-1, 8)
    Q = d["Q"].reshape(-1, 3)
    for i in range(v.shape[0]):
        E = sum(int(P[i, s]) << (8 * s) for s in range(8))
        assert E == sum(int(v[i, k]) * C.U_FP32[k] for k in range(6))
        z = sum(int(Q[i, t]) << (8 * t) for t in range(3))
        assert z == sum(int(v[i, k]) * C.W_FP32[k] for k in range(6))
        assert all(0 <= v[i, k] < C.MODULI_FP32[k] for k in range(6))


# --------------------------------------------------------------------------
# whole transforms: closed forms and the double-double DFT
# --------------------------------------------------------------------------
SPL = ((4, 4), (4, 4), (4, 4))


def test_fp32_impulse_gives_exact_constant():
    x = np.zeros((16, 16, 16), np.complex64)
    x[0, 0, 0] = 1
    y, mism = ref.obfft3d(x, SPL, prec="fp32")
    assert mism == 0 and y.dtype == np.complex64
    assert np.all(y == 1)


def test_fp32_single_mode_gives_delta():
    n = 16
    j = np.arange(n)
    k0 = (3, 5, 7)
    ph = np.exp(2j * np.pi * (np.add.outer(np.add.outer(j * k0[0], j * k0[1]), j * k0[2])) / n)
    y, _ = ref.obfft3d(ph.astype(np.complex64), SPL, prec="fp32")
    want = np.zeros_like(y)
    want[k0] = n ** 3
    assert np.max(np.abs(y - want)) < 1e-5 * n ** 3


def test_fp32_against_double_double_and_roundtrip():
    rng = np.random.default_rng(20260001)
    x = (rng.uniform(-1, 1, (16, 16, 16)) + 1j * rng.uniform(-1, 1, (16, 16, 16))).astype(np.complex64)
    y, mism = ref.obfft3d(x, SPL, prec="fp32")
    assert mism == 0
    yd = ref.dft3d_dd(x.astype(np.complex128))
    err = ref.normwise_error(y.astype(np.complex128), yd)
    # six roundings to binary32 (u = 2^-24) plus the 2^-24-relative constants
    assert err < 12 * 2.0 ** -24
    z, _ = ref.obfft3d(y, SPL, sign=+1, prec="fp32")
    rt = np.linalg.norm(z / 16 ** 3 - x) / np.linalg.norm(x)
    assert rt < 16 * 2.0 ** -24
    # Parseval
    assert abs(np.sum(np.abs(y.astype(np.complex128)) ** 2) / (16 ** 3 * np.sum(np.abs(x) ** 2)) - 1) < 1e-6
