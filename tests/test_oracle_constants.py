"""Pins of the oracle's constants against values the paper prints and against
number-theoretic facts (not against a retyped formula)."""
import json
import math
import os
import random
from fractions import Fraction

import pytest

from oracle import constants as C

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_modulus_set_matches_paper():
    assert list(C.MODULI) == GOLD["moduli_rev34"]["value"]


def test_pairwise_coprime():
    for i, a in enumerate(C.MODULI):
        for b in C.MODULI[i + 1:]:
            assert math.gcd(a, b) == 1


def test_log2_M_and_bit_length():
    assert abs(math.log2(C.M) - GOLD["log2_M"]["value"]) < GOLD["log2_M"]["tol"]
    assert C.M.bit_length() == GOLD["bitlen_M"]["value"]
    assert C.S_RAW == GOLD["S_raw"]["value"] == math.ceil(C.M.bit_length() / 8)
    assert C.S_FRAC == GOLD["S_frac"]["value"] == C.F_BITS // 8


def test_capacity_budget_and_margin():
    g = GOLD["capacity_rhs_bits"]
    assert C.capacity_bits(g["K"], g["k"]) == g["value"]
    margin = math.log2(C.M) - C.capacity_bits(32)
    assert abs(margin - GOLD["capacity_margin_bits"]["value"]) < GOLD["capacity_margin_bits"]["tol"]


def test_rev33_fails_budget_by_216_bits():
    m33 = C.modulus_product(C.MODULI_REV33)
    assert abs(math.log2(m33) - GOLD["log2_M_rev33"]["value"]) < GOLD["log2_M_rev33"]["tol"]
    deficit = C.capacity_bits(32) - math.log2(m33)
    assert abs(deficit - GOLD["rev33_deficit_bits"]["value"]) < GOLD["rev33_deficit_bits"]["tol"]


def test_idempotent_property():
    # u_k = 1 mod m_k and 0 mod every other modulus; 0 <= u_k < M
    for k, u in enumerate(C.U):
        assert 0 <= u < C.M
        for j, m in enumerate(C.MODULI):
            assert u % m == (1 if j == k else 0)


def test_accumulator_width_identities():
    """Eq. (accwidth): sum (m_k - 1) u_k = 4360 M - 1, sum (2 m_k - 1) u_k = 8724 M - 1."""
    assert sum((m - 1) * u for m, u in zip(C.MODULI, C.U)) == 4360 * C.M - 1
    assert sum((2 * m - 1) * u for m, u in zip(C.MODULI, C.U)) == 8724 * C.M - 1
    assert (8724 * C.M - 1).bit_length() == 131
    assert (8724 * C.M - 1).bit_length() + 1 == GOLD["twos_complement_bits"]["value"]


def test_phase_a_column_bound():
    """T6: canonical residue <= 2038, slice <= 255, 12-term sums < 2^23."""
    assert max(m - 1 for m in C.MODULI) * 255 == GOLD["phaseA_product_bound"]["value"]
    bound = len(C.MODULI) * max(m - 1 for m in C.MODULI) * 255
    assert bound == GOLD["phaseA_column_bound"]["value"] < 2 ** 23
    # every slice really is a byte and reassembles u_k / w_k
    for k in range(C.R):
        assert sum(b << (8 * s) for s, b in enumerate(C.U_SLICES[k])) == C.U[k]
        assert sum(b << (8 * t) for t, b in enumerate(C.W_SLICES[k])) == C.W[k]


def test_h1_column_bound():
    assert C.R * 255 * (128 + 8) == GOLD["h1_column_bound"]["value"]


def test_lift_weights_are_48_bit_and_error_below_quarter():
    for w in C.W:
        assert 0 < w < 2 ** 48
    # lift error sum_k v_k |w_k 2^-48 - u_k / M| < 1/4 for canonical v_k (worst case v = m - 1)
    err = sum((m - 1) * abs(Fraction(w, 2 ** 48) - Fraction(u, C.M))
              for m, u, w in zip(C.MODULI, C.U, C.W))
    assert err < Fraction(1, 4)
    # and for the signed |v_k| < 2 m_k bound the paper's ledger also covers
    err2 = sum((2 * m - 1) * abs(Fraction(w, 2 ** 48) - Fraction(u, C.M))
               for m, u, w in zip(C.MODULI, C.U, C.W))
    assert err2 < Fraction(1, 4)


def test_reduction_friendly_complements():
    g = GOLD["reduction_friendly"]
    for m in g["value"]:
        c = (2 ** 11 - m) if m > 1024 else (2 ** 9 - m if m < 1024 else 0)
        assert 0 <= c <= g["max_c"]
    for m in GOLD["perfect_squares"]["value"]:
        assert math.isqrt(m) ** 2 == m


def test_fixed_point_cos_sin_closed_forms():
    one = 1 << C.PREC
    assert C.cos_sin_2pi(0, 7) == (one, 0)
    assert C.cos_sin_2pi(1, 4) == (0, one)
    assert C.cos_sin_2pi(2, 4) == (-one, 0)
    assert C.cos_sin_2pi(3, 4) == (0, -one)
    c, s = C.cos_sin_2pi(1, 6)                 # cos 60 = 1/2
    assert abs(c - one // 2) < 16
    c, s = C.cos_sin_2pi(1, 8)                 # sqrt(2)/2 via integer square root
    r2 = math.isqrt(2 << (2 * C.PREC)) // 2
    assert abs(c - r2) < 16 and abs(s - r2) < 16
    rng = random.Random(5)
    for _ in range(200):
        N = rng.randint(1, 5000)
        m = rng.randint(0, N - 1)
        c, s = C.cos_sin_2pi(m, N)
        assert abs(c * c + s * s - one * one) < one * 64   # cos^2 + sin^2 = 1


def test_fixed_point_cos_sin_vs_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 300
    rng = random.Random(7)
    for _ in range(300):
        N = rng.choice([8, 12, 16, 24, 32, 64, 96, 128, 192, 256, 384, 1024, 4096, 7, 11])
        m = rng.randint(0, N - 1)
        c, s = C.cos_sin_2pi(m, N)
        th = 2 * mp.pi * m / N
        assert abs(mp.mpf(c) / 2 ** C.PREC - mp.cos(th)) < mp.mpf(2) ** (-C.PREC + 8)
        assert abs(mp.mpf(s) / 2 ** C.PREC - mp.sin(th)) < mp.mpf(2) ** (-C.PREC + 8)


def test_quantised_twiddle_special_points_and_rounding():
    two52 = 1 << 52
    assert C.quantised_twiddle(0, 32) == (two52, 0)
    assert C.quantised_twiddle(8, 32) == (0, -two52)          # exp(-i pi/2) = -i
    assert C.quantised_twiddle(8, 32, +1) == (0, two52)
    assert C.quantised_twiddle(1, 6) == (two52 // 2, C.quantised_twiddle(1, 6)[1])
    # 2^52 cos(pi/4) = 2^51.5 = sqrt(2^103): RNE by exact integer square root
    r = math.isqrt(2 ** 103)
    exp = r + 1 if (2 * r + 1) ** 2 < 4 * 2 ** 103 else r
    re, im = C.quantised_twiddle(1, 8)
    assert re == exp and im == -exp
    # |entry| <= 2^52 everywhere (53-bit signed significands)
    for N in (8, 16, 32, 96):
        for m in range(N):
            re, im = C.quantised_twiddle(m, N)
            assert abs(re) <= two52 and abs(im) <= two52


def test_quantised_twiddle_vs_mpmath_rne():
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 300
    for N in (8, 12, 16, 32, 64, 1024):
        for m in range(0, N, max(1, N // 64)):
            re, im = C.quantised_twiddle(m, N)
            th = 2 * mp.pi * m / N
            for got, val in ((re, mp.cos(th)), (im, -mp.sin(th))):
                x = val * 2 ** 52
                fl = int(mp.floor(x))
                frac = x - fl
                want = fl + 1 if frac > 0.5 else fl   # no exact ties off the exact points
                assert got == want


def test_fused_matrix_is_dft_times_twiddle():
    """F_p^(k2)[k1][j1] quantises omega_p^(j1 k1) omega_N^(j1 k2)."""
    p, q = 4, 8
    N = p * q
    Fp = C.fused_matrices_p(p, q)
    for k2 in range(q):
        for k1 in range(p):
            for j1 in range(p):
                # same exponent reduced mod N: j1 k1 q + j1 k2
                assert Fp[k2][k1][j1] == C.quantised_twiddle((j1 * k1 * q + j1 * k2) % N, N)


def test_default_split():
    assert C.default_split(1024) == (32, 32)
    assert C.default_split(64) == (8, 8)
    assert C.default_split(256) == (16, 16)
    p, q = C.default_split(384)
    assert p * q == 384 and p <= 64 and q <= 64
