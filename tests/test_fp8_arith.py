"""Host-side checks of the FP32 / integer arithmetic the FP8 stage kernel relies on.

The kernel reduces data residues lazily (Barrett without its correction step),
balances them with one rounded FP32 quotient, and reduces each output's class
sum to r with |r| <= m/2 + 1 before adding the offset 1024 (Sec. tcgarner:
FP16 operands below 2048 are exact; Algorithm 2 lifts any representative of
the residue class).  These tests emulate each step exactly (integers and
rationals, round-to-nearest-even where the kernel rounds) for every modulus.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import constants as C

MODULI = [int(m) for m in C.MODULI]
MAGIC_RANGE = 2 ** 22  # rint via the 1.5 * 2^23 magic add needs |value| < 2^22


def f32_recip(m: int) -> Fraction:
    """1/m as the kernel's constant: (float)(1.0 / (double)m)."""
    return Fraction(float(np.float32(1.0 / m)))


def rne(q: Fraction) -> int:
    """Round a rational to the nearest integer, ties to even."""
    f = q.numerator // q.denominator
    rem = q - f
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and f % 2 == 1):
        return f + 1
    return f


@pytest.mark.parametrize("m", MODULI)
def test_lazy_barrett_range(m):
    mu = (1 << 32) // m
    c20, c40 = pow(2, 20, m), pow(2, 40, m)
    tmax = (2 ** 20 - 1) + (2 ** 20 - 1) * c20 + (2 ** 16 - 1) * c40
    assert tmax < 2 ** 32
    rng = np.random.default_rng(m)
    ts = list(rng.integers(0, tmax + 1, 20000)) + [0, tmax, m - 1, m, 2 * m - 1]
    ts += [j * m + d for j in range(1, tmax // m, max(1, (tmax // m) // 5000)) for d in (-1, 0, 1)]
    for t in ts:
        t = int(t)
        if not 0 <= t <= tmax:
            continue
        r = t - ((t * mu) >> 32) * m
        assert 0 <= r < 2 * m and (r - t) % m == 0


@pytest.mark.parametrize("m", MODULI)
def test_data_balance_exact(m):
    """f in (-m, 2m) -> v = f - m RNE(f * fl(1/m)) is the round-half-even
    balanced residue: |v| <= m/2 and v = f (mod m), for every f."""
    im = f32_recip(m)
    for f in range(-m + 1, 2 * m):
        q = rne(f * im)
        assert abs(f * im) < MAGIC_RANGE
        v = f - m * q
        assert 2 * abs(v) <= m and (v - f) % m == 0
        assert q == rne(Fraction(f, m))  # the FP32 quotient is the exact one


@pytest.mark.parametrize("m", MODULI)
def test_offset_residue_range(m):
    """|x| < 2^24 -> x - m RNE(x * fl(1/m)) lies in [-m/2 - 1, m/2 + 1], so the
    offset value is in [2, 2046]; checked at every half-integer boundary of
    x/m near the largest magnitudes and on random x."""
    im = f32_recip(m)
    xs = []
    nmax = (2 ** 24 - 1) // m
    for n in list(range(0, 64)) + list(range(nmax - 64, nmax + 1)):
        c = (2 * n + 1) * m // 2
        xs += [c + d for d in range(-3, 4)]
    xs += list(np.random.default_rng(7 * m).integers(-(2 ** 24) + 1, 2 ** 24, 5000))
    for x in xs:
        for xx in (int(x), -int(x)):
            if abs(xx) >= 2 ** 24:
                continue
            q = rne(xx * im)
            r = xx - m * q
            assert 2 * abs(r) <= m + 2, (m, xx, r)
            assert 2 <= r + 1024 <= 2046
    # Phase-A deposits stay below 2^23 with twelve offset residues per slice
    assert 12 * 2046 * 255 < 2 ** 23


def test_offset_lifts_to_c_plus_offset():
    """Sum_k u_k = 1 (mod M): the CRT of r_k + 1024 is C + 1024."""
    M = C.M
    us = C.idempotents()
    assert sum(us) % M == 1
    rng = np.random.default_rng(3)
    for _ in range(20):
        c = int(rng.integers(-(2 ** 62), 2 ** 62)) * int(rng.integers(1, 2 ** 40))
        r = [(c % m) + 1024 for m in MODULI]
        e = sum(ri * ui for ri, ui in zip(r, us)) % M
        e = e - M if e >= M // 2 else e
        assert e == c + 1024


# --------------------------------------------------------------------------
# FP32-precision variant: data residues of the exact integers |x~| < 2^24
# --------------------------------------------------------------------------
@pytest.mark.parametrize("m", [int(v) for v in C.MODULI_FP32])
def test_fp32_variant_balanced_residue_exhaustive(m):
    """v1 = x - m RNE(x fl(1/m)), v = v1 - m RNE(v1 fl(1/m)) (RNE of the exact
    products, as the fused magic-number rounding computes them) is the balanced
    residue |v| <= m/2, v = x (mod m), for every integer |x| < 2^24."""
    f = float(np.float32(1.0 / m))                 # the kernel's rounded reciprocal
    step = 1 << 20
    for lo in range(-(1 << 24) + 1, 1 << 24, step):
        x = np.arange(lo, min(lo + step, 1 << 24), dtype=np.float64)
        q1 = np.rint(x * f)                           # x f is exact in float64 (24 x 24 bits)
        assert np.all(np.abs(x * f) < 2 ** 22)        # range of the magic-number rounding
        v1 = x - m * q1
        q2 = np.rint(v1 * f)
        v = v1 - m * q2
        assert np.all(2 * np.abs(v) <= m)
        assert np.all(np.mod(v - x, m) == 0)
    # FP16 carrier bound for the largest modulus
    assert m // 2 <= 1020
