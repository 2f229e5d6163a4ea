"""Pins of the oracle's integer pipeline and end-to-end transform.

The CRT stages are pinned by what fixes them independently of the oracle's
code: the exact integer the reconstruction must reach (Python big integers),
Garner's mixed-radix recursion and Bernstein's fractional form as two other
reconstructions, the paper's counterexamples (T3: P_0 = -1; T4: the lift
near +-M/2), Python's correctly rounded int -> float conversion for the pack,
and closed forms / double-double sums for the transform."""
import math
import random
from fractions import Fraction

import numpy as np
import pytest

from oracle import constants as C
from oracle import ref
from synth import inputs as S


def exact_float(R: int, e: int) -> float:
    """Correctly rounded R * 2^e by Python's exact rational conversion."""
    return float(Fraction(R) * Fraction(2) ** e) if e >= 0 else float(Fraction(R, 2 ** -e))


# ---------------------------------------------------------------- pack ----
@pytest.mark.parametrize("seed", range(4))
def test_pack_matches_exact_rounding(seed):
    rng = random.Random(seed)
    for _ in range(3000):
        bits = rng.randint(1, 117)
        R = rng.getrandbits(bits) * rng.choice((-1, 1))
        e = rng.randint(-1300, 800)
        assert ref.pack(R, e) == exact_float(R, e), (R, e)


def test_pack_ties_and_subnormals():
    # exact ties at the 53-bit boundary round to even
    for base in (2 ** 53 + 1, 2 ** 53 + 3):
        R = base * 2 + 1          # 55 bits, dropped half exactly
        assert ref.pack(R, 0) == exact_float(R, 0)
    for e in (-1074, -1075, -1076, -1100, -1130, -1180):
        for R in (1, 2, 3, 5, 2 ** 60 + 1, 2 ** 116 - 1, -(2 ** 70 + 12345)):
            assert ref.pack(R, e) == exact_float(R, e)
    assert ref.pack(0, 5) == 0.0
    assert ref.pack(2 ** 116, 1000) == math.inf


# ----------------------------------------------------------- CRT / lift ---
def residues(Cv: int, moduli=C.MODULI):
    return [Cv % m for m in moduli]


def phase_a(v, moduli=C.MODULI):
    us = [C.byte_slices(u, C.S_RAW) for u in C.idempotents(moduli)]
    ws = [C.byte_slices(w, C.S_FRAC) for w in C.lift_weights(moduli)]
    P = [sum(v[k] * us[k][s] for k in range(len(v))) for s in range(C.S_RAW)]
    Q = [sum(v[k] * ws[k][t] for k in range(len(v))) for t in range(C.S_FRAC)]
    return P, Q


def test_kulisch_T3_negative_deposit():
    """P_0 = -1 alone must reconstruct -1 (biased deposits, T3)."""
    P = np.zeros((1, 15), np.int64)
    P[0, 0] = -1
    Q = np.zeros((1, 6), np.int64)
    z, R = ref.kulisch(P, Q)
    assert R[0] == -1 and z[0] == 0


def test_kulisch_random_values_reconstruct_exactly():
    rng = random.Random(11)
    Cs = [rng.randrange(-C.M // 2, C.M // 2) for _ in range(2000)]
    Cs += [0, 1, -1, C.M // 2 - 1, -C.M // 2, 2 ** 112, -(2 ** 112)]
    Ps, Qs = zip(*[phase_a(residues(c)) for c in Cs])
    z, R = ref.kulisch(np.array(Ps), np.array(Qs))
    assert R == Cs


def test_two_sided_lift_T4_sweep_exercises_both_branches():
    """Near C = +-M/2 the rounded quotient can be one off either way; the
    two-sided correction must still return C, and the sweep must hit both
    correction branches (paper: July-30 counterexample, T4)."""
    half = C.M // 2
    Cs = []
    for t in range(1, 4000):
        Cs += [half - t, -half + t - 1]
    Cs += [-half]
    Ps, Qs = zip(*[phase_a(residues(c)) for c in Cs])
    z, R = ref.kulisch(np.array(Ps), np.array(Qs))
    assert R == Cs
    hits_low = hits_high = 0
    for c, zh in zip(Cs, z):
        E = sum(vk * u for vk, u in zip(residues(c), C.U))
        R0 = E - int(zh) * C.M
        hits_low += R0 >= half          # zhat one too small -> subtract M
        hits_high += R0 < -half         # zhat one too large -> add M
    assert hits_low > 0
    # with round-half-up w_k and canonical residues zhat is never too large near
    # +M/2; signed residues (|v| < 2m, also covered by the lift) reach it:
    signed_hits = 0
    rng = random.Random(3)
    for t in range(1, 3000):
        c = half - t
        v = [r - m if rng.random() < 0.5 else r for r, m in zip(residues(c), C.MODULI)]
        P, Q = phase_a(v)
        zz, RR = ref.kulisch(np.array([P]), np.array([Q]))
        assert RR[0] == c
        E = sum(vk * u for vk, u in zip(v, C.U))
        signed_hits += (E - int(zz[0]) * C.M) < -half
    assert hits_high + signed_hits > 0


def garner(v, moduli=C.MODULI):
    """Mixed-radix (Garner) reconstruction, the paper's recursive form."""
    digits = []
    for k, m in enumerate(moduli):
        acc = v[k]
        prod = 1
        for j in range(k):
            acc -= digits[j] * prod
            prod *= moduli[j]
        digits.append((acc * pow(prod % m, -1, m)) % m)
    x, prod = 0, 1
    for d, m in zip(digits, moduli):
        x += d * prod
        prod *= m
    return x  # in [0, M)


def bernstein(v, moduli=C.MODULI):
    """Fractional CRT with termwise reduction t_k = v_k y_k mod m_k."""
    Mp = C.modulus_product(moduli)
    s = Fraction(0)
    for vk, m in zip(v, moduli):
        y = pow(Mp // m, -1, m)
        t = (vk * y) % m
        assert 0 <= Fraction(t, m) < 1
        s += Fraction(t, m)
    f = s - math.floor(s)
    return int(Mp * f)  # in [0, M)


def test_oracle_stage_agrees_with_garner_and_bernstein():
    x = S.complex_uniform(99, (40, 16)).numpy()
    Ft = ref.table_q(16, -1)
    y, mism, d = ref.stage(x, Ft, dump=True)
    assert mism == 0
    half = C.M // 2
    rng = random.Random(1)
    for _ in range(300):
        c, k, part = rng.randrange(40), rng.randrange(16), rng.randrange(2)
        v = [int(t) for t in d["v"][c, k, part]]
        lo, hi = d["Rlimbs"][c, k, part]
        R = (int(hi) << 64) + (int(lo) & (2 ** 64 - 1))
        for rec in (garner(v), bernstein(v)):
            cen = rec - C.M if rec >= half else rec
            assert cen == R


def test_stage_residue_products_are_textbook_gemm_mod_m():
    """D, E, F of the dump equal int64 GEMMs mod m computed independently."""
    x = S.complex_uniform(5, (8, 32)).numpy()
    Ft = ref.table_q(32, -1)
    _, mism, d = ref.stage(x, Ft, dump=True)
    assert mism == 0
    xt = d["xt"].astype(object)
    F = Ft[0].astype(object)
    for c in range(8):
        for k in (0, 5, 31):
            for i, m in enumerate(C.MODULI):
                Dv = sum(F[k, j, 0] * xt[c, j, 0] for j in range(32)) % m
                Ev = sum(F[k, j, 1] * xt[c, j, 1] for j in range(32)) % m
                Fv = sum((F[k, j, 0] + F[k, j, 1]) * (xt[c, j, 0] + xt[c, j, 1]) for j in range(32)) % m
                assert tuple(int(t) for t in d["def"][c, k, i]) == (Dv, Ev, Fv)


def test_deconstruction_scale_rule():
    x = np.array([[0.75 + 0.1j, -0.3 - 0.5j, 1e-300 + 0j, 0.0 + 0j]])
    Ft = ref.table_q(4, -1)
    _, _, d = ref.stage(x, Ft, dump=True)
    assert d["col_exp"][0] == -1                       # ilogb(0.75)
    assert d["xt"][0, 0, 0] == int(0.75 * 2 ** 53)     # 0.75 * 2^(52+1) exact
    assert d["xt"][0, 2, 0] == 0                        # far below the column scale
    assert np.abs(d["xt"]).max() < 2 ** 53


def test_adversarial_columns_max_magnitude_and_dc():
    K = 64
    big = np.full((3, K), (1 - 2 ** -53) * (1 + 1j))
    big[1] = -big[1]
    big[2, ::2] *= -1
    Ft = ref.table_q(K, -1)
    _, mism, _ = ref.stage(big, Ft)
    assert mism == 0


def test_rev33_dc_column_reconstructs_wrong_by_M():
    """With the retired Rev-33 set a full-scale DC column overflows the CRT
    range: the lift returns the true value shifted by exactly M33."""
    K = 64
    x = np.full((1, K), (1 - 2 ** -53) * (1 + 1j))
    Ft = ref.table_q(K, -1)
    _, _, d33 = ref.stage(x, Ft, dump=True, moduli=C.MODULI_REV33)
    _, _, d34 = ref.stage(x, Ft, dump=True)
    M33 = C.modulus_product(C.MODULI_REV33)

    def R(d, part):
        lo, hi = d["Rlimbs"][0, 0, part]
        return (int(hi) << 64) + (int(lo) & (2 ** 64 - 1))

    true_re = sum(int(Ft[0, 0, j, 0]) * int(d34["xt"][0, j, 0]) for j in range(K))
    assert R(d34, 0) == true_re
    assert abs(R(d33, 0) - true_re) == M33


# --------------------------------------------------------- transforms -----
def test_impulse_gives_exact_constant():
    x = np.zeros((8, 12, 16), np.complex128)
    x[0, 0, 0] = 1.0
    y, mism = ref.obfft3d(x, ((2, 4), (3, 4), (4, 4)))
    assert mism == 0
    assert np.all(y == 1.0)


def test_constant_gives_scaled_delta():
    x = np.ones((8, 8, 8), np.complex128)
    y, _ = ref.obfft3d(x, ((2, 4), (2, 4), (2, 4)))
    ref_ = np.zeros_like(x)
    ref_[0, 0, 0] = 512
    assert np.abs(y - ref_).max() < 1e-12


def test_single_fourier_mode_gives_delta():
    n = (8, 16, 12)
    k = (3, 5, 7)
    j = np.indices(n)
    x = np.exp(2j * np.pi * sum(j[a] * k[a] / n[a] for a in range(3)))
    y, _ = ref.obfft3d(x, ((2, 4), (4, 4), (3, 4)))
    ref_ = np.zeros(n, np.complex128)
    ref_[k] = np.prod(n)
    assert np.abs(y - ref_).max() < 1e-11


def test_linearity_parseval_roundtrip():
    n = (16, 16, 16)
    sp = ((4, 4), (4, 4), (4, 4))
    a = S.complex_uniform(1, n).numpy()
    b = S.complex_gaussian(2, n).numpy()
    ya, _ = ref.obfft3d(a, sp)
    yb, _ = ref.obfft3d(b, sp)
    yab, _ = ref.obfft3d(a + 2 * b, sp)
    assert np.linalg.norm(yab - (ya + 2 * yb)) / np.linalg.norm(yab) < 1e-14
    N = np.prod(n)
    assert abs(np.sum(np.abs(ya) ** 2) - N * np.sum(np.abs(a) ** 2)) / (N * np.sum(np.abs(a) ** 2)) < 1e-14
    back, _ = ref.obfft3d(ya, sp, sign=+1)
    assert np.linalg.norm(back / N - a) / np.linalg.norm(a) < 1e-14


@pytest.mark.parametrize("shape,splits", [((16, 16, 16), ((4, 4), (4, 4), (4, 4))),
                                          ((8, 12, 24), ((2, 4), (3, 4), (4, 6))),
                                          ((2, 32, 5), ((1, 2), (4, 8), (1, 5)))])
def test_against_double_double_dft(shape, splits):
    x = S.complex_uniform(S.SEED_64, shape).numpy()
    y, mism = ref.obfft3d(x, splits)
    assert mism == 0
    yd = ref.dft3d_dd(x)
    err = ref.normwise_error(y, yd)
    assert err < 1e-15
    # a library FFT of the same input (pocketfft) lands at the same level
    assert err < 4 * ref.normwise_error(np.fft.fftn(x), yd) + 1e-16


def test_dd_reference_against_library_fft():
    x = S.complex_gaussian(4, (6, 10, 9)).numpy()
    yd = ref.dft3d_dd(x)
    assert ref.normwise_error(np.fft.fftn(x), yd) < 1e-15
    pt = ref.dft3d_dd_point(x, (1, 2, 3))
    assert abs((pt[0] + 1j * pt[2]) - ref.dd_to_complex(yd)[1, 2, 3]) < 1e-13


def test_wide_dynamic_range_input():
    x = S.complex_wide_range(S.SEED_256_WIDE, (16, 16, 16)).numpy()
    y, mism = ref.obfft3d(x, ((4, 4), (4, 4), (4, 4)))
    assert mism == 0
    err = ref.normwise_error(y, ref.dft3d_dd(x))
    assert err < 1e-14
