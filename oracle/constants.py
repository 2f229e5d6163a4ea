"""Ozaki-II / CRT / DFT constants, computed from their definitions with Python integers.

TEST INFRASTRUCTURE ONLY.  This package is the oracle: only tests/,
__graft_entry__.smoke() and bench.py's cpu_baseline / reference arm may
import it.  The GPU library computes every one of these constants with its
own host code; the two never share a table or a generator.

Sources (paper sections):
  * modulus set (Rev-34), M and its capacity budget: Background, "Ozaki
    Scheme II" paragraph, Eq. (capacity).
  * CRT idempotents u_k: Eq. (fcrt); byte slices u_k^(s), S = 15: Eq. (slicing).
  * fractional lift weights w_k = round(2^f u_k / M), f = 48, S_frac = 6:
    Sec. "Exact Phase B", paragraph on the two-sided modulo-M centered lift.
  * quantised DFT matrices F_q and twiddle-fused F_p^(k2): Bailey paragraph
    and Eq. (twiddle-fusion); 53-bit signed significands: Eq. (capacity).
"""
from __future__ import annotations

import math
from functools import lru_cache

# Rev-34 modulus set (Background, Ozaki Scheme II paragraph).
MODULI = (2039, 2029, 2027, 1089, 1024, 961, 841, 625, 529, 511, 491, 487)
# Retired Rev-33 set: 509, 503, 499 in place of the three 11-bit primes.
MODULI_REV33 = (509, 503, 499, 1089, 1024, 961, 841, 625, 529, 511, 491, 487)

R = len(MODULI)          # r = 12
S_RAW = 15               # S = ceil(118 / 8) byte slices of u_k
F_BITS = 48              # f = 48 fractional bits of the lift weights
S_FRAC = 6               # S_frac = f / 8 byte slices of w_k
SIGMA_F_EXP = 52         # quantised constants carry 2^52 (53-bit signed significands)
DATA_EXP = 52            # data columns scaled so that |x~| < 2^53


def modulus_product(moduli=MODULI) -> int:
    return math.prod(moduli)


M = modulus_product()


def idempotents(moduli=MODULI) -> list[int]:
    """u_k = (M/m_k) * ((M/m_k)^-1 mod m_k): u_k = 1 mod m_k, 0 mod m_j (j != k)."""
    Mp = modulus_product(moduli)
    out = []
    for m in moduli:
        Mk = Mp // m
        out.append(Mk * pow(Mk, -1, m))
    return out


U = idempotents()


def byte_slices(value: int, count: int) -> list[int]:
    assert 0 <= value < 256 ** count
    return [(value >> (8 * s)) & 0xFF for s in range(count)]


def lift_weights(moduli=MODULI, f=F_BITS) -> list[int]:
    """w_k = round(2^f u_k / M), rounding half up: floor((2^f u_k + M/2) / M)."""
    Mp = modulus_product(moduli)
    assert Mp % 2 == 0
    return [((u << f) + Mp // 2) // Mp for u in idempotents(moduli)]


W = lift_weights()
U_SLICES = [byte_slices(u, S_RAW) for u in U]      # [k][s]
W_SLICES = [byte_slices(w, S_FRAC) for w in W]     # [k][t]
# Compile-time deposit bias of the Kulisch accumulator: sum_s 2^23 * 256^s.
B_TOT = sum((1 << 23) << (8 * s) for s in range(S_RAW))


def capacity_bits(K: int, k: int = 53) -> float:
    """Right-hand side of Eq. (capacity): 1 + log2 K + 2 (k + 1)."""
    return 1 + math.log2(K) + 2 * (k + 1)


# --------------------------------------------------------------------------
# FP32-precision variant (Sec. "Ozaki-II for FP32" and the FP32 paragraph of
# the hardware-ladder section): k = 24-bit significands, capacity budget 56
# bits at K = 32, r = 6 moduli of the Rev-34 set with log2 M = 62.6, S = 8
# byte slices, a 77-bit accumulator.
# --------------------------------------------------------------------------
# The paper names the size of the set but not its members.  Among the six-member
# subsets of the Rev-34 set exactly one has log2 M = 62.6 (to +-0.05): this one.
MODULI_FP32 = (2039, 2029, 2027, 1024, 961, 841)
R_FP32 = len(MODULI_FP32)     # r = 6
S_RAW_FP32 = 8                # S = ceil(63 / 8) byte slices of u_k
# The paper fixes f only for the FP64 set.  Reading: f = 24 (three byte
# slices), for which the lift error r max(v) 2^-f stays far below the 1/4 that
# the two-sided correction needs (6 * 2047 * 2^-24 < 0.001).
F_BITS_FP32 = 24
S_FRAC_FP32 = 3
SIGMA_F_EXP_FP32 = 23         # quantised constants carry 2^23 (24-bit signed significands)
DATA_EXP_FP32 = 23            # data columns scaled so that |x~| < 2^24
M_FP32 = modulus_product(MODULI_FP32)
U_FP32 = idempotents(MODULI_FP32)
W_FP32 = lift_weights(MODULI_FP32, F_BITS_FP32)
U_SLICES_FP32 = [byte_slices(u, S_RAW_FP32) for u in U_FP32]
W_SLICES_FP32 = [byte_slices(w, S_FRAC_FP32) for w in W_FP32]


# --------------------------------------------------------------------------
# High-precision cos / sin of 2*pi*m/N in integer fixed point.
# --------------------------------------------------------------------------
PREC = 240  # fractional bits of the fixed-point evaluation


@lru_cache(maxsize=None)
def _pi_fixed(prec: int = PREC) -> int:
    """pi * 2^prec by Machin's formula, pi = 16 atan(1/5) - 4 atan(1/239)."""
    guard = 32
    one = 1 << (prec + guard)

    def atan_inv(x: int) -> int:
        total, term, n, sign = 0, one // x, 1, 1
        x2 = x * x
        while term:
            total += sign * (term // n)
            term //= x2
            n += 2
            sign = -sign
        return total

    return (16 * atan_inv(5) - 4 * atan_inv(239)) >> guard


def _cos_sin_small(phi: int, prec: int = PREC) -> tuple[int, int]:
    """Taylor series of cos, sin for |phi| <= pi/4, fixed point with prec bits."""
    one = 1 << prec
    neg = phi < 0
    phi = -phi if neg else phi        # terms stay non-negative: the loops end
    phi2 = (phi * phi) >> prec
    c, s = 0, 0
    term = one          # phi^(2n) / (2n)!
    n = 0
    while term > 0:
        c += term if n % 2 == 0 else -term
        term = (term * phi2 >> prec) // ((2 * n + 1) * (2 * n + 2))
        n += 1
    term = phi          # phi^(2n+1) / (2n+1)!
    n = 0
    while term > 0:
        s += term if n % 2 == 0 else -term
        term = (term * phi2 >> prec) // ((2 * n + 2) * (2 * n + 3))
        n += 1
    return c, (-s if neg else s)


@lru_cache(maxsize=None)
def cos_sin_2pi(m: int, N: int, prec: int = PREC) -> tuple[int, int]:
    """(cos, sin)(2 pi m / N) * 2^prec, to within a few units of 2^-prec.

    The argument is reduced exactly: m mod N, then the nearest multiple k of
    pi/2, phi = pi (4m - kN) / (2N) with |phi| <= pi/4.  Points where phi = 0
    come out exact (cos = 1, sin = 0).
    """
    m %= N
    k = (8 * m + N) // (2 * N)            # round(4m / N)
    num = 4 * m - k * N                   # phi = pi * num / (2N)
    phi = (_pi_fixed(prec) * num) // (2 * N) if num >= 0 else -((_pi_fixed(prec) * -num) // (2 * N))
    c, s = _cos_sin_small(phi, prec)
    q = k % 4
    return [(c, s), (-s, c), (-c, -s), (s, -c)][q]


def round_half_even_fixed(v: int, prec: int, scale_exp: int) -> int:
    """RNE of v * 2^(scale_exp - prec) (v a fixed-point integer)."""
    shift = prec - scale_exp
    if shift <= 0:
        return v << (-shift)
    q, r = divmod(v, 1 << shift)
    half = 1 << (shift - 1)
    if r > half or (r == half and (q & 1)):
        q += 1
    return q


def quantised_twiddle(m: int, N: int, sign: int = -1, scale_exp: int = SIGMA_F_EXP) -> tuple[int, int]:
    """RNE(2^scale_exp * omega) for omega = exp(sign * 2 pi i m / N): (Re, Im) integers
    (scale_exp = 52 for the FP64 method, 23 for its FP32 variant)."""
    c, s = cos_sin_2pi(m, N)
    re = round_half_even_fixed(c, PREC, scale_exp)
    im = round_half_even_fixed(s, PREC, scale_exp)
    return re, (im if sign > 0 else -im)


def dft_matrix_q(q: int, sign: int = -1, scale_exp: int = SIGMA_F_EXP) -> list[list[tuple[int, int]]]:
    """Quantised F_q[k2][j2] = RNE(2^scale_exp omega_q^(j2 k2))."""
    return [[quantised_twiddle(j2 * k2, q, sign, scale_exp) for j2 in range(q)] for k2 in range(q)]


def fused_matrices_p(p: int, q: int, sign: int = -1,
                     scale_exp: int = SIGMA_F_EXP) -> list[list[list[tuple[int, int]]]]:
    """Quantised twiddle-fused F_p^(k2)[k1][j1] = RNE(2^scale_exp omega_N^(j1 (q k1 + k2))), N = p q.

    omega_p^(j1 k1) omega_N^(j1 k2) = omega_N^(j1 (q k1 + k2)); the exponent is
    reduced mod N before evaluation (Eq. twiddle-fusion)."""
    N = p * q
    return [[[quantised_twiddle((j1 * (q * k1 + k2)) % N, N, sign, scale_exp) for j1 in range(p)]
             for k1 in range(p)] for k2 in range(q)]


def dd_twiddle(m: int, N: int, sign: int = -1) -> tuple[float, float, float, float]:
    """Double-double (re_hi, re_lo, im_hi, im_lo) of exp(sign 2 pi i m / N)."""
    from fractions import Fraction
    c, s = cos_sin_2pi(m, N)
    if sign < 0:
        s = -s
    out = []
    for v in (c, s):
        fr = Fraction(v, 1 << PREC)
        hi = float(fr)                    # correctly rounded
        lo = float(fr - Fraction(hi))
        out += [hi, lo]
    return tuple(out)


def default_split(N: int) -> tuple[int, int]:
    """Bailey split N = p * q used when the caller gives none: q is the smallest
    divisor >= sqrt(N), p = N / q.  Both must be <= 64 (K <= 64)."""
    if N == 1:
        return 1, 1
    for q in range(1, N + 1):
        if N % q == 0 and q * q >= N:
            return N // q, q
    raise ValueError(N)
