"""Exhaustive checks of the tensor-core operand layouts (TEST INFRASTRUCTURE ONLY).

The paper assumes each residue travels in E4M3 planes but proves no exact
layout for the 11-bit primes (Background, "Layout caveat").  The contract an
exact layout must meet: every operand an E4M3-exact value, every FP32 partial
sum an integer below 2^24, and the weighted recombination congruent to a*b
mod m.  This module states the build's layouts independently of the CUDA code
(written from the rules, not shared) and checks them for every residue of
every modulus with numpy.

Layouts (balanced residues v in (-m/2, m/2]):
  m = s^2 (1089, 1024, 961, 841, 625, 529): v = s h + l, h = RNE(v / s);
      a b = s (a_h b_l + a_l b_h) + a_l b_l  (mod m).
  511, 491, 487: v = d0 + 16 d1, d1 = RNE(v / 16).
  2039, 2029, 2027: v = d0 + 16 d1 + 256 d2, d2 = RNE(v / 256), d1 = RNE((v - 256 d2) / 16).
  Weight classes w = i + j of digit pairs accumulate in one FP32 register
  each; 16^3 and 16^4 are reduced mod m before the recombination.
INT8 two-limb split (Eq. h1-group): v = v0 + 256 v1, v0 in [-128, 128), v1 in [0, 8].
"""
from __future__ import annotations

import numpy as np

from .constants import MODULI


def e4m3_exact(x: np.ndarray) -> np.ndarray:
    """True where the integer x is exactly representable in E4M3 (|x| <= 448,
    at most 4 significant bits)."""
    a = np.abs(x.astype(np.int64))
    ok = a <= 448
    nz = a > 0
    lead = np.zeros_like(a)
    lead[nz] = np.floor(np.log2(a[nz])).astype(np.int64)
    shift = np.maximum(lead - 3, 0)
    ok &= (a >> shift) << shift == a
    return ok


def rne_div(v: np.ndarray, d: int) -> np.ndarray:
    """Round-half-even of v / d for integer arrays."""
    q = np.floor_divide(v, d)
    r = v - q * d
    up = (2 * r > d) | ((2 * r == d) & (q % 2 == 1))
    return q + up


def balanced(m: int) -> np.ndarray:
    """Every integer v with |v| <= m/2: the balanced representatives of all
    residues mod m, with both -m/2 and m/2 for even m (a round-half-even
    reduction v = x - m RNE(x/m) can give either)."""
    return np.arange(-(m // 2), m // 2 + 1, dtype=np.int64)


def digits(m: int, v: np.ndarray):
    """(digits list, weights list per class, class of pair (i, j))."""
    s = int(round(m ** 0.5))
    if s * s == m:
        h = rne_div(v, s)
        return [h, v - s * h], "square", s
    if m < 1024:
        d1 = rne_div(v, 16)
        return [v - 16 * d1, d1], "base16", None
    d2 = rne_div(v, 256)
    r = v - 256 * d2
    d1 = rne_div(r, 16)
    return [r - 16 * d1, d1, d2], "base16", None


def class_weights(m: int, kind: str, s):
    if kind == "square":
        return {0: 1, 1: s}
    return {w: pow(16, w, m) if w >= 3 else 16 ** w for w in range(5)}


def check_fp8_layout(m: int, K: int = 32) -> dict:
    """Exhaustive: digits reconstruct v and are E4M3-exact; worst-case class sums
    over K terms stay < 2^24; the recombination equals a*b mod m for every pair."""
    v = balanced(m)
    dg, kind, s = digits(m, v)
    # reconstruction and exactness of every digit of every residue
    if kind == "square":
        rec = s * dg[0] + dg[1]
    else:
        rec = sum(d * 16 ** i for i, d in enumerate(dg))
    assert np.array_equal(rec, v), m
    for d in dg:
        assert e4m3_exact(d).all(), m
    nd = len(dg)
    maxd = [int(np.abs(d).max()) for d in dg]
    # pairs per class (const digit i, data digit j)
    if kind == "square":
        pairs = {1: [(0, 1), (1, 0)], 0: [(1, 1)]}
    else:
        pairs = {}
        for i in range(nd):
            for j in range(nd):
                pairs.setdefault(i + j, []).append((i, j))
    wts = class_weights(m, kind, s)
    # worst-case class magnitude (K terms of the largest digit products)
    cls_max = {w: K * sum(maxd[i] * maxd[j] for i, j in pl) for w, pl in pairs.items()}
    assert max(cls_max.values()) < 2 ** 24
    comb_max = sum(wts[w] * cls_max[w] for w in pairs)
    assert comb_max < 2 ** 24, (m, comb_max)
    # exhaustive recombination for all (a, b): sum_w wts[w] sum_pairs a_i b_j == a b (mod m)
    a = v[:, None]
    b = v[None, :]
    da = [d[:, None] for d in dg]
    db = [d[None, :] for d in dg]
    n = v.size
    tot = np.zeros((n, n), dtype=np.int64)
    for w, pl in pairs.items():
        cw = sum(da[i] * db[j] for i, j in pl)
        tot += wts[w] * cw
    assert np.array_equal(np.mod(tot - a * b, m), np.zeros((n, n), np.int64)), m
    return {"modulus": m, "kind": kind, "planes": nd, "mmas_per_product": sum(len(p) for p in pairs.values()),
            "classes": len(pairs), "max_digit": maxd, "max_combined": int(comb_max)}


def check_fp16_carrier(m: int, K: int = 64) -> dict:
    """FP16-carrier layout: every balanced data residue v is one FP16 operand;
    every balanced constant residue a = c0 + 32 c1 with c1 = RNE(a / 32).
    Checks, for every residue of m: both digits and v are FP16-exact integers,
    c0 + 32 c1 = a, and over K terms (both halves of the real-form complex
    product, K = 64) the c0-class stays below 2^24 and the c1-class below 2^22
    (so its reduction mod m by one rounded FP32 quotient is exact), and the
    class-0 sum plus 32 times the reduced class-1 stays below 2^24."""
    a = balanced(m)
    c1 = rne_div(a, 32)
    c0 = a - 32 * c1
    assert np.array_equal(c0 + 32 * c1, a), m
    assert np.abs(c0).max() <= 16 and np.abs(c1).max() <= 32, m
    vmax = int(np.abs(a).max())  # data residues share the balanced range
    assert vmax <= 2048  # FP16 represents every integer up to 2048
    cls0 = K * int(np.abs(c0).max()) * vmax
    cls1 = K * int(np.abs(c1).max()) * vmax
    assert cls0 < 2 ** 24 and cls1 < 2 ** 22, (m, cls0, cls1)
    comb = cls0 + 32 * (m // 2 + 1)
    assert comb < 2 ** 24
    # the recombination is exact integer algebra: c0 v + 32 (c1 v) = a v
    v = a[:, None]
    assert np.array_equal(c0[None, :] * v + 32 * (c1[None, :] * v), a[None, :] * v)
    return {"modulus": m, "max_c0": int(np.abs(c0).max()), "max_c1": int(np.abs(c1).max()),
            "class0_max": cls0, "class1_max": cls1}


def check_int8_two_limb(m: int) -> None:
    """v = v0 + 256 v1 with v0 in [-128, 128), v1 in [0, 8] for every canonical residue."""
    v = np.arange(m, dtype=np.int64)
    v1 = (v + 128) >> 8
    v0 = v - 256 * v1
    assert np.array_equal(v0 + 256 * v1, v)
    assert v0.min() >= -128 and v0.max() < 128 and v1.min() >= 0 and v1.max() <= 8


def alpha_fp8() -> dict:
    """Issued E4M3 MMAs (K = 32 each) per real product, per modulus and in total,
    and per complex GEMM (three Karatsuba products)."""
    per = {m: check_fp8_layout(m)["mmas_per_product"] for m in MODULI}
    tot = sum(per.values())
    return {"per_modulus": per, "alpha_real": tot, "alpha_complex": 3 * tot}
