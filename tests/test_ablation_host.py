"""Host checks of the epilogue ablation's Kulisch word layouts (Strategy A of
Sec. "INT16 and INT8"): the word counts of the paper's substrate table, the
guard-bit capacity of every word, and an exact emulation of the packed-word
deposit and carry sweep the ablation kernel performs."""
import math

import numpy as np
import pytest

from oracle import constants as C

S_RAW = 15
P_BITS = 23                    # every slice sum P_s < 2^23
LAYOUTS = {32: 28, 16: 12, 8: 6}  # word width -> radix bits (rho)


def words_needed(rho, bits=130):
    return math.ceil(bits / rho)


def test_paper_substrate_table_word_counts():
    """Table 'Width-parameterised Kulisch Phase B': 130-bit accumulator in
    5 INT32 (radix ~28), 11 INT16 (~12), 22 INT8 (~6) words."""
    assert [words_needed(LAYOUTS[w]) for w in (32, 16, 8)] == [5, 11, 22]


def pieces(s, rho):
    """(word index, bit width of the piece) of a slice deposited at bit 8 s."""
    pos = 8 * s
    i0, o = divmod(pos, rho)
    out = []
    lo, hi = o, o + P_BITS          # bits of P << o
    j = 0
    while rho * j < hi:
        a, b = max(lo, rho * j), min(hi, rho * (j + 1))
        if b > a:
            out.append((i0 + j, b - a))
        j += 1
    return out


@pytest.mark.parametrize("wb", [32, 16, 8])
def test_guard_bits_absorb_every_deposit(wb):
    """The largest possible sum of pieces in any word stays below 2^wb, so the
    packed lanes never carry into each other before the sweep."""
    rho = LAYOUTS[wb]
    load = {}
    for s in range(S_RAW):
        for i, width in pieces(s, rho):
            load[i] = load.get(i, 0) + (2 ** width - 1)
    assert max(load.values()) < 2 ** wb
    top = 8 * (S_RAW - 1) + P_BITS
    nw = (top + rho - 1) // rho + 1
    assert max(load) < nw and rho * nw >= 131   # the exact magnitude fits (Eq. accwidth: 131 bits)


@pytest.mark.parametrize("wb", [32, 16, 8])
def test_packed_deposit_and_sweep_are_exact(wb):
    """Emulates the kernel: pieces added into 32-bit registers holding 32 / wb
    packed words, then the lane extraction, carry sweep and assembly."""
    rho = LAYOUTS[wb]
    lanes = 32 // wb
    top = 8 * (S_RAW - 1) + P_BITS
    nw = (top + rho - 1) // rho + 1
    nr = (nw + lanes - 1) // lanes
    rng = np.random.default_rng(wb)
    cases = [[2 ** P_BITS - 1] * S_RAW, [0] * S_RAW] + \
        [[int(v) for v in rng.integers(0, 2 ** P_BITS, S_RAW)] for _ in range(300)]
    for P in cases:
        regs = [0] * nr
        for s, p in enumerate(P):
            i0, o = divmod(8 * s, rho)
            v = p << o
            j = 0
            while rho * j < P_BITS + o:
                piece = (v >> (rho * j)) & ((1 << rho) - 1)
                i = i0 + j
                regs[i // lanes] = (regs[i // lanes] + (piece << (wb * (i % lanes)))) & 0xFFFFFFFF
                j += 1
        E, carry = 0, 0
        for i in range(nw):
            word = (regs[i // lanes] >> (wb * (i % lanes))) & ((1 << wb) - 1)
            t = word + carry
            carry = t >> rho
            E |= (t & ((1 << rho) - 1)) << (rho * i)
        assert E % 2 ** 128 == sum(p << (8 * s) for s, p in enumerate(P)) % 2 ** 128


# The H0 residue form (fold-and-add for the pseudo-Mersenne members of the
# modulus set, Sec. "Ozaki Scheme II" and the co-design ladder's rung H0): the
# paper names the seven friendly members, and the folds the kernel applies
# (two for a = 11, one for 1024, three for a = 9 from the dp4a bound
# 7 x 255 x (m - 1)) must leave every possible sum below 2m and congruent to it.
H0_FRIENDLY = {2039: (11, 2), 2029: (11, 2), 2027: (11, 2), 1024: (10, 1), 511: (9, 2), 491: (9, 3), 487: (9, 3)}


def test_h0_friendly_members_are_the_papers_seven():
    friendly = [m for m in C.MODULI if any(m == (1 << a) - c for a in (9, 10, 11) for c in range(0, 26))]
    assert sorted(friendly) == sorted(H0_FRIENDLY)
    assert len(friendly) == 7


@pytest.mark.parametrize("m", sorted(H0_FRIENDLY))
def test_h0_folds_reach_two_m_exhaustively(m):
    a, folds = H0_FRIENDLY[m]
    c = (1 << a) - m
    t0 = np.arange(0, 7 * 255 * (m - 1) + 1, dtype=np.int64)
    t = t0.copy()
    for _ in range(folds):
        t = (t >> a) * c + (t & ((1 << a) - 1))
    assert int(t.max()) < 2 * m
    assert np.array_equal(t % m, t0 % m)
