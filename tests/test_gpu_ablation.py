"""GPU parity of the epilogue ablation kernels: every Phase-B word layout and
every residue form gives the value its inputs define, bit for bit.

Phase-B inputs are built from chosen integers C (|C| < 2^116): the offset
residues r_k + 1024 of C, their byte-slice contractions P_s and Q_t with the
oracle's u_k and w_k, as FP32 bit patterns 2^23 + P.  The expected output is
the oracle's correctly rounded RNE(C 2^et)."""
import numpy as np
import pytest
import torch

from oracle import constants as C
from oracle import ref

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2606_23698_gb300 import build as B
    B.build()
    assert torch.cuda.is_available()


def balanced(c, m):
    r = c % m
    return r - m if 2 * r > m else r


def phase_b_inputs(values, ets):
    acc = np.zeros((len(values), 21), np.uint32)
    for i, c in enumerate(values):
        v = [balanced(c, m) + 1024 for m in C.MODULI]
        for s in range(C.S_RAW):
            acc[i, s] = 0x4B000000 + sum(vk * C.U_SLICES[k][s] for k, vk in enumerate(v))
        for t in range(C.S_FRAC):
            acc[i, C.S_RAW + t] = 0x4B000000 + sum(vk * C.W_SLICES[k][t] for k, vk in enumerate(v))
    return acc, np.asarray(ets, np.int32)


def test_phase_b_all_word_widths_exact():
    from paper_2606_23698_gb300 import _lib
    rng = np.random.default_rng(5)
    half = C.M // 2
    vals, ets = [], []
    for _ in range(3000):
        bits = int(rng.integers(1, 117))
        v = int(rng.integers(0, 2 ** 62)) * 2 ** 62 + int(rng.integers(0, 2 ** 62))
        vals.append((v % 2 ** bits) * (1 if rng.random() < 0.5 else -1))
        ets.append(int(rng.integers(-160, -60)))
    # lift-boundary cases (C and C + 1024 both in [-M/2, M/2), the range the
    # lift returns), zero, tiny, subnormal and overflowing results
    for t in range(0, 40):
        vals += [half - 1025 - t, -half + t]
        ets += [-104, -104]
    vals += [0, 1, -1, 2 ** 60, 3 ** 70, -(3 ** 70)]
    ets += [-104, -1074, -1080, -1100, 900, 920]
    acc, et = phase_b_inputs(vals, ets)
    want = np.array([ref.pack(c, e) for c, e in zip(vals, ets)])
    n = len(vals)
    dacc, det = torch.from_numpy(acc.view(np.int32)).cuda(), torch.from_numpy(et).cuda()
    sums = {}
    for variant in (0, 32, 16, 8):
        out = torch.empty(n, dtype=torch.float64, device="cuda")
        ck = torch.zeros(1, dtype=torch.int64, device="cuda")
        _lib.obfft_ablation_phase_b(variant, n, n, dacc.data_ptr(), det.data_ptr(), out.data_ptr(), ck.data_ptr())
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        bad = np.nonzero(got.view(np.uint64) != want.view(np.uint64))[0]
        assert bad.size == 0, (variant, [(vals[i], ets[i], got[i], want[i]) for i in bad[:3]])
        # a longer launch over the same inputs (item i uses input i mod n)
        ck2 = torch.zeros(1, dtype=torch.int64, device="cuda")
        _lib.obfft_ablation_phase_b(variant, n, 7 * n, dacc.data_ptr(), det.data_ptr(), None, ck2.data_ptr(), reps=3)
        torch.cuda.synchronize()
        sums[variant] = (int(ck.item()), int(ck2.item()))
    assert len(set(sums.values())) == 1


def test_residue_forms_exact():
    from paper_2606_23698_gb300 import _lib
    rng = np.random.default_rng(6)
    xs = [int(v) for v in rng.integers(-(2 ** 53) + 1, 2 ** 53, 5000)]
    xs += [0, 1, -1, 2 ** 53 - 1, -(2 ** 53) + 1, 2 ** 40, -(2 ** 40), 1024, -2039]
    n = len(xs)
    want = np.array([[x % m for m in C.MODULI] for x in xs], np.uint16)
    dx = torch.tensor(xs, dtype=torch.int64, device="cuda")
    sums = set()
    for variant in (0, 1, 2, 3):
        res = torch.empty((n, 12), dtype=torch.int16, device="cuda")
        ck = torch.zeros(1, dtype=torch.int64, device="cuda")
        _lib.obfft_ablation_residues(variant, n, n, dx.data_ptr(), res.data_ptr(), ck.data_ptr())
        torch.cuda.synchronize()
        got = res.cpu().numpy().view(np.uint16)
        assert np.array_equal(got, want), variant
        sums.add(int(ck.item()))
    assert len(sums) == 1


def test_ablation_argument_errors():
    from paper_2606_23698_gb300 import _lib
    with pytest.raises(_lib.ObfftError):
        _lib.obfft_ablation_phase_b(12, 1, 1, 0, 0, None, 0)
    with pytest.raises(_lib.ObfftError):
        _lib.obfft_ablation_residues(4, 1, 1, 0, None, 0)
