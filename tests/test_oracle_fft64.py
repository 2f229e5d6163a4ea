"""Pins of the oracle's plain FP64 mixed-radix FFT (the FP64 reference
transform): a library FFT (numpy's pocketfft) as the special case it must
match to rounding, the double-double direct DFT, and closed forms."""
import numpy as np
import pytest

from oracle import ref
from synth import inputs as S


@pytest.mark.parametrize("shape", [(8, 12, 10), (16, 16, 16), (3, 5, 7), (32, 6, 45), (1, 1, 64), (2, 96, 1)])
def test_fft3d_matches_library_fft(shape):
    x = S.complex_gaussian(31, shape).numpy()
    y = ref.fft3d(x)
    yn = np.fft.fftn(x)
    assert np.linalg.norm(y - yn) / np.linalg.norm(yn) < 2e-15
    z = ref.fft3d(x, sign=+1)
    zn = np.fft.ifftn(x) * x.size
    assert np.linalg.norm(z - zn) / np.linalg.norm(zn) < 2e-15


@pytest.mark.parametrize("shape", [(32, 32, 32), (12, 10, 9)])
def test_fft3d_against_double_double(shape):
    x = S.complex_uniform(32, shape).numpy()
    assert ref.normwise_error(ref.fft3d(x), ref.dft3d_dd(x)) < 1e-15


def test_fft3d_closed_forms():
    n = (8, 12, 10)
    x = np.zeros(n, np.complex128)
    x[0, 0, 0] = 1
    assert np.all(ref.fft3d(x) == 1)                       # impulse -> constant, exactly
    c = np.ones(n, np.complex128)
    y = ref.fft3d(c)
    want = np.zeros(n, np.complex128)
    want[0, 0, 0] = np.prod(n)
    assert np.max(np.abs(y - want)) < 1e-12                # constant -> N delta
    j = [np.arange(v) for v in n]
    k = (3, 5, 7)
    ph = np.exp(2j * np.pi * (j[0][:, None, None] * k[0] / n[0] + j[1][None, :, None] * k[1] / n[1]
                              + j[2][None, None, :] * k[2] / n[2]))
    y = ref.fft3d(ph)
    want = np.zeros(n, np.complex128)
    want[k] = np.prod(n)
    assert np.max(np.abs(y - want)) < 1e-11                # single mode -> delta
