"""Pins of the oracle's double-double references at double-double precision.

The accuracy of every Ozaki result is measured against the oracle's
double-double DFTs (`ref.dft_dd_lines`, `ref.dft3d_dd`, `ref.dft3d_dd_point`).
Comparing them with a library FFT only shows they are right to about 1e-16,
which a plain-double DFT also is.  Here they are compared with the exact DFT
of the same double inputs, evaluated by mpmath at 240-bit precision.

Error bound used: every double-double add or multiply has relative error
below about 8 u^2 (u = 2^-53, u^2 = 1.2e-32) and the twiddles carry one
double-double rounding, so an output of a length-N sum is within about
(N + 4) * 8 u^2 * sum_j |x_j| of the exact value; the separable 3-D sum
compounds that over its three axes.  The tests require 1e-29 * sum_j |x_j|
per output (2e-30 relative to the line sums at N = 32, with margin), which a
plain-double DFT (error about u * N * sum|x| = 1e-15 * sum|x|) misses by
fourteen orders of magnitude.  Negative controls: the same check fails once
the `lo` words of the twiddles or of the outputs are dropped.
"""
import mpmath
import numpy as np
import pytest

from oracle import ref
from synth import inputs as S

mpmath.mp.prec = 240
TOL = 1e-29


def _exact_twiddles(N, sign):
    # exp(sign 2 pi i m / N) at 240 bits, m < N
    return [mpmath.expjpi(mpmath.mpf(2 * sign * m) / N) for m in range(N)]


def _exact_dft_line(xs, sign):
    N = len(xs)
    w = _exact_twiddles(N, sign)
    return [mpmath.fsum(xs[j] * w[(j * k) % N] for j in range(N)) for k in range(N)]


def _mp(x):
    return [mpmath.mpc(float(v.real), float(v.imag)) for v in x]


def _dd_err(hi_lo, exact):
    """|(hi + lo) - exact| evaluated exactly in mpmath, per complex output."""
    re = mpmath.mpf(float(hi_lo[0])) + mpmath.mpf(float(hi_lo[1]))
    im = mpmath.mpf(float(hi_lo[2])) + mpmath.mpf(float(hi_lo[3]))
    return float(abs(mpmath.mpc(re, im) - exact))


@pytest.mark.parametrize("N", [3, 8, 12, 32])
@pytest.mark.parametrize("sign", [-1, 1])
def test_dd_lines_against_mpmath(N, sign):
    x = S.complex_uniform(900 + N, (4, N)).numpy()
    y = ref.dft_dd_lines(ref.to_dd(x), sign)
    worst = 0.0
    for l in range(x.shape[0]):
        ex = _exact_dft_line(_mp(x[l]), sign)
        scale = float(np.sum(np.abs(x[l])))
        for k in range(N):
            worst = max(worst, _dd_err(y[l, k], ex[k]) / scale)
    assert worst <= TOL, worst


def _exact_dft3(x, sign):
    """Exact separable 3-D DFT (axis 2, then 1, then 0) of a small grid in mpmath."""
    n0, n1, n2 = x.shape
    a = [[[mpmath.mpc(float(x[i, j, k].real), float(x[i, j, k].imag)) for k in range(n2)]
          for j in range(n1)] for i in range(n0)]
    w = {n: _exact_twiddles(n, sign) for n in (n0, n1, n2)}

    def dft(v, n):
        return [mpmath.fsum(v[j] * w[n][(j * k) % n] for j in range(n)) for k in range(n)]

    a = [[dft(a[i][j], n2) for j in range(n1)] for i in range(n0)]
    for i in range(n0):
        for k in range(n2):
            col = dft([a[i][j][k] for j in range(n1)], n1)
            for j in range(n1):
                a[i][j][k] = col[j]
    for j in range(n1):
        for k in range(n2):
            col = dft([a[i][j][k] for i in range(n0)], n0)
            for i in range(n0):
                a[i][j][k] = col[i]
    return a


@pytest.fixture(scope="module")
def grid_6_10_9():
    x = S.complex_uniform(977, (6, 10, 9)).numpy()
    return x, _exact_dft3(x, -1)


def test_dd_3d_against_mpmath(grid_6_10_9):
    x, ex = grid_6_10_9
    y = ref.dft3d_dd(x, -1)
    scale = float(np.sum(np.abs(x)))
    worst = max(_dd_err(y[i, j, k], ex[i][j][k]) / scale
                for i in range(6) for j in range(10) for k in range(9))
    assert worst <= TOL, worst


@pytest.mark.parametrize("k", [(0, 0, 0), (1, 2, 3), (5, 9, 8), (3, 0, 4)])
def test_dd_point_against_mpmath(grid_6_10_9, k):
    x, ex = grid_6_10_9
    pt = ref.dft3d_dd_point(x, k, -1)
    assert _dd_err(pt, ex[k[0]][k[1]][k[2]]) / float(np.sum(np.abs(x))) <= TOL


def test_negative_control_plain_double_twiddles(monkeypatch):
    """A double-double DFT whose twiddles lost their lo words is only
    double-accurate: the check above must reject it."""
    N = 12
    x = S.complex_uniform(912, (2, N)).numpy()
    full = ref.dd_twiddles(N, -1)
    plain = full.copy()
    plain[:, 1] = 0.0
    plain[:, 3] = 0.0
    monkeypatch.setattr(ref, "dd_twiddles", lambda n, s: plain if (n, s) == (N, -1) else full)
    y = ref.dft_dd_lines(ref.to_dd(x), -1)
    ex = _exact_dft_line(_mp(x[0]), -1)
    scale = float(np.sum(np.abs(x[0])))
    worst = max(_dd_err(y[0, k], ex[k]) / scale for k in range(N))
    assert worst > 1e3 * TOL


def test_negative_control_dropped_output_lo(grid_6_10_9):
    """The hi words alone (a correctly rounded double result at best) fail the bound."""
    x, ex = grid_6_10_9
    y = ref.dft3d_dd(x, -1).copy()
    y[..., 1] = 0.0
    y[..., 3] = 0.0
    scale = float(np.sum(np.abs(x)))
    worst = max(_dd_err(y[i, j, k], ex[i][j][k]) / scale
                for i in range(6) for j in range(10) for k in range(9))
    assert worst > 1e3 * TOL
