"""Pins for the oracle's scaled Bessel functions i_n(t) = exp(-2t) I_n(2t) (App. B).

The oracle computes them by Miller's backward recurrence (moderate t) or the
Hankel large-argument series (t > 5e7); mpmath's besseli at 30 digits is an
independent implementation.  The Neumann addition theorem
I_n(x + y) = sum_k I_k(x) I_{n-k}(y) checks the recurrence's normalisation
without any library."""
import numpy as np
import pytest

import oracle as O

CASES = [(1e-12, 4), (1e-6, 3), (0.025, 12), (0.05, 10), (0.5, 30), (1.0, 20), (7.5, 40),
         (37.0, 60), (512.0, 200), (1e4, 300), (3e6, 280), (4e7, 250), (1e9, 20), (5e11, 280)]


@pytest.mark.parametrize("t,nmax", CASES)
def test_bessel_vs_mpmath(t, nmax):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    b = O.bessel_scaled(t, nmax)
    for n in sorted({0, 1, 2, nmax // 3, nmax // 2, nmax}):
        ref = mp.besseli(n, 2 * mp.mpf(t)) * mp.e ** (-2 * mp.mpf(t))
        if ref < mp.mpf("1e-290"):
            continue
        rel = abs(mp.mpf(b[n]) - ref) / ref
        assert rel < 1e-13, (t, n, b[n], ref)


@pytest.mark.parametrize("a,b", [(0.05, 0.05), (0.1, 0.9), (0.3, 2.2), (5.0, 11.0)])
def test_neumann_addition(a, b):
    """exp(-2(a+b)) I_n(2(a+b)) = sum_k i_k(a) i_{n-k}(b), k over all integers (i_{-k} = i_k)."""
    M = 120
    ga, gb, gab = O.bessel_scaled(a, M), O.bessel_scaled(b, M), O.bessel_scaled(a + b, M)
    full_a = np.concatenate([ga[:0:-1], ga])  # k = -M..M
    full_b = np.concatenate([gb[:0:-1], gb])
    conv = np.convolve(full_a, full_b)  # index 0 <-> n = -2M
    for n in range(0, 20):
        assert abs(conv[2 * M + n] - gab[n]) <= 1e-15 + 1e-13 * gab[n]


def test_zero_argument():
    b = O.bessel_scaled(0.0, 5)
    assert b[0] == 1.0 and np.all(b[1:] == 0.0)


def test_bad_args():
    with pytest.raises(ValueError):
        O.bessel_scaled(-1.0, 3)
