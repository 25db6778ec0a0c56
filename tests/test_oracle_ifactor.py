"""Pins for the oracle's integrating factor E_Q(alpha) (Sec. 2.3, App. B eq. lgf_intfac).

* the footnote of Sec. 2.3: G_E(n,0,0)/G_E(0) first drops below 1e-10 at
  n = 7 for alpha = 0.1 and at n = 13 for alpha = 1.0 (this fixes the Bessel
  argument as 2 alpha);
* mass conservation sum_n g(n) = 1 (sigma(0) = 0 in eq. if_def);
* semigroup E(a) E(b) = E(a + b) (Sec. 3.2) through the 1-D factors;
* dE/dalpha = L E (eq. if_dt) through the 1-D factors, by finite differences;
* the plain 3-D sum keeps a constant field constant away from the box edge.
"""
import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("alpha", [0.1, 1.0])
def test_footnote_decay(alpha):
    from tests.helpers import golden
    expected = golden("ifactor_decay_n_alpha_%.1f" % alpha)
    g = O.bessel_scaled(alpha, 40)
    ratio = g / g[0]  # [G_E](n,0,0) / [G_E](0) = g(n) g(0)^2 / g(0)^3
    first = int(np.argmax(ratio < golden("ifactor_decay_threshold")))
    assert first == expected


@pytest.mark.parametrize("alpha", [0.05, 0.2, 1.0, 3.0])
def test_mass(alpha):
    g = O.bessel_scaled(alpha, 80)
    assert abs(g[0] + 2 * g[1:].sum() - 1.0) < 1e-15


def test_semigroup():
    a, b = 0.07, 0.33
    M = 40
    ga, gb, gab = (O.bessel_scaled(x, M) for x in (a, b, a + b))
    fa = np.concatenate([ga[:0:-1], ga])
    fb = np.concatenate([gb[:0:-1], gb])
    conv = np.convolve(fa, fb)[2 * M: 2 * M + 10]
    assert np.allclose(conv, gab[:10], rtol=1e-13, atol=1e-17)


def test_derivative_is_laplacian():
    a, h = 0.4, 1e-5
    M = 30
    gp, gm, g = O.bessel_scaled(a + h, M), O.bessel_scaled(a - h, M), O.bessel_scaled(a, M)
    dg = (gp - gm) / (2 * h)
    full = np.concatenate([g[:0:-1], g])
    lap = np.array([full[M + n - 1] + full[M + n + 1] - 2 * full[M + n] for n in range(10)])
    assert np.allclose(dg[:10], lap, rtol=1e-7, atol=1e-12)


def test_radius_reading():
    # truncation box radius for |E| < 1e-14 (3-D value along an axis)
    assert [O.ifactor_radius(a) for a in (0.05, 0.2, 1.0)] == [7, 9, 15]


def test_direct_constant_field():
    alpha = 0.2
    g = O.ifactor_taps(alpha)
    R = len(g) - 1
    n = 2 * R + 6
    x = np.ones((n, n, n))
    c = n // 2
    y = O.ifactor_direct(g, x, np.array([[c, c, c], [R, R, R]], dtype=np.int32))
    # full mass inside: 1 up to the truncated tail (each axis drops < 1e-13)
    assert abs(y[0] - 1.0) < 5e-13 and abs(y[1] - 1.0) < 5e-13
    y2 = O.ifactor_direct(g, x, np.array([[0, c, c]], dtype=np.int32))
    assert y2[0] < 1.0 - 0.1  # a box edge loses mass (mask M of Sec. 4.4)
