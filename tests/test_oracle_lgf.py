"""Pins for the oracle's unit-lattice LGF table G(n) (App. B, Bessel form).

* G(0) = -W/6, W = Watson's integral in Watson's closed Gamma-function form.
* L G = delta at every table entry (the defining property, Sec. 2.2 with the
  7-point stencil of App. A).  A constant offset would survive this, so it is
  paired with the G(0) pin and the decay pin below.
* |G - (two-term asymptotic)| * |n|^5 tends to a constant along rays
  (App. B expansion; the neglected term is O(|n|^-5)); a wrong sign in either
  printed term breaks the ratio test.
* the quadrature is converged: halving the panels and raising the order
  changes no entry by more than 1e-15 relative.
* the 48-fold symmetry of the dense expansion.
"""
import numpy as np
import pytest

import oracle as O


def test_watson_closed_form():
    # the closed form itself against the integral's known decimal expansion
    assert abs(O.WATSON_W - 1.516386059151978) < 1e-14


def test_G0_is_minus_watson_over_6():
    assert abs(O.lgf_value((0, 0, 0), 8) + O.WATSON_W / 6) < 2e-15


def test_G100():
    # L G (0) = 1  <=>  6 (G(1,0,0) - G(0)) = 1
    g0 = O.lgf_value((0, 0, 0), 8)
    g1 = O.lgf_value((1, 0, 0), 8)
    assert abs(g1 - g0 - 1.0 / 6.0) < 1e-15


def test_L_G_is_delta_everywhere():
    K = 48
    cube = O.lgf_cube(K)
    # full symmetric table on [-K, K]^3
    full = np.zeros((2 * K + 1,) * 3)
    idx = np.abs(np.arange(-K, K + 1))
    full[:] = cube[idx[:, None, None], idx[None, :, None], idx[None, None, :]]
    LG = O.op_L(full)[1:-1, 1:-1, 1:-1]
    delta = np.zeros_like(LG)
    delta[K - 1, K - 1, K - 1] = 1.0
    assert np.abs(LG - delta).max() < 5e-15


@pytest.mark.parametrize("direction", [(1, 0, 0), (1, 1, 0), (1, 1, 1), (3, 2, 1)])
def test_asymptotic_n_minus_5(direction):
    d = np.array(direction, dtype=float)
    errs = []
    for s in (16, 32, 64):
        n = (d * s).astype(int)
        r = np.linalg.norm(n)
        errs.append(abs(O.lgf_value(n, 200) - O.asymptotic_G(n)) * r ** 5)
    # error * |n|^5 approaches a constant: consecutive doublings change it by < 10 %
    assert abs(errs[1] / errs[2] - 1) < 0.1, errs
    assert abs(errs[0] / errs[1] - 1) < 0.2, errs


def test_asymptotic_absolute_far():
    n = np.array([150, 90, 40])
    assert abs(O.lgf_value(n, 200) - O.asymptotic_G(n)) < 1e-12


def test_quadrature_converged():
    K = 40
    a = O.lgf_octant(K)
    b = O.lgf_octant(K, panel=0.5, ngl=24)
    assert np.max(np.abs(a - b) / np.abs(b)) < 1e-15 * 10


def test_symmetry_of_cube():
    cube = O.lgf_cube(20)
    assert np.array_equal(cube, cube.transpose(1, 0, 2))
    assert np.array_equal(cube, cube.transpose(2, 1, 0))
    assert np.array_equal(cube, cube.transpose(0, 2, 1))


def test_monotone_and_negative():
    cube = O.lgf_cube(30)
    axis = cube[0, 0, :]
    assert np.all(axis < 0) and np.all(np.diff(axis) > 0)


def test_points_equal_table():
    rng = np.random.default_rng(1)
    o = rng.integers(-40, 41, size=(200, 3))
    cube = O.lgf_cube(40)
    a = np.abs(o)
    ref = cube[a[:, 2], a[:, 1], a[:, 0]]
    # same quadrature; the Miller start index follows the largest requested offset,
    # so agreement is to the last bits rather than bitwise
    assert np.max(np.abs(O.lgf_points(o) - ref) / np.abs(ref)) < 2e-15
