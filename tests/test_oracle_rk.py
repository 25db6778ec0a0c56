"""Pins for the oracle's IF-HERK step (Sec. 3.2 algorithm with Scheme A, Sec. 3.3
projection, Sec. 5 masks).

* With the nonlinear term switched off and a divergence-free start whose support
  stays far from the edge of D_xsoln, the three stages reduce to
  H^2 H^1 u = E(alpha/2) E(alpha/2) u = E(alpha) u (c~ = (1/2, 1, 1), H^3 = I,
  semigroup of Sec. 3.2): checked against one integrating factor of alpha.
* With the nonlinear term on, the last stage is a projection (H^3 = I), so
  G^T u_{k+1} vanishes on the D_supp cells (eq. proj_final with L_C = -G^T G).
* The shifted tableau of Scheme A (eq. herk_shift): a~ rows and c~ = (1/2, 1, 1).
"""
import math

import numpy as np
import pytest

import oracle as O
from tests.rk_cases import small_case


def test_shifted_tableau_scheme_a():
    at, ct, s = O.shifted_tableau()
    assert s == 3
    assert ct[1] == 0.5 and ct[2] == 1.0 and ct[3] == 1.0 and ct[0] == 0.0
    assert math.isclose(at[(1, 1)], 0.5)
    assert math.isclose(at[(2, 1)], math.sqrt(3) / 3) and math.isclose(at[(2, 2)], (3 - math.sqrt(3)) / 3)
    assert math.isclose(at[(3, 1)] + at[(3, 2)] + at[(3, 3)], 1.0)  # b sums to 1


@pytest.mark.parametrize("name", ["A", "B", "C"])
def test_tableau_order_conditions(name):
    """Row sums give c; the classical order conditions hold to the order the
    paper's table of scheme orders gives for y (A: 2, B and C: 3)."""
    tab = O.SCHEMES[name]
    A, b, c = tab["A"], tab["b"], tab["c"]
    assert np.allclose(A.sum(1), c, atol=1e-15)
    assert np.all(np.triu(A) == 0)                     # explicit
    assert math.isclose(b.sum(), 1.0)
    assert math.isclose(b @ c, 0.5)
    third = math.isclose(b @ c ** 2, 1 / 3) and math.isclose(b @ A @ c, 1 / 6)
    from tests.helpers import golden
    assert third == (golden("scheme_%s_y_order" % name) >= 3)


@pytest.mark.parametrize("name,ct", [("B", (1 / 3, 1.0, 1.0)), ("C", (8 / 15, 2 / 3, 1.0))])
def test_shifted_tableau_b_c(name, ct):
    at, c_t, s = O.shifted_tableau(O.SCHEMES[name])
    assert [c_t[i] for i in (1, 2, 3)] == pytest.approx(list(ct))
    tab = O.SCHEMES[name]
    assert at[(1, 1)] == pytest.approx(tab["A"][1, 0])
    assert [at[(3, j)] for j in (1, 2, 3)] == pytest.approx(list(tab["b"]))


def test_linear_step_is_one_integrating_factor():
    cs = small_case(B=8)
    u0 = cs["u0"]
    dt, re, dx = 0.5, 10.0, 1.0       # alpha = 0.05
    cube = O.lgf_cube(64)
    u1 = O.if_herk_step(u0, dt, re, dx, (0.0, 0.0, 0.0), cs["masks"], cube, nonlinear=False)
    ref = O.ifactor_masked(O.ifactor_taps(dt / (re * dx * dx)), u0, cs["masks"]["xsoln"])
    assert np.abs(u1 - ref).max() < 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("name", ["B", "C"])
def test_linear_step_b_c(name):
    """Schemes B and C, nonlinear term off: H^3 H^2 H^1 = E((c~_3 - c~_0) alpha) = E(alpha)."""
    cs = small_case(B=8)
    u0 = cs["u0"]
    dt, re, dx = 0.5, 10.0, 1.0
    u1 = O.if_herk_step(u0, dt, re, dx, (0.0, 0.0, 0.0), cs["masks"], O.lgf_cube(64), nonlinear=False,
                        tab=O.SCHEMES[name])
    ref = O.ifactor_masked(O.ifactor_taps(dt / (re * dx * dx)), u0, cs["masks"]["xsoln"])
    assert np.abs(u1 - ref).max() < 1e-10 * np.abs(ref).max()


def test_step_is_divergence_free_on_supp():
    cs = small_case(B=8)
    u0 = cs["u0"]
    dt, re, dx = 0.5, 10.0, 1.0
    cube = O.lgf_cube(64)
    u1 = O.if_herk_step(u0, dt, re, dx, (0.05, -0.02, 0.1), cs["masks"], cube, nonlinear=True)
    div = O.op_Gt(u1, dx)
    supp = cs["masks"]["supp"]
    assert np.abs(div[supp]).max() < 1e-11 * np.abs(u1).max() / dx
    assert np.abs(u1 - u0).max() > 1e-4 * np.abs(u0).max()  # the step did something


@pytest.mark.parametrize("alpha", [0.05, 0.3, 1.0])
def test_ifactor_tail_is_masked_convolution_error(alpha):
    """App. D: (I - M' E M') u at depth k for a uniform u kept on n > 0, by an explicit
    1-D convolution, equals the kernel tail; and tail(0) = (1 + g(0)) / 2 (kernel mass 1,
    symmetric)."""
    R = 120
    g = O.bessel_scaled(alpha, R)
    kern = np.concatenate([g[:0:-1], g])            # g(-R..R)
    n = np.arange(-300, 301)
    u = (n > 0).astype(float)                        # M' applied to the uniform field 1
    y = np.convolve(u, kern, mode="same") * (n > 0)   # M' E M' u
    for k in (1, 2, 5, 9):
        err = 1.0 - y[n == k][0]
        assert abs(err - O.ifactor_tail(k, alpha)) < 1e-15
    assert abs(O.ifactor_tail(0, alpha) - 0.5 * (1 + g[0])) < 1e-15


def test_rk_qmax_brackets_the_tolerance():
    for beta, depth, eps in [(0.05, 8, 1e-6), (0.086, 16, 1e-6), (0.02, 8, 1e-10)]:
        q = O.rk_qmax(beta, depth, eps)
        assert q >= 1
        assert O.ifactor_tail(depth, q * beta) <= eps < O.ifactor_tail(depth, (q + 1) * beta)


def test_vor2vel_recovers_divergence_free_velocity():
    """u0 = C^T a0 with compact a0: Vor2Vel(u0) = C^T(-L^{-1} C u0) reproduces u0 on D_soln
    (the identity -L = C C^T + D^T D on edges with D C u0 = 0; the masks only touch the
    outermost xsoln layer)."""
    cs = small_case(B=8)
    u0 = cs["u0"]
    u1 = O.vor2vel(u0, cs["masks"], O.lgf_cube(64), cs["dx"])
    so = cs["masks"]["soln"]
    assert np.abs(u1[:, so] - u0[:, so]).max() < 1e-10 * np.abs(u0).max()


def test_regrid_weights():
    """Weights of eq. weight_fun on D_xsoln: in [0, 1] with maximum 1; the blocks that
    hold the ring's vorticity outweigh the buffer; a field that vanishes except on the
    mask-edge layer (the contaminated cells) has zero vorticity weight."""
    cs = small_case(B=8, amp=3.0)
    B, org = cs["B"], cs["origin"]
    W = O.regrid_weights(cs["u0"], (0.05, -0.02, 0.1), cs["dx"], cs["masks"]["xsoln"], B, cs["xsoln"], org)
    assert W.max() == pytest.approx(1.0) and W.min() >= 0.0
    soln = set(map(tuple, cs["soln"].tolist()))
    ws = [W[i] for i, b in enumerate(cs["xsoln"].tolist()) if tuple(b) in soln]
    wb = [W[i] for i, b in enumerate(cs["xsoln"].tolist()) if tuple(b) not in soln]
    assert min(ws) > max(wb)
    # a uniform field: its masked curl and Lamb-vector divergence live only on the mask
    # edge's cell layer, which the weights leave out
    xs = cs["masks"]["xsoln"]
    uni = np.ones_like(cs["u0"]) * np.array([0.3, -0.2, 0.5]).reshape(3, 1, 1, 1) * xs
    with np.errstate(invalid="ignore"):
        W2 = O.regrid_weights(uni, (0.1, 0.0, 0.0), cs["dx"], xs, B, cs["xsoln"], org)
    assert np.all(np.isnan(W2) | (W2 == 0))
