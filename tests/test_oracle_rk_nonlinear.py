"""CPU pins of the oracle's nonlinear IF-HERK step and of the grid-update weights,
each against something other than the oracle's own code:

* temporal order: with the nonlinear term on, the velocity error of 4, 8 and 16
  steps against a 64-step run falls at the y-orders the paper's table of scheme
  orders prints (Sec. 3.2: Scheme A 2, Schemes B and C 3).  A wrong a~_ii weight
  in g, a misplaced w^{i,j} recursion or a wrong integrating-factor exponent drops
  the order;
* sign of g (eq. ifherk_g): a free Gaussian-core ring moves along its impulse I at
  about Saffman's speed (Sec. 6, eq. u_saffman); with the sign of g reversed it
  would move backwards;
* the weights of eq. weight_fun on a field whose curl and Lamb-vector divergence
  are known in closed form;
* the depth to which the masks of Sec. 5 corrupt the weight fields;
* the vorticity formulation of Sec. 4.1 against the curl of the primitive-variable step
  (the two are algebraically equivalent).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1601_00035_gb300 import inputs
from tests.helpers import golden
from tests.rk_cases import dilate, small_case


@pytest.mark.parametrize("name", ["A", "B", "C"])
def test_oracle_temporal_order_nonlinear(name):
    """Velocity error against a 64-step run over T = 2 (Re = 10, amplitude 3, B = 4):
    observed orders within 0.3 (A) or 0.4 (B, C) of the printed y-order."""
    cs = small_case(B=4, amp=3.0)
    cube = O.lgf_cube(40)
    re, T, uinf = 10.0, 2.0, (0.05, -0.02, 0.1)
    out = {}
    for nst in (4, 8, 16, 64):
        u = cs["u0"].copy()
        for _ in range(nst):
            u = O.if_herk_step(u, T / nst, re, cs["dx"], uinf, cs["masks"], cube, nonlinear=True,
                               tab=O.SCHEMES[name])
        out[nst] = u
    err = [np.linalg.norm(out[n] - out[64]) / np.linalg.norm(out[64]) for n in (4, 8, 16)]
    orders = [math.log2(err[0] / err[1]), math.log2(err[1] / err[2])]
    want = golden("scheme_%s_y_order" % name)
    tol = 0.3 if want < 3 else 0.4
    assert all(abs(o - want) <= tol for o in orders), (name, err, orders)


def _free_ring(B=4, R=4.0, sigma=1.0, axis=(0.3, -0.2, 1.0)):
    """A Gaussian-core ring (Gamma = 1) centred in a 4^3-block D_soln, its velocity by
    the oracle's Vor2Vel path (a = -L^{-1} w per component, u = C^T a, eq. vel_refresh)."""
    soln = np.array([[x, y, z] for z in range(1, 5) for y in range(1, 5) for x in range(1, 5)], dtype=np.int32)
    xsoln = dilate(soln)                       # blocks 0..5
    n = 8 * B                                  # dense box = blocks -1..6
    origin = np.array([-1, -1, -1])
    c = np.array([n / 2.0] * 3)
    axis = np.asarray(axis, dtype=float) / np.linalg.norm(axis)
    w = inputs.vortex_ring_edges(n, R, sigma, axis, centre=c)
    xs = O.block_mask((n, n, n), B, xsoln, origin)
    so = O.block_mask((n, n, n), B, soln, origin)
    cube = O.lgf_cube(2 * n)
    a = np.stack([-O.poisson_masked(cube, w[q] * so, so, xs, 1.0) for q in range(3)])
    u0 = O.op_Ct(a * xs, 1.0) * xs
    masks = {"supp": so, "soln": so, "xsoln": xs}
    return dict(u0=u0, masks=masks, cube=cube, axis=axis, origin_cells=origin * B, R=R, sigma=sigma)


def test_free_ring_moves_along_its_impulse():
    """Two steps of Scheme A at Re = 1000 (alpha = 1e-3): the ring position X . I/|I|
    (eq. int_quantities) advances along +I at 0.5-1.5 times Saffman's speed
    Gamma/(4 pi R) (ln(8R/delta) - beta_0), beta_0 from the paper (eq. u_saffman)."""
    r = _free_ring()
    xs, so = r["masks"]["xsoln"], r["masks"]["soln"]
    d0 = O.ring_diagnostics(r["u0"], 1.0, r["origin_cells"], xs, so)
    Ihat = d0["I"] / np.linalg.norm(d0["I"])
    assert float(Ihat @ r["axis"]) > 0.99          # the impulse lies along the ring axis
    dt, nst = 1.0, 2
    u = r["u0"]
    for _ in range(nst):
        u = O.if_herk_step(u, dt, 1000.0, 1.0, (0.0, 0.0, 0.0), r["masks"], r["cube"], nonlinear=True)
    d1 = O.ring_diagnostics(u, 1.0, r["origin_cells"], xs, so)
    speed = float((d1["X"] - d0["X"]) @ Ihat) / (dt * nst)
    saffman = 1.0 / (4 * math.pi * r["R"]) * (math.log(8 * r["R"] / r["sigma"]) - golden("saffman_beta0"))
    assert 0.5 * saffman < speed < 1.5 * saffman, (speed, saffman)


def _depth_map(xs):
    """Chebyshev depth of each D_xsoln cell: 1 on the outermost layer, 2 on the next, ..."""
    depth = np.zeros(xs.shape, dtype=int)
    inner, d = xs.copy(), 0
    while inner.any():
        d += 1
        er = inner.copy()
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dxx in (-1, 0, 1):
                    er &= O.shift(O.shift(O.shift(inner, 0, dxx), 1, dy), 2, dz)
        depth[inner & ~er] = d
        inner = er
    return depth


def test_regrid_weights_closed_form():
    """u = (0, 0, u_z(x)) with u_z(i) = sum_{k<i} s(k), s constant on each x-block column:
    App. A gives w_y(i) = u_z(i) - u_z(i+1) = -s(i) and, with uinf = 0, the Lamb-vector
    term N_x(i) = -s(i) (u_z(i) + u_z(i+1)) / 2 and q(i) = N_x(i) - N_x(i-1) (all other
    components vanish).  mu and nu of each block are the maxima of |w| and |q| over its
    cells deeper than 3 cells inside D_xsoln, written out here from those closed forms."""
    cs = small_case(B=8)
    B, org = cs["B"], cs["origin"]
    xs = cs["masks"]["xsoln"]
    n = xs.shape[0]
    slope = {0: 0.3, 1: -0.7, 2: 0.2, 3: 1.1}            # per x-block of D_xsoln (blocks 0..3)
    i0 = -org[0] * B                                     # dense index of x-block 0
    s = np.array([slope.get((i - i0) // B, 0.0) if 0 <= i - i0 < 4 * B else 0.0 for i in range(n)])
    uz = np.concatenate([[0.0], np.cumsum(s)])[:n] - 1.5  # u_z(i) = sum_{k<i} s(k) + const
    u = np.zeros((3, n, n, n))
    u[2] = uz[None, None, :]
    u *= xs
    W, mu, nu = O.regrid_weights(u, (0.0, 0.0, 0.0), 1.0, xs, B, cs["xsoln"], org, parts=True)
    # closed forms along x (the field is uniform in y and z)
    Nx = np.array([-s[i] * (uz[i] + (uz[i + 1] if i + 1 < n else 0.0)) / 2 for i in range(n)])
    q = np.array([Nx[i] - (Nx[i - 1] if i > 0 else 0.0) for i in range(n)])
    depth = _depth_map(xs)
    for k, (bx, by, bz) in enumerate(cs["xsoln"].tolist()):
        lo = (np.array([bx, by, bz]) - org) * B
        sl = (slice(lo[2], lo[2] + B), slice(lo[1], lo[1] + B), slice(lo[0], lo[0] + B))
        keep = depth[sl] > 3
        xs_idx = np.nonzero(keep.any(axis=(0, 1)))[0] + lo[0]
        assert len(xs_idx) > 0
        assert mu[k] == pytest.approx(np.abs(s[xs_idx]).max(), rel=1e-12)
        assert nu[k] == pytest.approx(np.abs(q[xs_idx]).max(), rel=1e-12)
    assert W == pytest.approx(np.maximum(mu / mu.max(), nu / nu.max()), rel=1e-12)
    # the block columns order as their slopes do
    assert mu.max() == pytest.approx(1.1)


def test_mask_contamination_depth():
    """The masks corrupt w = M C M u and q = -M G^T M N~(M (u + uinf)) on the outermost
    D_xsoln cell layer only: against the same operators on the unmasked smooth field, the
    values differ (by O(|u|)) at depth 1 and agree exactly at every depth >= 2.  The grid
    update leaves out 3 layers (the reading of 'significantly contaminated' taken for
    Sec. 5): a margin of two layers beyond this one."""
    cs = small_case(B=8)
    xs = cs["masks"]["xsoln"]
    n = xs.shape[0]
    z, y, x = np.meshgrid(*[np.arange(n)] * 3, indexing="ij")
    u = np.stack([0.3 * np.sin(0.2 * y + 0.1 * z) + 0.1, 0.2 * np.cos(0.15 * x) - 0.05 * (z - n / 2) / n,
                  0.25 * np.sin(0.1 * x + 0.2 * y)])
    uinf = np.array([0.05, -0.02, 0.1]).reshape(3, 1, 1, 1)
    w_m = O.op_C(u * xs) * xs
    w_u = O.op_C(u) * xs
    q_m = -O.op_Gt(O.op_N((u + uinf) * xs) * xs) * xs
    q_u = -O.op_Gt(O.op_N(u + uinf)) * xs
    depth = _depth_map(xs)
    dw = np.abs(w_m - w_u).max(0)
    dq = np.abs(q_m - q_u)
    assert dw[depth == 1].max() > 0.1 and dq[depth == 1].max() > 0.1
    assert dw[depth >= 2].max() == 0.0 and dq[depth >= 2].max() == 0.0


@pytest.mark.parametrize("name", ["A", "B", "C"])
def test_vorticity_step_is_curl_of_primitive_step(name):
    """Sec. 4.1: the vorticity formulation (curl of eq. dnstp, velocity from eq. vel_vor, no
    projection) is algebraically the primitive-variable one: one step of each from w0 = C u0
    agrees on D_soln to far below the step's own change (the masks of Sec. 5 differ slightly
    in the two forms, within 1e-6 here)."""
    cs = small_case(B=8, amp=3.0)
    cube = O.lgf_cube(64)
    m, dx = cs["masks"], cs["dx"]
    uinf = (0.05, -0.02, 0.1)
    u0 = cs["u0"]
    w0 = O.op_C(u0 * m["xsoln"], dx) * m["xsoln"]
    u1 = O.if_herk_step(u0, 0.5, 10.0, dx, uinf, m, cube, nonlinear=True, tab=O.SCHEMES[name])
    w1 = O.if_herk_step_vorticity(w0, 0.5, 10.0, dx, uinf, m, cube, tab=O.SCHEMES[name])
    wc = O.op_C(u1 * m["xsoln"], dx) * m["xsoln"]
    so = m["soln"]
    diff = np.linalg.norm((w1 - wc)[:, so]) / np.linalg.norm(wc[:, so])
    change = np.linalg.norm((w1 - w0)[:, so]) / np.linalg.norm(w0[:, so])
    assert change > 0.1 and diff < 1e-6, (diff, change)
