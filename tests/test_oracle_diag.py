"""Pins for the oracle's ring diagnostics (Sec. 6 eq. int_quantities on the lattice).

A Gaussian-core ring (eq. initial_omega_gauss read as in the input recipe),
u = C^T a with a = -L^{-1} w0 (the free-space velocity, direct sums):
* impulse |I| = pi Gamma (R^2 + sigma^2 / 2) along the axis (Gaussian moments);
* enstrophy E = Gamma^2 R / (2 sigma^2) (leading order in sigma / R);
* centroid: along the axis, X at the ring centre (the printed formula's transverse
  components are 3/2 of the centre's, from int x_i w_j = eps_ijk I_k); helicity J = 0;
* K = sum u . (x cross w) equals the kinetic energy 1/2 sum |u|^2, the identity
  of the integrals for decaying fields (less the box's far-field tail).
* I, E and J are unchanged when the field is moved by whole cells.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1601_00035_gb300 import inputs


@pytest.fixture(scope="module")
def ring():
    n, R, sig = 48, 10.0, 2.0
    c = np.array([n / 2.0 + 0.3, n / 2.0 - 0.2, n / 2.0 + 0.1])
    axis = np.array([0.0, 0.0, 1.0])
    w0 = inputs.vortex_ring_edges(n, R, sig, axis, centre=c)
    K = n
    cube = O.lgf_cube(K)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    pts = np.stack([x.ravel(), y.ravel(), z.ravel()], 1).astype(np.int32)
    a = np.zeros_like(w0)
    for q in range(3):
        v = w0[q].ravel()
        nz = np.abs(v) > 1e-10 * np.abs(w0).max()
        a[q] = -O.direct_conv(cube, pts[nz], v[nz], pts).reshape(n, n, n)
    u = O.op_Ct(a, 1.0)
    xs = np.ones((n, n, n), dtype=bool)
    xs[:1] = xs[-1:] = False
    xs[:, :1] = xs[:, -1:] = False
    xs[:, :, :1] = xs[:, :, -1:] = False
    so = np.zeros((n, n, n), dtype=bool)                 # the vorticity's support, away from the mask edge
    so[6:-6, 6:-6, 6:-6] = True
    return dict(n=n, R=R, sig=sig, c=c, u=u * xs, xs=xs, so=so)


def test_closed_forms(ring):
    d = O.ring_diagnostics(ring["u"], 1.0, (0, 0, 0), ring["xs"], ring["so"])
    R, sig = ring["R"], ring["sig"]
    assert abs(d["I"][2] / (math.pi * (R * R + sig * sig / 2)) - 1) < 0.01, d["I"]
    assert np.abs(d["I"][:2]).max() < 1e-6 * abs(d["I"][2])
    assert abs(d["E"] / (R / (2 * sig * sig)) - 1) < 0.05, d["E"]
    # X as printed is covariant only along I: for a symmetric ring centred at c,
    # int x_i w_j = eps_ijk I_k gives X = 3c/2 - (I^ . c) I^/2, i.e. the centre along
    # the axis (the component the ring speed is read from)
    ih = d["I"] / np.linalg.norm(d["I"])
    want = 1.5 * ring["c"] - 0.5 * (ih @ ring["c"]) * ih
    assert np.abs(d["X"] - want).max() < 0.05, (d["X"], want)
    assert abs(d["X"] @ ih - ring["c"] @ ih) < 0.05
    uc = np.abs(ring["u"]).max()
    assert abs(d["J"]) < 1e-3 * d["E"] * uc * 10
    ke = 0.5 * float((ring["u"] ** 2).sum())   # over the box: the dipole tail beyond it is missed
    assert abs(d["K"] / ke - 1) < 0.1, (d["K"], ke)


def test_shift_invariance(ring):
    u = ring["u"]
    d0 = O.ring_diagnostics(u, 1.0, (0, 0, 0), ring["xs"], ring["so"])
    d1 = O.ring_diagnostics(u, 1.0, (1, -2, 3), ring["xs"], ring["so"])   # moved by (1, -2, 3) cells
    for k in ("E", "J"):
        assert abs(d1[k] - d0[k]) <= 1e-12 * abs(d0["E"])
    # I moves by c x (sum of w over the mask), which the mask edge leaves at ~1e-9 of I
    assert np.abs(d1["I"] - d0["I"]).max() < 1e-7 * np.abs(d0["I"]).max()
