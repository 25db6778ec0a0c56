"""Pins for the oracle's staggered-grid operators (App. A) and mimetic identities (Sec. 2.1).

Random fields with a zero border (so that the mask of the finite box drops
nothing) are used for the exact identities; the nonlinear term is pinned by
its second-order convergence to (curl f) x f for a smooth field, which a
wrong index, sign or averaging weight would break.
"""
import numpy as np

import oracle as O

rng = np.random.default_rng(5)


def _rand(shape, pad=3):
    a = np.zeros(shape)
    sl = tuple(slice(pad, s - pad) for s in shape[-3:])
    a[(Ellipsis,) + sl] = rng.standard_normal(a[(Ellipsis,) + sl].shape)
    return a


def test_adjoint_G():
    c = _rand((12, 12, 12))
    f = _rand((3, 12, 12, 12))
    assert abs((O.op_G(c) * f).sum() - (c * O.op_Gt(f)).sum()) < 1e-12


def test_adjoint_C():
    f = _rand((3, 12, 12, 12))
    e = _rand((3, 12, 12, 12))
    assert abs((O.op_C(f) * e).sum() - (f * O.op_Ct(e)).sum()) < 1e-12


def test_Dbar_is_minus_Gt():
    f = _rand((3, 10, 10, 10))
    assert np.allclose(O.op_Dbar(f), -O.op_Gt(f))


def test_curl_grad_zero_div_curl_zero():
    c = _rand((12, 12, 12))
    f = _rand((3, 12, 12, 12))
    assert np.abs(O.op_C(O.op_G(c))).max() < 1e-12
    assert np.abs(O.op_D(O.op_C(f))).max() < 1e-12


def test_laplacians_mimetic():
    c = _rand((12, 12, 12))
    assert np.allclose(O.op_L(c), -O.op_Gt(O.op_G(c)), atol=1e-12)
    f = _rand((3, 12, 12, 12))
    assert np.allclose(O.op_L(f), -O.op_G(O.op_Gt(f)) - O.op_Ct(O.op_C(f)), atol=1e-12)


def test_nonlinear_second_order():
    """N(f) -> (curl f) x f at face positions with O(dx^2) error."""
    errs = []
    for n in (24, 48):
        dx = 1.0 / n
        f = np.zeros((3, n, n, n))
        z, y, x = np.meshgrid(*[np.arange(n) * dx] * 3, indexing="ij")

        def field(px, py, pz):
            return np.stack([np.sin(2 * np.pi * py) * np.cos(2 * np.pi * pz),
                             np.sin(2 * np.pi * pz) * np.cos(2 * np.pi * px),
                             np.sin(2 * np.pi * px) * np.cos(2 * np.pi * py)])

        # face (q) position: vertex shifted -1/2 in the two directions != q
        for q in range(3):
            s = [-0.5 * dx] * 3
            s[q] = 0.0
            f[q] = field(x + s[0], y + s[1], z + s[2])[q]
        N = O.op_N(f, dx)
        # exact (curl f) x f at face positions, per component
        ex = np.zeros_like(N)
        for q in range(3):
            s = [-0.5 * dx] * 3
            s[q] = 0.0
            px, py, pz = x + s[0], y + s[1], z + s[2]
            k = 2 * np.pi
            F = field(px, py, pz)
            w = np.stack([
                -k * np.sin(k * px) * np.sin(k * py) - k * np.cos(k * pz) * np.cos(k * px),
                -k * np.sin(k * py) * np.sin(k * pz) - k * np.cos(k * px) * np.cos(k * py),
                -k * np.sin(k * pz) * np.sin(k * px) - k * np.cos(k * py) * np.cos(k * pz),
            ])
            ex[q] = np.cross(w, F, axis=0)[q]
        inner = (slice(None),) + (slice(3, n - 3),) * 3
        errs.append(np.abs(N - ex)[inner].max())
    order = np.log2(errs[0] / errs[1])
    assert 1.8 < order < 2.3, errs
