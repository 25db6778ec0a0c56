"""CPU study of the far-field approximation the block-sparse solve makes (the LGF-FMM of
Sec. 2.2 evaluates the convolution "to a tolerance"), computed with the oracle's own
FP64 tables and no GPU code:

* the split of the Bessel form at time a, G = G_near + G_far with
  G_far(n) = -int_a^inf prod_i i_{n_i}(t) dt, reproduces G and leaves G_near < 1e-8 |G(0)|
  beyond 32 cells (a = 20), so near offsets up to two 16^3 blocks suffice;
* the far part replaced by its 10-point Lagrange interpolant on the spacing-2 coarse
  lattice (anterpolation, coarse convolution, interpolation) stays below 1e-6 relative L2
  for a white-noise source block (the worst case for interpolation) and a smooth one;
  the error falls with a and with the order p (the parameter study behind the plan's
  a = 20, p = 10: p = 8 leaves 1.6e-6 on white noise at a = 20).
"""
import numpy as np
import pytest
import scipy.fft as sf

import oracle as O


def _sym(cube):
    K = cube.shape[0] - 1
    idx = np.abs(np.arange(-K, K + 1))
    return cube[np.ix_(idx, idx, idx)]


def _conv(k, f):
    """Linear convolution of f (box at 0) with a kernel given on offsets -K..K, output on f's box."""
    K = k.shape[0] // 2
    L = [sf.next_fast_len(s + 2 * K, real=True) for s in f.shape]
    u = sf.irfftn(sf.rfftn(f, L) * sf.rfftn(k, L), L)
    return u[K:K + f.shape[0], K:K + f.shape[1], K:K + f.shape[2]]


def _interp_matrix(nf, p=10):
    """1-D P[n][j]: fine n of [0, nf), coarse node j - p/2 at fine 2 (j - p/2); even n takes its
    node, odd n = 2i + 1 the p-point Lagrange midpoint weights on nodes i - p/2 + 1 .. i + p/2."""
    h = p // 2
    x = np.arange(float(p))
    w = np.array([np.prod([((p - 1) / 2 - x[m]) / (x[k] - x[m]) for m in range(p) if m != k]) for k in range(p)])
    P = np.zeros((nf, nf // 2 + 2 * h))
    for n in range(nf):
        if n % 2 == 0:
            P[n, n // 2 + h] = 1.0
        else:
            P[n, n // 2 + 1:n // 2 + 1 + p] = w
    return P


def _split_error(alpha, f, K, p=10):
    G = O.lgf_cube(K)
    Gf = O.lgf_cube(K, t_lo=alpha)
    u = _conv(_sym(G), f)
    u_near = _conv(_sym(G - Gf), f)
    P = _interp_matrix(f.shape[0], p)
    q = np.einsum("ai,bj,ck,ijk->abc", P.T, P.T, P.T, f, optimize=True)
    Kc = q.shape[0] - 1
    assert 2 * Kc <= K
    kc = _sym(Gf[::2, ::2, ::2][:Kc + 1, :Kc + 1, :Kc + 1])
    v = _conv(kc, q)
    u_far = np.einsum("ia,jb,kc,abc->ijk", P, P, P, v, optimize=True)
    return np.linalg.norm(u_near + u_far - u) / np.linalg.norm(u), G, Gf


@pytest.fixture(scope="module")
def sources():
    n = 48
    rng = np.random.default_rng(1601)
    noise = np.zeros((n, n, n))
    noise[16:32, 16:32, 16:32] = rng.uniform(-1, 1, (16, 16, 16))
    z, y, x = np.meshgrid(*[np.arange(n)] * 3, indexing="ij")
    c = n / 2 + 0.3
    smooth = np.exp(-((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2) / 18.0)
    return noise, smooth


def test_split_reproduces_G_and_near_part_is_compact():
    K = 60
    G = O.lgf_cube(K)
    Gf = O.lgf_cube(K, t_lo=20.0)
    Gn = G - Gf
    a, b, c = np.meshgrid(*[np.arange(K + 1)] * 3, indexing="ij")
    far = np.maximum(np.maximum(a, b), c) > 32
    assert np.abs(Gn[far]).max() < 1e-8 * abs(G[0, 0, 0])
    assert Gn[0, 0, 0] < 0 and Gf[0, 0, 0] < 0 and abs(Gf[0, 0, 0]) < 0.05 * abs(G[0, 0, 0])
    # G_far = e^{aL} G, so L G_far = e^{aL} L G = E(a), the time-a heat kernel of
    # eq. lgf_intfac, on the table interior
    L = sum(np.roll(Gf, s, ax) for ax in range(3) for s in (1, -1)) - 6 * Gf
    g = O.bessel_scaled(20.0, K)                  # e^{-2a} I_n(2a)
    E = g[a] * g[b] * g[c]
    inner = (a >= 1) & (b >= 1) & (c >= 1) & (a < K) & (b < K) & (c < K)
    assert np.abs(L[inner] - E[inner]).max() < 1e-12 * abs(E[1, 1, 1])


@pytest.mark.parametrize("kind", [0, 1])
def test_far_interpolation_error_below_fp32_target(sources, kind):
    f = sources[kind]
    err, _, _ = _split_error(20.0, f, 84)
    assert err < 1e-6, err


def test_far_interpolation_error_falls_with_split_time_and_order(sources):
    errs = [_split_error(a, sources[0], 84)[0] for a in (8.0, 20.0)]
    assert errs[1] < errs[0] / 5, errs
    assert _split_error(20.0, sources[0], 84, p=8)[0] > 2 * errs[1]
