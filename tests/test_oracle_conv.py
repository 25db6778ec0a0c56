"""Pins for the oracle's direct convolution u(n) = sum_m G(n - m) f(m) (Sec. 2.2, eq. dpoisson_conv).

* a single unit point source reproduces the shifted table exactly;
* L u = f on every point whose stencil stays inside the evaluated box, to
  1e-12 relative (the discrete identity the method solves);
* agreement with an independent algorithm: a zero-padded FP64 FFT circular
  convolution of the same kernel samples (brute-force check on small boxes);
* linearity and translation invariance.
"""
import numpy as np

import oracle as O


def _box_targets(lo, hi):
    z, y, x = np.meshgrid(*[np.arange(l, h) for l, h in zip(lo[::-1], hi[::-1])], indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], 1).astype(np.int32)


def test_point_source_is_shifted_table():
    K = 30
    cube = O.lgf_cube(K)
    src = np.array([[5, 7, 9]], dtype=np.int32)
    tgt = _box_targets((0, 0, 0), (12, 12, 12))
    u = O.direct_conv(cube, src, np.array([1.0]), tgt)
    d = np.abs(tgt - src)
    assert np.array_equal(u, cube[d[:, 2], d[:, 1], d[:, 0]])


def test_discrete_poisson_identity():
    rng = np.random.default_rng(7)
    K = 40
    cube = O.lgf_cube(K)
    n = 10
    f = np.zeros((n, n, n))
    f[2:8, 3:7, 1:9] = rng.standard_normal((6, 4, 8))
    # evaluate u on a box two cells larger on each side
    tgt = _box_targets((-2, -2, -2), (n + 2, n + 2, n + 2))
    u = O.direct_conv_box(cube, f, tgt).reshape(n + 4, n + 4, n + 4)
    Lu = O.op_L(u)[1:-1, 1:-1, 1:-1]          # valid on the box grown by one
    fbig = np.zeros((n + 2,) * 3)
    fbig[1:-1, 1:-1, 1:-1] = f
    assert np.abs(Lu - fbig).max() / np.abs(f).max() < 1e-12


def test_against_fft_convolution():
    rng = np.random.default_rng(3)
    K = 40
    cube = O.lgf_cube(K)
    n = 12
    f = rng.standard_normal((n, n, n))
    tgt = _box_targets((0, 0, 0), (n, n, n))
    u = O.direct_conv_box(cube, f, tgt).reshape(n, n, n)
    # circular convolution on a 2n grid with the kernel placed at wrapped offsets
    N = 2 * n
    j = np.arange(N)
    off = np.abs(np.where(j < N // 2, j, j - N))
    kern = cube[off[:, None, None], off[None, :, None], off[None, None, :]]
    F = np.zeros((N, N, N))
    F[:n, :n, :n] = f
    conv = np.fft.irfftn(np.fft.rfftn(F) * np.fft.rfftn(kern), s=(N, N, N), axes=(0, 1, 2))[:n, :n, :n]
    assert np.abs(conv - u).max() / np.abs(u).max() < 1e-13


def test_linearity_translation():
    rng = np.random.default_rng(11)
    cube = O.lgf_cube(30)
    src = rng.integers(0, 10, size=(20, 3)).astype(np.int32)
    a, b = rng.standard_normal(20), rng.standard_normal(20)
    tgt = rng.integers(0, 12, size=(50, 3)).astype(np.int32)
    ua = O.direct_conv(cube, src, a, tgt)
    ub = O.direct_conv(cube, src, b, tgt)
    uab = O.direct_conv(cube, src, 2 * a - 3 * b, tgt)
    assert np.allclose(uab, 2 * ua - 3 * ub, rtol=1e-13, atol=1e-15)
    sh = np.array([3, -2, 5], dtype=np.int32)
    assert np.allclose(O.direct_conv(cube, src + sh, a, tgt + sh), ua, rtol=0, atol=1e-15)


def test_fft_conv_matches_direct_sum():
    """oracle.fft_conv (FFT-based linear convolution) agrees with the direct sum
    (an independent algorithm) at every target of a box that overlaps the source box
    on one side and lies beyond it on another, to FP64 rounding."""
    rng = np.random.default_rng(9)
    f = rng.standard_normal((7, 9, 11))                  # [z, y, x], origin (x, y, z) = (3, -2, 5)
    src_origin, tgt_origin, tgt_shape = (3, -2, 5), (-4, 4, 9), (6, 8, 10)
    u = O.fft_conv(f, src_origin, tgt_origin, tgt_shape, workers=2)
    z, y, x = np.meshgrid(*[np.arange(s) for s in tgt_shape], indexing="ij")
    tgt = np.stack([x.ravel() + tgt_origin[0], y.ravel() + tgt_origin[1], z.ravel() + tgt_origin[2]], 1)
    zs, ys, xs = np.meshgrid(*[np.arange(s) for s in f.shape], indexing="ij")
    src = np.stack([xs.ravel() + src_origin[0], ys.ravel() + src_origin[1], zs.ravel() + src_origin[2]], 1)
    K = int(np.abs(tgt[:, None, :] - src[None, :, :]).max())
    ref = O.direct_conv(O.lgf_cube(K), src.astype(np.int32), f.ravel(), tgt.astype(np.int32))
    assert np.abs(u.ravel() - ref).max() < 1e-14 * np.abs(ref).max()
