"""GPU parity of the device FP64 tables and of the integrating factor.

* The device LGF octant (its own quadrature and Bessel code) against the
  oracle's, to 1e-13 relative: two independent FP64 evaluations of App. B.
* The integrating-factor taps g(k) = e^{-2a} I_k(2a) and radius R against the
  oracle.
* y = M E_Q(alpha) M x (Sec. 2.3, Sec. 4.4) against the oracle's plain 3-D sum,
  for alpha in {0.05, 0.2, 1.0} on a holed block set, full comparison; FP32
  tolerance relative L2 <= 1e-6.
"""
import numpy as np
import pytest

import oracle as O
from paper_1601_00035_gb300 import inputs
from tests.helpers import built, rel_l2, rel_linf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_lgf_octant_matches_oracle():
    lgf = built()
    K = 64
    t = lgf.Table(lgf.LAPLACE7, max_offset=K)
    dev = t.values()
    ref = O.lgf_octant(K)
    assert dev.shape == ref.shape
    assert np.max(np.abs(dev - ref) / np.abs(ref)) < 1e-13
    assert abs(dev[0] + O.WATSON_W / 6) < 1e-14


def test_lgf_octant_large_offsets():
    lgf = built()
    K = 300
    dev = lgf.Table(lgf.LAPLACE7, max_offset=K).values()
    ref = O.lgf_octant(K)
    idx = np.random.default_rng(0).choice(len(ref), 4000, replace=False)
    assert np.max(np.abs(dev[idx] - ref[idx]) / np.abs(ref[idx])) < 1e-13


@pytest.mark.parametrize("alpha", [0.05, 0.1, 0.2, 1.0, 3.0])
def test_if_taps(alpha):
    lgf = built()
    t = lgf.Table(lgf.IFACTOR, alpha=alpha)
    ref = O.ifactor_taps(alpha)
    assert t.radius == len(ref) - 1
    assert np.max(np.abs(t.values() - ref) / ref) < 1e-14


@pytest.mark.parametrize("B,alpha", [(16, 0.05), (16, 0.2), (16, 1.0), (16, 0.002), (8, 0.05), (8, 0.002)])
def test_ifactor_holed_set(B, alpha):
    """A 3 x 3 x 3 block box with holes, 2 components, radii 4, 7, 9 and 15 (instantiated
    radii 4, 8, 12 and 16), B = 16 and B = 8."""
    lgf = built()
    rng = np.random.default_rng(int(alpha * 1000) + B)
    box = np.array([[x, y, z] for z in range(3) for y in range(3) for x in range(3)], dtype=np.int32)
    keep = rng.random(len(box)) < 0.75
    keep[13] = True  # centre block
    blocks = box[keep]
    x = rng.standard_normal((len(blocks), 2, B, B, B)).astype(np.float32)
    t = lgf.Table(lgf.IFACTOR, alpha=alpha)
    assert t.radius == {0.002: 4, 0.05: 7, 0.2: 9, 1.0: 15}[alpha]
    plan = lgf.Plan(t, [lgf.Solve(B, 2, blocks, None)])
    dx = torch.from_numpy(x).cuda()
    dy = torch.zeros_like(dx)
    plan.ifactor(dx, dy)
    torch.cuda.synchronize()
    y = dy.cpu().numpy()
    g = O.ifactor_taps(alpha)
    pts = inputs.block_points(blocks, B)
    sub = rng.choice(len(pts), size=6000, replace=False)
    for c in range(2):
        dense = inputs.from_blocks(x[:, c:c + 1], B, blocks, (3 * B,) * 3)[0]
        ref = O.ifactor_direct(g, dense, pts[sub])
        got = y[:, c].reshape(-1)[sub]
        assert rel_l2(got, ref) < 1e-6
        assert rel_linf(got, ref) < 1e-5


@pytest.mark.parametrize("alpha", [0.05, 0.2, 1.0])
def test_ifactor_velocity_128_sampled(alpha):
    """3-component 128^3 two-ring velocity, dense block set, alpha in {0.05, 0.2, 1.0}
    (R = 7, 9, 15): the integrating-factor configuration of the benchmark."""
    lgf = built()
    B = 16
    u = inputs.two_ring_velocity()
    blocks = inputs.block_grid(u.shape[1:], B)
    xb = inputs.to_blocks(u, B, blocks)
    t = lgf.Table(lgf.IFACTOR, alpha=alpha)
    plan = lgf.Plan(t, [lgf.Solve(B, 3, blocks, None)])
    dx = torch.from_numpy(xb).cuda()
    dy = torch.zeros_like(dx)
    plan.ifactor(dx, dy)
    torch.cuda.synchronize()
    y = dy.cpu().numpy()
    g = O.ifactor_taps(alpha)
    rng = np.random.default_rng(4)
    pts = rng.integers(0, 128, size=(3000, 3)).astype(np.int32)
    lut = {tuple(c): i for i, c in enumerate(blocks.tolist())}
    for c in range(3):
        ref = O.ifactor_direct(g, u[c], pts)
        got = np.array([y[lut[(p[0] // B, p[1] // B, p[2] // B)], c, p[2] % B, p[1] % B, p[0] % B] for p in pts])
        assert rel_l2(got, ref) < 1e-6


def test_ifactor_constant_interior():
    """A constant field stays constant where the full kernel box lies inside the set (mass, sigma(0) = 0)."""
    lgf = built()
    B = 16
    blocks = inputs.block_grid((48, 48, 48), B)
    t = lgf.Table(lgf.IFACTOR, alpha=0.2)
    plan = lgf.Plan(t, [lgf.Solve(B, 1, blocks, None)])
    dx = torch.ones((len(blocks), 1, B, B, B), device="cuda")
    dy = torch.zeros_like(dx)
    plan.ifactor(dx, dy)
    y = dy.cpu().numpy()
    centre = [i for i, c in enumerate(blocks.tolist()) if c == [1, 1, 1]][0]
    assert np.abs(y[centre] - 1.0).max() < 2e-6


def test_errors_are_reported():
    lgf = built()
    with pytest.raises(lgf.LGFError) as e:
        lgf.Table(lgf.LAPLACE7, max_offset=0)
    assert e.value.status == lgf.LGF_ERR_ARG
    t = lgf.Table(lgf.LAPLACE7, max_offset=8)
    blocks = np.array([[0, 0, 0], [3, 0, 0]], dtype=np.int32)
    with pytest.raises(lgf.LGFError) as e:  # table too small for the needed FFT grid
        lgf.Plan(t, [lgf.Solve(16, 1, blocks, blocks)])
    assert e.value.status == lgf.LGF_ERR_ARG and "max_offset" in str(e.value)
    with pytest.raises(lgf.LGFError):  # duplicate blocks
        lgf.Plan(t, [lgf.Solve(8, 1, np.array([[0, 0, 0], [0, 0, 0]]), blocks)])
    with pytest.raises(lgf.LGFError):  # bad block size
        lgf.Plan(t, [lgf.Solve(12, 1, blocks, blocks)])
    ti = lgf.Table(lgf.IFACTOR, alpha=3.0)   # R > 8
    with pytest.raises(lgf.LGFError) as e:
        lgf.Plan(ti, [lgf.Solve(8, 1, blocks, None)])
    assert "radius" in str(e.value)
