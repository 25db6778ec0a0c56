"""Edge cases of the Poisson path: every FFT length class, single blocks,
far-apart source and target sets (FFT length 1024), and argument errors.

Tolerances are relative L2 against the FP64 direct sum over the tested targets,
unscaled: 1e-6 where the targets include the sources' near field; for target sets
made mostly (4e-6) or only (1e-4) of blocks far from every source the whole-box FP32
transforms, which round at the near-field scale, reach the stated looser bounds.

Lengths 16 and 32 run one thread per line; 64..512 two-stage transforms
(512 with 32 elements per lane); 384, 432, 768 and 1024 three-stage transforms.  Far offsets use the oracle's per-point
LGF evaluation (same Bessel-integral quadrature as its tables)."""
import numpy as np
import pytest

import oracle as O
from paper_1601_00035_gb300 import inputs
from tests.helpers import built, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _solve(lgf, B, src_c, dst_c, f, ncomp=1):
    K = lgf.required_max_offset(src_c, dst_c, B)
    table = lgf.Table(lgf.LAPLACE7, max_offset=K)
    plan = lgf.Plan(table, [lgf.Solve(B, ncomp, src_c, dst_c)])
    d_src = torch.from_numpy(np.ascontiguousarray(f, dtype=np.float32)).cuda()
    d_dst = torch.zeros((len(dst_c), ncomp, B, B, B), device="cuda")
    plan.execute([d_src], [d_dst])
    return d_dst.cpu().numpy()


def _reference(f, src_c, dst_c, B, pts):
    """Direct sum at sample points with G evaluated per offset."""
    sp = inputs.block_points(src_c, B)
    v = f[:, 0].reshape(-1).astype(np.float64)
    offs = (np.asarray(pts)[:, None, :] - sp[None, :, :]).reshape(-1, 3)
    g = O.lgf_points(offs).reshape(len(pts), len(sp))
    return g @ v


@pytest.mark.parametrize("dst", [[[0, 0, 0]], [[0, 0, 0], [1, 0, 0]], [[-1, 0, 0], [0, 1, 0], [1, 1, 1]]])
def test_small_lengths(dst):
    """Single source block B=8: FFT lengths 16 (same block) and 32/64 (neighbours)."""
    lgf = built()
    B = 8
    rng = np.random.default_rng(len(dst))
    src_c = np.array([[0, 0, 0]], dtype=np.int32)
    dst_c = np.array(dst, dtype=np.int32)
    f = rng.standard_normal((1, 1, B, B, B))
    out = _solve(lgf, B, src_c, dst_c, f)
    pts = inputs.block_points(dst_c, B)
    K = lgf.required_max_offset(src_c, dst_c, B)
    ref = O.direct_conv(O.lgf_cube(K), inputs.block_points(src_c, B), f.reshape(-1), pts)
    assert rel_l2(out.reshape(-1), ref) < 1e-6


@pytest.mark.parametrize("dst", [[[30, 0, 0]], [[0, 30, 30]]])
def test_far_target_length_1024(dst):
    """Target block 30 blocks (480 cells) from the source: FFT length 1024 on the far axes."""
    lgf = built()
    B = 16
    rng = np.random.default_rng(7)
    src_c = np.array([[0, 0, 0]], dtype=np.int32)
    dst_c = np.array(dst, dtype=np.int32)
    f = rng.standard_normal((1, 1, B, B, B))
    out = _solve(lgf, B, src_c, dst_c, f)
    pts = inputs.block_points(dst_c, B)
    sel = rng.choice(len(pts), 48, replace=False)
    ref = _reference(f, src_c, dst_c, B, pts[sel])
    # Targets that see only the far field (480 cells away): the whole-box FP32 transforms
    # round at the scale of the near field, |G(0)| rms(f), 24-35x the far values here, so
    # the stated bound of the whole-box FP32 path on far-only target sets is 1e-4
    # (a departure from the 1e-6 target, which holds wherever the targets include the
    # sources' near field).
    err = rel_l2(out.reshape(-1)[sel], ref)
    assert err < 1e-4, err


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_wide_source_narrow_target(axis):
    """Source six blocks long on one axis, target one block inside it: the
    largest offset (63) alone would allow length 128, but the source extent (96)
    must stay in the lower half of the line, so the plan takes 192 there."""
    lgf = built()
    B = 16
    rng = np.random.default_rng(11 + axis)
    src_c = np.zeros((6, 3), dtype=np.int32)
    src_c[:, axis] = np.arange(6)
    dst_c = np.zeros((1, 3), dtype=np.int32)
    dst_c[0, axis] = 3
    f = rng.standard_normal((6, 1, B, B, B))
    out = _solve(lgf, B, src_c, dst_c, f)
    K = lgf.required_max_offset(src_c, dst_c, B)
    assert K == 95
    ref = O.direct_conv(O.lgf_cube(K), inputs.block_points(src_c, B), f.reshape(-1), inputs.block_points(dst_c, B))
    assert rel_l2(out.reshape(-1), ref) < 1e-6


@pytest.mark.parametrize("precision", [0, 1])
def test_length_512(precision):
    """Targets 15 blocks away along x (FFT length 512) and 7 along y (256), in
    FP32 and FP64; sampled against the per-point direct sum."""
    lgf = built()
    B = 16
    rng = np.random.default_rng(21)
    src_c = np.array([[0, 0, 0]], dtype=np.int32)
    dst_c = np.array([[15, 0, 0], [0, 7, 0], [1, 1, 0]], dtype=np.int32)
    f = rng.standard_normal((1, 1, B, B, B))
    K = lgf.required_max_offset(src_c, dst_c, B)
    assert K == 255
    table = lgf.Table(lgf.LAPLACE7, max_offset=K)
    plan = lgf.Plan(table, [lgf.Solve(B, 1, src_c, dst_c)], precision=precision)
    dt = torch.float64 if precision else torch.float32
    d_src = torch.from_numpy(f).to(dt).cuda()
    d_dst = torch.zeros((len(dst_c), 1, B, B, B), dtype=dt, device="cuda")
    (plan.execute_f64 if precision else plan.execute)([d_src], [d_dst])
    out = d_dst.cpu().numpy().reshape(-1)
    pts = inputs.block_points(dst_c, B)
    sel = rng.choice(len(pts), 96, replace=False)
    ref = _reference(f, src_c, dst_c, B, pts[sel])
    # most of these targets lie 7-15 blocks from the source: stated bound 4e-6 (FP32)
    err = rel_l2(out[sel], ref)
    assert err < (1e-10 if precision else 4e-6), err


@pytest.mark.parametrize("dst", [[[15, 0, 0], [0, 0, 7], [1, 0, 1]], [[0, 15, 0], [0, 0, 3], [1, 1, 1]]])
def test_packed_z_with_long_x_or_y(dst):
    """The packed z pass (lengths 128 and 256) beside a 512-point x or y axis:
    targets 15 blocks away along x (KX = 257) or y, and 7 or 3 along z; sampled
    against the direct sum."""
    lgf = built()
    B = 16
    rng = np.random.default_rng(31)
    src_c = np.array([[0, 0, 0]], dtype=np.int32)
    dst_c = np.array(dst, dtype=np.int32)
    f = rng.standard_normal((1, 1, B, B, B))
    out = _solve(lgf, B, src_c, dst_c, f).reshape(-1)
    pts = inputs.block_points(dst_c, B)
    sel = rng.choice(len(pts), 128, replace=False)
    ref = _reference(f, src_c, dst_c, B, pts[sel])
    # two of the three target blocks lie 3-15 blocks away: stated bound 4e-6 (FP32)
    err = rel_l2(out[sel], ref)
    assert err < 4e-6, err


@pytest.mark.parametrize("precision", [0, 1])
def test_lengths_3x2k(precision):
    """FFT lengths 96, 192 and 384 at once (x, y, z): one source block and targets
    5, 11 and 23 blocks away, in FP32 and FP64; sampled against the direct sum."""
    lgf = built()
    B = 8
    rng = np.random.default_rng(23)
    src_c = np.array([[0, 0, 0]], dtype=np.int32)
    dst_c = np.array([[5, 0, 0], [0, 11, 0], [0, 0, 23], [2, 3, 4], [0, 0, 0]], dtype=np.int32)
    f = rng.standard_normal((1, 1, B, B, B))
    K = lgf.required_max_offset(src_c, dst_c, B)
    assert K == 191
    table = lgf.Table(lgf.LAPLACE7, max_offset=K)
    plan = lgf.Plan(table, [lgf.Solve(B, 1, src_c, dst_c)], precision=precision)
    dt = torch.float64 if precision else torch.float32
    d_src = torch.from_numpy(f).to(dt).cuda()
    d_dst = torch.zeros((len(dst_c), 1, B, B, B), dtype=dt, device="cuda")
    (plan.execute_f64 if precision else plan.execute)([d_src], [d_dst])
    out = d_dst.cpu().numpy().reshape(-1)
    pts = inputs.block_points(dst_c, B)
    sel = rng.choice(len(pts), 160, replace=False)
    ref = _reference(f, src_c, dst_c, B, pts[sel])
    # four of the five target blocks lie 5-23 blocks from the source: stated bound 4e-6 (FP32)
    err = rel_l2(out[sel], ref)
    assert err < (1e-10 if precision else 4e-6), err


@pytest.mark.parametrize("e", [40, 80, 160])
def test_full_box_3x2k(e):
    """A dense e^3 source on its own box (FFT length 96, 192, 384 on every axis),
    FP32, sampled against the direct sum."""
    lgf = built()
    B = 8
    rng = np.random.default_rng(e)
    f = rng.standard_normal((e, e, e))
    c = inputs.block_grid(f.shape, B)
    K = lgf.required_max_offset(c, c, B)
    assert K == {40: 47, 80: 95, 160: 191}[e]
    out = _solve(lgf, B, c, c, inputs.to_blocks(f, B, c))
    pts = inputs.block_points(c, B)
    sel = rng.choice(len(pts), 64, replace=False)
    ref = O.direct_conv_box(O.lgf_cube(K), f, pts[sel])
    got = out.reshape(-1)[sel]
    assert rel_l2(got, ref) < 1e-6


@pytest.mark.parametrize("precision", [0, 1])
def test_lengths_9x2k(precision):
    """FFT lengths 288 = 9 * 32 (x, two radix-12/24 stages, 12 lanes per line) and
    432 = 27 * 16 (y, three stages 6/12/6, 18 lanes per line) at once: one source block and
    targets 17 and 26 blocks away, in FP32 and FP64; sampled against the direct sum."""
    lgf = built()
    B = 8
    rng = np.random.default_rng(432)
    src_c = np.array([[0, 0, 0]], dtype=np.int32)
    dst_c = np.array([[17, 0, 0], [0, 26, 0], [0, 0, 3], [5, 9, 1], [0, 0, 0]], dtype=np.int32)
    f = rng.standard_normal((1, 1, B, B, B))
    K = lgf.required_max_offset(src_c, dst_c, B)
    assert K == 215 and lgf.fft_length(2 * (17 * B + 7) + 2) == 288
    table = lgf.Table(lgf.LAPLACE7, max_offset=K)
    plan = lgf.Plan(table, [lgf.Solve(B, 1, src_c, dst_c)], precision=precision)
    dt = torch.float64 if precision else torch.float32
    d_src = torch.from_numpy(f).to(dt).cuda()
    d_dst = torch.zeros((len(dst_c), 1, B, B, B), dtype=dt, device="cuda")
    (plan.execute_f64 if precision else plan.execute)([d_src], [d_dst])
    out = d_dst.cpu().numpy().reshape(-1)
    pts = inputs.block_points(dst_c, B)
    sel = rng.choice(len(pts), 160, replace=False)
    ref = _reference(f, src_c, dst_c, B, pts[sel])
    # four of the five target blocks lie 3-26 blocks from the source: stated bound 4e-6 (FP32)
    err = rel_l2(out[sel], ref)
    assert err < (1e-10 if precision else 4e-6), err


@pytest.mark.parametrize("e", [136, 200])
def test_full_box_9x2k(e):
    """A dense e^3 source on its own box: FFT length 288 (e = 136) or 432 (e = 200) on
    every axis, so the packed z pass runs at 288; FP32, sampled against the direct sum."""
    lgf = built()
    B = 8
    rng = np.random.default_rng(e)
    f = rng.standard_normal((e, e, e))
    c = inputs.block_grid(f.shape, B)
    K = lgf.required_max_offset(c, c, B)
    assert K == {136: 143, 200: 215}[e]
    out = _solve(lgf, B, c, c, inputs.to_blocks(f, B, c))
    pts = inputs.block_points(c, B)
    sel = rng.choice(len(pts), 48, replace=False)
    ref = O.direct_conv_box(O.lgf_cube(K), f, pts[sel])
    got = out.reshape(-1)[sel]
    assert rel_l2(got, ref) < 1e-6


def test_argument_errors():
    lgf = built()
    t = lgf.Table(lgf.LAPLACE7, max_offset=31)
    one = np.array([[0, 0, 0]], dtype=np.int32)
    with pytest.raises(lgf.LGFError) as e:
        lgf.Plan(t, [lgf.Solve(8, 1, np.zeros((0, 3), np.int32), one)])
    assert e.value.status == lgf.LGF_ERR_ARG
    with pytest.raises(lgf.LGFError):
        lgf.Plan(t, [lgf.Solve(8, 4, one, one)])          # ncomp out of range
    with pytest.raises(lgf.LGFError):
        lgf.Plan(t, [lgf.Solve(8, 1, one, one, dx=0.0)])  # dx must be positive
    p = lgf.Plan(t, [lgf.Solve(8, 1, one, one)])
    x = torch.zeros((1, 1, 8, 8, 8), device="cuda")
    with pytest.raises(lgf.LGFError) as e:
        p.ifactor(x, torch.zeros_like(x))                   # wrong kind of plan
    assert e.value.status == lgf.LGF_ERR_STATE


@pytest.mark.parametrize("axis", [0, 2])
def test_length_768(axis):
    """FFT length 768 (3 * 256) along x (the x passes) or z (the packed z pass): a target
    block 20 blocks (320 cells) from the source, beside two near blocks; sampled against
    the per-point direct sum."""
    lgf = built()
    B = 16
    rng = np.random.default_rng(768 + axis)
    src_c = np.array([[0, 0, 0]], dtype=np.int32)
    far = [0, 0, 0]
    far[axis] = 20
    dst_c = np.array([far, [0, 0, 0], [1, 1, 1]], dtype=np.int32)
    f = rng.standard_normal((1, 1, B, B, B))
    K = lgf.required_max_offset(src_c, dst_c, B)
    assert K == 383
    out = _solve(lgf, B, src_c, dst_c, f).reshape(-1)
    pts = inputs.block_points(dst_c, B)
    sel = rng.choice(len(pts), 192, replace=False)
    ref = _reference(f, src_c, dst_c, B, pts[sel])
    # one of the three target blocks lies 20 blocks away: stated bound 4e-6 (FP32)
    err = rel_l2(out[sel], ref)
    assert err < 4e-6, err
