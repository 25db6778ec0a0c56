"""GPU parity of the block-sparse split solve (lgf_plan_opts.method = 1; Sec. 2.2: the
LGF-FMM's near field by block pairs and far field by interpolation, evaluated to a
tolerance) against the FP64 direct sum of eq. dpoisson_conv.

The split G = G_near + G_far at time a = 20 of the Bessel form, near offsets up to two
16^3 blocks and 10-point Lagrange interpolation on the spacing-2 coarse lattice give a
relative L2 error of a few 1e-7 on smooth and on white-noise sources (the committed CPU
study tests/test_oracle_split_study.py); the FP32 bound 1e-6 is applied unscaled, also
to a target set that sees only the far field.
"""
import numpy as np
import pytest

import oracle as O
from paper_1601_00035_gb300 import inputs
from tests.helpers import block_values_at, built, oracle_poisson_blocks, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPLIT = 1


def _plan(lgf, src_c, dst_c, ncomp=1, scale=1.0, dx=1.0, method=SPLIT, use_graph=False, far_precision=0, near_form=0):
    # the split plan builds its own tables; the whole-box plan (methods 0 and 2) samples
    # this one up to half its FFT length (a box beyond the FFT limit gets the largest table)
    K = 31 if method == SPLIT else max(31, lgf.required_max_offset(src_c, dst_c, 16))
    t = lgf.Table(lgf.LAPLACE7, max_offset=min(K, 1024))
    return t, lgf.Plan(t, [lgf.Solve(16, ncomp, src_c, dst_c, dx=dx, scale=scale)], method=method,
                       use_graph=use_graph, far_precision=far_precision, near_form=near_form)


def _dilate(blocks, r=1):
    s = set(map(tuple, np.asarray(blocks).tolist()))
    out = set()
    for (x, y, z) in s:
        for dz in range(-r, r + 1):
            for dy in range(-r, r + 1):
                for dx in range(-r, r + 1):
                    out.add((x + dx, y + dy, z + dz))
    return np.array(sorted(out), dtype=np.int32)


@pytest.mark.parametrize("seed,near_form", [(0, 0), (1, 0), (0, 1), (0, 2), (0, 3), (1, 3)])
def test_split_random_blocks_full(seed, near_form):
    """White-noise sources on a holed set of 16^3 blocks, targets on their two-block
    dilation (every near offset and the far field), two components, dx != 1, scale -1:
    every target point against the direct sum; with the near-field multiply-accumulate
    chosen at plan time, and in each of its forms (pairs, runs of 4 targets, quads of 4 x 2)."""
    lgf = built()
    B = 16
    rng = np.random.default_rng(200 + seed)
    box = np.array([[x, y, z] for z in range(3) for y in range(3) for x in range(4)], dtype=np.int32)
    src_c = box[rng.random(len(box)) < 0.45]
    dst_c = _dilate(src_c, 2)
    dst_c = dst_c[rng.random(len(dst_c)) < 0.5]
    f = rng.standard_normal((len(src_c), 2, B, B, B)).astype(np.float32)
    dx, scale = 0.5, -1.0
    _, plan = _plan(lgf, src_c, dst_c, ncomp=2, scale=scale, dx=dx, near_form=near_form)
    d_dst = torch.zeros((len(dst_c), 2, B, B, B), device="cuda")
    plan.execute([torch.from_numpy(f).cuda()], [d_dst])
    out = d_dst.cpu().numpy()
    pts = inputs.block_points(dst_c, B)
    K = lgf.required_max_offset(src_c, dst_c, B)
    for c in range(2):
        ref = oracle_poisson_blocks(f, src_c, B, pts, K, comp=c, scale=scale, dx=dx)
        err = rel_l2(out[:, c].reshape(-1), ref)
        assert err < 1e-6, (c, err)
    assert plan.method()[0] == SPLIT
    plan.check()            # no bounded tensor-core wait gave up


def test_split_ring128_whole_field():
    """The 128^3 vector ring (as benchmarked, 3 components) by the split method: the whole
    3 x 128^3 field against the oracle's FP64 FFT convolution."""
    lgf = built()
    B = 16
    w, _ = inputs.ring_128()
    src_c = inputs.active_blocks(w, B, 1e-14)
    dst_c = inputs.block_grid(w.shape[1:], B)
    f = inputs.to_blocks(w, B, src_c)
    _, plan = _plan(lgf, src_c, dst_c, ncomp=3, scale=-1.0, use_graph=True)
    d_src = torch.from_numpy(f).cuda()
    d_dst = torch.zeros((len(dst_c), 3, B, B, B), device="cuda")
    for _ in range(2):
        plan.execute([d_src], [d_dst])
    torch.cuda.synchronize()
    got = inputs.from_blocks(d_dst.cpu().numpy(), B, dst_c, (128, 128, 128))
    s0 = src_c.min(0) * B
    s1 = (src_c.max(0) + 1) * B
    dense = inputs.from_blocks(f.astype(np.float64), B, src_c - src_c.min(0), tuple((s1 - s0)[::-1]))
    ref = -O.fft_conv(dense, s0, (0, 0, 0), (128, 128, 128))
    err = rel_l2(got, ref)
    assert err < 1e-6, err


def test_split_shell_256_sampled():
    """The 256^3 Re = 500 ring shell (542 D_supp / 1186 D_xsoln blocks, Sec. 6.4
    parameters): 2048 sampled targets against the direct sum."""
    lgf = built()
    B, n = 16, 256
    axis = inputs.random_axis_tilted(inputs.rng_for(4))
    w = inputs.vortex_ring_edges(n, 50.0, 10.0, axis)[0]
    src_c = inputs.active_blocks(w, B, 1e-6)
    dst_c = _dilate(src_c)
    f = inputs.to_blocks(w, B, src_c)
    _, plan = _plan(lgf, src_c, dst_c, scale=-1.0)
    d_dst = torch.zeros((len(dst_c), 1, B, B, B), device="cuda")
    plan.execute([torch.from_numpy(f).cuda()], [d_dst])
    out = d_dst.cpu().numpy()
    rng = np.random.default_rng(9)
    pts_all = inputs.block_points(dst_c, B)
    pts = pts_all[rng.choice(len(pts_all), 2048, replace=False)]
    ref = oracle_poisson_blocks(f, src_c, B, pts, lgf.required_max_offset(src_c, dst_c, B), scale=-1.0)
    err = rel_l2(block_values_at(out, dst_c, B, pts), ref)
    assert err < 1e-6, err


@pytest.mark.parametrize("dst", [[[30, 0, 0]], [[0, 30, 30]]])
def test_split_far_only_targets(dst):
    """A target block 30 blocks from a white-noise source block sees only G_far: the split
    solve meets the unscaled 1e-6 there (the whole-box FP32 path's stated bound is 1e-4)."""
    lgf = built()
    B = 16
    rng = np.random.default_rng(7)
    src_c = np.array([[0, 0, 0]], dtype=np.int32)
    dst_c = np.array(dst, dtype=np.int32)
    f = rng.standard_normal((1, 1, B, B, B)).astype(np.float32)
    _, plan = _plan(lgf, src_c, dst_c)
    d_dst = torch.zeros((1, 1, B, B, B), device="cuda")
    plan.execute([torch.from_numpy(f).cuda()], [d_dst])
    out = d_dst.cpu().numpy().reshape(-1)
    pts = inputs.block_points(dst_c, B)
    sel = rng.choice(len(pts), 96, replace=False)
    sp = inputs.block_points(src_c, B)
    offs = (pts[sel][:, None, :] - sp[None, :, :]).reshape(-1, 3)
    ref = O.lgf_points(offs).reshape(len(sel), len(sp)) @ f.reshape(-1).astype(np.float64)
    err = rel_l2(out[sel], ref)
    assert err < 1e-6, err


def test_split_beyond_whole_box_limit():
    """Source and target blocks 40 blocks (640 cells) apart along x and 30 along y: the
    whole-box embedding would need FFT lengths above 1024 and is refused; the split plan
    runs (its coarse lattice halves the box).  Stated bounds: 1e-6 on the target blocks
    beside the sources; 3e-6 on the two blocks 30-40 blocks away, which see only G_far
    and carry the FP32 rounding of the coarse transforms (scale |G_far(0)| ~ 0.009, ~70x
    the far values; the whole-box path's bound on far-only sets is 1e-4)."""
    lgf = built()
    B = 16
    rng = np.random.default_rng(17)
    src_c = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=np.int32)
    dst_c = np.array([[40, 0, 0], [40, 30, 0], [1, 1, 0], [2, 0, 0]], dtype=np.int32)
    f = rng.standard_normal((len(src_c), 1, B, B, B)).astype(np.float32)
    with pytest.raises(lgf.LGFError):
        _plan(lgf, src_c, dst_c, method=0)
    _, plan = _plan(lgf, src_c, dst_c)
    d_dst = torch.zeros((len(dst_c), 1, B, B, B), device="cuda")
    plan.execute([torch.from_numpy(f).cuda()], [d_dst])
    out = d_dst.cpu().numpy()
    for b in range(len(dst_c)):
        pts = inputs.block_points(dst_c[b:b + 1], B)
        sel = rng.choice(len(pts), 64, replace=False)
        sp = inputs.block_points(src_c, B)
        offs = (pts[sel][:, None, :] - sp[None, :, :]).reshape(-1, 3)
        ref = O.lgf_points(offs).reshape(len(sel), len(sp)) @ f.reshape(-1).astype(np.float64)
        err = rel_l2(out[b, 0].reshape(-1)[sel], ref)
        assert err < (3e-6 if b < 2 else 1e-6), (b, err)


def test_split_host_buffers_residual_and_autotune():
    """lgf_conv_execute_host on a split plan equals the device execution bit for bit; the
    FP64 residual of the split result is at the FP32 floor; an autotuned plan (method 2)
    records both candidate times and its result matches the chosen method's."""
    lgf = built()
    B = 16
    w, _ = inputs.ring_128()
    src_c = inputs.active_blocks(w, B, 1e-14)
    dst_c = inputs.block_grid(w.shape[1:], B)
    f = inputs.to_blocks(w, B, src_c)
    _, plan = _plan(lgf, src_c, dst_c, ncomp=3, scale=-1.0)
    d_src = torch.from_numpy(f).cuda()
    d_dst = torch.zeros((len(dst_c), 3, B, B, B), device="cuda")
    plan.execute([d_src], [d_dst])
    h_dst = np.zeros((len(dst_c), 3, B, B, B), dtype=np.float32)
    plan.execute_host([np.ascontiguousarray(f)], [h_dst])
    assert np.array_equal(h_dst, d_dst.cpu().numpy())
    r = plan.residual(0, d_src, d_dst)
    assert r < 1e-4, r
    t, auto = _plan(lgf, src_c, dst_c, ncomp=3, scale=-1.0, method=2)
    m, ms0, ms1 = auto.method()
    assert m in (0, 1) and ms0 > 0 and ms1 > 0
    a_dst = torch.zeros_like(d_dst)
    auto.execute([d_src], [a_dst])
    torch.cuda.synchronize()
    if m == SPLIT:
        assert torch.equal(a_dst, d_dst)
    else:
        assert rel_l2(a_dst.cpu().numpy(), d_dst.cpu().numpy()) < 2e-6


def test_split_tensor_core_far_field():
    """The reduced-precision far field (far_precision = 1): interpolation and anterpolation
    as tcgen05 TF32 GEMMs on operands split into two TF32 parts.  On the 256^3 shell the
    solve stays within the 1e-5 stated for it against the FP64 direct sum, and within 2e-6
    of the FP32 CUDA-core far field; no bounded tensor-core wait gives up."""
    lgf = built()
    B, n = 16, 256
    axis = inputs.random_axis_tilted(inputs.rng_for(4))
    w = inputs.vortex_ring_edges(n, 50.0, 10.0, axis)[0]
    src_c = inputs.active_blocks(w, B, 1e-6)
    dst_c = _dilate(src_c)
    f = inputs.to_blocks(w, B, src_c)
    d_src = torch.from_numpy(f).cuda()
    outs = []
    for fp in (0, 1):
        _, plan = _plan(lgf, src_c, dst_c, scale=-1.0, far_precision=fp)
        d = torch.zeros((len(dst_c), 1, B, B, B), device="cuda")
        plan.execute([d_src], [d])
        plan.check()
        outs.append(d.cpu().numpy())
    assert rel_l2(outs[1], outs[0]) < 2e-6, rel_l2(outs[1], outs[0])
    rng = np.random.default_rng(19)
    pts_all = inputs.block_points(dst_c, B)
    pts = pts_all[rng.choice(len(pts_all), 1024, replace=False)]
    ref = oracle_poisson_blocks(f, src_c, B, pts, lgf.required_max_offset(src_c, dst_c, B), scale=-1.0)
    err = rel_l2(block_values_at(outs[1], dst_c, B, pts), ref)
    assert err < 1e-5, err


@pytest.mark.parametrize("far_precision", [0, 1])
def test_split_thin_ring_sampled(far_precision):
    """The thinnest ring of Sec. 6 (delta / R0 = 0.0125: R0 = 400 cells, 5-cell core, tilted),
    whose bounding box (about 750 cells across) the whole-box embedding cannot take: the
    split solve on its 1616 source blocks and their dilation (two levels: its coarse box is a
    768^3 FFT grid), 512 sampled targets against the direct sum; 1e-6 with the FP32 far
    field, 1e-5 with the tensor-core far field on both levels."""
    lgf = built()
    B = 16
    src_c, vals = inputs.thin_ring_blocks()
    dst_c = _dilate(src_c)
    if far_precision == 0:
        with pytest.raises(lgf.LGFError):
            _plan(lgf, src_c, dst_c, method=0)
    _, plan = _plan(lgf, src_c, dst_c, scale=-1.0, far_precision=far_precision)
    d_dst = torch.zeros((len(dst_c), 1, B, B, B), device="cuda")
    plan.execute([torch.from_numpy(vals).cuda()], [d_dst])
    plan.check()
    out = d_dst.cpu().numpy()
    rng = np.random.default_rng(400)
    pts_all = inputs.block_points(dst_c, B)
    pts = pts_all[rng.choice(len(pts_all), 512, replace=False)]
    sp = inputs.block_points(src_c, B)
    v = vals.reshape(-1).astype(np.float64)
    nz = v != 0
    offs_max = int(max(np.abs(pts.max(0) - sp.min(0)).max(), np.abs(sp.max(0) - pts.min(0)).max()))
    ref = -O.direct_conv(O.lgf_cube(offs_max), sp[nz], v[nz], pts)
    err = rel_l2(block_values_at(out, dst_c, B, pts), ref)
    assert err < (1e-6 if far_precision == 0 else 1e-5), err


def test_bounded_wait_reports_timeout_and_context_survives():
    """Failure detection without a fault: the tensor-core kernels' mbarrier wait, run on a
    barrier nothing arrives on, gives up after its poll limit and the host reads
    LGF_ERR_TIMEOUT; a split solve on the same context afterwards is still correct."""
    lgf = built()
    with pytest.raises(lgf.LGFError) as e:
        lgf.wait_probe(1000)
    assert e.value.status == lgf.LGF_ERR_TIMEOUT
    B = 16
    rng = np.random.default_rng(3)
    src_c = np.array([[0, 0, 0], [1, 0, 0]], dtype=np.int32)
    dst_c = np.array([[0, 0, 0], [1, 1, 0], [3, 0, 0]], dtype=np.int32)
    f = rng.standard_normal((2, 1, B, B, B)).astype(np.float32)
    _, plan = _plan(lgf, src_c, dst_c, far_precision=1)
    d = torch.zeros((3, 1, B, B, B), device="cuda")
    plan.execute([torch.from_numpy(f).cuda()], [d])
    plan.check()
    pts = inputs.block_points(dst_c, B)
    ref = oracle_poisson_blocks(f, src_c, B, pts, lgf.required_max_offset(src_c, dst_c, B))
    assert rel_l2(d.cpu().numpy().reshape(-1), ref) < 1e-5
