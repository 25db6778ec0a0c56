"""GPU parity of the benchmarked workloads in the form bench.py runs them, against the
FP64 oracle:

* the 128^3 vector ring streamfunction a = -L^{-1} w (three component streams, one
  captured graph): the whole 3 x 128^3 result against the oracle's FP64 zero-padded
  FFT convolution (oracle.fft_conv, pinned to the direct sum);
* the ragged batch of 64 scalar ring solves (one plan, one graph) at every block edge
  the library takes (8, 16, 32): every solve on sampled targets against the direct sum;
* the integrating factor at alpha = 0.05, 0.2, 1.0 and the 32^3 Poisson solve in one
  captured graph, on the velocity u = C^T a, a = -L^{-1} w of two seeded rings (u from
  the oracle);
* the stage operators C, G^T, N~ and one integrating factor on the full D_xsoln of the
  256^3 Re = 500 ring (542 D_supp / 1186 D_xsoln blocks), on sampled points.
Tolerance: relative L2 <= 1e-6 (the FP32 target), L_inf <= 1e-5 where the whole field is
compared.
"""
import numpy as np
import pytest

import oracle as O
from paper_1601_00035_gb300 import inputs
from tests.helpers import built, rel_l2, rel_linf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_ring128_whole_field_as_benchmarked():
    lgf = built()
    B = 16
    w, _ = inputs.ring_128()
    src_c = inputs.active_blocks(w, B, 1e-14)
    dst_c = inputs.block_grid(w.shape[1:], B)
    f = inputs.to_blocks(w, B, src_c)
    table = lgf.Table(lgf.LAPLACE7, max_offset=lgf.required_max_offset(src_c, dst_c, B))
    plan = lgf.Plan(table, [lgf.Solve(B, 3, src_c, dst_c, scale=-1.0)], use_graph=True)
    d_src = torch.from_numpy(f).cuda()
    d_dst = torch.zeros((len(dst_c), 3, B, B, B), device="cuda")
    for _ in range(2):                      # capture, then replay
        plan.execute([d_src], [d_dst])
    torch.cuda.synchronize()
    got = inputs.from_blocks(d_dst.cpu().numpy(), B, dst_c, (128, 128, 128))
    # the oracle on the same sources (w on the source blocks), every target point
    s0 = src_c.min(0) * B
    s1 = (src_c.max(0) + 1) * B
    dense = inputs.from_blocks(f.astype(np.float64), B, src_c - src_c.min(0), tuple((s1 - s0)[::-1]))
    ref = -O.fft_conv(dense, s0, (0, 0, 0), (128, 128, 128))
    assert rel_l2(got, ref) < 1e-6, rel_l2(got, ref)
    assert rel_linf(got, ref) < 1e-5, rel_linf(got, ref)


@pytest.fixture(scope="module")
def ragged_reference():
    """The 64 ragged sources and, per solve, 256 sampled targets with the FP64 direct sum there."""
    fs = inputs.ragged_ring_sources(nsolve=64)
    cube = O.lgf_cube(max(f.shape[0] for f in fs) + 1)
    rng = np.random.default_rng(64)
    refs = []
    for f in fs:
        pts = rng.integers(0, f.shape[0], size=(256, 3)).astype(np.int32)
        refs.append((pts, -O.direct_conv_box(cube, f, pts)))
    return fs, refs


@pytest.mark.parametrize("B", [8, 16, 32])
def test_ragged64_all_solves_as_benchmarked(B, ragged_reference):
    lgf = built()
    fs, refs = ragged_reference
    solves, srcs, dsts = [], [], []
    for f in fs:
        sc = inputs.active_blocks(f, B, 1e-14)
        dc = inputs.block_grid(f.shape, B)
        solves.append(lgf.Solve(B, 1, sc, dc, scale=-1.0))
        srcs.append(torch.from_numpy(inputs.to_blocks(f, B, sc)).cuda())
        dsts.append(torch.zeros((len(dc), 1, B, B, B), device="cuda"))
    K = max(lgf.required_max_offset(s_.src_blocks, s_.dst_blocks, B) for s_ in solves)
    table = lgf.Table(lgf.LAPLACE7, max_offset=K)
    plan = lgf.Plan(table, solves, use_graph=True)
    for _ in range(2):
        plan.execute(srcs, dsts)
    torch.cuda.synchronize()
    worst = 0.0
    for j, (s_, d, (pts, ref)) in enumerate(zip(solves, dsts, refs)):
        u = inputs.from_blocks(d.cpu().numpy(), B, s_.dst_blocks, fs[j].shape)[0]
        got = u[pts[:, 2], pts[:, 1], pts[:, 0]]
        worst = max(worst, rel_l2(got, ref))
    assert worst < 1e-6, (B, worst)


def test_ifactor_three_alphas_and_poisson_in_one_graph():
    """The if128 workload as benchmarked: three integrating-factor plans over the 128^3 box
    and the 32^3 Poisson plan, captured in one CUDA graph and replayed.  The velocity is
    u = C^T a with a = -L^{-1} w of the two seeded rings, computed by the oracle in FP64;
    each y_alpha = M E(alpha) M u is compared on 2048 sampled faces per component against
    the oracle's plain 3-D sum, and the Poisson result on every point."""
    lgf = built()
    B, n = 16, 128
    w = inputs.two_rings_vorticity()
    a = -O.fft_conv(w, (0, 0, 0), (0, 0, 0), (n, n, n))
    u = O.op_Ct(a)                                  # faces; zero outside the box (mask)
    c = inputs.block_grid((n, n, n), B)
    x = torch.from_numpy(inputs.to_blocks(u, B, c)).cuda()
    alphas = (0.05, 0.2, 1.0)
    ys = [torch.zeros_like(x) for _ in alphas]
    tabs = [lgf.Table(lgf.IFACTOR, alpha=al) for al in alphas]
    plans = [lgf.Plan(tb, [lgf.Solve(B, 3, c, None)]) for tb in tabs]
    fb = inputs.gaussian_blobs(32)
    cb = inputs.block_grid(fb.shape, B)
    tp = lgf.Table(lgf.LAPLACE7, max_offset=lgf.required_max_offset(cb, cb, B))
    pp = lgf.Plan(tp, [lgf.Solve(B, 1, cb, cb)])
    fs = torch.from_numpy(inputs.to_blocks(fb, B, cb)).cuda()
    fd = torch.zeros_like(fs)

    def step():
        for pl, y in zip(plans, ys):
            pl.ifactor(x, y)
        pp.execute([fs], [fd])
    step()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    for y in ys:
        y.zero_()
    fd.zero_()
    g.replay()
    torch.cuda.synchronize()
    rng = np.random.default_rng(33)
    pts = rng.integers(0, n, size=(2048, 3)).astype(np.int32)
    for al, y in zip(alphas, ys):
        taps = O.ifactor_taps(al)
        got_all = inputs.from_blocks(y.cpu().numpy(), B, c, (n, n, n))
        for q in range(3):
            ref = O.ifactor_direct(taps, u[q], pts)
            got = got_all[q][pts[:, 2], pts[:, 1], pts[:, 0]]
            assert rel_l2(got, ref) < 1e-6, (al, q, rel_l2(got, ref))
    up = inputs.from_blocks(fd.cpu().numpy(), B, cb, fb.shape)[0]
    z, yy, xx = np.meshgrid(*[np.arange(32)] * 3, indexing="ij")
    tp_ = np.stack([xx.ravel(), yy.ravel(), z.ravel()], 1).astype(np.int32)
    ref = O.direct_conv_box(O.lgf_cube(40), fb, tp_).reshape(32, 32, 32)
    assert rel_l2(up, ref) < 1e-6


def _windows(vals, coords, B, centres, r):
    """Values of a block-contiguous field [nblk, nc, B, B, B] on the cubes of half-width r
    around each centre (zero off the listed blocks), and the matching block-set mask:
    returns ([m, nc, 2r+1, 2r+1, 2r+1], [m, 2r+1, 2r+1, 2r+1] bool)."""
    coords = np.asarray(coords)
    lo = coords.min(0)
    ext = coords.max(0) - lo + 1
    lut = -np.ones(ext[::-1], dtype=np.int64)
    lut[coords[:, 2] - lo[2], coords[:, 1] - lo[1], coords[:, 0] - lo[0]] = np.arange(len(coords))
    o = np.arange(-r, r + 1)
    oz, oy, ox = np.meshgrid(o, o, o, indexing="ij")
    p = centres[:, None, :] + np.stack([ox.ravel(), oy.ravel(), oz.ravel()], 1)[None]   # [m, W, 3] (x, y, z)
    b = p // B - lo
    inside = np.all((b >= 0) & (b < ext), axis=-1)
    bi = np.where(inside, lut[np.clip(b[..., 2], 0, ext[2] - 1), np.clip(b[..., 1], 0, ext[1] - 1),
                              np.clip(b[..., 0], 0, ext[0] - 1)], -1)
    loc = p % B
    v = vals[np.maximum(bi, 0), :, loc[..., 2], loc[..., 1], loc[..., 0]]          # [m, W, nc]
    v = np.where((bi >= 0)[..., None], v, 0.0).astype(np.float64)
    w = 2 * r + 1
    return (np.moveaxis(v, -1, 1).reshape(len(centres), -1, w, w, w),
            (bi >= 0).reshape(len(centres), w, w, w))


def test_stage_operators_full_size_sampled():
    """C, G^T and the nonlinear term (coef M^soln N~(M^xsoln (u + uinf))) on the 1186-block
    D_xsoln of the 256^3 ring, and one integrating factor E(alpha/2) (Scheme A's H^1) over
    the same block set, on 1024 sampled points each; the oracle applies the App. A
    operators on a small window around each point (they reach 2 cells) and the plain 3-D
    integrating-factor sum."""
    lgf = built()
    B, n, R0c, dcells = 16, 256, 50.0, 10.0
    dx = 1.0 / R0c
    dt, re = 0.01721, 500.0
    axis = inputs.random_axis_tilted(inputs.rng_for(4))
    w = inputs.vortex_ring_edges(n, R0c, dcells, axis) / dx ** 2
    supp = inputs.active_blocks(w, B, 1e-6)
    rk = lgf.RKPlan(B, supp, dx, dt, re, scheme=0)
    xs = rk.blocks(0)
    assert (len(supp), len(xs)) == (542, 1186)
    rng = np.random.default_rng(44)
    f = rng.standard_normal((len(xs), 3, B, B, B)).astype(np.float32)
    d_f = torch.from_numpy(f).cuda()
    pts_all = inputs.block_points(xs, B)
    centres = pts_all[rng.choice(len(pts_all), 1024, replace=False)].astype(np.int64)
    win, mask = _windows(f, xs, B, centres, 2)
    soln = set(map(tuple, np.asarray(supp).tolist()))
    in_soln = np.array([tuple(p) in soln for p in (centres // B).tolist()])
    uinf = (0.0, 0.0, -0.18686)
    coef = -0.37
    cases = [(lgf.OP_CURL, 3, lambda v, m: O.op_C(v * m, dx)),
             (lgf.OP_DIV_T, 1, lambda v, m: O.op_Gt(v * m, dx)[None]),
             (lgf.OP_NONLINEAR, 3, lambda v, m: coef * O.op_N((v + np.reshape(uinf, (3, 1, 1, 1))) * m, dx))]
    for op, nout, fn in cases:
        d_out = torch.zeros((len(xs), nout, B, B, B), device="cuda")
        rk.op(op, d_f, d_out, coef=coef if op == lgf.OP_NONLINEAR else 1.0, uinf=uinf)
        out = d_out.cpu().numpy()
        got, _ = _windows(out, xs, B, centres, 0)
        got = got[:, :, 0, 0, 0]
        ref = np.stack([fn(win[i], mask[i])[:, 2, 2, 2] for i in range(len(centres))])
        if op == lgf.OP_NONLINEAR:
            ref = ref * in_soln[:, None]
        assert rel_l2(got, ref) < 1e-6, (op, rel_l2(got, ref))
    # one integrating factor over D_xsoln, alpha/2 of the step
    al = dt / (re * dx * dx) / 2
    t_if = lgf.Table(lgf.IFACTOR, alpha=al)
    p_if = lgf.Plan(t_if, [lgf.Solve(B, 3, xs, None)])
    d_y = torch.zeros_like(d_f)
    p_if.ifactor(d_f, d_y)
    y = d_y.cpu().numpy()
    R = t_if.radius
    win, mask = _windows(f, xs, B, centres, R)
    taps = O.ifactor_taps(al)
    c0 = np.array([[R, R, R]], dtype=np.int32)
    ref = np.stack([[O.ifactor_direct(taps, win[i, q] * mask[i], c0)[0] for q in range(3)]
                    for i in range(len(centres))])
    got, _ = _windows(y, xs, B, centres, 0)
    assert rel_l2(got[:, :, 0, 0, 0], ref) < 1e-6, rel_l2(got[:, :, 0, 0, 0], ref)
