"""FP64 GPU path (plans built with precision = 1) against the FP64 oracle.

The 32^3 scalar Gaussian-blob solve is specified in FP64; with FP64 data,
transforms and spectrum the GPU result must agree with the direct sum to
within FP64 rounding of the transforms: relative L2 <= 1e-12 (reading of the
target: the FP64 instantiation is held to the oracle's own residual bar).
"""
import numpy as np
import pytest

import oracle as O
from paper_1601_00035_gb300 import inputs
from tests.helpers import built, oracle_poisson_blocks, rel_l2, rel_linf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run64(lgf, solve, f):
    K = lgf.required_max_offset(solve.src_blocks, solve.dst_blocks, solve.B)
    table = lgf.Table(lgf.LAPLACE7, max_offset=K)
    plan = lgf.Plan(table, [solve], precision=1)
    src = torch.from_numpy(np.ascontiguousarray(f, dtype=np.float64)).cuda()
    dst = torch.zeros((len(solve.dst_blocks), solve.ncomp, solve.B, solve.B, solve.B), dtype=torch.float64,
                      device="cuda")
    plan.execute_f64([src], [dst])
    torch.cuda.synchronize()
    with pytest.raises(lgf.LGFError):  # an FP64 plan refuses the FP32 entry
        plan.execute([src.float()], [dst.float()])
    return dst.cpu().numpy()


def test_blobs32_fp64_full():
    lgf = built()
    B = 16
    f = inputs.gaussian_blobs(32)
    blocks = inputs.block_grid(f.shape, B)
    out = _run64(lgf, lgf.Solve(B, 1, blocks, blocks), inputs.to_blocks(f, B, blocks, dtype=np.float64))
    u = inputs.from_blocks(out, B, blocks, f.shape)[0]
    z, y, x = np.meshgrid(*[np.arange(32)] * 3, indexing="ij")
    pts = np.stack([x.ravel(), y.ravel(), z.ravel()], 1).astype(np.int32)
    ref = O.direct_conv_box(O.lgf_cube(40), f, pts).reshape(32, 32, 32)
    assert rel_l2(u, ref) < 1e-12, rel_l2(u, ref)
    assert rel_linf(u, ref) < 1e-11


def test_sparse_fp64():
    lgf = built()
    rng = np.random.default_rng(12)
    B = 8
    box = np.array([[x, y, z] for z in range(-1, 2) for y in range(0, 3) for x in range(-1, 3)], dtype=np.int32)
    src_c = box[rng.choice(len(box), size=11, replace=False)]
    dst_c = box[rng.random(len(box)) < 0.7]
    f = rng.standard_normal((len(src_c), 2, B, B, B))
    out = _run64(lgf, lgf.Solve(B, 2, src_c, dst_c, dx=0.3, scale=-2.0), f)
    pts = inputs.block_points(dst_c, B)
    K = lgf.required_max_offset(src_c, dst_c, B)
    for c in range(2):
        ref = oracle_poisson_blocks(f, src_c, B, pts, K, comp=c, scale=-2.0, dx=0.3)
        assert rel_l2(out[:, c].reshape(-1), ref) < 1e-12
