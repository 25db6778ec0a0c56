"""GPU parity at the sizes of the larger workloads, on sampled outputs.

* Shell-shaped sparse support on a 256^3 bounding box (a Re=500 ring of radius
  50 cells and core 10 cells, Sec. 6.4 parameters): sources on blocks where
  |w| > 1e-6 max (the support threshold of Sec. 6), targets = sources dilated
  by one block (D_xsoln with N_b = 1, Sec. 4.2 eq. def_xsoln); scalar source
  w_x; 1536 sampled targets against the direct sum.
(The ragged batch of 64 solves is checked solve by solve, at every block edge, in
tests/test_gpu_configs_asrun.py.)
"""
import numpy as np
import pytest

from paper_1601_00035_gb300 import inputs
from tests.helpers import block_values_at, built, oracle_poisson_blocks, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dilate(blocks):
    s = set(map(tuple, np.asarray(blocks).tolist()))
    out = set()
    for (x, y, z) in s:
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    out.add((x + dx, y + dy, z + dz))
    return np.array(sorted(out), dtype=np.int32)


def test_shell_256_sparse_sampled():
    lgf = built()
    B, n = 16, 256
    axis = inputs.random_axis_tilted(inputs.rng_for(4))
    w = inputs.vortex_ring_edges(n, 50.0, 10.0, axis)[0]          # w_x, scalar source
    src_c = inputs.active_blocks(w, B, 1e-6)
    dst_c = _dilate(src_c)
    f = inputs.to_blocks(w, B, src_c)
    K = lgf.required_max_offset(src_c, dst_c, B)
    table = lgf.Table(lgf.LAPLACE7, max_offset=K)
    plan = lgf.Plan(table, [lgf.Solve(B, 1, src_c, dst_c, scale=-1.0)])
    d_src = torch.from_numpy(f).cuda()
    d_dst = torch.zeros((len(dst_c), 1, B, B, B), device="cuda")
    plan.execute([d_src], [d_dst])
    out = d_dst.cpu().numpy()
    assert 300 < len(src_c) < 1500 and len(dst_c) > len(src_c)
    rng = np.random.default_rng(5)
    pts_all = inputs.block_points(dst_c, B)
    pts = pts_all[rng.choice(len(pts_all), 1536, replace=False)]
    ref = oracle_poisson_blocks(f, src_c, B, pts, K, scale=-1.0)
    got = block_values_at(out, dst_c, B, pts)
    assert rel_l2(got, ref) < 1e-6, rel_l2(got, ref)
