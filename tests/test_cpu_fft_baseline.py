"""bench.py's fast-CPU reference point (an FP64 zero-padded FFT convolution on
the host) against the oracle's direct sum on the benchmarked 128^3 ring: the two
independent algorithms agree to FP64 rounding at 4096 sampled targets."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_cpu_fft_matches_direct_sum():
    sys.path.insert(0, ROOT)
    import bench
    import oracle as O
    from paper_1601_00035_gb300 import inputs
    f, src_c, dst_c, _ = bench.workload()
    B = bench.B
    # the direct sum at the targets cpu_fft_rate samples, in the place of the GPU field
    tgt = inputs.block_points(dst_c, B)
    sel = np.random.default_rng(5).choice(len(tgt), 4096, replace=False)
    u = np.zeros((len(dst_c), 3, B, B, B))
    cube = O.lgf_cube(127)
    pts = inputs.block_points(src_c, B)
    for c in range(3):
        v = f[:, c].reshape(-1).astype(np.float64)
        nz = v != 0
        flat = u[:, c].reshape(len(dst_c), -1)
        flat[sel // B ** 3, sel % B ** 3] = O.direct_conv(cube, pts[nz], -v[nz], tgt[sel].astype(np.int32))
    rate, dt, threads, diff = bench.cpu_fft_rate(f, src_c, dst_c, u, reps=1)
    assert diff < 1e-13 and rate > 0
