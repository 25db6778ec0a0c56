"""Test helpers: build-once fixtures and comparisons (tests only)."""
import functools

import numpy as np

import oracle as O
from paper_1601_00035_gb300 import inputs


@functools.lru_cache(maxsize=1)
def built():
    from paper_1601_00035_gb300 import build
    build.build()
    from paper_1601_00035_gb300 import lgf
    lgf.load()
    return lgf


def rel_l2(got, ref):
    return float(np.linalg.norm(np.ravel(got) - np.ravel(ref)) / np.linalg.norm(np.ravel(ref)))


def rel_linf(got, ref):
    return float(np.abs(np.ravel(got) - np.ravel(ref)).max() / np.abs(np.ravel(ref)).max())


def oracle_poisson_blocks(src_blocks_vals, src_coords, B, tgt_pts, K, comp=0, scale=1.0, dx=1.0):
    """FP64 direct sum (eq. dpoisson_conv) with sources given block-contiguously.

    src_blocks_vals: [nblk, ncomp, B, B, B]; returns u at tgt_pts ([n,3] x,y,z)."""
    pts = inputs.block_points(src_coords, B)
    vals = np.asarray(src_blocks_vals[:, comp], dtype=np.float64).reshape(-1)
    nz = vals != 0
    cube = O.lgf_cube(K)
    return scale * dx * dx * O.direct_conv(cube, pts[nz], vals[nz], tgt_pts)


def block_values_at(blocks_vals, coords, B, pts, comp=0):
    """Values of a block-contiguous field at integer points (must lie in listed blocks)."""
    lut = {tuple(c): i for i, c in enumerate(np.asarray(coords).tolist())}
    out = np.empty(len(pts))
    for j, (x, y, z) in enumerate(np.asarray(pts).tolist()):
        i = lut[(x // B, y // B, z // B)]
        out[j] = blocks_vals[i, comp, z % B, y % B, x % B]
    return out


def golden(name: str):
    """A value printed in the paper (tests/golden/paper_values.txt, which gives the
    passage of each).  Numbers come back as float; comma lists as lists of floats;
    the entries may use fractions and sqrt3."""
    import math
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_values.txt")
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        key, val = line.split()[:2]
        if key != name:
            continue

        def num(t):
            return float(eval(t.replace("sqrt3", "math.sqrt(3)"), {"math": math}))
        parts = val.split(",")
        return [num(t) for t in parts] if len(parts) > 1 else num(val)
    raise KeyError(name)
