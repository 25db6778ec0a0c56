"""Shared set-up of the IF-HERK test cases (tests only)."""
import numpy as np

import oracle as O
from paper_1601_00035_gb300 import inputs


def dilate(blocks):
    s = set(map(tuple, np.asarray(blocks).tolist()))
    out = []
    for (x, y, z) in s:
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    out.append((x + dx, y + dy, z + dz))
    return np.array(sorted(set(out)), dtype=np.int32)


def small_case(B=8, dx=1.0, amp=1.0, seed=0):
    """Soln = supp = the 2x2x2 central blocks of a 4^3 block box; xsoln = their dilation
    (the whole 4^3 box); the dense box adds a one-block margin of zeros on every side.
    u0 = C^T a with a a compact ring-like vector potential centred in the box, so that
    G^T u0 = 0 exactly (Im C^T = Null G^T)."""
    soln = np.array([[x, y, z] for z in (1, 2) for y in (1, 2) for x in (1, 2)], dtype=np.int32)
    xsoln = dilate(soln)                  # blocks 0..3 on each axis
    n = 6 * B                             # dense box = blocks -1..4
    origin = np.array([-1, -1, -1])
    rng = np.random.default_rng(seed)
    axis = inputs.random_axis_sphere(rng)
    c = np.array([n / 2.0] * 3)
    a = np.zeros((3, n, n, n))
    for q in range(3):
        pts = inputs.edge_points((n, n, n), q)
        a[q] = amp * inputs.ring_vorticity(pts, c, axis, 0.35 * B, 0.12 * B)[..., q]
    # compact support: cut a to a cube inside the soln blocks
    lo, hi = int(n / 2 - 0.8 * B), int(n / 2 + 0.8 * B)
    cut = np.zeros((n, n, n), dtype=bool)
    cut[lo:hi, lo:hi, lo:hi] = True
    a *= cut
    u0 = O.op_Ct(a, dx)
    xs_mask = O.block_mask((n, n, n), B, xsoln, origin)
    so_mask = O.block_mask((n, n, n), B, soln, origin)
    masks = {"supp": so_mask, "soln": so_mask, "xsoln": xs_mask}
    return dict(B=B, n=n, origin=origin, soln=soln, xsoln=xsoln, u0=u0 * xs_mask, masks=masks, dx=dx)


def to_blocks_dense(f, B, blocks, origin):
    """Dense [c, z, y, x] box (block (0,0,0) of the box at `origin`) -> [nblk, c, B, B, B]."""
    sh = np.asarray(blocks) - np.asarray(origin)
    return inputs.to_blocks(f, B, sh)


def from_blocks_dense(blk, B, blocks, origin, shape):
    sh = np.asarray(blocks) - np.asarray(origin)
    return inputs.from_blocks(blk, B, sh, shape)
