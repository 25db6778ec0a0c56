"""Seeded synthetic inputs shaped like the paper's vortex-ring workloads.

This module is shared by the tests, the benchmark and the CPU oracle checks.
It holds none of the convolution / integrating-factor arithmetic: only
analytic source fields sampled on the staggered grid and the block layout
helpers (dense box <-> block-contiguous arrays).

Grid positions (staggered grid of Sec. 2.1; the figure is missing from the
paper, so the positions are derived from the App. A operators): vertex
(i, j, k) sits at (i, j, k); a cell centre at (i-1/2, j-1/2, k-1/2); an edge
(q) value at the vertex shifted by -1/2 along x_q.

Seeds: numpy.random.default_rng(160100035 + cfg), with +1000*j for the j-th
solve of the ragged batch.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 160100035


def rng_for(cfg: int, sub: int = 0) -> np.random.Generator:
    return np.random.default_rng(SEED_BASE + cfg + 1000 * sub)


# ---------------------------------------------------------------------------
# analytic fields
# ---------------------------------------------------------------------------
def _rotation(axis: np.ndarray) -> np.ndarray:
    """Rotation matrix taking e_z to the unit vector `axis`."""
    a = np.asarray(axis, dtype=float)
    a = a / np.linalg.norm(a)
    z = np.array([0.0, 0.0, 1.0])
    v = np.cross(z, a)
    s = np.linalg.norm(v)
    c = float(np.dot(z, a))
    if s < 1e-15:
        return np.eye(3) if c > 0 else np.diag([1.0, -1.0, -1.0])
    vx = np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]])
    return np.eye(3) + vx + vx @ vx * ((1 - c) / s ** 2)


def ring_vorticity(points: np.ndarray, centre, axis, R: float, sigma: float, gamma: float = 1.0) -> np.ndarray:
    """Gaussian-core vortex ring (Sec. 6, eq. initial_omega_gauss, read with the
    negative exponent and rho = sqrt(x^2 + y^2)):
        omega_theta = Gamma/(pi sigma^2) exp(-(z^2 + (rho - R)^2)/sigma^2),
    expressed in the ring frame (axis -> z) and returned as Cartesian vectors."""
    Rm = _rotation(axis)
    p = (np.asarray(points, dtype=float) - np.asarray(centre, dtype=float)) @ Rm  # ring frame
    x, y, z = p[..., 0], p[..., 1], p[..., 2]
    rho = np.sqrt(x * x + y * y)
    w = gamma / (math.pi * sigma ** 2) * np.exp(-(z * z + (rho - R) ** 2) / sigma ** 2)
    with np.errstate(invalid="ignore", divide="ignore"):
        ex = np.where(rho > 0, -y / rho, 0.0)
        ey = np.where(rho > 0, x / rho, 0.0)
    v = np.stack([w * ex, w * ey, np.zeros_like(w)], axis=-1)
    return v @ Rm.T


def ring_velocity_like(points: np.ndarray, centre, axis, R: float, s: float, amp: float = 1.0) -> np.ndarray:
    """Smooth divergence-free ring-shaped field u = curl(psi e_theta),
    psi = amp * exp(-((rho - R)^2 + z^2)/s^2), with the curl taken in closed form:
        u_rho = -d psi/dz,  u_z = (1/rho) d(rho psi)/d rho."""
    Rm = _rotation(axis)
    p = (np.asarray(points, dtype=float) - np.asarray(centre, dtype=float)) @ Rm
    x, y, z = p[..., 0], p[..., 1], p[..., 2]
    rho = np.sqrt(x * x + y * y)
    psi = amp * np.exp(-((rho - R) ** 2 + z * z) / s ** 2)
    u_rho = 2.0 * z / s ** 2 * psi
    with np.errstate(invalid="ignore", divide="ignore"):
        u_z = np.where(rho > 0, psi / rho, 0.0) - 2.0 * (rho - R) / s ** 2 * psi
        cx = np.where(rho > 0, x / rho, 0.0)
        cy = np.where(rho > 0, y / rho, 0.0)
    v = np.stack([u_rho * cx, u_rho * cy, u_z], axis=-1)
    return v @ Rm.T


def _grid_points(n, shift):
    nz, ny, nx = n
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack([x + shift[0], y + shift[1], z + shift[2]], axis=-1).astype(float)


def edge_points(n, q):
    s = [0.0, 0.0, 0.0]
    s[q] = -0.5
    return _grid_points(n, s)


def face_points(n, q):
    s = [-0.5, -0.5, -0.5]
    s[q] = 0.0
    return _grid_points(n, s)


def cell_points(n):
    return _grid_points(n, [-0.5, -0.5, -0.5])


def random_axis_tilted(rng: np.random.Generator) -> np.ndarray:
    """Axis tilted from e_z by theta ~ U[0, pi/2] about a horizontal axis at azimuth phi ~ U[0, 2 pi)."""
    theta = rng.uniform(0.0, math.pi / 2)
    phi = rng.uniform(0.0, 2 * math.pi)
    h = np.array([math.cos(phi), math.sin(phi), 0.0])  # rotation axis
    # rotate e_z about h by theta (Rodrigues)
    ez = np.array([0.0, 0.0, 1.0])
    return ez * math.cos(theta) + np.cross(h, ez) * math.sin(theta) + h * np.dot(h, ez) * (1 - math.cos(theta))


def random_axis_sphere(rng: np.random.Generator) -> np.ndarray:
    v = rng.standard_normal(3)
    return v / np.linalg.norm(v)


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def gaussian_blobs(n: int = 32, nblob: int = 3, sigma: float = 3.0, spread: float = 8.0, cfg: int = 1) -> np.ndarray:
    """Scalar source: sum of Gaussian blobs A exp(-|x-c|^2/(2 sigma^2)), A ~ U[-1,1],
    c = box centre + U[-spread, spread]^3, sampled at cell centres. Returns f[z, y, x]."""
    rng = rng_for(cfg)
    pts = cell_points((n, n, n))
    f = np.zeros((n, n, n))
    for _ in range(nblob):
        A = rng.uniform(-1.0, 1.0)
        c = n / 2 + rng.uniform(-spread, spread, size=3)
        f += A * np.exp(-((pts - c) ** 2).sum(-1) / (2 * sigma ** 2))
    return f


def vortex_ring_edges(n: int, R: float, sigma: float, axis, centre=None, gamma: float = 1.0) -> np.ndarray:
    """Edge-sampled vorticity of one ring; returns w[q, z, y, x] (q = component)."""
    if centre is None:
        centre = np.array([n / 2.0] * 3)
    out = np.zeros((3, n, n, n))
    for q in range(3):
        out[q] = ring_vorticity(edge_points((n, n, n), q), centre, axis, R, sigma, gamma)[..., q]
    return out


def ring_128(cfg: int = 2, n: int = 128, R: float = 32.0, sigma: float = 3.0):
    """Vector source of the 128^3 streamfunction solve: one tilted ring at the box centre."""
    rng = rng_for(cfg)
    axis = random_axis_tilted(rng)
    return vortex_ring_edges(n, R, sigma, axis), axis


def two_ring_velocity(cfg: int = 3, n: int = 128):
    """Face-sampled smooth ring-shaped velocity of two seeded rings: u[q, z, y, x].

    Stand-in for the velocity of two Gaussian vortex rings (centres within 16
    cells of the box centre, R ~ U[16, 28], tilted as in the 128^3 ring case);
    the field is the closed-form curl of a Gaussian ring potential, so it
    carries no Poisson-solve arithmetic."""
    rng = rng_for(cfg)
    u = np.zeros((3, n, n, n))
    for _ in range(2):
        c = n / 2 + rng.uniform(-16, 16, size=3)
        R = rng.uniform(16, 28)
        axis = random_axis_tilted(rng)
        for q in range(3):
            u[q] += ring_velocity_like(face_points((n, n, n), q), c, axis, R, s=6.0)[..., q]
    return u


def two_rings_vorticity(cfg: int = 3, n: int = 128, sigma: float = 3.0):
    """Edge-sampled vorticity of the two seeded Gaussian-core rings of the 128^3
    integrating-factor workload (circulation 1 each, centres within 16 cells of the
    box centre, R ~ U[16, 28], sigma = 3, tilted as in the 128^3 ring case): w[q, z, y, x].
    The velocity u = C^T a, a = -L^{-1} w, is left to the caller (it needs the Poisson
    solve)."""
    rng = rng_for(cfg)
    w = np.zeros((3, n, n, n))
    for _ in range(2):
        c = n / 2 + rng.uniform(-16, 16, size=3)
        R = rng.uniform(16, 28)
        axis = random_axis_tilted(rng)
        w += vortex_ring_edges(n, R, sigma, axis, centre=c)
    return w


def thin_ring_vorticity(R: float = 400.0, sigma: float = 5.0, B: int = 16, rel_thresh: float = 1e-6, cfg: int = 6):
    """All three components of the thin ring of thin_ring_blocks (component q at edge(q)
    centres, Gamma = 1), on the blocks where any component exceeds rel_thresh * max.
    Returns (block coordinates [n, 3], values [n, 3, B, B, B] float32)."""
    rng = rng_for(cfg)
    axis = random_axis_tilted(rng)
    reach = 6.0 * sigma + B
    span = int(math.ceil((R + reach) / B)) + 1
    g = np.arange(-span, span)
    bz, by, bx = np.meshgrid(g, g, g, indexing="ij")
    cen = (np.stack([bx.ravel(), by.ravel(), bz.ravel()], 1) + 0.5) * B
    p = cen @ _rotation(axis)
    near = np.hypot(np.hypot(p[:, 0], p[:, 1]) - R, p[:, 2]) < reach
    cand = np.stack([bx.ravel(), by.ravel(), bz.ravel()], 1)[near].astype(np.int32)
    k, j, i = np.meshgrid(np.arange(B), np.arange(B), np.arange(B), indexing="ij")
    base = np.stack([i.ravel(), j.ravel(), k.ravel()], 1).astype(float)
    vals = np.zeros((len(cand), 3, B, B, B), dtype=np.float32)
    for q in range(3):
        shift = np.zeros(3)
        shift[q] = -0.5
        for n, c in enumerate(cand):
            vals[n, q] = ring_vorticity(c * B + base + shift, np.zeros(3), axis, R, sigma)[:, q].reshape(B, B, B)
    mx = np.abs(vals).reshape(len(cand), -1).max(1)
    keep = mx > rel_thresh * mx.max()
    return cand[keep], vals[keep], axis


def thin_ring_blocks(R: float = 400.0, sigma: float = 5.0, B: int = 16, rel_thresh: float = 1e-6, cfg: int = 6):
    """A thin Gaussian-core ring of radius R cells and core sigma (delta/R0 = 0.0125 at the
    defaults, the thinnest ring of Sec. 6) centred at the origin, axis tilted as in the 128^3
    ring case; the scalar source is the x-component of its vorticity at edge(1) centres,
    kept on the blocks whose |w| exceeds rel_thresh * max.  Only blocks near the torus are
    sampled, so the box (about 2R + 12 sigma across) is never held densely.
    Returns (block coordinates [n, 3], values [n, 1, B, B, B] float32)."""
    rng = rng_for(cfg)
    axis = random_axis_tilted(rng)
    reach = 6.0 * sigma + B                       # torus half-thickness plus one block
    span = int(math.ceil((R + reach) / B)) + 1
    g = np.arange(-span, span)
    bz, by, bx = np.meshgrid(g, g, g, indexing="ij")
    cen = (np.stack([bx.ravel(), by.ravel(), bz.ravel()], 1) + 0.5) * B
    Rm = _rotation(axis)
    p = cen @ Rm
    rho = np.hypot(p[:, 0], p[:, 1])
    near = np.hypot(rho - R, p[:, 2]) < reach
    cand = np.stack([bx.ravel(), by.ravel(), bz.ravel()], 1)[near].astype(np.int32)
    k, j, i = np.meshgrid(np.arange(B), np.arange(B), np.arange(B), indexing="ij")
    loc = np.stack([i.ravel(), j.ravel(), k.ravel()], 1).astype(float) + np.array([-0.5, 0.0, 0.0])  # edge(1)
    vals = np.zeros((len(cand), 1, B, B, B), dtype=np.float32)
    for n, c in enumerate(cand):
        w = ring_vorticity(c * B + loc, np.zeros(3), axis, R, sigma)[:, 0]
        vals[n, 0] = w.reshape(B, B, B)
    mx = np.abs(vals).reshape(len(cand), -1).max(1)
    keep = mx > rel_thresh * mx.max()
    return cand[keep], vals[keep]


def ragged_ring_sources(nsolve: int = 64, emin: int = 24, emax: int = 192, cfg: int = 5):
    """Ragged batch: per solve an edge e ~ round(exp(U[ln emin, ln emax])), a ring with
    R ~ U[4, min(40, (e/2 - 2)/1.75)], sigma = R/8, axis uniform on S^2, centred in the box;
    the scalar source is its x-component sampled at edge(1) centres. Returns a list of f[z,y,x]."""
    out = []
    for j in range(nsolve):
        rng = rng_for(cfg, j)
        e = int(round(math.exp(rng.uniform(math.log(emin), math.log(emax)))))
        rmax = min(40.0, (e / 2 - 2) / 1.75)
        R = rng.uniform(4.0, max(4.0, rmax))
        axis = random_axis_sphere(rng)
        w = ring_vorticity(edge_points((e, e, e), 0), np.array([e / 2.0] * 3), axis, R, R / 8)[..., 0]
        out.append(w)
    return out


# ---------------------------------------------------------------------------
# block layout helpers
# ---------------------------------------------------------------------------
def pad_to_blocks(f: np.ndarray, B: int) -> np.ndarray:
    """Zero-pad the trailing spatial dims of f[..., z, y, x] up to multiples of B."""
    shp = f.shape[-3:]
    pad = [(0, 0)] * (f.ndim - 3) + [(0, (-s) % B) for s in shp]
    return np.pad(f, pad)


def block_grid(shape, B: int) -> np.ndarray:
    """All block coordinates (bx, by, bz) covering a box of shape (nz, ny, nx)."""
    nbz, nby, nbx = [(s + B - 1) // B for s in shape]
    bz, by, bx = np.meshgrid(np.arange(nbz), np.arange(nby), np.arange(nbx), indexing="ij")
    return np.stack([bx.ravel(), by.ravel(), bz.ravel()], axis=1).astype(np.int32)


def active_blocks(f: np.ndarray, B: int, rel_thresh: float) -> np.ndarray:
    """Blocks holding any |f| > rel_thresh * max|f| (f[..., z, y, x]; the max
    runs over leading component axes too)."""
    a = np.abs(f)
    if a.ndim == 4:
        a = a.max(axis=0)
    a = pad_to_blocks(a, B)
    nbz, nby, nbx = [s // B for s in a.shape]
    m = a.reshape(nbz, B, nby, B, nbx, B).max(axis=(1, 3, 5))
    thr = rel_thresh * a.max()
    bz, by, bx = np.nonzero(m > thr)
    return np.stack([bx, by, bz], axis=1).astype(np.int32)


def to_blocks(f: np.ndarray, B: int, coords: np.ndarray, dtype=np.float32) -> np.ndarray:
    """Dense f[(c,) z, y, x] -> block-contiguous [nblk, ncomp, B, B, B] (x fastest)."""
    if f.ndim == 3:
        f = f[None]
    f = pad_to_blocks(f, B)
    nc = f.shape[0]
    out = np.zeros((len(coords), nc, B, B, B), dtype=dtype)
    for i, (bx, by, bz) in enumerate(np.asarray(coords)):
        out[i] = f[:, bz * B:(bz + 1) * B, by * B:(by + 1) * B, bx * B:(bx + 1) * B]
    return out


def from_blocks(blocks: np.ndarray, B: int, coords: np.ndarray, shape) -> np.ndarray:
    """Block-contiguous [nblk, ncomp, B, B, B] -> dense [ncomp, *shape] (zeros where no block)."""
    blocks = np.asarray(blocks)
    nc = blocks.shape[1]
    nz, ny, nx = shape
    pz, py, px = [((s + B - 1) // B) * B for s in shape]
    out = np.zeros((nc, pz, py, px), dtype=np.float64)
    for i, (bx, by, bz) in enumerate(np.asarray(coords)):
        out[:, bz * B:(bz + 1) * B, by * B:(by + 1) * B, bx * B:(bx + 1) * B] = blocks[i]
    return out[:, :nz, :ny, :nx]


def block_points(coords: np.ndarray, B: int) -> np.ndarray:
    """Integer (x, y, z) of every point of the listed blocks, in block-contiguous order."""
    k, j, i = np.meshgrid(np.arange(B), np.arange(B), np.arange(B), indexing="ij")
    loc = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)
    coords = np.asarray(coords, dtype=np.int64)
    return (coords[:, None, :] * B + loc[None]).reshape(-1, 3).astype(np.int32)
