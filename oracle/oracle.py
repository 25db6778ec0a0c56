"""FP64 CPU oracle (test infrastructure only; see the package docstring).

Heavy loops (table quadrature, direct sums) live in ``lgf_oracle.c``; the
staggered-grid operators of App. A and the residual are plain numpy.

Conventions
-----------
* Dense boxes are numpy arrays indexed ``[z, y, x]`` (x fastest in memory);
  vector fields carry a leading component axis ``q = 0, 1, 2`` for the
  paper's superscripts (1), (2), (3), i.e. the x, y, z components.
* Values outside a box are zero (the mask operator M of Sec. 4.2).
* The unit-lattice LGF ``G`` is returned; the physical kernel is
  ``G_L = dx**2 * G`` (reading of App. B: the 7-point Laplacian carries
  ``1/dx**2``, so its fundamental solution carries ``dx**2``).
"""
from __future__ import annotations

import ctypes
import functools
import math
import os

import numpy as np

from . import build as _build

__all__ = [
    "lib", "gauss_legendre", "bessel_scaled", "lgf_octant", "lgf_cube", "lgf_value",
    "octant_size", "asymptotic_G", "ifactor_taps", "ifactor_radius", "direct_conv",
    "direct_conv_box", "ifactor_direct", "shift", "op_G", "op_Gt", "op_C", "op_Ct", "op_D",
    "op_Dbar", "op_L", "op_N", "residual_L", "WATSON_W", "num_threads", "SCHEME_A", "SCHEME_B", "SCHEME_C",
    "SCHEMES", "shifted_tableau",
    "block_mask", "ifactor_masked", "poisson_masked", "if_herk_step", "lgf_points", "ifactor_tail", "rk_qmax",
    "vor2vel", "ring_diagnostics", "regrid_weights", "fft_conv", "vel_from_vort", "if_herk_step_vorticity",
]

# Watson's integral for the simple cubic lattice, closed form (Watson 1939):
#   W = sqrt(6) / (32 pi^3) * Gamma(1/24) Gamma(5/24) Gamma(7/24) Gamma(11/24)
WATSON_W = (math.sqrt(6.0) / (32.0 * math.pi ** 3) * math.gamma(1 / 24) * math.gamma(5 / 24)
            * math.gamma(7 / 24) * math.gamma(11 / 24))

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)


@functools.lru_cache(maxsize=1)
def lib() -> ctypes.CDLL:
    path = _build.build()
    L = ctypes.CDLL(path)
    L.oracle_gauss_legendre.argtypes = [ctypes.c_int, _dp, _dp]
    L.oracle_bessel_scaled.argtypes = [ctypes.c_double, ctypes.c_int, _dp]
    L.oracle_octant_size.argtypes = [ctypes.c_int]
    L.oracle_octant_size.restype = ctypes.c_int64
    L.oracle_lgf_octant.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_int, _dp]
    L.oracle_octant_to_cube.argtypes = [ctypes.c_int, _dp, _dp]
    L.oracle_lgf_points.argtypes = [ctypes.c_int64, _ip, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_int, _dp]
    L.oracle_direct_conv.argtypes = [ctypes.c_int, _dp, ctypes.c_int64, _ip, _dp,
                                     ctypes.c_int64, _ip, _dp]
    L.oracle_ifactor_direct.argtypes = [ctypes.c_int, _dp, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, _dp, ctypes.c_int64, _ip, _dp]
    return L


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def _d(a):
    return a.ctypes.data_as(_dp)


def _i(a):
    return a.ctypes.data_as(_ip)


def gauss_legendre(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().oracle_gauss_legendre(n, _d(x), _d(w))
    return x, w


def bessel_scaled(t: float, nmax: int) -> np.ndarray:
    """exp(-2t) I_n(2t) for n = 0..nmax (Miller recurrence / Hankel series)."""
    out = np.zeros(nmax + 1)
    rc = lib().oracle_bessel_scaled(float(t), int(nmax), _d(out))
    if rc != 0:
        raise ValueError("bessel_scaled: bad arguments")
    return out


def octant_size(K: int) -> int:
    return int(lib().oracle_octant_size(K))


# Default quadrature: Gauss-Legendre in s = ln t on [ln 1e-18, ln 1e12],
# panels of width 1, 16 nodes each, plus the closed-form tail beyond 1e12.
QUAD_DEFAULT = dict(t_lo=1e-18, T=1e12, panel=1.0, ngl=16)


@functools.lru_cache(maxsize=8)
def lgf_octant(K: int, t_lo: float = QUAD_DEFAULT["t_lo"], T: float = QUAD_DEFAULT["T"],
               panel: float = QUAD_DEFAULT["panel"], ngl: int = QUAD_DEFAULT["ngl"]) -> np.ndarray:
    """Unit-lattice G on the sorted octant K >= a >= b >= c >= 0 (App. B, Bessel form)."""
    out = np.zeros(octant_size(K))
    rc = lib().oracle_lgf_octant(int(K), t_lo, T, panel, int(ngl), _d(out))
    if rc != 0:
        raise RuntimeError("oracle_lgf_octant failed (%d)" % rc)
    out.setflags(write=False)
    return out


@functools.lru_cache(maxsize=4)
def lgf_cube(K: int, t_lo: float = QUAD_DEFAULT["t_lo"]) -> np.ndarray:
    """Dense table D[|dz|, |dy|, |dx|] = G(dx, dy, dz), 0..K on each axis.  With t_lo above
    its default the Bessel-form integral starts there: -int_{t_lo}^inf prod_i i_{n_i}(t) dt
    (the far part of a split of G at time t_lo)."""
    oct_ = np.ascontiguousarray(lgf_octant(K, t_lo=t_lo))
    cube = np.zeros((K + 1, K + 1, K + 1))
    lib().oracle_octant_to_cube(int(K), _d(oct_), _d(cube))
    cube.setflags(write=False)
    return cube


def lgf_points(offsets) -> np.ndarray:
    """G at explicit integer offsets [n, 3] (App. B Bessel form, same quadrature as the table)."""
    o = np.ascontiguousarray(offsets, dtype=np.int32).reshape(-1, 3)
    nmax = int(np.abs(o).max()) if len(o) else 0
    out = np.zeros(len(o))
    q = QUAD_DEFAULT
    rc = lib().oracle_lgf_points(len(o), _i(o), nmax, q["t_lo"], q["T"], q["panel"], int(q["ngl"]), _d(out))
    if rc != 0:
        raise RuntimeError("oracle_lgf_points failed (%d)" % rc)
    return out


def lgf_value(n, K: int | None = None) -> float:
    a, b, c = sorted((abs(int(v)) for v in n), reverse=True)
    if K is None:
        K = max(a, 8)
    oct_ = lgf_octant(K)
    return float(oct_[a * (a + 1) * (a + 2) // 6 + b * (b + 1) // 2 + c])


def asymptotic_G(n) -> np.ndarray:
    """Two-term large-|n| expansion of the unit LGF (App. B)."""
    n = np.asarray(n, dtype=float)
    r2 = (n ** 2).sum(-1)
    r = np.sqrt(r2)
    n4 = (n ** 4).sum(-1)
    cross = n[..., 0] ** 2 * n[..., 1] ** 2 + n[..., 0] ** 2 * n[..., 2] ** 2 + n[..., 1] ** 2 * n[..., 2] ** 2
    return -1.0 / (4 * np.pi * r) - (n4 - 3 * cross) / (16 * np.pi * r ** 7)


def ifactor_radius(alpha: float, tol: float = 1e-14) -> int:
    """Largest on-axis offset r with g(r) g(0)^2 >= tol.

    Reading of the truncation rule 'drop the kernel where |E_Q| < tol': the
    retained support is the box |n_i| <= R (App. B eq. lgf_intfac)."""
    g = bessel_scaled(alpha, 200)
    r = 0
    while r + 1 <= 200 and g[r + 1] * g[0] ** 2 >= tol:
        r += 1
    return r


def ifactor_taps(alpha: float, tol: float = 1e-14) -> np.ndarray:
    """1-D factors g(k) = exp(-2 alpha) I_k(2 alpha), k = 0..R (App. B eq. lgf_intfac)."""
    R = ifactor_radius(alpha, tol)
    return bessel_scaled(alpha, R)


def direct_conv(cube: np.ndarray, src_xyz: np.ndarray, val: np.ndarray, tgt_xyz: np.ndarray) -> np.ndarray:
    """u(t_j) = sum_i G(t_j - s_i) val_i (Sec. 2.2 eq. dpoisson_conv), FP64, unit lattice."""
    K = cube.shape[0] - 1
    cube = np.ascontiguousarray(cube, dtype=np.float64)
    src = np.ascontiguousarray(src_xyz, dtype=np.int32).reshape(-1, 3)
    tgt = np.ascontiguousarray(tgt_xyz, dtype=np.int32).reshape(-1, 3)
    v = np.ascontiguousarray(val, dtype=np.float64).reshape(-1)
    out = np.zeros(len(tgt))
    rc = lib().oracle_direct_conv(K, _d(cube), len(src), _i(src), _d(v), len(tgt), _i(tgt), _d(out))
    if rc != 0:
        raise ValueError("direct_conv: offset beyond the table (K=%d)" % K)
    return out


def direct_conv_box(cube: np.ndarray, f: np.ndarray, tgt_xyz: np.ndarray, origin=(0, 0, 0)) -> np.ndarray:
    """Direct sum with the source given as a dense box f[z, y, x] (zeros skipped)."""
    z, y, x = np.nonzero(f)
    src = np.stack([x, y, z], axis=1).astype(np.int32) + np.asarray(origin, dtype=np.int32)
    return direct_conv(cube, src, f[z, y, x], tgt_xyz)


def fft_conv(f: np.ndarray, src_origin, tgt_origin, tgt_shape, workers: int | None = None) -> np.ndarray:
    """u(n) = sum_m G(n - m) f(m) (eq. dpoisson_conv on the unit lattice) for every n of
    the box tgt_origin + [0, tgt_shape), by one FP64 linear convolution through
    zero-padded FFTs (the FFT is a library step; G comes from lgf_cube over every offset
    the two boxes produce, so nothing wraps).

    f: dense [z, y, x] sources whose point (0, 0, 0) is src_origin (x, y, z), or
    [c, z, y, x] for c independent components (the kernel is transformed once);
    tgt_shape: (nz, ny, nx).  Returns u[z, y, x] (or [c, z, y, x]).  Pinned against
    direct_conv."""
    import scipy.fft as sf
    f = np.asarray(f, dtype=np.float64)
    if f.ndim == 4:
        return np.stack(list(_fft_conv_many(f, src_origin, tgt_origin, tgt_shape, workers)))
    return next(_fft_conv_many(f[None], src_origin, tgt_origin, tgt_shape, workers))


def _fft_conv_many(fs, src_origin, tgt_origin, tgt_shape, workers):
    import scipy.fft as sf
    f = fs[0]
    S0 = np.asarray(src_origin, dtype=np.int64)
    T0 = np.asarray(tgt_origin, dtype=np.int64)
    Sn = np.array(f.shape[::-1], dtype=np.int64)          # (x, y, z) extents
    Tn = np.array(tuple(tgt_shape)[::-1], dtype=np.int64)
    dmin = T0 - (S0 + Sn - 1)                              # smallest offset n - m per axis
    dmax = T0 + Tn - 1 - S0                                # largest
    cube = lgf_cube(int(max(np.abs(dmin).max(), np.abs(dmax).max())))
    ax = [np.abs(np.arange(dmin[a], dmax[a] + 1)) for a in range(3)]
    k = cube[np.ix_(ax[2], ax[1], ax[0])]                  # k[i] = G(dmin + i), [z, y, x]
    # full linear convolution; lengths rounded up to fast FFT sizes (extra zeros change nothing)
    L = [sf.next_fast_len(f.shape[i] + k.shape[i] - 1, real=True) for i in range(3)]
    w = workers or os.cpu_count() or 1
    kh = sf.rfftn(k, L, workers=w)
    st = (Sn - 1)[::-1]                                    # index of n = T0: n - S0 - dmin
    for fc in fs:
        U = sf.irfftn(sf.rfftn(fc, L, workers=w) * kh, L, workers=w)
        yield U[st[0]:st[0] + tgt_shape[0], st[1]:st[1] + tgt_shape[1], st[2]:st[2] + tgt_shape[2]].copy()


def ifactor_direct(g: np.ndarray, x: np.ndarray, tgt_xyz: np.ndarray) -> np.ndarray:
    """y(n) = sum_m prod_i g(|n_i - m_i|) x(m) over the box |n_i - m_i| <= R (plain 3-D sum)."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    tgt = np.ascontiguousarray(tgt_xyz, dtype=np.int32).reshape(-1, 3)
    nz, ny, nx = x.shape
    out = np.zeros(len(tgt))
    lib().oracle_ifactor_direct(len(g) - 1, _d(g), nx, ny, nz, _d(x), len(tgt), _i(tgt), _d(out))
    return out


# ---------------------------------------------------------------------------
# Staggered-grid operators, App. A point-operator forms.  Axis map: paper
# component (1),(2),(3) = x,y,z = numpy axis 2,1,0 of a [z,y,x] array.
# ---------------------------------------------------------------------------
_AX = {0: 2, 1: 1, 2: 0}


def shift(a: np.ndarray, q: int, s: int) -> np.ndarray:
    """b(n) = a(n + s e_q) with zeros beyond the box (mask semantics)."""
    ax = _AX[q]
    b = np.zeros_like(a)
    n = a.shape[ax]
    if abs(s) >= n:
        return b
    src = [slice(None)] * a.ndim
    dst = [slice(None)] * a.ndim
    if s > 0:
        src[ax] = slice(s, n)
        dst[ax] = slice(0, n - s)
    else:
        src[ax] = slice(0, n + s)
        dst[ax] = slice(-s, n)
    b[tuple(dst)] = a[tuple(src)]
    return b


def op_G(c: np.ndarray, dx: float = 1.0) -> np.ndarray:
    """cells -> faces: dx [G c]^(q)_n = c_{n+e_q} - c_n."""
    return np.stack([(shift(c, q, 1) - c) / dx for q in range(3)])


def op_Gt(f: np.ndarray, dx: float = 1.0) -> np.ndarray:
    """faces -> cells, the adjoint of G:  G^T f = -Dbar f."""
    return -op_Dbar(f, dx)


def op_Dbar(f: np.ndarray, dx: float = 1.0) -> np.ndarray:
    """faces -> cells: dx [Dbar f]_n = sum_q (f^(q)_n - f^(q)_{n-e_q})."""
    return sum((f[q] - shift(f[q], q, -1)) for q in range(3)) / dx


def op_C(f: np.ndarray, dx: float = 1.0) -> np.ndarray:
    """faces -> edges: dx [C f]^(1) = f2_n - f2_{n+e3} + f3_{n+e2} - f3_n, cyclic in (1,2,3)."""
    out = []
    for q in range(3):
        r, s = (q + 1) % 3, (q + 2) % 3
        out.append((f[r] - shift(f[r], s, 1) + shift(f[s], r, 1) - f[s]) / dx)
    return np.stack(out)


def op_Ct(e: np.ndarray, dx: float = 1.0) -> np.ndarray:
    """edges -> faces: dx [Cbar e]^(1) = e2_{n-e3} - e2_n + e3_n - e3_{n-e2}, cyclic."""
    out = []
    for q in range(3):
        r, s = (q + 1) % 3, (q + 2) % 3
        out.append((shift(e[r], s, -1) - e[r] + e[s] - shift(e[s], r, -1)) / dx)
    return np.stack(out)


def op_D(e: np.ndarray, dx: float = 1.0) -> np.ndarray:
    """edges -> vertices: dx [D e]_n = sum_q (e^(q)_{n+e_q} - e^(q)_n)."""
    return sum((shift(e[q], q, 1) - e[q]) for q in range(3)) / dx


def op_L(a: np.ndarray, dx: float = 1.0) -> np.ndarray:
    """7-point Laplacian: dx^2 [L a]_n = -6 a_n + sum_{q, +-1} a_{n +- e_q} (per component)."""
    if a.ndim == 4:
        return np.stack([op_L(a[q], dx) for q in range(a.shape[0])])
    return (sum(shift(a, q, 1) + shift(a, q, -1) for q in range(3)) - 6.0 * a) / (dx * dx)


def op_N(f: np.ndarray, dx: float = 1.0) -> np.ndarray:
    """Rotational nonlinear term of App. A eq. opr_def_nonlin, e = C f:
    [N f]^(1) = 1/4 sum_{m in {-1,0}} [ e2_{n+m e3} (f3 + f3_{+e1})_{n+m e3}
                                         - e3_{n+m e2} (f2 + f2_{+e1})_{n+m e2} ], cyclic."""
    e = op_C(f, dx)
    out = []
    for q in range(3):
        r, s = (q + 1) % 3, (q + 2) % 3
        a = e[r] * (f[s] + shift(f[s], q, 1))
        b = e[s] * (f[r] + shift(f[r], q, 1))
        out.append(0.25 * sum(shift(a, s, m) - shift(b, r, m) for m in (-1, 0)))
    return np.stack(out)


def residual_L(u: np.ndarray, f: np.ndarray, interior: np.ndarray, dx: float = 1.0) -> float:
    """||L u - f||_2 / ||f||_2 over the points flagged `interior` (App. A stencil)."""
    r = op_L(u, dx) - f
    den = np.sqrt((f[interior] ** 2).sum())
    return float(np.sqrt((r[interior] ** 2).sum()) / den)


# ---------------------------------------------------------------------------
# IF-HERK step on a finite block set (Sec. 3.2 algorithm, Sec. 3.3 eq.
# proj_final, Sec. 5 xIF-HERK masks), FP64, written in the paper's order:
# q and w recursions, one integrating factor per quantity.
# ---------------------------------------------------------------------------
SCHEME_A = {
    "A": np.array([[0.0, 0.0, 0.0],
                   [0.5, 0.0, 0.0],
                   [math.sqrt(3) / 3, (3 - math.sqrt(3)) / 3, 0.0]]),
    "b": np.array([(3 + math.sqrt(3)) / 6, -math.sqrt(3) / 3, (3 + math.sqrt(3)) / 6]),
    "c": np.array([0.0, 0.5, 1.0]),
}
# Schemes B and C of eq. ifherk_schemes (Sec. 3.2)
SCHEME_B = {
    "A": np.array([[0.0, 0.0, 0.0],
                   [1.0 / 3.0, 0.0, 0.0],
                   [-1.0, 2.0, 0.0]]),
    "b": np.array([0.0, 0.75, 0.25]),
    "c": np.array([0.0, 1.0 / 3.0, 1.0]),
}
SCHEME_C = {
    "A": np.array([[0.0, 0.0, 0.0],
                   [8.0 / 15.0, 0.0, 0.0],
                   [0.25, 5.0 / 12.0, 0.0]]),
    "b": np.array([0.25, 0.0, 0.75]),
    "c": np.array([0.0, 8.0 / 15.0, 2.0 / 3.0]),
}
SCHEMES = {"A": SCHEME_A, "B": SCHEME_B, "C": SCHEME_C}


def shifted_tableau(tab=SCHEME_A):
    """Shifted coefficients of eq. herk_shift: a~_{i,j} = a_{i+1,j} (i < s), b_j (i = s);
    c~_i = c_{i+1} (i < s), 1 (i = s).  Returned 1-based as dicts for readability."""
    A, b, c = tab["A"], tab["b"], tab["c"]
    s = len(b)
    at = {}
    for i in range(1, s + 1):
        for j in range(1, i + 1):
            at[(i, j)] = A[i, j - 1] if i < s else b[j - 1]
    ct = {i: (c[i] if i < s else 1.0) for i in range(1, s + 1)}
    ct[0] = c[0]  # reading: c~_0 = c_1 (the first stage starts at t_k)
    return at, ct, s


def block_mask(shape, B, blocks, origin_blocks=(0, 0, 0)):
    """Boolean mask [z,y,x] of the listed blocks inside a dense box whose block (0,0,0)
    is origin_blocks."""
    m = np.zeros(shape, dtype=bool)
    o = np.asarray(origin_blocks)
    for bx, by, bz in (np.asarray(blocks) - o).tolist():
        m[bz * B:(bz + 1) * B, by * B:(by + 1) * B, bx * B:(bx + 1) * B] = True
    return m


def ifactor_masked(g, f, mask):
    """M E(alpha) M f on a dense box (per component), plain 3-D sum over all points."""
    z, y, x = np.nonzero(mask)
    tgt = np.stack([x, y, z], 1).astype(np.int32)
    if f.ndim == 4:
        return np.stack([ifactor_masked(g, f[q], mask) for q in range(f.shape[0])])
    out = np.zeros_like(f)
    out[z, y, x] = ifactor_direct(g, np.where(mask, f, 0.0), tgt)
    return out


def poisson_masked(cube, f, supp_mask, xsoln_mask, dx):
    """M^xsoln L^{-1} M^supp f by the direct sum (eq. dpoisson_conv), G_L = dx^2 G."""
    z, y, x = np.nonzero(xsoln_mask)
    tgt = np.stack([x, y, z], 1).astype(np.int32)
    out = np.zeros_like(f)
    out[z, y, x] = dx * dx * direct_conv_box(cube, np.where(supp_mask, f, 0.0), tgt)
    return out


def ifactor_tail(k: int, alpha: float, nmax: int = 400) -> float:
    """Truncation error of the integrating factor at depth k inside a masked
    region (App. D): for a uniform field kept only on n > 0, the relative
    difference between E(alpha) u and M E(alpha) M u at n = k is the kernel's
    mass beyond the mask edge, sum_{n >= k} g(n), g(n) = exp(-2 alpha) I_n(2 alpha).
    (Reading: the App. D sum is written with index k - j + 1; the mass that the
    mask removes at depth k is the tail n >= k of the 1-D kernel.)"""
    g = bessel_scaled(alpha, nmax)
    return float(g[k:].sum()) if k <= nmax else 0.0


def rk_qmax(beta: float, depth: int, eps: float, qcap: int = 1 << 16) -> int:
    """Largest number of steps q (>= 1 when possible, else 0) over which the
    integrating factors of a step, E(q beta) with beta = dt / (dx^2 Re), keep the
    truncation error at depth n_E = depth below eps relative to max |u| (Sec. 5
    velocity refresh, App. D)."""
    q = 0
    while q < qcap and ifactor_tail(depth, (q + 1) * beta) <= eps:
        q += 1
    return q


def ring_diagnostics(u, dx, origin_cells, xs_mask, int_mask):
    """The volume integrals of Sec. 6 eq. int_quantities on the lattice: impulse
    I = 1/2 sum x cross w, K = sum u . (x cross w), E = 1/2 sum |w|^2, J = sum u . w
    and the centroid X = 1/2 sum ((x cross w) . I / |I|^2) x (without the
    freestream term), each times dx^3, over int_mask (D_soln: the integrands'
    support, Sec. 6; the mask edge of D_xsoln carries a spurious vortex sheet that
    these sums must not see).
    Readings: w = M C M u on edges (eq. w_k of the algorithm summary, M = M^xsoln).
    I, E and X are sums over edges, each vorticity component at its own edge
    (edge (q) of vertex n at n - e_q / 2); K and J pair u with w at cell centres,
    averaging the 2 faces / 4 edges around each cell (cell n at n - (1,1,1)/2).
    Positions add origin_cells; an edge or face belongs to the cell of its index."""
    w = op_C(u * xs_mask, dx) * xs_mask * int_mask
    nz, ny, nx = int_mask.shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    vert = [(i + origin_cells[0]) * dx, (j + origin_cells[1]) * dx, (k + origin_cells[2]) * dx]
    dv = dx ** 3
    # x cross w, term by term at the edges of the vorticity component involved
    def x_at_edge(a, q):  # coordinate a of edge (q)
        return vert[a] - (0.5 * dx if a == q else 0.0)
    I = np.zeros(3)
    M = np.zeros((3, 3))
    for a_ in range(3):
        b_, c_ = (a_ + 1) % 3, (a_ + 2) % 3
        # (x cross w)_a = x_b w_c - x_c w_b
        t1, t2 = x_at_edge(b_, c_) * w[c_], x_at_edge(c_, b_) * w[b_]
        I[a_] = 0.5 * (t1.sum() - t2.sum()) * dv
        for bb in range(3):
            M[a_, bb] = 0.5 * ((t1 * x_at_edge(bb, c_)).sum() - (t2 * x_at_edge(bb, b_)).sum()) * dv
    E = float(0.5 * (w * w).sum() * dv)
    X = (M.T @ I) / float(I @ I) if float(I @ I) > 0 else np.zeros(3)
    # cell-centred products for K and J
    uc = np.stack([0.5 * (u[q] + shift(u[q], q, -1)) for q in range(3)]) * int_mask
    wc = []
    for q in range(3):
        r, s_ = (q + 1) % 3, (q + 2) % 3
        wc.append(0.25 * (w[q] + shift(w[q], r, -1) + shift(w[q], s_, -1) + shift(shift(w[q], r, -1), s_, -1)))
    wc = np.stack(wc) * int_mask
    pos = [v - 0.5 * dx for v in vert]
    xw = np.stack([pos[1] * wc[2] - pos[2] * wc[1], pos[2] * wc[0] - pos[0] * wc[2], pos[0] * wc[1] - pos[1] * wc[0]])
    K = float((uc * xw).sum() * dv)
    J = float((uc * wc).sum() * dv)
    return {"I": I, "K": K, "E": E, "J": J, "X": X}


def regrid_weights(u, uinf, dx, xs_mask, B, blocks, origin_blocks, parts=False):
    """Block weights of Sec. 5 eq. weight_fun on D_xsoln: W = max(mu / mu_global,
    nu / nu_global), mu = max |C u| and nu = max |G^T N~(u + u_inf)| over the block,
    from w = M C M u and q = -M G^T M N~(M (u + u_inf)) (algorithm summary, step 1).
    Reading of 'contaminated by finite boundary errors': w and q are zeroed on the
    cells within 3 cells of the outside of D_xsoln.  The masked curl is spurious on the
    last cell layer; N~ and G^T each reach one cell further, so q carries that error
    3 cells deep.
    blocks: [n][3] block coordinates (the dense box's block (0,0,0) at origin_blocks);
    returns W per listed block (with parts=True: W, mu, nu)."""
    xs = xs_mask
    w = op_C(u * xs, dx) * xs
    uf = (u + np.asarray(uinf, dtype=float).reshape(3, 1, 1, 1)) * xs
    q = -op_Gt(op_N(uf, dx) * xs, dx) * xs
    inner = xs.copy()
    for _ in range(3):  # erode by one cell (26-neighbourhood) three times
        prev = inner.copy()
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dxx in (-1, 0, 1):
                    inner &= shift(shift(shift(prev, 0, dxx), 1, dy), 2, dz)
    w = w * inner
    q = q * inner
    mu, nu = [], []
    for bx, by, bz in (np.asarray(blocks) - np.asarray(origin_blocks)).tolist():
        sl = (slice(bz * B, (bz + 1) * B), slice(by * B, (by + 1) * B), slice(bx * B, (bx + 1) * B))
        mu.append(np.abs(w[(slice(None),) + sl]).max())
        nu.append(np.abs(q[sl]).max())
    mu, nu = np.array(mu), np.array(nu)
    W = np.maximum(mu / mu.max(), nu / nu.max() if nu.max() > 0 else 0.0 * nu)
    return (W, mu, nu) if parts else W


def vor2vel(u, masks, cube, dx):
    """Velocity refresh of Sec. 5 (eq. vel_refresh): w = M^xsoln C M^xsoln u,
    a = -M^xsoln L^{-1} M^supp w (per component, eq. vel_vor), u' = M^xsoln C^T M^xsoln a."""
    xs = masks["xsoln"]
    w = op_C(u * xs, dx) * xs
    a = np.stack([-poisson_masked(cube, w[q], masks["supp"], xs, dx) for q in range(3)])
    return op_Ct(a * xs, dx) * xs


def if_herk_step(u, dt, re, dx, uinf, masks, cube, nonlinear=True, tab=SCHEME_A):
    """One xIF-HERK step u_k -> u_{k+1} on a dense box.

    u: face velocity [3, z, y, x] (zero outside D_xsoln); masks: dict of boolean
    [z,y,x] arrays 'supp', 'soln', 'xsoln'; uinf: constant freestream (3,).
    Integrating factors H^i = E((c~_i - c~_{i-1}) dt / (dx^2 Re)) (eq. ifherk_aux_1);
    g^i = -a~_{ii} dt M^soln N~(M^xsoln(u^{i-1} + u_inf)) (eq. ifherk_g, with the
    sign of eq. ifherk_g rather than eq. rhs_final); projection eq. proj_final with
    d^ = -M^xsoln L^{-1} M^supp G^T M^xsoln r (eq. dpoisson_final)."""
    at, ct, s = shifted_tableau(tab)
    xs = masks["xsoln"]
    alpha = dt / (dx * dx * re)
    H = {}
    for i in range(1, s + 1):
        a = (ct[i] - ct[i - 1]) * alpha
        H[i] = None if a == 0.0 else ifactor_taps(a)

    def applyH(i, f):
        return f * xs if H[i] is None else ifactor_masked(H[i], f, xs)

    uinf = np.asarray(uinf, dtype=float).reshape(3, 1, 1, 1)
    q = {1: u.copy()}
    w = {}
    u_prev = u
    for i in range(1, s + 1):
        if nonlinear:
            g = -at[(i, i)] * dt * op_N((u_prev + uinf) * xs, dx) * masks["soln"]
        else:
            g = np.zeros_like(u)
        r = q[i] + g
        for j in range(1, i):
            r = r + dt * at[(i, j)] * w[(i, j)]
        r = r * xs
        dhat = -poisson_masked(cube, op_Gt(r, dx), masks["supp"], xs, dx)
        gd = op_G(dhat, dx) * xs
        u_i = applyH(i, r - gd)
        w[(i, i)] = (g - gd) / (at[(i, i)] * dt)
        if i < s:
            q[i + 1] = applyH(i, q[i])
            for j in range(1, i + 1):
                w[(i + 1, j)] = applyH(i, w[(i, j)])
        u_prev = u_i
    return u_prev


def vel_from_vort(w, masks, cube, dx):
    """u = M^xsoln C^T M^xsoln a, a = -M^xsoln L^{-1} M^supp w per component (Sec. 4.1 eq. vel_vor
    with the masks of Sec. 5), for an edge field w on D_xsoln."""
    xs = masks["xsoln"]
    a = np.stack([-poisson_masked(cube, w[q], masks["supp"], xs, dx) for q in range(3)])
    return op_Ct(a * xs, dx) * xs


def if_herk_step_vorticity(w, dt, re, dx, uinf, masks, cube, tab=SCHEME_A):
    """One step of the vorticity formulation of Sec. 4.1: the discrete curl of eq. dnstp,
        dw/dt = (1/Re) L w - C N~(u + u_inf),   u = -C^T L^{-1} w   (eq. vel_vor),
    integrated with the IF-HERK algorithm of Sec. 3.2 in the paper's q / w recursions; there is no
    constraint, so each stage value is the integrating factor applied to r^i (no projection).
    Masks (reading: Sec. 5 carried over): w lives on D_xsoln, the integrating factors are
    M^xsoln E M^xsoln, the velocity takes its Poisson source on D_supp, and the stage term is
    g^i = -a~_ii dt M^soln C M^soln N~(M^xsoln (u^{i-1} + u_inf))."""
    at, ct, s = shifted_tableau(tab)
    xs, so = masks["xsoln"], masks["soln"]
    alpha = dt / (dx * dx * re)
    H = {}
    for i in range(1, s + 1):
        a = (ct[i] - ct[i - 1]) * alpha
        H[i] = None if a == 0.0 else ifactor_taps(a)

    def applyH(i, f):
        return f * xs if H[i] is None else ifactor_masked(H[i], f, xs)

    uinf = np.asarray(uinf, dtype=float).reshape(3, 1, 1, 1)
    q = {1: w.copy()}
    z = {}
    w_prev = w
    for i in range(1, s + 1):
        u = vel_from_vort(w_prev, masks, cube, dx)
        g = -at[(i, i)] * dt * op_C(op_N((u + uinf) * xs, dx) * so, dx) * so
        r = q[i] + g
        for j in range(1, i):
            r = r + dt * at[(i, j)] * z[(i, j)]
        w_i = applyH(i, r * xs)
        z[(i, i)] = g / (at[(i, i)] * dt)
        if i < s:
            q[i + 1] = applyH(i, q[i])
            for j in range(1, i + 1):
                z[(i + 1, j)] = applyH(i, z[(i, j)])
        w_prev = w_i
    return w_prev
