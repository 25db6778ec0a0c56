"""Thin ctypes binding of liblgf.so (the C-ABI in include/lgf.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Device buffers are torch CUDA tensors (float32, contiguous) passed by
data pointer; streams default to torch's current stream.  There is no CPU
fallback: if the library is missing or fails to load, `load()` raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liblgf.so")

LGF_OK = 0
LGF_ERR_ARG = -1
LGF_ERR_OOM = -2
LGF_ERR_CUDA = -3
LGF_ERR_TIMEOUT = -4
LGF_ERR_TOL = -5
LGF_ERR_STATE = -6

LAPLACE7 = 0
IFACTOR = 1


class LGFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("lgf status %d: %s" % (status, msg))
        self.status = status


class _SolveDesc(ctypes.Structure):
    _fields_ = [
        ("B", ctypes.c_int),
        ("ncomp", ctypes.c_int),
        ("n_src", ctypes.c_int),
        ("n_dst", ctypes.c_int),
        ("src_blocks", ctypes.POINTER(ctypes.c_int32)),
        ("dst_blocks", ctypes.POINTER(ctypes.c_int32)),
        ("dx", ctypes.c_double),
        ("scale", ctypes.c_double),
    ]


class _RkDesc(ctypes.Structure):
    _fields_ = [
        ("B", ctypes.c_int),
        ("n_soln", ctypes.c_int),
        ("soln_blocks", ctypes.POINTER(ctypes.c_int32)),
        ("dx", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("re", ctypes.c_double),
        ("scheme", ctypes.c_int),
        ("use_graph", ctypes.c_int),
        ("poisson_method", ctypes.c_int),
        ("reserved", ctypes.c_int * 1),
    ]


class _PlanOpts(ctypes.Structure):
    _fields_ = [("use_graph", ctypes.c_int), ("precision", ctypes.c_int), ("method", ctypes.c_int),
                ("far_precision", ctypes.c_int), ("split_alpha", ctypes.c_double), ("near_form", ctypes.c_int),
                ("reserved", ctypes.c_int * 1)]


METHOD_WHOLE_BOX, METHOD_SPLIT, METHOD_AUTOTUNE = 0, 1, 2


_lib = None

# name -> (restype, argtypes); every function declared in include/lgf.h
_SIGS = {
    "lgf_table_build": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.POINTER(ctypes.c_void_p)]),
    "lgf_table_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "lgf_table_copy": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int64]),
    "lgf_table_size": (ctypes.c_int64, [ctypes.c_void_p]),
    "lgf_table_destroy": (None, [ctypes.c_void_p]),
    "lgf_conv_plan": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(_SolveDesc), ctypes.c_int,
                                     ctypes.POINTER(_PlanOpts), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "lgf_plan_workspace_bytes": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    "lgf_plan_method": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]),
    "lgf_plan_check": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "lgf_wait_probe": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p]),
    "lgf_conv_execute": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p]),
    "lgf_conv_execute_f64": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p),
                                            ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p]),
    "lgf_conv_execute_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p),
                                             ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p]),
    "ifactor_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "ifactor_apply_noalloc": (ctypes.c_int, [ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p]),
    "lgf_residual_fp64": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "lgf_plan_set_profiling": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "lgf_plan_kernel_count": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "lgf_plan_kernel_times": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p),
                                             ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double)]),
    "lgf_rk_plan": (ctypes.c_int, [ctypes.POINTER(_RkDesc), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "lgf_rk_block_count": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "lgf_rk_blocks": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int32), ctypes.c_int]),
    "lgf_rk_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                   ctypes.c_void_p]),
    "lgf_rk_step_vorticity": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "lgf_op_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                    ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "lgf_rk_refresh": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "lgf_rk_qmax": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "lgf_rk_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_void_p]),
    "lgf_rk_diagnostics": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                          ctypes.c_void_p]),
    "lgf_rk_regrid_blocks": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                            ctypes.c_double, ctypes.POINTER(ctypes.c_int32), ctypes.c_int,
                                            ctypes.c_void_p]),
    "lgf_rk_transfer": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "lgf_plan_destroy": (None, [ctypes.c_void_p]),
    "lgf_last_error": (ctypes.c_char_p, []),
    "lgf_version": (ctypes.c_char_p, []),
    "lgf_fft_length": (ctypes.c_int, [ctypes.c_int]),
    "lgf_measure_peak": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                        ctypes.c_void_p]),
}


def load() -> ctypes.CDLL:
    """Load liblgf.so; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("liblgf.so not built (expected %s); run paper_1601_00035_gb300/build.py "
                           "or __graft_entry__.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(st: int):
    if st != LGF_OK:
        raise LGFError(st, load().lgf_last_error().decode())


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError("expected a contiguous float32 CUDA tensor")
    return t.data_ptr()


class Table:
    """FP64 kernel table on the device (lgf_table_build)."""

    def __init__(self, kind: int, alpha: float = 0.0, max_offset: int = 0, stream=None):
        L = load()
        h = ctypes.c_void_p()
        _check(L.lgf_table_build(kind, float(alpha), int(max_offset), _stream(stream), ctypes.byref(h)))
        self._h = h
        k, a, K, R = ctypes.c_int(), ctypes.c_double(), ctypes.c_int(), ctypes.c_int()
        _check(L.lgf_table_info(h, ctypes.byref(k), ctypes.byref(a), ctypes.byref(K), ctypes.byref(R)))
        self.kind, self.alpha, self.max_offset, self.radius = k.value, a.value, K.value, R.value

    def values(self) -> np.ndarray:
        L = load()
        n = L.lgf_table_size(self._h)
        out = np.zeros(n)
        _check(L.lgf_table_copy(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n))
        return out

    def close(self):
        if getattr(self, "_h", None):
            load().lgf_table_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class Solve:
    """One independent problem (lgf_solve_desc)."""
    B: int
    ncomp: int
    src_blocks: np.ndarray            # [n_src, 3] int (bx, by, bz)
    dst_blocks: Optional[np.ndarray]  # [n_dst, 3] (Poisson) or None (IF)
    dx: float = 1.0
    scale: float = 1.0


class Plan:
    """lgf_conv_plan over one or more solves.

    The keyword options are the fields of lgf_plan_opts: method 0 (whole-box FFT convolution),
    1 (block-sparse split solve) or 2 (plan both, keep the faster); split_alpha, far_precision
    (0 CUDA cores, 1 tensor cores) and near_form (0 time the forms, 1 pairs, 2 runs of 4 targets,
    3 quads of 4 x 2 targets) for the split solve."""

    def __init__(self, table: Table, solves: Sequence[Solve], use_graph: bool = False, stream=None,
                 precision: int = 0, method: int = 0, split_alpha: float = 0.0, far_precision: int = 0,
                 near_form: int = 0):
        L = load()
        self.table = table  # keep alive
        self.solves = list(solves)
        descs = (_SolveDesc * len(self.solves))()
        self._keep = []
        for d, s in zip(descs, self.solves):
            src = np.ascontiguousarray(s.src_blocks, dtype=np.int32).reshape(-1, 3)
            dst = src if s.dst_blocks is None else np.ascontiguousarray(s.dst_blocks, dtype=np.int32).reshape(-1, 3)
            self._keep += [src, dst]
            d.B, d.ncomp, d.n_src, d.n_dst = s.B, s.ncomp, len(src), len(dst)
            d.src_blocks = src.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            d.dst_blocks = dst.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            d.dx, d.scale = float(s.dx), float(s.scale)
        opts = _PlanOpts()
        opts.use_graph = 1 if use_graph else 0
        opts.precision = int(precision)
        opts.method = int(method)
        opts.split_alpha = float(split_alpha)
        opts.far_precision = int(far_precision)
        opts.near_form = int(near_form)
        h = ctypes.c_void_p()
        _check(L.lgf_conv_plan(table._h, descs, len(self.solves), ctypes.byref(opts), _stream(stream), ctypes.byref(h)))
        self._h = h

    def method(self):
        """(executed method, autotune ms of the whole-box plan, autotune ms of the split plan)."""
        a, b = ctypes.c_double(), ctypes.c_double()
        m = load().lgf_plan_method(self._h, ctypes.byref(a), ctypes.byref(b))
        return m, a.value, b.value

    def check(self, stream=None):
        """Synchronise and raise LGFError(LGF_ERR_TIMEOUT) if a bounded device wait gave up."""
        _check(load().lgf_plan_check(self._h, _stream(stream)))

    def workspace_bytes(self) -> int:
        b = ctypes.c_size_t()
        _check(load().lgf_plan_workspace_bytes(self._h, ctypes.byref(b)))
        return b.value

    def execute(self, src, dst, stream=None):
        """Poisson: dst[i] = scale dx^2 G * src[i] (device tensors)."""
        n = len(self.solves)
        a = (ctypes.c_void_p * n)(*[_ptr(t) for t in src])
        b = (ctypes.c_void_p * n)(*[_ptr(t) for t in dst])
        _check(load().lgf_conv_execute(self._h, a, b, _stream(stream)))

    def execute_f64(self, src, dst, stream=None):
        """FP64 plans (precision=1): float64 device tensors."""
        import torch

        def p64(t):
            if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
                raise TypeError("expected a contiguous float64 CUDA tensor")
            return t.data_ptr()
        n = len(self.solves)
        a = (ctypes.c_void_p * n)(*[p64(t) for t in src])
        b = (ctypes.c_void_p * n)(*[p64(t) for t in dst])
        _check(load().lgf_conv_execute_f64(self._h, a, b, _stream(stream)))

    def execute_host(self, src: Sequence[np.ndarray], dst: Sequence[np.ndarray], stream=None):
        """Poisson with host float32 arrays (pinned for full bandwidth); synchronous."""
        n = len(self.solves)

        def hp(x):
            if hasattr(x, "data_ptr"):
                return x.data_ptr()
            assert x.dtype == np.float32 and x.flags.c_contiguous
            return x.ctypes.data

        a = (ctypes.c_void_p * n)(*[hp(t) for t in src])
        b = (ctypes.c_void_p * n)(*[hp(t) for t in dst])
        _check(load().lgf_conv_execute_host(self._h, a, b, _stream(stream)))

    def ifactor(self, x, y, stream=None):
        """IF plan: y = M E_Q(alpha) M x."""
        _check(load().ifactor_apply(self._h, _ptr(x), _ptr(y), _stream(stream)))

    def residual(self, solve: int, src, dst, stream=None) -> float:
        out = ctypes.c_double()
        _check(load().lgf_residual_fp64(self._h, int(solve), _ptr(src), _ptr(dst), ctypes.byref(out), _stream(stream)))
        return out.value

    def set_profiling(self, enable: int):
        """1: record per-kernel device times; 0: stop; 2: clear totals and record."""
        _check(load().lgf_plan_set_profiling(self._h, int(enable)))

    def kernel_times(self) -> dict:
        """{kernel name: (launches, total device ms)} accumulated while profiling."""
        L = load()
        n = ctypes.c_int()
        _check(L.lgf_plan_kernel_count(self._h, ctypes.byref(n)))
        out = {}
        for i in range(n.value):
            nm, la, ms = ctypes.c_char_p(), ctypes.c_longlong(), ctypes.c_double()
            _check(L.lgf_plan_kernel_times(self._h, i, ctypes.byref(nm), ctypes.byref(la), ctypes.byref(ms)))
            out[nm.value.decode()] = (la.value, ms.value)
        return out

    def close(self):
        if getattr(self, "_h", None):
            load().lgf_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


OP_CURL, OP_CURL_T, OP_DIV_T, OP_GRAD, OP_NONLINEAR = 0, 1, 2, 3, 4


SCHEME_A, SCHEME_B, SCHEME_C = 0, 1, 2


class RKPlan:
    """One IF-HERK step (Scheme A, B or C) on a block set (lgf_rk_plan / lgf_rk_step)."""

    def __init__(self, B: int, soln_blocks, dx: float, dt: float, re: float, stream=None, scheme: int = SCHEME_A,
                 use_graph: bool = False, poisson_method: int = 0):
        """poisson_method: 0 whole box where its FFT lengths reach, else the split solve;
        1 whole box; 2 block-sparse split solve (B = 16)."""
        L = load()
        self._soln = np.ascontiguousarray(soln_blocks, dtype=np.int32).reshape(-1, 3)
        d = _RkDesc()
        d.B, d.n_soln = int(B), len(self._soln)
        d.soln_blocks = self._soln.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        d.dx, d.dt, d.re, d.scheme = float(dx), float(dt), float(re), int(scheme)
        d.use_graph = int(bool(use_graph))
        d.poisson_method = int(poisson_method)
        h = ctypes.c_void_p()
        _check(L.lgf_rk_plan(ctypes.byref(d), _stream(stream), ctypes.byref(h)))
        self._h = h
        self.B = B

    def blocks(self, which: int = 0) -> np.ndarray:
        """Block coordinates of D_xsoln (which=0, field order) or D_soln (which=1)."""
        L = load()
        n = L.lgf_rk_block_count(self._h, which)
        out = np.zeros((n, 3), dtype=np.int32)
        _check(L.lgf_rk_blocks(self._h, which, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), n))
        return out

    def set_profiling(self, enable: int):
        _check(load().lgf_plan_set_profiling(self._h, int(enable)))

    kernel_times = Plan.kernel_times

    def step(self, u_in, u_out, uinf=(0.0, 0.0, 0.0), stream=None):
        ui = (ctypes.c_double * 3)(*[float(v) for v in uinf])
        _check(load().lgf_rk_step(self._h, _ptr(u_in), _ptr(u_out), ui, _stream(stream)))

    def step_vorticity(self, w_in, w_out, uinf=(0.0, 0.0, 0.0), stream=None):
        """One step of the vorticity formulation (lgf_rk_step_vorticity): edge vorticity on D_xsoln."""
        ui = (ctypes.c_double * 3)(*[float(v) for v in uinf])
        _check(load().lgf_rk_step_vorticity(self._h, _ptr(w_in), _ptr(w_out), ui, _stream(stream)))

    def refresh(self, u_in, u_out, stream=None):
        """Velocity refresh (lgf_rk_refresh); u_out may be u_in."""
        _check(load().lgf_rk_refresh(self._h, _ptr(u_in), _ptr(u_out), _stream(stream)))

    def qmax(self, eps: float) -> int:
        q = load().lgf_rk_qmax(self._h, float(eps))
        if q < 0:
            raise LGFError(LGF_ERR_ARG, load().lgf_last_error().decode())
        return int(q)

    def regrid_blocks(self, u, uinf=(0.0, 0.0, 0.0), eps_supp: float = 1e-6, stream=None) -> np.ndarray:
        """New D_supp from the weights of the current field (lgf_rk_regrid_blocks)."""
        L = load()
        ui = (ctypes.c_double * 3)(*[float(v) for v in uinf])
        cap = L.lgf_rk_block_count(self._h, 0)
        out = np.zeros((max(cap, 1), 3), dtype=np.int32)
        n = L.lgf_rk_regrid_blocks(self._h, _ptr(u), ui, float(eps_supp),
                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), cap, _stream(stream))
        if n < 0:
            raise LGFError(LGF_ERR_ARG, L.lgf_last_error().decode())
        return out[:n].copy()

    def transfer_to(self, u_from, other: "RKPlan", u_to, stream=None):
        """Vorticity copy + velocity refresh onto another plan's grid (lgf_rk_transfer)."""
        _check(load().lgf_rk_transfer(self._h, _ptr(u_from), other._h, _ptr(u_to), _stream(stream)))

    def diagnostics(self, u, stream=None) -> dict:
        """Ring diagnostics over D_soln (lgf_rk_diagnostics): I, K, E, J, X."""
        out = (ctypes.c_double * 9)()
        _check(load().lgf_rk_diagnostics(self._h, _ptr(u), out, _stream(stream)))
        v = list(out)
        return {"I": np.array(v[0:3]), "K": v[3], "E": v[4], "J": v[5], "X": np.array(v[6:9])}

    def run(self, u_in, u_out, nsteps: int, uinf=(0.0, 0.0, 0.0), qmax: int = 0, stream=None):
        """nsteps steps with a refresh every qmax steps (lgf_rk_run)."""
        ui = (ctypes.c_double * 3)(*[float(v) for v in uinf])
        _check(load().lgf_rk_run(self._h, _ptr(u_in), _ptr(u_out), int(nsteps), ui, int(qmax), _stream(stream)))

    def op(self, op: int, inp, out, coef: float = 1.0, uinf=(0.0, 0.0, 0.0), stream=None):
        ui = (ctypes.c_double * 3)(*[float(v) for v in uinf])
        _check(load().lgf_op_apply(self._h, int(op), _ptr(inp), _ptr(out), float(coef), ui, _stream(stream)))

    def close(self):
        if getattr(self, "_h", None):
            load().lgf_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ifactor_apply_noalloc(alpha: float, B: int, ncomp: int, blocks, x, y, stream=None):
    """y = M E_Q(alpha) M x without any device allocation (static 64 MiB scratch
    inside the library; for callers that cannot allocate device memory)."""
    b = np.ascontiguousarray(blocks, dtype=np.int32).reshape(-1, 3)
    need = len(b) * int(ncomp) * int(B) ** 3
    if x.numel() != need or y.numel() != need:
        raise ValueError("ifactor_apply_noalloc: x and y must hold len(blocks) * ncomp * B^3 = %d floats "
                         "(got %d and %d)" % (need, x.numel(), y.numel()))
    _check(load().ifactor_apply_noalloc(float(alpha), int(B), int(ncomp), len(b),
                                        b.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _ptr(x), _ptr(y),
                                        _stream(stream)))


PEAK_FP32, PEAK_FP32X2, PEAK_FP64 = 0, 1, 2


def measure_peak(kind: int, ms: float = 200.0, stream=None) -> float:
    """Measured FMA rate of the current GPU in TFLOP/s (lgf_measure_peak)."""
    out = ctypes.c_double()
    _check(load().lgf_measure_peak(int(kind), float(ms), ctypes.byref(out), _stream(stream)))
    return out.value


def wait_probe(polls: int = 1000, stream=None):
    """Run a bounded device wait that cannot complete (lgf_wait_probe): raises LGFError with
    LGF_ERR_TIMEOUT when the wait gives up."""
    _check(load().lgf_wait_probe(int(polls), _stream(stream)))


def version() -> str:
    return load().lgf_version().decode()


# FFT lengths the library supports, ascending (powers of two, 3 times a power of two,
# 288 = 9 * 32 and 432 = 27 * 16)
FFT_LENGTHS = (16, 32, 64, 96, 128, 192, 256, 288, 384, 432, 512, 768, 1024)


def fft_length(need: int) -> int:
    """Smallest supported FFT length >= need (0 if none)."""
    for n in FFT_LENGTHS:
        if n >= need:
            return n
    return 0


def required_max_offset(src_blocks: np.ndarray, dst_blocks: np.ndarray, B: int) -> int:
    """Smallest table max_offset a Poisson plan over these block lists needs
    (half the zero-padded FFT length minus one, per the plan's size rule)."""
    s = np.asarray(src_blocks).reshape(-1, 3)
    t = np.asarray(dst_blocks).reshape(-1, 3)
    need = 0
    for a in range(3):
        S0, S1 = s[:, a].min() * B, (s[:, a].max() + 1) * B - 1
        T0, T1 = t[:, a].min() * B, (t[:, a].max() + 1) * B - 1
        m = max(abs(T0 - S1), abs(T1 - S0))
        n = fft_length(max(2 * m + 2, 2 * (S1 - S0 + 1)))
        need = max(need, n // 2 - 1)
    return int(need)
