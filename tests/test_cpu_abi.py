"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, and
exports every function declared in include/lgf.h (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lgf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*([a-z_0-9]+)\s*\(", src, flags=re.M)))


def test_header_declares_entry_points():
    names = _declared()
    for n in ["lgf_table_build", "lgf_conv_plan", "lgf_conv_execute", "ifactor_apply", "lgf_residual_fp64",
              "lgf_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    if not os.path.exists("/usr/local/cuda/bin/nvcc") and not os.environ.get("NVCC"):
        pytest.skip("no CUDA toolkit")
    from paper_1601_00035_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for n in _declared():
        assert hasattr(lib, n), n
    from paper_1601_00035_gb300 import lgf
    lgf.load()
    assert set(lgf._SIGS) == set(_declared())


def test_required_max_offset():
    import numpy as np
    from paper_1601_00035_gb300 import lgf
    b = np.array([[0, 0, 0], [7, 7, 7]])
    assert lgf.required_max_offset(b, b, 16) == 127
    # a target inside a long source: the offsets alone allow length 128, the
    # source extent (96 points) needs 192 so that it fills at most half a line
    s = np.array([[i, 0, 0] for i in range(6)])
    t = np.array([[3, 0, 0]])
    assert lgf.required_max_offset(s, t, 16) == 95
    # far target: the offsets decide
    assert lgf.required_max_offset(np.array([[0, 0, 0]]), np.array([[30, 0, 0]]), 16) == 511
    # lengths 3 * 2^k: a 40-point box needs 2 * 39 + 2 = 80 -> 96; 80 points -> 160 -> 192;
    # 160 points -> 320 -> 384; 200 points -> 400 -> 512
    for e, n in ((40, 96), (80, 192), (160, 384), (200, 512)):
        c = np.array([[0, 0, 0], [e // 8 - 1, 0, 0]])
        assert lgf.required_max_offset(c, c, 8) == n // 2 - 1, e
    assert [lgf.fft_length(v) for v in (1, 17, 65, 97, 129, 193, 257, 385, 513, 1025)] == \
        [16, 32, 96, 128, 192, 256, 384, 512, 1024, 0]


def test_size_rule_matches_the_library():
    """lgf.fft_length (used by required_max_offset on the host) and the library's
    own size rule agree for every need up to past the largest length."""
    if not os.path.exists("/usr/local/cuda/bin/nvcc") and not os.environ.get("NVCC"):
        pytest.skip("no CUDA toolkit")
    from paper_1601_00035_gb300 import lgf
    L = lgf.load()
    for need in range(1, 1100):
        assert L.lgf_fft_length(need) == lgf.fft_length(need), need
