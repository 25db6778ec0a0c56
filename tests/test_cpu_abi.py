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
    # lengths 3 * 2^k, 9 * 2^5, 27 * 2^4: a 40-point box needs 2 * 39 + 2 = 80 -> 96;
    # 80 points -> 160 -> 192; 136 points -> 272 -> 288; 160 points -> 320 -> 384;
    # 200 points -> 400 -> 432; 232 points -> 464 -> 512
    for e, n in ((40, 96), (80, 192), (136, 288), (160, 384), (200, 432), (232, 512)):
        c = np.array([[0, 0, 0], [e // 8 - 1, 0, 0]])
        assert lgf.required_max_offset(c, c, 8) == n // 2 - 1, e
    assert [lgf.fft_length(v) for v in (1, 17, 65, 97, 129, 193, 257, 289, 385, 433, 513, 769, 1025)] == \
        [16, 32, 96, 128, 192, 256, 288, 384, 432, 512, 768, 1024, 0]


def test_size_rule_matches_the_library():
    """lgf.fft_length (used by required_max_offset on the host) and the library's
    own size rule agree for every need up to past the largest length."""
    if not os.path.exists("/usr/local/cuda/bin/nvcc") and not os.environ.get("NVCC"):
        pytest.skip("no CUDA toolkit")
    from paper_1601_00035_gb300 import lgf
    L = lgf.load()
    for need in range(1, 1100):
        assert L.lgf_fft_length(need) == lgf.fft_length(need), need


def _noalloc_status(blocks, B=16, ncomp=1, alpha=0.2):
    """Call ifactor_apply_noalloc with placeholder device pointers: the argument
    checks under test all run on the host before any CUDA call."""
    import numpy as np
    from paper_1601_00035_gb300 import lgf
    L = lgf.load()
    b = np.ascontiguousarray(blocks, dtype=np.int32).reshape(-1, 3)
    st = L.ifactor_apply_noalloc(alpha, B, ncomp, len(b), b.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                 ctypes.c_void_p(256), ctypes.c_void_p(512), None)
    return st, L.lgf_last_error().decode()


def test_noalloc_rejects_bad_block_sets_on_the_host():
    if not os.path.exists("/usr/local/cuda/bin/nvcc") and not os.environ.get("NVCC"):
        pytest.skip("no CUDA toolkit")
    from paper_1601_00035_gb300 import lgf
    m = (1 << 20) - 1
    # two far corners: each extent is 2^21 + 2 blocks; the product would overflow a 64-bit long
    st, msg = _noalloc_status([[-m, -m, -m], [m, m, m]])
    assert st == lgf.LGF_ERR_ARG and "extent" in msg
    # extents within range but the box too large
    st, msg = _noalloc_status([[0, 0, 0], [200, 200, 200]])
    assert st == lgf.LGF_ERR_ARG and "bounding box" in msg
    # duplicate blocks
    st, msg = _noalloc_status([[0, 0, 0], [1, 0, 0], [0, 0, 0]])
    assert st == lgf.LGF_ERR_ARG and "duplicate" in msg
    # coordinates outside +-2^20
    st, msg = _noalloc_status([[1 << 20, 0, 0]])
    assert st == lgf.LGF_ERR_ARG and "coordinate" in msg


def test_struct_layouts_match_header(tmp_path):
    """The binding's ctypes structures have the size and field offsets that a C compiler
    gives the header's structures (lgf_solve_desc, lgf_plan_opts, lgf_rk_desc)."""
    import ctypes
    import shutil
    import subprocess
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_1601_00035_gb300 import lgf
    structs = {"lgf_solve_desc": lgf._SolveDesc, "lgf_plan_opts": lgf._PlanOpts, "lgf_rk_desc": lgf._RkDesc}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "lgf.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in py._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, fname))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([gcc, "-I", inc, str(src), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
