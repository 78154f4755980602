"""C-ABI checks that need no GPU: the library loads, exports every function
include/gfbp.h declares, and rejects bad arguments on the host before any
CUDA call."""
import ctypes as C
import os
import re
import shutil

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gfbp():
    from paper_cs_0605069_gb300 import build, gfbp as G
    if not os.path.exists(G.LIB_PATH):
        if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
            pytest.skip("libgfbp.so not built and nvcc unavailable")
        build.build()
    G.lib()
    return G


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(gfbp_[a-z0-9_]+)\s*\(", src))
    return names


def test_every_declared_function_is_exported(gfbp):
    names = declared_functions()
    assert {"gfbp_code_create", "gfbp_decode", "gfbp_step"} <= names
    lib = C.CDLL(gfbp.LIB_PATH)
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert names == set(gfbp.EXPORTS) | (names - set(gfbp.EXPORTS))
    assert set(gfbp.EXPORTS) <= names


def _create(gfbp, q, M, N, rows, cols, vals, poly=0):
    r = np.ascontiguousarray(rows, np.int32)
    c = np.ascontiguousarray(cols, np.int32)
    v = np.ascontiguousarray(vals, np.int32)
    h = C.c_void_p()
    rc = gfbp.lib().gfbp_code_create(q, M, N, r.size, r.ctypes.data, c.ctypes.data, v.ctypes.data, poly, C.byref(h))
    return rc, gfbp.last_error()


def test_code_create_validates_on_host(gfbp):
    rc, msg = _create(gfbp, 3, 1, 2, [0], [0], [1])
    assert rc == gfbp.GFBP_EINVAL and "q must be" in msg
    rc, msg = _create(gfbp, 4, 1, 2, [0], [0], [4])
    assert rc == gfbp.GFBP_EINVAL and "out of range" in msg
    rc, msg = _create(gfbp, 4, 1, 2, [0, 0], [1, 1], [1, 2])
    assert rc == gfbp.GFBP_EINVAL and "duplicate" in msg
    rc, msg = _create(gfbp, 16, 1, 2, [0], [0], [1], poly=0x1F)
    assert rc == gfbp.GFBP_EINVAL and "primitive" in msg
    rc, msg = _create(gfbp, 4, 1, 20, [0] * 17, list(range(17)), [1] * 17)
    assert rc == gfbp.GFBP_EUNSUPPORTED
    rc, msg = _create(gfbp, 4, 0, 0, [], [], [])
    assert rc == gfbp.GFBP_EINVAL


def test_decode_rejects_null_code(gfbp):
    ch = gfbp.gfbp_channel(0, 0.1, None)
    rc = gfbp.lib().gfbp_decode(None, 1, None, ch, 0, None, 10, None, None, None, None, None)
    assert rc == gfbp.GFBP_EINVAL and "NULL code" in gfbp.last_error()
    n = C.c_size_t()
    assert gfbp.lib().gfbp_workspace_size(None, 1, 0, None, 0, C.byref(n)) == gfbp.GFBP_EINVAL


def test_binding_has_no_cpu_path():
    src = open(os.path.join(ROOT, "paper_cs_0605069_gb300", "gfbp.py")).read()
    assert "oracle" not in src
    for f in os.listdir(os.path.join(ROOT, "paper_cs_0605069_gb300")):
        if f.endswith(".py"):
            assert "import oracle" not in open(os.path.join(ROOT, "paper_cs_0605069_gb300", f)).read()
