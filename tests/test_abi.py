"""The C ABI library builds, loads and exports every function the header declares.

No compute call is made here (this container has no GPU): only symbol
resolution, struct layouts and host-side argument checks that fail before any
CUDA call.
"""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mstress.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|const char\*)\s+(mstress_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2411_12690_gb300 import build as b
    b.build()
    from paper_2411_12690_gb300 import _lib
    return _lib.load()


def test_header_and_binding_agree(lib):
    from paper_2411_12690_gb300 import _lib
    decl = declared_functions()
    assert len(decl) >= 20
    assert sorted(_lib.SIGNATURES) == decl
    for name in decl:
        assert hasattr(lib, name), name


def test_struct_layouts_match_c():
    from paper_2411_12690_gb300 import _lib as L
    # sizes follow the C layout rules for the declared member order
    assert C.sizeof(L.mstress_material) == 24
    assert C.sizeof(L.mstress_block_mesh) == 3 * 8 + 3 * 4 + 4 + 8
    assert C.sizeof(L.mstress_layout) == 4 + 4 + 8 + 8 + 8
    assert C.sizeof(L.mstress_bc) == 4 + 4 + 8 + 8 + 8
    assert C.sizeof(L.mstress_opts) == 8 * 8


def test_defaults_and_null_handles(lib):
    from paper_2411_12690_gb300 import _lib as L
    o = L.mstress_opts()
    assert lib.mstress_opts_default(C.byref(o)) == 0
    assert o.precision == L.MSTRESS_FP64 and o.rtol == 1e-13 and o.max_iter == 20000
    assert lib.mstress_opts_default(None) == L.MSTRESS_EINVAL
    assert lib.mstress_sync(None) == L.MSTRESS_EINVAL
    assert lib.mstress_solve(None, None, 0.0, None, None) == L.MSTRESS_EINVAL
    assert lib.mstress_sol_info(None, 0, None, None, None, None) == L.MSTRESS_EINVAL
    assert lib.mstress_last_error(None) == b"null context"
    lib.mstress_free_sol(None)
    lib.mstress_free_block(None)
    lib.mstress_free_ctx(None)
