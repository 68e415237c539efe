"""The C-ABI library loads, exports every function include/sense.h declares,
and rejects bad arguments on the host before touching the GPU (CPU only)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sense.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2202_14005_b300 import _lib, build
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    return _lib.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s+([a-z_][a-z0-9_]*)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["sense_plan_create", "sense_forward", "sense_adjoint", "sense_normal",
              "cg_dc_solve", "cg_dc_solve_backward", "sense_get_status", "sense_strerror"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for n in declared_functions():
        assert hasattr(lib, n), f"{n} declared in sense.h but not exported"


def test_strerror_covers_codes(lib):
    for code in range(0, -9, -1):
        s = lib.sense_strerror(code).decode()
        assert s and s != "unknown error code"
    assert lib.sense_strerror(-99).decode() == "unknown error code"


def _create(lib, B, Cc, H, W, maps, mask, lines=1):
    h = C.c_void_p()
    return lib.sense_plan_create(C.byref(h), B, Cc, H, W, maps, mask, lines, None), h


def test_plan_create_rejects_bad_shapes_on_host(lib):
    buf = (C.c_byte * 64)()
    base = (C.addressof(buf) + 15) & ~15
    p = C.c_void_p(base)
    assert _create(lib, 0, 2, 8, 8, p, p)[0] == -1
    assert _create(lib, 1, 0, 8, 8, p, p)[0] == -1
    assert _create(lib, 1, 2, 7, 8, p, p)[0] == -1      # odd H
    assert _create(lib, 1, 2, 8, 9, p, p)[0] == -1      # odd W
    assert _create(lib, 1, 2, 8, 8, None, p)[0] == -2   # NULL maps
    assert _create(lib, 1, 2, 8, 8, C.c_void_p(base + 4), p)[0] == -2  # misaligned
    assert _create(lib, 1, 2, 8, 8, p, p, lines=2)[0] == -7
    assert _create(lib, 1, 2, 8, 74, p, p)[0] == -4     # 74 = 2 * 37: prime factor > 31


def test_calls_reject_null_plan(lib):
    assert lib.sense_normal(None, None, None, C.c_float(0.0)) == -2
    assert lib.sense_forward(None, None, None) == -2
    assert lib.sense_adjoint(None, None, None) == -2
    assert lib.cg_dc_solve(None, None, None, None, None, 1, 1, None) == -2
    v = C.c_int()
    assert lib.sense_get_status(None, C.byref(v)) == -2
    assert lib.sense_plan_destroy(None) == -2
