"""The C ABI library builds, loads and exports every entry point that
include/pic.h declares; argument errors are reported without any GPU work."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pic.h")


def declared_entry_points():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1612_03369_gb300 import build

    path = build.build()
    return C.CDLL(path)


def test_header_declares_the_paper_calls():
    names = declared_entry_points()
    for n in ("pic_create_mesh", "pic_seed_particles", "pic_set_velocity_dofs", "pic_advect", "pic_locate",
              "pic_rebin", "pic_interpolate_to_cells"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_entry_points():
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol(lib):
    from paper_1612_03369_gb300 import pic

    assert set(pic.SIGNATURES) >= set(declared_entry_points())
    assert pic.pic_version().startswith("pic-gb300")


def test_argument_errors_without_gpu(lib):
    lib.pic_create_mesh.restype = C.c_int
    lib.pic_last_error.restype = C.c_char_p
    out = C.c_void_p()
    n = (C.c_int * 3)(4, 4, 4)
    # dim 5 is rejected before any CUDA call
    assert lib.pic_create_mesh(5, n, C.c_void_p(1), 0, None, C.byref(out)) == 1
    assert b"dim" in lib.pic_last_error()
    assert out.value is None
    bad = (C.c_int * 2)(4, 0)
    assert lib.pic_create_mesh(2, bad, C.c_void_p(1), 0, None, C.byref(out)) == 1
    lib.pic_advect.restype = C.c_int
    lib.pic_advect.argtypes = [C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.c_int, C.c_int, C.c_void_p]
    assert lib.pic_advect(None, None, 0.1, 4, 0, 1, None) == 1
    assert lib.pic_rebin(None, None) == 1
    lib.pic_get_state.restype = C.c_int
    assert lib.pic_get_state(None, None, None, None) == 1


def test_no_oracle_on_product_path():
    """The library sources and the binding never reference the oracle."""
    pkg = os.path.join(ROOT, "paper_1612_03369_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")) and f != "workloads.py":
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "pic_oracle" not in text and "liboracle" not in text, f
