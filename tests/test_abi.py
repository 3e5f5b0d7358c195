"""CPU checks of the C-ABI boundary: the library builds, loads and exports every
entry point that include/rihv.h declares (no compute calls without a GPU)."""
import os
import re

import pytest

from paper_1904_04884_gb300 import build as B
from paper_1904_04884_gb300 import rihv

INC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


def declared():
    names = set()
    for f in os.listdir(INC):
        if f.endswith(".h"):
            names |= set(re.findall(r"\b(rihv_[a-z0-9_]+)\s*\(", open(os.path.join(INC, f)).read()))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    B.build()
    return rihv.load_library()


def test_header_declares_the_boundary():
    names = declared()
    for n in ("rihv_create", "rihv_forward", "rihv_adjoint", "rihv_prox_fused_lasso",
              "rihv_solve", "rihv_detect", "rihv_destroy", "rihv_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(rihv.EXPORTS) <= set(declared())


def test_errors_without_device_are_reported(lib):
    # Unsupported sizes are rejected before any CUDA call.
    import ctypes
    h = ctypes.c_void_p()
    st = lib.rihv_create(100, 64, 4, 532e-9, 5e-6, 5e-3, 50e-6, ctypes.byref(h))
    assert st == 6
    assert b"unsupported size" in lib.rihv_last_error(None)
    st = lib.rihv_create(64, 64, 4, -1.0, 5e-6, 5e-3, 50e-6, ctypes.byref(h))
    assert st == 1


def test_default_options(lib):
    o = rihv.Options()
    lib.rihv_default_options(o)
    assert (o.tv_dims, o.restart, o.accelerate, o.n_inner, o.check_every) == (3, 1, 1, 20, 10)
    assert (o.tv_steps_per_launch, o.fuse_finalize, o.skip_empty_planes) == (2, 1, 0)


def test_options_binding_mirrors_the_header():
    """The ctypes mirror lists the header's rihv_options fields in order."""
    text = open(os.path.join(INC, "rihv.h")).read()
    body = re.search(r"typedef struct \{(.*?)\} rihv_options;", text, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(int|double)\s+(\w+)\s*;", body)
    names = [n for _, n in fields]
    assert names == [n for n, _ in rihv.Options._fields_]
    import ctypes
    for (ty, _), (_, cty) in zip(fields, rihv.Options._fields_):
        assert cty is (ctypes.c_int if ty == "int" else ctypes.c_double)
