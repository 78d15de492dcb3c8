"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol
(no compute call: runs without a GPU)."""
import ctypes
import os
import re

from paper_2507_09730_gb300 import binding as B
from conftest import ROOT


def declared_functions():
    src = open(os.path.join(ROOT, "include", "frw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(frw_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    names = declared_functions()
    assert len(names) >= 12
    L = B.lib()
    for n in names:
        assert hasattr(L, n), n
    assert set(B.EXPORTS) == set(names)


def test_checked_library_exports_the_same_symbols():
    from paper_2507_09730_gb300 import build as bld
    L = ctypes.CDLL(bld.build(checked=True))
    for n in declared_functions():
        assert hasattr(L, n), n


def test_options_layout_and_defaults():
    assert ctypes.sizeof(B.frw_options) == 80
    assert ctypes.sizeof(B.frw_block) == 56
    assert ctypes.sizeof(B.frw_job) == 40
    o = B.frw_default_options()
    assert o.N == 24 and o.hybrid == 1 and o.max_hops == 100000 and o.precision == B.FRW_FP64_GEOM


def test_strerror_and_bad_create():
    assert B.frw_strerror(0) == "ok"
    assert "sigma" in B.frw_strerror(B.FRW_ENOTCONV)
    # invalid options are rejected before any device call
    o = B.frw_default_options(N=7)
    ctx = ctypes.c_void_p()
    assert B.lib().frw_create(ctypes.byref(ctx), 0, ctypes.byref(o)) == B.FRW_EINVAL
