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


def _prototypes():
    """name -> parameter count of every function prototype in include/frw.h"""
    src = open(os.path.join(ROOT, "include", "frw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(frw_[a-z_]+)\s*\(([^;{]*?)\)\s*;", src, flags=re.S):
        params = m.group(2).strip()
        out[m.group(1)] = 0 if params in ("", "void") else len(params.split(","))
    return out


def test_binding_argument_counts_match_the_header():
    protos = _prototypes()
    L = B.lib()
    assert set(protos) == set(B.EXPORTS)
    for name, n in protos.items():
        at = getattr(L, name).argtypes
        assert at is not None and len(at) == n, (name, n, at)


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """sizeof and field offsets of the public structs as gcc lays them out against
    the ctypes declarations of the binding."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        import pytest
        pytest.skip("no C compiler")
    structs = [n for n in ("frw_box", "frw_block", "frw_options", "frw_extract_params", "frw_stats", "frw_job",
                           "frw_tuning", "frw_serve_info", "frw_structure")]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "frw.h"', "int main(void) {"]
    for n in structs:
        lines.append(f'    printf("{n} %zu\\n", sizeof({n}));')
        for f, _ in getattr(B, n)._fields_:
            lines.append(f'    printf("{n}.{f} %zu\\n", offsetof({n}, {f}));')
    lines += ["    return 0;", "}"]
    c = tmp_path / "layout.c"
    c.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for n in structs:
        cls = getattr(B, n)
        assert int(got[n]) == ctypes.sizeof(cls), n
        for f, _ in cls._fields_:
            assert int(got[f"{n}.{f}"]) == getattr(cls, f).offset, (n, f)
