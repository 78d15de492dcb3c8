"""bench.py runs on the GPU machine only; check on the CPU that every global name its
functions use is defined (a renamed or deleted helper would otherwise surface
only there), and that the reference arm's JSON line has the contract's keys."""
import builtins
import json
import os
import subprocess
import sys
import symtable

from tests.conftest import ROOT


def _globals_used(table, out):
    if table.get_type() == "function":
        for sym in table.get_symbols():
            if sym.is_global() and sym.is_referenced():
                out.add((table.get_name(), sym.get_name()))
    for child in table.get_children():
        _globals_used(child, out)


def test_bench_names_resolve():
    path = os.path.join(ROOT, "bench.py")
    src = open(path).read()
    top = symtable.symtable(src, path, "exec")
    defined = {s.get_name() for s in top.get_symbols() if s.is_assigned() or s.is_imported()}
    used = set()
    _globals_used(top, used)
    missing = sorted((f, n) for f, n in used if n not in defined and not hasattr(builtins, n))
    assert not missing, missing


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT,
                         env=dict(os.environ, FRW_BENCH_REF_WALKS="20"))
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "dtype", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0
