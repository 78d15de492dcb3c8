"""Uniform-grid candidate lists of the max-cube query (Sec. II-A), built on the
device at structure load (k_grid_lists) against the same lists built on the
host's cores (FRW_INDEX_HOST=1): both must give the walk kernel the same nearest
conductor everywhere, so per-walk records and rows are bit-identical, in FP32
and FP64 geometry, on structures from 2 to 200 conductors, with multi-box
conductors and with a voxel map.  The parity tests hold the same records to the
oracle (they load with the device-built lists).  Needs a GB300.
"""
import os
import time

import numpy as np
import pytest

from paper_2507_09730_gb300 import binding as B
from paper_2507_09730_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _structures():
    fam = W.batched_family(64)
    big = max(fam, key=lambda s: s.n_cond)
    return [("interconnect0", W.interconnect(0)), ("interconnect3", W.interconnect(3)),
            ("l_shape", W.l_shape_pair()), ("voxel", W.voxel_interconnect(1)), ("family_largest", big)]


def _records(s, precision, host_lists):
    if host_lists:
        os.environ["FRW_INDEX_HOST"] = "1"
    else:
        os.environ.pop("FRW_INDEX_HOST", None)
    try:
        c = B.Context(0, N=16, precision=precision, seed=9)
        t0 = time.perf_counter()
        sid = c.load(s)
        t_load = time.perf_counter() - t0
        m = s.masters[0]
        rec = c.walk_records(sid, m, 6000, request_id=4)
        C, se, st, _ = c.extract(sid, m, 60_000, 0.0, 5)
        c.close()
    finally:
        os.environ.pop("FRW_INDEX_HOST", None)
    return rec, C, se, st["walks"], t_load


@pytest.mark.parametrize("precision", [B.FRW_FP32_GEOM, B.FRW_FP64_GEOM])
def test_device_lists_equal_host_lists(torch_cuda, precision):
    for name, s in _structures():
        rd, Cd, sd, wd, td = _records(s, precision, False)
        rh, Ch, sh, wh, th = _records(s, precision, True)
        for k in rd:
            assert np.array_equal(rd[k], rh[k]), (name, k)
        assert np.array_equal(Cd, Ch) and np.array_equal(sd, sh) and wd == wh, name
        print(f"{name}: {s.n_cond} conductors, load {1e3 * td:.2f} ms (device lists) vs {1e3 * th:.2f} ms (host)")
