"""MicroWalk-E on the GPU (needs a GB300): with FP64 geometry the walk kernel's
walks are the oracle's walks, record for record (same Philox streams, same
expanded cubes, same absorptions by conductors inside them), and the rows equal
the oracle's; with FP32 geometry the rows stay within the statistics."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2507_09730_gb300 import binding as B
from paper_2507_09730_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _records_match(g, o):
    np.testing.assert_array_equal(g["k"], o.k)
    np.testing.assert_array_equal(g["hops"], o.hops)
    np.testing.assert_array_equal(g["steps"], o.steps)
    np.testing.assert_array_equal(g["branch"], o.branch)
    np.testing.assert_allclose(g["omega"], o.omega, rtol=1e-12, atol=0)


@pytest.mark.parametrize("N,master,n", [(16, 11, 600), (8, 3, 1500), (24, 19, 200)])
def test_mwe_walk_records_interconnect_fp64(torch_cuda, N, master, n):
    s = W.interconnect(0)
    with B.Context(0, N=N, slots=1 << 15, mwe_factor=5) as c:
        sid = c.load(s)
        g = c.walk_records(sid, master, n, request_id=3, walk_begin=50)
    o = O.frw_run(s, master, n, N=N, seed=0, request=3, walk_begin=50, mwe=5)
    assert o.stats[9] > 0                                    # expanded cubes were used
    _records_match(g, o)


def test_mwe_walk_records_tiny_fp64(torch_cuda):
    s = W.tiny_two_plate()
    with B.Context(0, N=8, slots=1 << 15, mwe_factor=5) as c:
        sid = c.load(s)
        g = c.walk_records(sid, 1, 4000, request_id=4)
    o = O.frw_run(s, 1, 4000, N=8, seed=0, request=4, mwe=5)
    _records_match(g, o)


def test_mwe_extract_matches_oracle_fp64(torch_cuda):
    s = W.interconnect(1)
    with B.Context(0, N=16, slots=1 << 16, mwe_factor=5) as c:
        sid = c.load(s)
        C, se, st, _ = c.extract(sid, 3, 6000, request_id=8)
    o = O.frw_run(s, 3, 6000, N=16, seed=0, request=8, records=False, mwe=5)
    np.testing.assert_allclose(C, o.C, rtol=1e-9, atol=1e-15)
    assert st["walks"] == 6000 and st["hops"] == o.stats[0] and st["micro_steps"] == o.stats[1]


def test_mwe_fp32_within_statistics(torch_cuda):
    s = W.interconnect(0)
    rows = {}
    for prec in (B.FRW_FP32_GEOM, B.FRW_FP64_GEOM):
        with B.Context(0, N=16, precision=prec, mwe_factor=5) as c:
            sid = c.load(s)
            rows[prec] = c.extract(sid, 11, 200_000, request_id=9 + prec)
    (C32, se32, _, _), (C64, se64, _, _) = rows[B.FRW_FP32_GEOM], rows[B.FRW_FP64_GEOM]
    for k in (11, 3, 19):
        assert abs(C32[k] - C64[k]) <= 3.0 * np.hypot(se32[k], se64[k]), (k, C32[k], C64[k])
