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
    """FP32 geometry on MicroWalk-E cubes, paired with FP64 on the same walk ids:
    the rows agree within 3 combined standard errors and the paired difference
    (walks differ only where an FP32 decision differs) is within 3 of its own
    standard errors and below 0.1 % of the FP64 value (of the self term for the
    couplings below the largest)."""
    s = W.interconnect(0)
    n = 200_000
    recs = {}
    for prec in (B.FRW_FP32_GEOM, B.FRW_FP64_GEOM):
        with B.Context(0, N=16, precision=prec, mwe_factor=5) as c:
            sid = c.load(s)
            recs[prec] = c.walk_records(sid, 11, n, request_id=9)
    r32, r64 = recs[B.FRW_FP32_GEOM], recs[B.FRW_FP64_GEOM]
    col = lambda r, k: np.where(r["k"] == k, r["omega"], 0.0)
    c64 = np.array([col(r64, j).mean() for j in range(s.n_cond)])
    coup = sorted((j for j in range(s.n_cond) if j != 11), key=lambda j: -abs(c64[j]))[:3]
    for k in (11, *coup):
        x32, x64 = col(r32, k), col(r64, k)
        se32, se64 = x32.std(ddof=1) / np.sqrt(n), x64.std(ddof=1) / np.sqrt(n)
        assert abs(x32.mean() - x64.mean()) <= 3.0 * np.hypot(se32, se64), (k, x32.mean(), x64.mean())
        dd = x32 - x64
        d, sd = dd.mean(), dd.std(ddof=1) / np.sqrt(n)
        assert abs(d) <= 3.0 * sd + 1e-15 * abs(x64.mean()), (k, d, sd)
        # 0.1 %: of the entry for the self term and the largest coupling, of the self term otherwise
        scale = abs(x64.mean()) if k in (11, coup[0]) else abs(c64[11])
        assert abs(d) < 1e-3 * scale, (k, d / x64.mean())
