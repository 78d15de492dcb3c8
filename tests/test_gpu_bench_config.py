"""Parity in the benchmark's own configuration (needs a GB300): the interconnect
structure at N = 24 with the launch settings the autotuner picks for it (2 CTAs x
448 threads per SM, 2048 slots per CTA, 2 analytical hops per epoch, MicroWalk
lanes parked after 64 steps once the queue is empty).

- FP64 geometry: walks sampled deep into a full-size run (walk ids around 2.5 M,
  the ids a benchmark step reaches) have exactly the oracle's records; the oracle
  computes any walk id on its own (counter-based random numbers).
- FP32 geometry (what the benchmark times): its rows at the benchmark's budget
  agree with the FP64 rows within their combined standard errors (the walks
  differ only where an FP32 geometric decision differs).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2507_09730_gb300 import binding as B
from paper_2507_09730_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TUNING = dict(pool_per_cta=2048, hops_per_epoch=2, suspend_lanes=32, suspend_min_steps=64)


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("master,n", [(11, 160), (3, 80), (19, 80)])
def test_sampled_walks_at_bench_scale_fp64(torch_cuda, master, n):
    s = W.interconnect(0)
    begin = 2_500_000 + 7919 * master
    request = 4_000_001 * 4 + master % 3
    with B.Context(0, N=24, seed=0) as c:
        c.set_tuning(**TUNING)
        sid = c.load(s)
        g = c.walk_records(sid, master, n, request_id=request, walk_begin=begin)
    o = O.frw_run(s, master, n, N=24, seed=0, request=request, walk_begin=begin)
    assert o.stats[4] > 0 and o.stats[2] + o.stats[3] > 0     # both transition routes taken
    np.testing.assert_array_equal(g["k"], o.k)
    np.testing.assert_array_equal(g["hops"], o.hops)
    np.testing.assert_array_equal(g["steps"], o.steps)
    np.testing.assert_array_equal(g["branch"], o.branch)
    np.testing.assert_allclose(g["omega"], o.omega, rtol=1e-12, atol=0)


def test_fp32_rows_at_bench_scale(torch_cuda):
    s = W.interconnect(0)
    rows = {}
    for prec in (B.FRW_FP32_GEOM, B.FRW_FP64_GEOM):
        with B.Context(0, N=24, precision=prec, seed=0) as c:
            c.set_tuning(**TUNING)
            sid = c.load(s)
            res, _ = c.extract_batch([dict(structure_id=sid, master=m, walk_budget=1_500_000, request_id=70 + i)
                                      for i, m in enumerate(s.masters)])
            rows[prec] = res
    for m, (C32, se32, st32), (C64, se64, st64) in zip(s.masters, rows[B.FRW_FP32_GEOM], rows[B.FRW_FP64_GEOM]):
        assert st32["walks"] == st64["walks"] == 1_500_000
        for k in (m, 3, 11, 19):
            assert abs(C32[k] - C64[k]) <= 4.0 * np.hypot(se32[k], se64[k]), (m, k, C32[k], C64[k])
