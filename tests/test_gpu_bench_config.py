"""Parity in the benchmark's own configuration (needs a GB300): the interconnect
structure at N = 24 with the launch settings the autotuner picks for it (2 CTAs x
448 threads per SM, 2048 slots per CTA, 2 analytical hops per epoch, MicroWalk
lanes parked after 64 steps once the queue is empty).

- FP64 geometry: walks sampled deep into a full-size run (walk ids around 2.5 M,
  the ids a benchmark step reaches) have exactly the oracle's records; the oracle
  computes any walk id on its own (counter-based random numbers).
- FP32 geometry (what the benchmark times), on 1.5 M walks per master: the FP32
  rows lie within 3 combined standard errors of the FP64 rows, and the paired
  difference of the two estimators on the same walk ids (the walks differ only
  where an FP32 geometric decision differs) is within 3 of its own standard
  errors and below 0.1 % of the FP64 value for the self term and the largest
  coupling (the two the stop rule converges; 0.1 % of the self term for the
  smaller couplings).  The FP64 walks are the oracle's:
  a prefix of those very walk ids is compared with the oracle record by record.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2507_09730_gb300 import binding as B
from paper_2507_09730_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TUNING = dict(pool_per_cta=2048, hops_per_epoch=1, suspend_lanes=32, suspend_min_steps=128)


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


def _col(rec, j):
    """Per-walk contributions X_i = omega_i [k_i = j] to row entry j (ground = n_cond)."""
    return np.where(rec["k"] == j, rec["omega"], 0.0)


def _mean_se(x):
    return x.mean(), x.std(ddof=1) / np.sqrt(x.shape[0])


def test_fp32_rows_at_bench_scale(torch_cuda):
    s = W.interconnect(0)
    n, prefix = 1_500_000, 40
    recs = {}
    for prec in (B.FRW_FP32_GEOM, B.FRW_FP64_GEOM):
        with B.Context(0, N=24, precision=prec, seed=0) as c:
            c.set_tuning(**TUNING)
            sid = c.load(s)
            recs[prec] = [c.walk_records(sid, m, n, request_id=70 + i) for i, m in enumerate(s.masters)]
    pooled_d, pooled_c = 0.0, 0.0
    for i, m in enumerate(s.masters):
        r32, r64 = recs[B.FRW_FP32_GEOM][i], recs[B.FRW_FP64_GEOM][i]
        # the FP64 walks are the oracle's (same walk ids, same streams)
        o = O.frw_run(s, m, prefix, N=24, seed=0, request=70 + i)
        for f in ("k", "hops", "steps", "branch"):
            np.testing.assert_array_equal(r64[f][:prefix], getattr(o, f))
        np.testing.assert_allclose(r64["omega"][:prefix], o.omega, rtol=1e-12, atol=0)
        # self term and the three largest couplings (ground excluded); the stop rule
        # converges the self term and the largest coupling, so the 0.1 % bias bound
        # applies to those two; smaller couplings (whose paired error exceeds 0.1 % of
        # their own value at this budget) are held to 0.1 % of the row's self term
        C64_all = np.array([_col(r64, j).mean() for j in range(s.n_cond)])
        coup = sorted((j for j in range(s.n_cond) if j != m), key=lambda j: -abs(C64_all[j]))[:3]
        c_self = C64_all[m]
        for k in (m, *coup):
            x32, x64 = _col(r32, k), _col(r64, k)
            (c32, se32), (c64, se64) = _mean_se(x32), _mean_se(x64)
            d, sd = _mean_se(x32 - x64)
            assert abs(c32 - c64) <= 3.0 * np.hypot(se32, se64), (m, k, c32, c64, se32, se64)
            assert abs(d) <= 3.0 * sd + 1e-15 * abs(c64), (m, k, d, sd)
            scale = abs(c64) if k in (m, coup[0]) else abs(c_self)
            assert abs(d) < 1e-3 * scale, (m, k, d / c64)
            if k in (m, coup[0]):
                # the bias bound is resolvable: the paired standard error is well below 0.1 %
                assert sd < 5e-4 * abs(c64), (m, k, sd / c64)
            if k == m:
                pooled_d += d
                pooled_c += c64
    assert abs(pooled_d) < 1e-3 * abs(pooled_c)
