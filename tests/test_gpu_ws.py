"""The warp-specialised walk kernel (tuning geo_warps > 0: geometry warps and
MicroWalk warps of a CTA running at the same time) against the oracle and
against the phased kernel (needs a GB300).  Only the schedule differs, so walk
records equal the oracle's and rows, sigma stops and batched rows equal the
phased kernel's bit for bit."""
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
    for f in ("k", "hops", "steps", "branch"):
        np.testing.assert_array_equal(g[f], getattr(o, f))
    np.testing.assert_allclose(g["omega"], o.omega, rtol=1e-12, atol=0)


@pytest.mark.parametrize("geo", [1, 4, 13])
def test_ws_records_match_oracle(torch_cuda, geo):
    s = W.interconnect(0)
    with B.Context(0, N=16, slots=1 << 16) as c:
        c.set_tuning(geo_warps=geo)
        sid = c.load(s)
        g = c.walk_records(sid, 11, 400, request_id=1)
    o = O.frw_run(s, 11, 400, N=16, seed=0, request=1)
    assert o.stats[4] > 0
    _records_match(g, o)
    t = W.tiny_two_plate()
    with B.Context(0, N=8, slots=1 << 14) as c:
        c.set_tuning(geo_warps=geo)
        g = c.walk_records(c.load(t), 0, 3000, request_id=5, walk_begin=100)
    _records_match(g, O.frw_run(t, 0, 3000, N=8, seed=0, request=5, walk_begin=100))


@pytest.mark.parametrize("mwe", [0, 5])
def test_ws_rows_equal_phased_kernel(torch_cuda, mwe):
    """sigma-stopped rows of the benchmark's kind (N = 24, FP32 geometry, three
    masters in one run) and the records of MicroWalk-E walks."""
    s = W.interconnect(0)
    rows = {}
    for geo in (0, 5):
        with B.Context(0, N=24, precision=B.FRW_FP32_GEOM, seed=0, mwe_factor=mwe) as c:
            c.set_tuning(geo_warps=geo)
            sid = c.load(s)
            res, conv = c.extract_batch([dict(structure_id=sid, master=m, walk_budget=2_000_000, sigma_target=0.01,
                                              request_id=30 + i) for i, m in enumerate(s.masters)])
            rec = c.walk_records(sid, 3, 300, request_id=8)
            rows[geo] = (res, conv, rec)
    (ra, ca, ga), (rb, cb, gb) = rows[0], rows[5]
    assert ca == cb
    for (C0, se0, st0), (C1, se1, st1) in zip(ra, rb):
        np.testing.assert_array_equal(C0, C1)
        np.testing.assert_array_equal(se0, se1)
        assert st0["walks"] == st1["walks"] and st0["micro_steps"] == st1["micro_steps"]
    for f in ("k", "hops", "steps", "branch", "omega"):
        np.testing.assert_array_equal(ga[f], gb[f])


def test_ws_batched_and_matrix(torch_cuda):
    """many jobs of several structures in one run, and the full matrix"""
    fam = W.batched_family(6, seed=3)
    out = {}
    for geo in (0, 3):
        with B.Context(0, N=16, precision=B.FRW_FP32_GEOM, seed=0) as c:
            c.set_tuning(geo_warps=geo)
            sids = [c.load(st) for st in fam]
            jobs = [dict(structure_id=sid, master=m, walk_budget=40000, sigma_target=0.02, request_id=7 + 31 * k + m)
                    for k, (sid, st) in enumerate(zip(sids, fam)) for m in range(st.n_cond)]
            res, conv = c.extract_batch(jobs)
            M = c.matrix(sids[0], 20000, request_id=40)
            out[geo] = (res, M)
    (ra, Ma), (rb, Mb) = out[0], out[3]
    for (C0, se0, st0), (C1, se1, st1) in zip(ra, rb):
        np.testing.assert_array_equal(C0, C1)
        assert st0["walks"] == st1["walks"]
    np.testing.assert_array_equal(Ma[0], Mb[0])
    np.testing.assert_array_equal(Ma[2], Mb[2])


def test_ws_tuning_range(torch_cuda):
    with B.Context(0, N=8, slots=1 << 14) as c:
        with pytest.raises(B.FRWError):
            c.set_tuning(geo_warps=14)
        with pytest.raises(B.FRWError):
            c.set_tuning(geo_warps=-1)
