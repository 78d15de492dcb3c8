"""Batching tools (need a GB300): a plan replays its captured launch (CUDA graph)
and must give exactly what frw_extract_batch gives for the same request ids; the
autotuner may change only speed, never a result."""
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


def _rows_equal(a, b):
    for (C, se, st), (C2, se2, st2) in zip(a, b):
        np.testing.assert_array_equal(C, C2)
        np.testing.assert_array_equal(se, se2)
        assert st["walks"] == st2["walks"]


def _jobs(sids):
    a, b = sids
    return [dict(structure_id=a, master=0, walk_budget=30000, request_id=1, batch=4096),
            dict(structure_id=b, master=3, walk_budget=200000, sigma_target=0.02, request_id=2, batch=4096),
            dict(structure_id=b, master=11, walk_budget=0, request_id=3),
            dict(structure_id=a, master=1, walk_budget=50000, sigma_target=0.03, request_id=4, batch=2048)]


def test_plan_replays_equal_extract_batch(torch_cuda):
    with B.Context(0, N=16, precision=B.FRW_FP32_GEOM, seed=11, slots=1 << 16) as c:
        sids = (c.load(W.tiny_two_plate()), c.load(W.interconnect(3)))
        jobs = _jobs(sids)
        plan = c.plan(jobs)
        try:
            for off in (0, 1000, 0):
                got, _ = plan.run(off)
                ref, _ = c.extract_batch([dict(j, request_id=j["request_id"] + off) for j in jobs])
                _rows_equal(got, ref)
            assert got[2][2]["walks"] == 0 and not got[2][0].any()
        finally:
            plan.close()


def test_autotune_changes_speed_only(torch_cuda):
    with B.Context(0, N=16, precision=B.FRW_FP32_GEOM, seed=12, slots=1 << 18) as c:
        sids = (c.load(W.tiny_two_plate()), c.load(W.interconnect(3)))
        jobs = _jobs(sids)
        before, _ = c.extract_batch(jobs)
        t = c.autotune(jobs, sample_walks=60000)
        assert t["pool_per_cta"] % 256 == 0 and 256 <= t["pool_per_cta"] <= 4096 and 1 <= t["hops_per_epoch"] <= 16
        assert t["walks_per_s"] > 0 and t["mw_steps_per_s"] > 0
        assert c.tuning() == t
        after, _ = c.extract_batch(jobs)
        _rows_equal(before, after)
        c.set_tuning(pool_per_cta=256, hops_per_epoch=1, mw_warps_per_cta=4, mw_ctas_per_sm=1)
        _rows_equal(before, c.extract_batch(jobs)[0])
        with pytest.raises(B.FRWError):
            c.set_tuning(pool_per_cta=300)


def test_autotune_cache(torch_cuda, tmp_path):
    cache = str(tmp_path / "tune.json")
    with B.Context(0, N=16, precision=B.FRW_FP32_GEOM, seed=12, slots=1 << 18) as c:
        sids = (c.load(W.tiny_two_plate()), c.load(W.interconnect(3)))
        t1 = c.autotune(_jobs(sids), sample_walks=40000, cache=cache)
        c.set_tuning(pool_per_cta=256, hops_per_epoch=1)
        t2 = c.autotune(_jobs(sids), sample_walks=40000, cache=cache)   # from the cache, no tuning
        for k in ("pool_per_cta", "hops_per_epoch", "suspend_lanes", "suspend_min_steps"):
            assert t2[k] == t1[k]
    import json
    data = json.load(open(cache))
    assert len(data) == 1 and list(data)[0].endswith("|N=16|precision=1|mwe=0")
