"""Serving form (needs a GB300): requests submitted while others run are admitted
into the running walk kernel as its job table and arenas allow, and each result
is exactly the one the same job gives alone (exact integer accumulation and a
stop rule read on walk-id prefixes make the mix invisible)."""
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


def _same(served, alone):
    C, se, st, conv = served
    Ca, sea, sta, conva = alone
    np.testing.assert_array_equal(C, Ca)
    np.testing.assert_array_equal(se, sea)
    assert st["walks"] == sta["walks"]
    assert st["hops"] == sta["hops"] and st["micro_steps"] == sta["micro_steps"]
    assert conv == conva


def _alone(c, j):
    return c.extract(j["structure_id"], j["master"], j["walk_budget"], j.get("sigma_target", 0.0),
                     j["request_id"], j.get("batch", 0))


def test_served_results_equal_alone(torch_cuda):
    with B.Context(0, N=16, precision=B.FRW_FP32_GEOM, seed=5, slots=1 << 17, serve_jobs=64,
                   serve_arena_mb=512) as c:
        a = c.load(W.tiny_two_plate())
        b = c.load(W.interconnect(0))
        d = c.load(W.interconnect(2))
        jobs = []
        rid = 100
        for sid, masters in ((a, (0, 1)), (b, (3, 11, 19)), (d, (2, 10))):
            for m in masters:
                for sigma, budget in ((0.02, 2_000_000), (0.0, 40_000)):
                    jobs.append(dict(structure_id=sid, master=m, walk_budget=budget, sigma_target=sigma,
                                     request_id=rid, batch=4096))
                    rid += 1
        # three waves: later requests arrive while earlier ones are on the device
        tickets = []
        for w in range(3):
            for j in jobs[w::3]:
                tickets.append((j, c.submit(j)))
            time.sleep(0.003)
        served = [(j, c.wait(t, timeout_s=300)) for j, t in tickets]
        for j, r in served:
            assert r is not None
            assert r[2]["seconds"] > 0.0
            _same(r, _alone(c, j))


def test_admission_by_memory(torch_cuda):
    # an arena of 4 MB holds 131072 walks of budget: requests of 100000 walks run
    # one at a time, a request of 10^6 walks can never be admitted
    with B.Context(0, N=8, seed=9, slots=1 << 14, serve_jobs=8, serve_arena_mb=4) as c:
        a = c.load(W.tiny_two_plate())
        jobs = [dict(structure_id=a, master=i % 2, walk_budget=100_000, request_id=200 + i, batch=4096)
                for i in range(4)]
        tickets = [c.submit(j) for j in jobs]
        big = c.submit(dict(structure_id=a, master=0, walk_budget=1_000_000, request_id=300))
        results = [c.wait(t, timeout_s=300) for t in tickets]
        with pytest.raises(B.FRWError) as e:
            c.wait(big, timeout_s=300)
        assert e.value.code == B.FRW_ENOMEM
        for j, r in zip(jobs, results):
            _same(r, _alone(c, j))


def test_poll_and_wait_timeout(torch_cuda):
    with B.Context(0, N=8, seed=1, slots=1 << 14) as c:
        a = c.load(W.tiny_two_plate())
        t = c.submit(dict(structure_id=a, master=0, walk_budget=4_000_000, request_id=7))
        assert c.wait(t, timeout_s=0.0) is None          # still running: the ticket stays valid
        r = c.wait(t, timeout_s=300)
        assert r is not None and r[2]["walks"] == 4_000_000
        with pytest.raises(B.FRWError) as e:
            c.poll(t)                                    # collected: unknown now
        assert e.value.code == B.FRW_ENOTFOUND
        t2 = c.submit(dict(structure_id=a, master=1, walk_budget=1000, request_id=8))
        for _ in range(20000):
            if c.poll(t2):
                break
            time.sleep(0.001)
        assert c.poll(t2)
        assert c.wait(t2)[2]["walks"] == 1000
