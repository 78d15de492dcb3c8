"""Failure paths of the serving loop, made on the host (needs a GB300; nothing here
faults, traps or hangs the GPU): a cancelled request, a request that is cancelled
while queued, and a device wait that runs out (the walk kernel's idle limit,
set short) -- the kernel returns an error status, the host reads it, and the
next request is served by a new run with the right result."""
import time

import numpy as np
import pytest

from paper_2507_09730_gb300 import binding as B
from paper_2507_09730_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ERR_IDLE_TIMEOUT = 64


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _alone(c, j):
    return c.extract(j["structure_id"], j["master"], j["walk_budget"], j.get("sigma_target", 0.0),
                     j["request_id"], j.get("batch", 0))


def test_cancel_running_and_queued(torch_cuda):
    with B.Context(0, N=8, seed=2, slots=1 << 16, serve_jobs=2, serve_arena_mb=4096) as c:
        a = c.load(W.tiny_two_plate())
        big = c.submit(dict(structure_id=a, master=0, walk_budget=60_000_000, request_id=1))
        small = dict(structure_id=a, master=1, walk_budget=20_000, request_id=2)
        ts = c.submit(small)
        queued = c.submit(dict(structure_id=a, master=0, walk_budget=1000, request_id=3))   # table full: waits
        c.cancel(queued)
        time.sleep(0.03)
        was_done = c.poll(big)
        c.cancel(big)
        if not was_done:
            with pytest.raises(B.FRWError) as e:
                c.wait(big, 120)
            assert e.value.code == B.FRW_ECANCELED
        with pytest.raises(B.FRWError) as e:
            c.wait(queued, 120)
        assert e.value.code == B.FRW_ECANCELED
        r = c.wait(ts, 120)
        Ca, sea, sta, _ = _alone(c, small)
        np.testing.assert_array_equal(r[0], Ca)
        assert r[2]["walks"] == sta["walks"]
        # a completed request keeps its result
        t4 = c.submit(dict(small, request_id=4))
        while not c.poll(t4):
            time.sleep(0.001)
        c.cancel(t4)
        assert c.wait(t4, 10)[2]["walks"] == 20_000
        info = c.serve_info()
        assert info["cancelled"] >= 1 + (0 if was_done else 1) and info["submitted"] == 4


def test_device_idle_limit_runs_out_and_context_recovers(torch_cuda):
    with B.Context(0, N=8, seed=3, slots=1 << 14, idle_timeout_ms=200) as c:
        a = c.load(W.tiny_two_plate())
        j1 = dict(structure_id=a, master=0, walk_budget=30_000, request_id=5)
        r1 = c.wait(c.submit(j1), 60)
        # the open run now has nothing to do: its kernel gives up after 0.2 s, before
        # the host would close it (0.5 s), and ends the run with an error status
        deadline = time.time() + 20
        while c.serve_info()["runs_failed"] == 0 and time.time() < deadline:
            time.sleep(0.05)
        info = c.serve_info()
        assert info["runs_failed"] == 1 and info["last_status"] & ERR_IDLE_TIMEOUT
        # the context stays usable: the next request starts a new run
        j2 = dict(structure_id=a, master=1, walk_budget=30_000, request_id=6)
        r2 = c.wait(c.submit(j2), 60)
        assert c.serve_info()["runs"] == 2
        for j, r in ((j1, r1), (j2, r2)):
            Ca, _, sta, _ = _alone(c, j)
            np.testing.assert_array_equal(r[0], Ca)
            assert r[2]["walks"] == sta["walks"]
