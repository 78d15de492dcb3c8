"""Batched form (needs a GB300): 64 structures of 2-200 conductors with every
master (3024 jobs) in one run of the persistent walk kernel, FP32 geometry and
exact accumulation.  Each job's row must be the one it gives alone, and every
row must be physical (positive self term, zero row sum within its errors)."""
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


def test_all_masters_of_64_structures(torch_cuda):
    fam = W.batched_family(64)
    with B.Context(0, N=16, precision=B.FRW_FP32_GEOM, seed=4) as c:
        sids = [c.load(s) for s in fam]
        jobs = []
        for sid, s in zip(sids, fam):
            for m in range(s.n_cond):
                jobs.append(dict(structure_id=sid, master=m, walk_budget=32768, sigma_target=0.01,
                                 request_id=len(jobs), batch=8192))
        assert len(jobs) == sum(s.n_cond for s in fam) == 3024
        rows, _ = c.extract_batch(jobs)
        bad = 0
        for j, (C, se, st) in zip(jobs, rows):
            m = j["master"]
            assert 8192 <= st["walks"] <= 32768
            assert C[m] > 0.0
            if abs(C.sum()) > 5.0 * np.sqrt(np.sum(se ** 2)) + 1e-12:
                bad += 1
        assert bad <= len(jobs) // 100          # 5-sigma outliers: essentially none
        # alone == in the batch, for a spread of jobs
        for i in (0, 1, 777, 1500, 2222, len(jobs) - 1):
            j = jobs[i]
            Ca, sea, sta, _ = c.extract(j["structure_id"], j["master"], j["walk_budget"], j["sigma_target"],
                                        j["request_id"], j["batch"])
            np.testing.assert_array_equal(rows[i][0], Ca)
            np.testing.assert_array_equal(rows[i][1], sea)
            assert rows[i][2]["walks"] == sta["walks"]
