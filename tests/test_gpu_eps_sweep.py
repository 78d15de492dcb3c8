"""Permittivity sweep (the robustness study of Fig. 5b, on the two-plate structure
instead of the paper's Case 1): the high-k block between the plates takes eps_high
in {3.9, 10, 100} (25 is the structure's own value, tested elsewhere), and the
GPU rows of master 0 are compared with the independent whole-structure finite-
difference solve (tests/fdm_reference.py) at h = 0.05 and 0.025 um.

FRW-MW (N = 16) and FRW-FDM (N = 16) must agree with the h = 0.025 solve within
3 standard errors + |C(h = 0.05) - C(h = 0.025)| (the grid error of the reference),
as the paper finds FRW-MW accurate across the range.  FRW-MWE (expansion 5) is
reported, not asserted: its expanded cubes resolve the 0.4 um block on a 5x
coarser lattice (see the module's printed rows).  Needs a GB300; the reference
solves run in a spawned process pool (about a minute).
"""
import concurrent.futures as cf
import dataclasses
import json
import multiprocessing as mp

import numpy as np
import pytest

from paper_2507_09730_gb300 import binding as B
from paper_2507_09730_gb300 import workloads as W

pytestmark = pytest.mark.gpu

EPS_HIGH = (3.9, 10.0, 100.0)


def _structure(eh):
    return dataclasses.replace(W.tiny_two_plate(), eps=[3.9, float(eh)])


def _reference_row(eh, h):
    from tests import fdm_reference as F
    return F.capacitance_row(_structure(eh), 0, h, rtol=1e-8)


@pytest.fixture(scope="module")
def reference_rows():
    with cf.ProcessPoolExecutor(2 * len(EPS_HIGH), mp_context=mp.get_context("spawn")) as ex:
        futs = {(eh, h): ex.submit(_reference_row, eh, h) for eh in EPS_HIGH for h in (0.05, 0.025)}
        return {k: np.asarray(f.result()) for k, f in futs.items()}


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _row(eh, budget, **opts):
    c = B.Context(0, N=16, seed=0, **opts)
    sid = c.load(_structure(eh))
    C, se, st, _ = c.extract(sid, 0, budget, 0.0, 9)
    c.close()
    return C, se, st


@pytest.mark.parametrize("eh", EPS_HIGH)
def test_rows_follow_the_whole_structure_solve(torch_cuda, reference_rows, eh):
    c1, c2 = reference_rows[(eh, 0.05)], reference_rows[(eh, 0.025)]
    report = {"eps_high": eh, "fd_h0.05": c1.tolist(), "fd_h0.025": c2.tolist()}
    for name, budget, opts, check in (("frw_mw", 2_000_000, {}, True),
                                      ("frw_fdm", 40_000, {"transition": B.FRW_TRANSITION_FDM}, True),
                                      ("frw_mwe", 2_000_000, {"mwe_factor": 5}, False)):
        C, se, st = _row(eh, budget, **opts)
        assert st["walks"] == budget
        report[name] = {"C": C[:2].tolist(), "se": se[:2].tolist(),
                        "dev_in_sigma": ((C[:2] - c2) / se[:2]).tolist()}
        if check:
            for k in range(2):
                tol = 3.0 * se[k] + abs(c1[k] - c2[k])
                assert abs(C[k] - c2[k]) <= tol, (name, eh, k, C[k], c2[k], tol)
    print(json.dumps(report))
