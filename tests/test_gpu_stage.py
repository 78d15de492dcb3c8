"""Shared-memory copy of the structure geometry in the walk kernel (the max-cube
query of Sec. II-A and the cube classification read conductor boxes, dielectric
blocks and slab masks from it when every job of a run uses one structure).

The copy changes where the kernel reads the geometry, never a result: rows,
standard errors, walk counts and per-walk records must be bit-identical with the
copy (tuning unstaged = 0, the default) and without it (unstaged = 1), in FP32
and FP64 geometry, for plain MicroWalk and MicroWalk-E, in closed runs and in a
captured plan; the statistics report the copy's size, and a run that mixes
structures makes none.  The records themselves are held to the oracle by the
parity tests, which run with the copy.  Needs a GB300.
"""
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


def _round16(b):
    return (b + 15) // 16 * 16


def _stage_groups(s, tsize):
    """Sizes of the copy's groups: boxes, blocks (coordinates, then material
    bytes), slab masks (256 slabs per axis, one bit per block), each rounded up to
    16 bytes."""
    n_c, n_b = len(s.cond_lo), len(s.block_lo)
    words = max(1, (n_b + 31) // 32)
    blocks = _round16(6 * n_b * tsize) + _round16(n_b) if n_b else 0
    return [_round16(6 * n_c * tsize), blocks, _round16(2 * 3 * 256 * words * 4)]


def _greedy_sums(groups):
    """Copy sizes the greedy choice can give: groups taken in order, each when it
    still fits (for some capacity)."""
    out = set()
    for cap in range(0, sum(groups) + 16, 16):
        used = 0
        for g in groups:
            if g and used + g <= cap:
                used += g
        out.add(used)
    return out


def _run(s, N, precision, unstaged, sigma=0.01, budget=400_000, **opts):
    c = B.Context(0, N=N, precision=precision, seed=3, **opts)
    c.set_tuning(unstaged=unstaged)
    sid = c.load(s)
    jobs = [dict(structure_id=sid, master=m, walk_budget=budget, sigma_target=sigma, request_id=7 + i)
            for i, m in enumerate(s.masters)]
    rows, _ = c.extract_batch(jobs)
    rec = c.walk_records(sid, s.masters[0], 4096, request_id=11)
    c.close()
    return rows, rec


def _same(a, b):
    (ra, reca), (rb, recb) = a, b
    for (Ca, sa, ta), (Cb, sb, tb) in zip(ra, rb):
        assert np.array_equal(Ca, Cb) and np.array_equal(sa, sb)
        assert ta["walks"] == tb["walks"] and ta["micro_steps"] == tb["micro_steps"] and ta["hops"] == tb["hops"]
    for k in reca:
        assert np.array_equal(reca[k], recb[k]), k


@pytest.mark.parametrize("precision,tsize", [(B.FRW_FP32_GEOM, 4), (B.FRW_FP64_GEOM, 8)])
def test_copy_changes_no_result(torch_cuda, precision, tsize):
    s = W.interconnect(0)
    staged = _run(s, 24, precision, 0)
    plain = _run(s, 24, precision, 1)
    _same(staged, plain)
    groups = _stage_groups(s, tsize)
    got = {t["stage_bytes"] for _, _, t in staged[0]}
    assert len(got) == 1 and got.pop() in _greedy_sums(groups) - {0}
    assert all(t["stage_bytes"] == 0 for _, _, t in plain[0])


def test_copy_changes_no_result_mwe(torch_cuda):
    s = W.interconnect(1)
    staged = _run(s, 16, B.FRW_FP32_GEOM, 0, mwe_factor=5)
    plain = _run(s, 16, B.FRW_FP32_GEOM, 1, mwe_factor=5)
    _same(staged, plain)
    assert staged[0][0][2]["stage_bytes"] > 0


def test_mixed_structures_read_global_memory(torch_cuda):
    c = B.Context(0, N=16, precision=B.FRW_FP32_GEOM, seed=3)
    a, b = W.interconnect(0), W.interconnect(2)
    sa, sb = c.load(a), c.load(b)
    mixed, _ = c.extract_batch([dict(structure_id=sa, master=a.masters[0], walk_budget=65536, request_id=1),
                                dict(structure_id=sb, master=b.masters[0], walk_budget=65536, request_id=2)])
    alone, _ = c.extract_batch([dict(structure_id=sa, master=a.masters[0], walk_budget=65536, request_id=1)])
    c.close()
    assert all(t["stage_bytes"] == 0 for _, _, t in mixed)
    assert alone[0][2]["stage_bytes"] > 0
    assert np.array_equal(mixed[0][0], alone[0][0]) and np.array_equal(mixed[0][1], alone[0][1])


def test_plan_with_copy_equals_plan_without(torch_cuda):
    s = W.interconnect(3)
    out = []
    for unstaged in (0, 1):
        c = B.Context(0, N=16, precision=B.FRW_FP32_GEOM, seed=5)
        c.set_tuning(unstaged=unstaged)
        sid = c.load(s)
        p = c.plan([dict(structure_id=sid, master=m, walk_budget=200_000, sigma_target=0.02, request_id=i)
                    for i, m in enumerate(s.masters)])
        out.append(p.run(request_offset=100)[0])
        p.close()
        c.close()
    for (Ca, sa, ta), (Cb, sb, tb) in zip(*out):
        assert np.array_equal(Ca, Cb) and np.array_equal(sa, sb) and ta["walks"] == tb["walks"]
        assert ta["stage_bytes"] > 0 and tb["stage_bytes"] == 0
