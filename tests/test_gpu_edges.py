"""Edge cases of the GPU path against the oracle: the largest lattice edge the
kernels take (N = 32: the mask rows, the table fill and the walk kernel's shared
memory at their limit), the smallest inputs (one sample, one walk, no cubes) and
walk counts that end in a ragged, partial batch.  Needs a GB300.
"""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_2507_09730_gb300 import binding as B
from paper_2507_09730_gb300 import workloads as W

pytestmark = pytest.mark.gpu

_ctx = {}


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def ctx_for(N):
    if N not in _ctx:
        _ctx[N] = B.Context(0, N=N, slots=1 << 16)
    return _ctx[N]


def _cubes(torch, c, cubes, spc, request):
    rec = torch.from_numpy(B.pack_cubes(cubes)).cuda()
    n = max(1, cubes.n * spc)
    ex = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    st = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    B.frw_microwalk_cubes(c.ctx, cubes.N, cubes.n, rec.data_ptr(), cubes.eps, spc, request, ex.data_ptr(),
                          st.data_ptr())
    torch.cuda.synchronize()
    return ex.cpu().numpy().view(np.uint32), st.cpu().numpy().view(np.uint32)


def test_microwalk_paths_at_the_largest_edge(torch_cuda):
    N, spc = 32, 40
    cubes = W.random_cubes(12, N=N, seed=4)
    ex, st = _cubes(torch_cuda, ctx_for(N), cubes, spc, 3)
    nodes = B.decode_exit(ex)
    for ci in range(cubes.n):
        lat = O.lattice_from_ranges(N, cubes.bg[ci], cubes.ranges[ci, :cubes.nblk[ci]], cubes.mat[ci, :cubes.nblk[ci]])
        nodes_o, steps_o = O.microwalk_many(N, lat, cubes.eps, 0, 3, ci * spc, spc)
        np.testing.assert_array_equal(nodes[ci * spc:(ci + 1) * spc], nodes_o)
        np.testing.assert_array_equal(st[ci * spc:(ci + 1) * spc].astype(np.uint64), steps_o)


def test_microwalk_one_sample_and_no_cubes(torch_cuda):
    N = 16
    c = ctx_for(N)
    cubes = W.random_cubes(1, N=N, seed=9)
    ex, st = _cubes(torch_cuda, c, cubes, 1, 8)
    lat = O.lattice_from_ranges(N, cubes.bg[0], cubes.ranges[0, :cubes.nblk[0]], cubes.mat[0, :cubes.nblk[0]])
    nodes_o, steps_o = O.microwalk_many(N, lat, cubes.eps, 0, 8, 0, 1)
    np.testing.assert_array_equal(B.decode_exit(ex), nodes_o)
    assert int(st[0]) == int(steps_o[0])
    # no cubes: a valid call that writes nothing
    empty = dataclasses.replace(cubes, bg=cubes.bg[:0], nblk=cubes.nblk[:0], ranges=cubes.ranges[:0],
                                mat=cubes.mat[:0])
    assert empty.n == 0
    ex0, st0 = _cubes(torch_cuda, c, empty, 5, 8)
    assert (ex0.view(np.int32) == -7).all() and (st0.view(np.int32) == -7).all()


def test_walk_records_at_the_largest_edge_fp64(torch_cuda):
    s = W.interconnect(0)
    c = ctx_for(32)
    sid = c.load(s)
    n = 40
    g = c.walk_records(sid, 11, n, request_id=2)
    o = O.frw_run(s, 11, n, N=32, seed=0, request=2)
    np.testing.assert_array_equal(g["k"], o.k)
    np.testing.assert_array_equal(g["hops"], o.hops)
    np.testing.assert_array_equal(g["steps"], o.steps)
    np.testing.assert_array_equal(g["branch"], o.branch)
    np.testing.assert_allclose(g["omega"], o.omega, rtol=1e-12, atol=0)
    assert o.stats[2] + o.stats[3] > 0 and o.stats[4] > 0   # both routes exercised
    c.unload(sid)


@pytest.mark.parametrize("n", [1, 16384 + 37])
def test_extract_single_walk_and_ragged_batch_fp64(torch_cuda, n):
    """One walk, and a budget that ends 37 walks into its second batch of 16384:
    the rows and their standard errors equal the oracle's over the same walks."""
    s = W.tiny_two_plate()
    c = ctx_for(8)
    sid = c.load(s)
    C, se, st, _ = c.extract(sid, 0, n, request_id=3)
    o = O.frw_run(s, 0, n, N=8, seed=0, request=3, records=False)
    assert st["walks"] == n and st["hops"] == o.stats[0] and st["micro_steps"] == o.stats[1]
    np.testing.assert_allclose(C, o.C, rtol=1e-9, atol=0)
    if n > 1:
        np.testing.assert_allclose(se, o.stderr, rtol=1e-6)
    c.unload(sid)
