"""Multi-box conductors on the GPU against the oracle, through the C ABI (needs a
GB300): walk records of FRW-MW and FRW-MWE on structures whose conductors are
unions of boxes equal the oracle's; multi-box masters and malformed box lists
are refused."""
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
    np.testing.assert_array_equal(g["k"], o.k)
    np.testing.assert_array_equal(g["hops"], o.hops)
    np.testing.assert_array_equal(g["steps"], o.steps)
    np.testing.assert_array_equal(g["branch"], o.branch)
    np.testing.assert_allclose(g["omega"], o.omega, rtol=1e-12, atol=0)


def test_l_shape_records(torch_cuda):
    s = W.l_shape_pair()
    with B.Context(0, N=8, slots=1 << 16) as c:
        sid = c.load(s)
        g = c.walk_records(sid, 0, 500, request_id=61)
    o = O.frw_run(s, 0, 500, N=8, seed=0, request=61)
    assert (o.k == 1).any()
    _records_match(g, o)


@pytest.mark.parametrize("mwe", [0, 5])
def test_cut_interconnect_records(torch_cuda, mwe):
    s = W.split_conductor(W.split_conductor(W.interconnect(0), 3, 3, axis=0), 12, 2, axis=1)
    n = 120 if mwe else 150
    with B.Context(0, N=16, slots=1 << 16, mwe_factor=mwe) as c:
        sid = c.load(s)
        g = c.walk_records(sid, 11, n, request_id=62)
    o = O.frw_run(s, 11, n, N=16, seed=0, request=62, mwe=mwe)
    if mwe:
        assert o.stats[9] > 0
    _records_match(g, o)


def test_multibox_master_and_matrix_refused(torch_cuda):
    with B.Context(0, N=8, slots=1 << 14) as c:
        sid = c.load(W.l_shape_pair())
        with pytest.raises(B.FRWError) as e:
            c.extract(sid, 1, 1000, 0.0, 1)
        assert e.value.code == B.FRW_EINVAL
        with pytest.raises(B.FRWError):
            c.matrix(sid, 1000)
        C, se, st, _ = c.extract(sid, 0, 2000, 0.0, 2)      # the single-box master is fine
        assert st["walks"] == 2000 and C[0] > 0 and C[1] < 0


def test_box_lists_are_validated(torch_cuda):
    s = W.l_shape_pair()
    mk = lambda name, cid: W.Structure(name, s.domain_lo, s.domain_hi, s.cond_lo, s.cond_hi, s.eps, s.background,
                                       cond_id=cid)
    bad = [mk("leg touches the other conductor", [0, 1, 0]),   # the leg (box 2) touches box 1 of conductor 1
           mk("conductor without a box", [0, 2, 2]),
           mk("negative conductor id", [0, -1, 1])]
    with B.Context(0, N=8, slots=1 << 14) as c:
        for t in bad:
            with pytest.raises(B.FRWError) as e:
                c.load(t)
            assert e.value.code == B.FRW_EINVAL, t.name
        c.unload(c.load(s))                                     # the L itself is fine
