"""Permittivity voxel maps through frw_load_structure_ex on the GPU (needs a
GB300): walk records equal the oracle's on the interconnect structure with a
random voxel map under its blocks (FRW-MW at N = 8, 16, 24), the map that
reproduces the two-plate block gives that structure's records, and malformed
descriptors are refused."""
import ctypes

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


def _match(g, o):
    for f in ("k", "hops", "steps", "branch"):
        np.testing.assert_array_equal(g[f], getattr(o, f))
    np.testing.assert_allclose(g["omega"], o.omega, rtol=1e-12, atol=0)


@pytest.mark.parametrize("N,n,master", [(8, 600, 11), (16, 300, 3), (24, 120, 19)])
def test_voxel_interconnect_records_match_oracle(torch_cuda, N, n, master):
    s = W.voxel_interconnect(0)
    with B.Context(0, N=N, slots=1 << 16) as c:
        sid = c.load(s)
        g = c.walk_records(sid, master, n, request_id=41)
    o = O.frw_run(s, master, n, N=N, seed=0, request=41)
    assert o.stats[4] > 0                                  # MicroWalk cubes were walked
    _match(g, o)


def test_voxel_two_plate_equals_block_structure(torch_cuda):
    with B.Context(0, N=8, slots=1 << 14) as c:
        a = c.walk_records(c.load(W.tiny_two_plate()), 0, 3000, request_id=5)
        b = c.walk_records(c.load(W.voxel_two_plate()), 0, 3000, request_id=5)
    for f in ("k", "hops", "steps", "branch", "omega"):
        np.testing.assert_array_equal(a[f], b[f])


def _desc(s, **over):
    d = B.frw_structure()
    d.domain = B.frw_box((ctypes.c_double * 3)(*s.domain_lo), (ctypes.c_double * 3)(*s.domain_hi))
    cond = (B.frw_box * s.n_boxes)()
    for k in range(s.n_boxes):
        cond[k].lo = (ctypes.c_double * 3)(*s.cond_lo[k])
        cond[k].hi = (ctypes.c_double * 3)(*s.cond_hi[k])
    eps = np.ascontiguousarray(s.eps)
    vm = np.ascontiguousarray(over.pop("vm", s.voxel_mat), np.uint8)
    d.grounded_walls = over.pop("grounded_walls", 1)
    d.n_boxes = d.n_cond = s.n_boxes
    d.n_mat, d.background_mat, d.n_blocks = len(eps), s.background, 0
    d.vox_dims = (ctypes.c_int32 * 3)(*over.pop("dims", vm.shape))
    d.boxes = ctypes.cast(cond, ctypes.c_void_p)
    d.eps_r = eps.ctypes.data
    d.voxel_mat = vm.ctypes.data
    return d, (cond, eps, vm)


def test_voxel_descriptor_errors(torch_cuda):
    s = W.voxel_two_plate()
    with B.Context(0, N=8, slots=1 << 14) as c:
        sid = ctypes.c_int32(-1)
        L = B.lib()
        d, keep = _desc(s)
        assert L.frw_load_structure_ex(c.ctx, ctypes.byref(d), ctypes.byref(sid)) == B.FRW_OK
        d, keep = _desc(s, grounded_walls=0)
        assert L.frw_load_structure_ex(c.ctx, ctypes.byref(d), ctypes.byref(sid)) == B.FRW_EINVAL
        d, keep = _desc(s, dims=(20, 20, 0))
        assert L.frw_load_structure_ex(c.ctx, ctypes.byref(d), ctypes.byref(sid)) == B.FRW_EINVAL
        bad = s.voxel_mat.copy()
        bad[0, 0, 0] = 2                                   # only materials 0 and 1 exist
        d, keep = _desc(s, vm=bad)
        assert L.frw_load_structure_ex(c.ctx, ctypes.byref(d), ctypes.byref(sid)) == B.FRW_EINVAL
        big = np.full((257, 256, 256), O.VOXEL_NONE, np.uint8)
        d, keep = _desc(s, vm=big)
        assert L.frw_load_structure_ex(c.ctx, ctypes.byref(d), ctypes.byref(sid)) == B.FRW_ECAPACITY
        # an empty map is no map: the same walks as the structure without one
        none = np.full((3, 4, 5), O.VOXEL_NONE, np.uint8)
        e = W.Structure("empty_map", s.domain_lo, s.domain_hi, s.cond_lo, s.cond_hi, s.eps, s.background,
                        masters=s.masters, voxel_mat=none)
        s_plain = W.Structure("plain", s.domain_lo, s.domain_hi, s.cond_lo, s.cond_hi, s.eps, s.background,
                              masters=s.masters)
        a = c.walk_records(c.load(e), 0, 1000, request_id=9)
        b = c.walk_records(c.load(s_plain), 0, 1000, request_id=9)
        for f in ("k", "hops", "steps", "omega"):
            np.testing.assert_array_equal(a[f], b[f])
