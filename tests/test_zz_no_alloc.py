"""The allocation-free MicroWalk entry point, for callers that cannot allocate
device memory (their device memory belongs to a host application's allocator, or
they run with a fixed budget and must not pay the device-wide synchronisation of
cudaMalloc / cudaFree).  Its output must equal the context entry point's, call
after call, although both calls share one fixed scratch array.

Kept in a file of its own that pytest collects last.
"""
import numpy as np
import pytest

from paper_2507_09730_gb300 import binding as B
from paper_2507_09730_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_matches_context_entry_point_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    N = 16
    cubes = W.random_cubes(96, N=N, seed=123)
    spc = 512
    n = cubes.n * spc
    rec = torch.from_numpy(B.pack_cubes(cubes)).cuda()
    stream = torch.cuda.current_stream()

    # reference: the context entry point (allocates its own scratch)
    with B.Context(0, N=N, slots=1 << 12) as c:
        B.frw_set_stream(c.ctx, stream.cuda_stream)
        ref = {}
        for request in (7, 8):
            ex = torch.zeros(n, dtype=torch.int32, device="cuda")
            st = torch.zeros(n, dtype=torch.int32, device="cuda")
            B.frw_microwalk_cubes(c.ctx, N, cubes.n, rec.data_ptr(), cubes.eps, spc, request, ex.data_ptr(),
                                  st.data_ptr())
            torch.cuda.synchronize()
            ref[request] = (ex.cpu().numpy(), st.cpu().numpy())

    # two calls in a row of the allocation-free entry point (same scratch array)
    for request in (7, 8):
        ex = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        st = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        rc = B.frw_microwalk_cubes_noalloc(N, cubes.n, rec.data_ptr(), cubes.eps, 0, spc, request, ex.data_ptr(),
                                           st.data_ptr(), stream.cuda_stream)
        assert rc == B.FRW_OK
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ex.cpu().numpy(), ref[request][0])
        np.testing.assert_array_equal(st.cpu().numpy(), ref[request][1])


def test_noalloc_rejects_sizes_beyond_its_limits():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rec = torch.zeros(64, dtype=torch.int32, device="cuda")
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    eps16 = np.linspace(1.0, 16.0, 16)
    assert B.frw_microwalk_cubes_noalloc(8, 1, rec.data_ptr(), eps16, 0, 4, 0, out.data_ptr(), 0) == B.FRW_ECAPACITY
    assert B.frw_microwalk_cubes_noalloc(7, 1, rec.data_ptr(), [1.0], 0, 4, 0, out.data_ptr(), 0) == B.FRW_EINVAL
    assert B.frw_microwalk_cubes_noalloc(34, 1, rec.data_ptr(), [1.0], 0, 4, 0, out.data_ptr(), 0) == B.FRW_EINVAL


def test_noalloc_and_context_reject_malformed_records():
    """A record with a material id >= n_mat, more than 8 blocks or an empty range is
    refused by both entry points (FRW_EINVAL) instead of being walked with zero
    weights; the well-formed cubes of the same call keep their samples."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    N, spc = 8, 64
    cubes = W.random_cubes(4, N=N, seed=9)
    good = B.pack_cubes(cubes)
    n_mat = len(cubes.eps)
    bad_mat = good[0].copy()
    bad_mat[8] = n_mat                      # block 0's material id: one past the table
    bad_bg = good[0].copy()
    bad_bg[0] = 15                          # background id aliasing the boundary slot
    bad_k = good[0].copy()
    bad_k[1] = 9                            # more blocks than a 64-word record holds
    bad_rng = good[0].copy()
    bad_rng[2], bad_rng[3] = 5, 5           # empty range on axis 0
    stream = torch.cuda.current_stream().cuda_stream
    for bad in (bad_mat, bad_bg, bad_k, bad_rng):
        recs = np.concatenate([good[1:2], bad[None, :]])
        d = torch.from_numpy(recs).cuda()
        ex = torch.full((2 * spc,), -1, dtype=torch.int32, device="cuda")
        st = torch.full((2 * spc,), -1, dtype=torch.int32, device="cuda")
        rc = B.frw_microwalk_cubes_noalloc(N, 2, d.data_ptr(), cubes.eps, 0, spc, 3, ex.data_ptr(), st.data_ptr(),
                                           stream)
        assert rc == B.FRW_EINVAL
        torch.cuda.synchronize()
        assert (ex[spc:] == 0).all() and (st[spc:] == 0).all()
        ex_ok = torch.zeros(spc, dtype=torch.int32, device="cuda")
        st_ok = torch.zeros(spc, dtype=torch.int32, device="cuda")
        d1 = torch.from_numpy(np.ascontiguousarray(good[1:2])).cuda()
        assert B.frw_microwalk_cubes_noalloc(N, 1, d1.data_ptr(), cubes.eps, 0, spc, 3, ex_ok.data_ptr(),
                                             st_ok.data_ptr(), stream) == B.FRW_OK
        torch.cuda.synchronize()
        assert torch.equal(ex[:spc], ex_ok) and torch.equal(st[:spc], st_ok)
        with B.Context(0, N=N, slots=1 << 12) as c:
            with pytest.raises(B.FRWError) as ei:
                B.frw_microwalk_cubes(c.ctx, N, 2, d.data_ptr(), cubes.eps, spc, 3, ex.data_ptr(), st.data_ptr())
            assert ei.value.code == B.FRW_EINVAL
    inf_eps = np.array(cubes.eps, np.float64)
    inf_eps[0] = np.inf
    d1 = torch.from_numpy(np.ascontiguousarray(good[1:2])).cuda()
    assert B.frw_microwalk_cubes_noalloc(N, 1, d1.data_ptr(), inf_eps, 0, spc, 3, ex_ok.data_ptr(), 0,
                                         stream) == B.FRW_EINVAL
