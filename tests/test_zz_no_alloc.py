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
