"""GPU FD-based transitions (Algorithm 2, FRW-FDM) vs the CPU oracle, through the
C ABI (needs a GB300).

Tolerance of the panel values: the device solve stops when its FP64 residual is
at most 1e-12 of ||e_c||_2 and the oracle's at 1e-15; the error of y, and so of
P_b = eps_v y_v, is then bounded by the condition number of the Jacobi-scaled FD
system (about 4 N^2 / pi^2 times the permittivity contrast, below 10^4 for N <= 24
and contrast 10) times 1e-12, i.e. below 1e-8 of max |P|; that is the bound used.
Sampled panels: both sides draw the same 32-bit word and compare it with
thresholds floor(2^32 cum / total) that the two solves agree on to a few units,
so the samples must agree except where the word lies that close to a threshold.
"""
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


def _lattices(cubes, N):
    return [O.lattice_from_ranges(N, cubes.bg[c], cubes.ranges[c, :cubes.nblk[c]], cubes.mat[c, :cubes.nblk[c]])
            for c in range(cubes.n)]


def _near_threshold(P, u, slack=64):
    cum = np.cumsum(P.reshape(-1))
    thr = np.minimum(np.floor(cum / cum[-1] * 4294967296.0), 4294967295.0)
    return np.abs(thr - float(u)).min() <= slack


@pytest.mark.parametrize("N,n_cubes", [(8, 48), (16, 12), (24, 4)])
def test_fdm_cubes_match_oracle(torch_cuda, N, n_cubes):
    torch = torch_cuda
    cubes = W.random_cubes(n_cubes, N=N, seed=70 + N)
    c = B.Context(0, N=N, slots=1 << 12)
    rec = torch.from_numpy(B.pack_cubes(cubes)).cuda()
    u_h = np.random.default_rng([7, N]).integers(0, 1 << 32, n_cubes, dtype=np.uint64).astype(np.uint32)
    u = torch.from_numpy(u_h.view(np.int32)).cuda()
    P = torch.zeros(n_cubes * 6 * N * N, dtype=torch.float64, device="cuda")
    ex = torch.zeros(n_cubes, dtype=torch.int32, device="cuda")
    it = torch.zeros(n_cubes, dtype=torch.int32, device="cuda")
    B.frw_fdm_cubes(c.ctx, N, n_cubes, rec.data_ptr(), cubes.eps, u.data_ptr(), P.data_ptr(), ex.data_ptr(),
                    it.data_ptr())
    torch.cuda.synchronize()
    Pg = P.cpu().numpy().reshape(n_cubes, 6, N, N)
    nodes = B.decode_exit(ex.cpu().numpy().view(np.uint32))
    iters = it.cpu().numpy().view(np.uint32)
    assert ((iters >> 24) >= 1).all() and ((iters >> 24) <= 12).all()
    for ci, lat in enumerate(_lattices(cubes, N)):
        Po = O.sgf(N, cubes.eps[lat])
        assert np.abs(Pg[ci] - Po).max() <= 1e-8 * np.abs(Po).max(), (ci, np.abs(Pg[ci] - Po).max())
        assert abs(Pg[ci].sum() - 1.0) < 1e-8
        no = O.fdm_transitions(N, lat, cubes.eps, u_h[ci:ci + 1])[0]
        if not (nodes[ci] == no).all():
            assert _near_threshold(Po, u_h[ci]), (ci, nodes[ci], no)
    c.close()


def test_fdm_cubes_homogeneous_faces_and_symmetry(torch_cuda):
    """A homogeneous cube: each face carries 1/6 and P is symmetric under the
    cube's reflections (a check of the device solve that needs no oracle)."""
    torch = torch_cuda
    N = 16
    rec = np.zeros((1, 64), np.int32)           # background only, material 0
    c = B.Context(0, N=N, slots=1 << 12)
    d = torch.from_numpy(rec).cuda()
    P = torch.zeros(6 * N * N, dtype=torch.float64, device="cuda")
    B.frw_fdm_cubes(c.ctx, N, 1, d.data_ptr(), np.array([3.9]), 0, P.data_ptr())
    Pg = P.cpu().numpy().reshape(6, N, N)
    np.testing.assert_allclose(Pg.sum(axis=(1, 2)), 1.0 / 6.0, rtol=0, atol=1e-10)
    np.testing.assert_allclose(Pg[0], Pg[0][::-1, :], rtol=0, atol=1e-12)
    np.testing.assert_allclose(Pg[0], Pg[0].T, rtol=0, atol=1e-12)
    np.testing.assert_allclose(Pg[0], Pg[5], rtol=0, atol=1e-12)
    c.close()


@pytest.mark.parametrize("N,n", [(8, 600), (16, 80)])
def test_frw_fdm_walk_records_match_oracle(torch_cuda, N, n):
    s = W.interconnect(0)
    c = B.Context(0, N=N, transition=B.FRW_TRANSITION_FDM)
    sid = c.load(s)
    g = c.walk_records(sid, 11, n, request_id=31)
    o = O.frw_run(s, 11, n, N=N, seed=0, request=31, fdm=True)
    assert o.stats[4] > 0                      # FD transitions were taken
    same = (g["k"] == o.k) & (g["hops"] == o.hops) & (g["branch"] == o.branch)
    # a walk may part from the oracle's only at a sampled word lying within a few
    # threshold units of a panel boundary: about 1e-6 per FD transition
    assert same.sum() >= n - 1, (n - same.sum())
    np.testing.assert_array_equal(g["steps"], np.zeros(n))
    np.testing.assert_allclose(g["omega"][same], o.omega[same], rtol=1e-12, atol=0)
    c.close()


def test_frw_fdm_extract_agrees_with_frw_mw(torch_cuda):
    """Theorem 1 on the device: FRW-FDM and FRW-MW estimate the same row."""
    s = W.interconnect(0)
    rows = []
    for tr in (B.FRW_TRANSITION_FDM, B.FRW_TRANSITION_MICROWALK):
        c = B.Context(0, N=16, precision=B.FRW_FP32_GEOM, transition=tr)
        sid = c.load(s)
        C, se, st, _ = c.extract(sid, 11, 20000, 0.0, 40 + tr)
        rows.append((C, se, st))
        c.close()
    (Cf, sef, stf), (Cm, sem, stm) = rows
    assert stf["mw_hops"] > 0 and stf["micro_steps"] == 0 and stm["micro_steps"] > 0
    for k in (11, 3, 19):
        assert abs(Cf[k] - Cm[k]) <= 3.0 * np.hypot(sef[k], sem[k]), (k, Cf[k], Cm[k])


def test_fdm_option_validation(torch_cuda):
    with pytest.raises(B.FRWError):
        B.Context(0, N=26, transition=B.FRW_TRANSITION_FDM)
    with pytest.raises(B.FRWError):
        B.Context(0, N=16, transition=B.FRW_TRANSITION_FDM, mwe_factor=5)
    with pytest.raises(B.FRWError):
        B.Context(0, N=16, transition=2)


def test_fdm_cubes_edge_cases(torch_cuda):
    """N = 2 (every node a centre node) against the oracle; no cubes is a no-op;
    a context with N above the FD solve's limit refuses FD transitions."""
    torch = torch_cuda
    N = 2
    rec = np.zeros((3, 64), np.int32)
    rec[1, 1] = 1
    rec[1, 2:9] = [0, 1, 0, 2, 0, 2, 1]        # one block on the low-x half, material 1
    rec[2, 0] = 1                              # background material 1
    eps = np.array([3.9, 25.0])
    c = B.Context(0, N=N, slots=1 << 12)
    d = torch.from_numpy(rec).cuda()
    P = torch.zeros(3 * 6 * N * N, dtype=torch.float64, device="cuda")
    B.frw_fdm_cubes(c.ctx, N, 3, d.data_ptr(), eps, 0, P.data_ptr())
    Pg = P.cpu().numpy().reshape(3, 6, N, N)
    lats = [np.zeros((N, N, N), np.uint8), np.zeros((N, N, N), np.uint8), np.ones((N, N, N), np.uint8)]
    lats[1][0:1, 0:2, 0:2] = 1
    for i, lat in enumerate(lats):
        Po = O.sgf(N, eps[lat])
        assert np.abs(Pg[i] - Po).max() <= 1e-10, i
    B.frw_fdm_cubes(c.ctx, N, 0, d.data_ptr(), eps)           # nothing to do
    c.close()
    big = B.Context(0, N=26, slots=1 << 12)
    with pytest.raises(B.FRWError) as e:
        B.frw_fdm_cubes(big.ctx, 26, 1, d.data_ptr(), eps)
    assert e.value.code == B.FRW_EINVAL
    big.close()
