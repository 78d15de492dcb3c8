"""GPU path vs the CPU oracle, through the C ABI (needs a GB300)."""
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


_ctx_cache = {}


def ctx_for(N, **kw):
    key = (N, tuple(sorted(kw.items())))
    if key not in _ctx_cache:
        _ctx_cache[key] = B.Context(0, N=N, slots=1 << 16, **kw)
    return _ctx_cache[key]


# ---------------------------------------------------------------------------
# Analytical tables: device separable solve vs oracle CG on the explicit lattice
@pytest.mark.parametrize("N", [8, 16, 24])
def test_tables_match_oracle(torch_cuda, N):
    c = ctx_for(N)
    eps = np.array([2.7, 7.0, 5.0, 25.0])
    rng = np.random.default_rng(N)
    prof = rng.integers(0, 4, N)
    cases = [(B.FRW_TAB_SGF, 2, 0), (B.FRW_TAB_SGF, 0, 0), (B.FRW_TAB_SGF, 1, 0),
             (B.FRW_TAB_FLUX_PAR, 2, 2), (B.FRW_TAB_FLUX_PAR, 0, 0),
             (B.FRW_TAB_FLUX_PERP, 2, 0), (B.FRW_TAB_FLUX_PERP, 0, 1), (B.FRW_TAB_FLUX_PERP, 1, 2),
             (B.FRW_TAB_SGF_HOM, 2, 0), (B.FRW_TAB_FLUX_HOM, 0, 2)]
    for kind, axis, naxis in cases:
        thr_g, neg_g, tot_g, vals = c.table(kind, prof, eps)
        thr_o, neg_o, tot_o = O.table(N, kind, axis, naxis, prof.astype(np.uint8), eps)
        assert abs(tot_g - tot_o) <= 1e-11 * abs(tot_o), (kind, axis, naxis, tot_g, tot_o)
        d = np.abs(thr_g.astype(np.int64) - thr_o.astype(np.int64))
        assert d.max() <= 2 and (d > 0).mean() < 0.02, (kind, axis, naxis, d.max(), (d > 0).mean())
        big = np.abs(vals) > 1e-12 * tot_o
        assert (neg_g[big] == neg_o[big]).all()
        if kind in (B.FRW_TAB_SGF, B.FRW_TAB_SGF_HOM):
            assert abs(vals.sum() - 1.0) < 1e-12


# ---------------------------------------------------------------------------
# MicroWalk kernel alone: bit-exact lattice paths vs the oracle
def _run_cubes(torch, c, cubes, spc, request=3):
    rec = torch.from_numpy(B.pack_cubes(cubes)).cuda()
    n = cubes.n * spc
    ex = torch.zeros(n, dtype=torch.int32, device="cuda")
    st = torch.zeros(n, dtype=torch.int32, device="cuda")
    B.frw_microwalk_cubes(c.ctx, cubes.N, cubes.n, rec.data_ptr(), cubes.eps, spc, request, ex.data_ptr(),
                          st.data_ptr())
    torch.cuda.synchronize()
    return ex.cpu().numpy().view(np.uint32), st.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("N", [8, 16])
def test_microwalk_paths_bit_exact(torch_cuda, N):
    c = ctx_for(N)
    cubes = W.random_cubes(48, N=N, seed=N)
    spc = 128
    ex, st = _run_cubes(torch_cuda, c, cubes, spc)
    nodes_g = B.decode_exit(ex)
    for ci in range(cubes.n):
        lat = O.lattice_from_ranges(N, cubes.bg[ci], cubes.ranges[ci, :cubes.nblk[ci]], cubes.mat[ci, :cubes.nblk[ci]])
        nodes_o, steps_o = O.microwalk_many(N, lat, cubes.eps, 0, 3, ci * spc, spc)
        np.testing.assert_array_equal(nodes_g[ci * spc:(ci + 1) * spc], nodes_o)
        np.testing.assert_array_equal(st[ci * spc:(ci + 1) * spc].astype(np.uint64), steps_o)


def test_microwalk_chunks_across_cubes_bit_exact(torch_cuda):
    """Warps of the MicroWalk kernel claim chunks of consecutive sample ids (up to
    512): at 997 cubes x 10007 samples (both prime) the chunks straddle cube
    boundaries, lanes change cubes mid-chunk and the last chunk runs past the end.
    Every sample must still be the oracle's walk for its id: checked on the ids
    around every 97th cube boundary, around chunk boundaries, the last ids and
    random ones; every sample must also have been written (steps > 0)."""
    N, n_cubes, spc = 8, 997, 10007
    c = ctx_for(N)
    cubes = W.random_cubes(n_cubes, N=N, seed=5)
    ex, st = _run_cubes(torch_cuda, c, cubes, spc, request=6)
    assert (st > 0).all()
    nodes_g = B.decode_exit(ex)
    total = n_cubes * spc
    rng = np.random.default_rng(1)
    ids = set(rng.integers(0, total, 300).tolist())
    for ci in range(0, n_cubes, 97):
        ids.update(j for j in (ci * spc - 1, ci * spc, ci * spc + 1) if 0 <= j < total)
    for k in range(1, total // 512, 977):
        ids.update((k * 512 - 1, k * 512))
    ids.update(range(total - 40, total))
    lats = {}
    for j in sorted(ids):
        ci = j // spc
        if ci not in lats:
            lats[ci] = O.lattice_from_ranges(N, cubes.bg[ci], cubes.ranges[ci, :cubes.nblk[ci]],
                                             cubes.mat[ci, :cubes.nblk[ci]])
        nodes_o, steps_o = O.microwalk_many(N, lats[ci], cubes.eps, 0, 6, j, 1)
        np.testing.assert_array_equal(nodes_g[j:j + 1], nodes_o)
        assert int(st[j]) == int(steps_o[0]), j


def test_microwalk_theorem1_on_gpu(torch_cuda):
    """Theorem 1: the GPU exit histogram follows e_c^T A_II^{-1} A_IB (exact chain solve)."""
    from scipy import stats
    N = 8
    c = ctx_for(N)
    cubes = W.random_cubes(4, N=N, seed=77)
    spc = 1 << 20
    ex, st = _run_cubes(torch_cuda, c, cubes, spc, request=9)
    nodes = B.decode_exit(ex)
    for ci in range(cubes.n):
        lat = O.lattice_from_ranges(N, cubes.bg[ci], cubes.ranges[ci, :cubes.nblk[ci]], cubes.mat[ci, :cubes.nblk[ci]])
        Pq, Et = O.absorption_exact(N, lat, cubes.eps, quantised=True)
        pan = O.node_to_panel(N, nodes[ci * spc:(ci + 1) * spc])
        hist = np.bincount(pan, minlength=6 * N * N)
        exp = Pq.reshape(-1) * spc
        big = exp >= 5
        obs_b = np.concatenate([hist[big], [hist[~big].sum()]])
        exp_b = np.concatenate([exp[big], [exp[~big].sum()]])
        keep = exp_b > 0
        chi = ((obs_b[keep] - exp_b[keep]) ** 2 / exp_b[keep]).sum()
        assert stats.chi2.sf(chi, keep.sum() - 1) > 1e-3
        s = st[ci * spc:(ci + 1) * spc].astype(np.float64)
        assert abs(s.mean() - Et) < 4 * s.std() / np.sqrt(spc)


# ---------------------------------------------------------------------------
# Whole walks (Algorithm 1), FP64 geometry: identical walks, identical records
def _records_match(g, o, rtol=1e-12):
    np.testing.assert_array_equal(g["k"], o.k)
    np.testing.assert_array_equal(g["hops"], o.hops)
    np.testing.assert_array_equal(g["steps"], o.steps)
    np.testing.assert_array_equal(g["branch"], o.branch)
    np.testing.assert_allclose(g["omega"], o.omega, rtol=rtol, atol=0)


@pytest.mark.parametrize("master", [0, 1])
def test_walk_records_tiny_fp64(torch_cuda, master):
    s = W.tiny_two_plate()
    c = ctx_for(8)
    sid = c.load(s)
    n = 3000
    g = c.walk_records(sid, master, n, request_id=5, walk_begin=100)
    o = O.frw_run(s, master, n, N=8, seed=0, request=5, walk_begin=100)
    _records_match(g, o)
    c.unload(sid)


def test_walk_records_interconnect_fp64(torch_cuda):
    s = W.interconnect(0)
    c = ctx_for(16)
    sid = c.load(s)
    n = 400
    g = c.walk_records(sid, 11, n, request_id=1)
    o = O.frw_run(s, 11, n, N=16, seed=0, request=1)
    _records_match(g, o)
    assert o.stats[4] > 0 and o.stats[2] + o.stats[3] > 0   # both routes exercised
    c.unload(sid)


@pytest.mark.parametrize("N,n", [(8, 3000), (16, 600), (24, 200)])
def test_walk_records_overflow_cubes_fp64(torch_cuda, N, n):
    """Cubes that list more than 14 blocks are halved on both sides (reading R3):
    the two-plate structure with its high-k cube cut into 32 blocks."""
    s = W.split_blocks(W.tiny_two_plate(), (4, 4, 2))
    c = ctx_for(N)
    sid = c.load(s)
    g = c.walk_records(sid, 0, n, request_id=23)
    o = O.frw_run(s, 0, n, N=N, seed=0, request=23)
    assert o.stats[10] > 0                     # the overflow rule was taken
    _records_match(g, o)
    c.unload(sid)


def test_extract_matches_oracle_fp64(torch_cuda):
    s = W.tiny_two_plate()
    c = ctx_for(8)
    sid = c.load(s)
    n = 100_000
    C, se, st, conv = c.extract(sid, 0, n, request_id=0)
    o = O.frw_run(s, 0, n, N=8, seed=0, request=0, records=False)
    np.testing.assert_allclose(C, o.C, rtol=1e-9, atol=0)
    np.testing.assert_allclose(se, o.stderr, rtol=1e-6)
    assert st["walks"] == n and st["hops"] == o.stats[0] and st["micro_steps"] == o.stats[1]
    c.unload(sid)


def test_sigma_stop_matches_oracle(torch_cuda):
    s = W.tiny_two_plate()
    c = ctx_for(8)
    sid = c.load(s)
    C, se, st, conv = c.extract(sid, 0, 400_000, sigma_target=0.03, request_id=2, batch=2000)
    o = O.frw_run(s, 0, 400_000, N=8, seed=0, request=2, sigma_target=0.03, batch=2000, records=False)
    assert conv and st["walks"] == o.n
    np.testing.assert_allclose(C, o.C, rtol=1e-9)
    c.unload(sid)


def test_batch_equals_alone(torch_cuda):
    """Continuous batching: each job's result is the same alone and in the mix."""
    s1 = W.tiny_two_plate()
    s2 = W.interconnect(1)
    c = ctx_for(8)
    a = c.load(s1)
    b = c.load(s2)
    jobs = [dict(structure_id=a, master=0, walk_budget=20000, request_id=1),
            dict(structure_id=b, master=3, walk_budget=3000, request_id=2),
            dict(structure_id=a, master=1, walk_budget=15000, request_id=3, sigma_target=0.05, batch=1000)]
    mix, _ = c.extract_batch(jobs)
    for j, (C, se, st) in zip(jobs, mix):
        Ca, sea, sta, _ = c.extract(j["structure_id"], j["master"], j["walk_budget"], j.get("sigma_target", 0.0),
                                    j["request_id"], j.get("batch", 0))
        np.testing.assert_array_equal(C, Ca)
        np.testing.assert_array_equal(se, sea)
        assert st["walks"] == sta["walks"]
    c.unload(a)
    c.unload(b)


def test_fp32_geometry_within_statistics(torch_cuda):
    s = W.tiny_two_plate()
    c64 = ctx_for(8)
    c32 = ctx_for(8, precision=B.FRW_FP32_GEOM)
    a = c64.load(s)
    b = c32.load(s)
    n = 400_000
    C64, se64, _, _ = c64.extract(a, 0, n, request_id=7)
    C32, se32, _, _ = c32.extract(b, 0, n, request_id=7)
    assert (np.abs(C32 - C64) <= 3 * np.hypot(se32, se64)).all()
    assert abs(C32[0] - C64[0]) <= 1e-3 * abs(C64[0]) + 3 * se64[0]
    c64.unload(a)
    c32.unload(b)


def test_edge_cases(torch_cuda):
    s = W.tiny_two_plate()
    c = ctx_for(8)
    sid = c.load(s)
    C, se, st, conv = c.extract(sid, 0, 0)
    assert st["walks"] == 0 and (C == 0).all()
    g = c.walk_records(sid, 0, 1, request_id=0)
    o = O.frw_run(s, 0, 1, N=8)
    _records_match(g, o)
    with pytest.raises(B.FRWError):
        c.extract(sid, 5, 10)
    with pytest.raises(B.FRWError):
        c.extract(sid + 17, 0, 10)
    c.unload(sid)
    # N = 2 lattice (every node central)
    c2 = ctx_for(2)
    sid = c2.load(s)
    g = c2.walk_records(sid, 0, 500)
    o = O.frw_run(s, 0, 500, N=2)
    _records_match(g, o)
    c2.unload(sid)


def test_capacitance_matrix_and_symmetrisation(torch_cuda):
    """Full matrix (every master in one run): rows as frw_extract gives them,
    reciprocity C_ij = C_ji within the errors, symmetrised matrix = the average."""
    s = W.interconnect(2)
    c = ctx_for(8)
    sid = c.load(s)
    C, se, Cs, st, _ = c.matrix(sid, 20000, request_id=40)
    n = s.n_cond
    assert C.shape == (n, n + 1) and Cs.shape == (n, n)
    for i in (0, 7, n - 1):
        Ci, sei, _, _ = c.extract(sid, i, 20000, request_id=40 + i)
        np.testing.assert_array_equal(C[i], Ci)
        np.testing.assert_array_equal(se[i], sei)
    assert (np.diag(C[:, :n]) > 0).all()
    off = ~np.eye(n, dtype=bool)
    sd = np.hypot(se[:, :n], se[:, :n].T)[off]
    dC = (C[:, :n] - C[:, :n].T)[off]
    # a pair that no walk of either row reached has both entries exactly 0
    # (no hits, zero standard error): check that, then test the others by z-score
    none = sd == 0.0
    assert (dC[none] == 0.0).all() and (C[:, :n][off][none] == 0.0).all()
    assert (~none).sum() >= n              # most rows reach several neighbours
    z = dC[~none] / sd[~none]
    assert np.isfinite(z).all()
    assert np.mean(np.abs(z) > 4.0) < 0.01
    np.testing.assert_allclose(Cs, 0.5 * (C[:, :n] + C[:, :n].T) * off + np.diag(np.diag(C[:, :n])), rtol=0, atol=0)
    c.unload(sid)


def test_expected_steps_study_cubes_match_eq11(torch_cuda):
    """The E(tau) study's random cubes (permittivities ~ Exp, mean 10): the mean
    walk length the MicroWalk kernel measures equals Eq. 11 solved by the oracle."""
    from paper_2507_09730_gb300 import studies
    N, samples = 8, 40000
    rng = np.random.default_rng([6, 99, N])
    for g in range(3):
        recs, eps = studies._cube_pair(rng, N, 2)
        d = torch_cuda.from_numpy(recs).cuda()
        st = torch_cuda.empty(2 * samples, dtype=torch_cuda.int32, device="cuda")
        ex = torch_cuda.empty(2 * samples, dtype=torch_cuda.int32, device="cuda")
        rc = B.frw_microwalk_cubes_noalloc(N, 2, d.data_ptr(), eps, 0, samples, 70 + g, ex.data_ptr(), st.data_ptr(),
                                           torch_cuda.cuda.current_stream().cuda_stream)
        assert rc == B.FRW_OK
        steps = st.view(2, samples).to(torch_cuda.float64).cpu().numpy()
        for c in range(2):
            K = recs[c, 1]
            ranges = recs[c, 2:2 + 7 * K].reshape(K, 7)
            lat = O.lattice_from_ranges(N, recs[c, 0], ranges[:, :6], ranges[:, 6])
            Et = O.expected_steps(N, eps[lat])
            m, se = steps[c].mean(), steps[c].std() / np.sqrt(samples)
            assert abs(m - Et) < 4.0 * se + 1e-3 * Et, (g, c, m, Et, se)
