"""Pins of the oracle's FD-based transition (Algorithm 2, FRW-FDM): the
non-stratified transitions sample the cube's discrete SGF of Eq. 8 instead of
running MicroWalk.  The SGF solve itself is pinned elsewhere (closed forms and the
chain solve of Theorem 1); here the walk around it:

- walks that meet no non-stratified cube make exactly the same decisions as
  FRW-MW (the branch changes nothing else, the draws are shared);
- the FD transition lands where the exact absorbing chain of Theorem 1 puts
  it: exit panels of one cube over many words, by chi-square;
- the whole FRW-FDM estimator agrees with the independent whole-structure
  finite-difference solve of the two-plate structure and, by Theorem 1, with
  FRW-MW on the interconnect structure.
"""
import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
from paper_2507_09730_gb300 import workloads as W


def test_fdm_changes_only_non_stratified_transitions():
    s = W.interconnect(0)
    a = O.frw_run(s, 11, 1500, N=8, seed=0, request=21, fdm=True)
    b = O.frw_run(s, 11, 1500, N=8, seed=0, request=21)
    plain = b.steps == 0                      # no MicroWalk transition in the FRW-MW walk
    assert 0.1 < plain.mean() < 0.9
    np.testing.assert_array_equal(a.k[plain], b.k[plain])
    np.testing.assert_array_equal(a.hops[plain], b.hops[plain])
    np.testing.assert_array_equal(a.omega[plain], b.omega[plain])
    np.testing.assert_array_equal(a.branch, b.branch)          # first transitions are shared
    assert (a.steps == 0).all() and a.stats[4] > 0             # FD transitions take no lattice steps


@pytest.mark.parametrize("seed", [0, 1])
def test_fdm_transition_hits_exact_chain(seed):
    """The oracle's FD transition (solve, thresholds, panel -> node) over many
    words against the exit law of the exact absorbing chain (Theorem 1, built
    from the unquantised jump law and solved by sparse LU: a separate route),
    by chi-square over the boundary panels."""
    N = 8
    cubes = W.random_cubes(2, N=N, seed=40 + seed)
    c = seed % 2
    lat = O.lattice_from_ranges(N, cubes.bg[c], cubes.ranges[c, :cubes.nblk[c]], cubes.mat[c, :cubes.nblk[c]])
    Pc, _ = O.absorption_exact(N, lat, cubes.eps, quantised=False)
    n = 200_000
    u = np.random.default_rng([9, seed]).integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    nodes = O.fdm_transitions(N, lat, cubes.eps, u)
    assert (((nodes == -1) | (nodes == N)).sum(axis=1) == 1).all()
    obs = np.bincount(O.node_to_panel(N, nodes), minlength=6 * N * N)
    exp = np.asarray(Pc).reshape(-1) * n
    big = exp >= 5
    ob = np.concatenate([obs[big], [obs[~big].sum()]])
    ex = np.concatenate([exp[big], [exp[~big].sum()]])
    keep = ex > 0
    chi = ((ob[keep] - ex[keep]) ** 2 / ex[keep]).sum()
    assert stats.chi2.sf(chi, keep.sum() - 1) > 1e-3


def test_frw_fdm_against_whole_structure_fdm(two_plate_fdm):
    s, (c1, _), c2 = two_plate_fdm
    r = O.frw_run(s, 0, 60000, N=8, seed=0, request=22, records=False, fdm=True)
    assert r.stats[4] > 0
    for k in range(2):
        tol = 3.0 * r.stderr[k] + abs(c1[k] - c2[k])
        assert abs(r.C[k] - c2[k]) <= tol, (k, r.C[k], c2[k], tol)


def test_frw_fdm_agrees_with_frw_mw_on_interconnect():
    s = W.interconnect(0)
    a = O.frw_run(s, 11, 4000, N=8, seed=0, request=23, records=False, fdm=True)
    b = O.frw_run(s, 11, 4000, N=8, seed=0, request=24, records=False)
    for k in (11, 3, 19):
        se = np.hypot(a.stderr[k], b.stderr[k])
        assert abs(a.C[k] - b.C[k]) <= 4.0 * se, (k, a.C[k], b.C[k], se)
