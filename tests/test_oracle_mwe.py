"""Pins of the oracle's MicroWalk-E (expanded transition cubes that may hold
conductors; reading R8 of the oracle, Sec. III-B and Fig. 3b of the paper).

- The walk on a lattice with conductor nodes has exactly the exit / absorption law
  and the mean length of its absorbing chain (Theorem 1 and Eq. 11 carried over to
  a lattice whose conductor nodes are Dirichlet nodes), by chi-square.
- A lattice with no conductor node is plain MicroWalk, walk for walk.
- The whole estimator with expanded cubes agrees with the independent
  whole-structure finite-difference solve of the two-plate structure, and with
  plain FRW-MW on the interconnect structure.
"""
import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
from paper_2507_09730_gb300 import workloads as W


def _lattice(N, seed):
    rng = np.random.default_rng([5, seed])
    lat = np.zeros((N, N, N), np.uint8)
    i0, i1 = sorted(rng.integers(0, N, 2))
    lat[i0:i1 + 1, :, 2:N - 1] = 1
    lat[:, 1:N // 2, :] = 2
    cond = -np.ones((N, N, N), np.int16)
    cond[0:2, 0:3, :] = 0                     # conductor 0 in one corner slab
    cond[N - 2:, N - 3:, N - 3:] = 3          # conductor 3 in another corner
    cond[:, :, N - 1] = 7                     # a grounded wall as the last layer
    c = N // 2
    assert (cond[c - 1:c + 1, c - 1:c + 1, c - 1:c + 1] < 0).all()
    return lat, cond


@pytest.mark.parametrize("seed", [0, 1])
def test_microwalk_e_hits_exact_chain(seed):
    N = 8
    eps = np.array([2.5, 7.0, 25.0])
    lat, cond = _lattice(N, seed)
    P, Q, Et = O.absorption_exact_e(N, lat, cond, eps)
    assert abs(P.sum() + Q.sum() - 1.0) < 1e-12
    n = 200_000
    co, nodes, steps = O.microwalk_e_many(N, lat, cond, eps, seed=3, request=seed, walk0=0, n=n)
    hit = co >= 0
    assert set(np.unique(co[hit])) <= {0, 3, 7}
    # exit nodes lie on the boundary; absorbed walks end on a node of their conductor
    nb = nodes[~hit]
    assert (((nb == -1) | (nb == N)).sum(axis=1) == 1).all()
    na = nodes[hit]
    assert (cond[na[:, 0], na[:, 1], na[:, 2]] == co[hit]).all()
    # chi-square over panels and conductors together
    obs = np.concatenate([np.bincount(O.node_to_panel(N, nb), minlength=6 * N * N),
                          np.bincount(co[hit], minlength=Q.size)])
    exp = np.concatenate([P.reshape(-1), Q]) * n
    big = exp >= 5
    obs_b = np.concatenate([obs[big], [obs[~big].sum()]])
    exp_b = np.concatenate([exp[big], [exp[~big].sum()]])
    keep = exp_b > 0
    chi = ((obs_b[keep] - exp_b[keep]) ** 2 / exp_b[keep]).sum()
    assert stats.chi2.sf(chi, keep.sum() - 1) > 1e-3
    m, se = steps.mean(), steps.std() / np.sqrt(n)
    assert abs(m - Et) < 4 * se, (m, Et, se)


def test_microwalk_e_without_conductors_is_microwalk():
    N = 8
    cubes = W.random_cubes(2, N=N, seed=9)
    lat = O.lattice_from_ranges(N, cubes.bg[0], cubes.ranges[0, :cubes.nblk[0]], cubes.mat[0, :cubes.nblk[0]])
    cond = -np.ones((N, N, N), np.int16)
    co, nodes, steps = O.microwalk_e_many(N, lat, cond, cubes.eps, seed=1, request=2, walk0=0, n=2000)
    n2, s2 = O.microwalk_many(N, lat, cubes.eps, seed=1, request=2, walk0=0, n=2000)
    assert (co == -1).all()
    np.testing.assert_array_equal(nodes, np.asarray(n2).reshape(-1, 3))
    np.testing.assert_array_equal(steps, s2)


def test_frw_mwe_against_whole_structure_fdm(two_plate_fdm):
    s, (c1, _), c2 = two_plate_fdm
    r = O.frw_run(s, 0, 400000, N=8, seed=0, request=12, records=False, mwe=5)
    assert r.stats[9] > 0                        # expanded cubes were used
    for k in range(2):
        tol = 3.0 * r.stderr[k] + abs(c1[k] - c2[k])
        assert abs(r.C[k] - c2[k]) <= tol, (k, r.C[k], c2[k], tol)


def test_frw_mwe_agrees_with_frw_mw_on_interconnect():
    s = W.interconnect(0)
    a = O.frw_run(s, 11, 3000, N=16, seed=0, request=13, records=False)
    b = O.frw_run(s, 11, 3000, N=16, seed=0, request=14, records=False, mwe=5)
    assert b.stats[9] > 0 and b.stats[0] < a.stats[0]     # fewer hops with expanded cubes
    for k in (11, 3, 19):
        se = np.hypot(a.stderr[k], b.stderr[k])
        assert abs(a.C[k] - b.C[k]) <= 4.0 * se, (k, a.C[k], b.C[k], se)
