"""Pins of the oracle's multi-box conductors (a conductor is the union of its
boxes; only single-box conductors are masters):

- cutting a conductor into touching boxes changes nothing: the distance to the
  union equals the distance to the uncut box bit for bit, so every walk of FRW-MW
  makes the same decisions (records identical), and the whole-structure FD solve
  gives the same row;
- an L-shaped conductor (two boxes) agrees with the independent whole-structure
  finite-difference solve;
- a multi-box master is refused (its Gaussian surface is not defined).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2507_09730_gb300 import workloads as W
from tests import fdm_reference as F


def test_cut_conductor_gives_identical_walks():
    s = W.interconnect(0)
    t = W.split_conductor(W.split_conductor(s, 3, 3, axis=0), 12, 2, axis=1)
    assert t.n_boxes == s.n_boxes + 3 and t.n_cond == s.n_cond
    a = O.frw_run(s, 11, 400, N=8, seed=0, request=51)
    b = O.frw_run(t, 11, 400, N=8, seed=0, request=51)
    np.testing.assert_array_equal(a.k, b.k)
    np.testing.assert_array_equal(a.hops, b.hops)
    np.testing.assert_array_equal(a.steps, b.steps)
    np.testing.assert_array_equal(a.omega, b.omega)
    assert ((a.k == 3) | (a.k == 12)).any()                 # walks end on the cut conductors too
    np.testing.assert_array_equal(a.S1, b.S1)


def test_cut_conductor_in_the_fd_reference():
    s = W.tiny_two_plate()
    t = W.split_conductor(s, 1, 2, axis=0)
    np.testing.assert_array_equal(F.capacitance_row(s, 0, 0.1 / 2), F.capacitance_row(t, 0, 0.1 / 2))


@pytest.fixture(scope="module")
def l_shape_fdm():
    s = W.l_shape_pair()
    return s, F.capacitance_row(s, 0, 0.05), F.capacitance_row(s, 0, 0.025, rtol=1e-8)


def test_l_shape_against_whole_structure_fdm(l_shape_fdm):
    s, c1, c2 = l_shape_fdm
    r = O.frw_run(s, 0, 150000, N=8, seed=0, request=52, records=False)
    # the leg adds to the coupling of the plain two plates (same geometry otherwise)
    base = F.capacitance_row(W.tiny_two_plate(), 0, 0.05)
    assert abs(c1[1]) > abs(base[1])
    for k in range(2):
        tol = 3.0 * r.stderr[k] + abs(c1[k] - c2[k])
        assert abs(r.C[k] - c2[k]) <= tol, (k, r.C[k], c2[k], tol)


def test_multibox_master_is_refused():
    with pytest.raises(ValueError):
        O.frw_run(W.l_shape_pair(), 1, 10, N=8)
