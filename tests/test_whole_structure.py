"""The random-walk estimator against an independent whole-structure
finite-difference solve (Eq. 1 with the interface rule of Eq. 4-5) on the
two-plate structure: the oracle's capacitances must agree with the solve at
grid h/2 within 3 standard errors plus the solve's own discretisation change
from h to h/2.  This fixes the absolute scale of the weight omega (eps0, the
permittivity at the Gaussian surface, K / h), which symmetry, reciprocity and
scaling tests cannot see."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2507_09730_gb300 import workloads as W
from tests import fdm_reference as F


H = 0.05     # every face of the two-plate structure lies on the planes of h and h / 2


@pytest.fixture(scope="module")
def fdm_rows(two_plate_fdm):
    return two_plate_fdm


def test_fdm_reference_is_consistent(fdm_rows):
    s, (c1, u1), c2 = fdm_rows
    # charge on the master at 1 V equals the discrete field energy (x2)
    assert abs(c1[0] - u1) <= 1e-7 * u1
    # mirror symmetry about y = 2: C12 from master 0 equals C21 from master 1
    r = F.capacitance_row(s, 1, H)
    assert abs(r[1] - c1[0]) <= 1e-7 * c1[0]
    assert abs(r[0] - c1[1]) <= 1e-7 * abs(c1[1])
    # the solve converges: refining moves C11 up (more field resolved near the edges) by < 5 %
    assert c1[0] < c2[0] < 1.05 * c1[0]
    # a grid that cannot hold the plates' faces is refused
    with pytest.raises(ValueError):
        F.capacitance_row(s, 0, 0.1)


def test_oracle_matches_whole_structure_fdm(fdm_rows):
    s, (c1, _), c2 = fdm_rows
    O.build()
    r = O.frw_run(s, 0, 400000, N=8, seed=0, request=11, records=False)
    for k in range(2):
        tol = 3.0 * r.stderr[k] + abs(c1[k] - c2[k])
        assert abs(r.C[k] - c2[k]) <= tol, (k, r.C[k], c2[k], tol)
    g1, g2 = -c1.sum(), -c2.sum()        # ground (walls) takes the remaining charge
    assert abs(r.C[2] - g2) <= 3.0 * r.stderr[2] + abs(g1 - g2)
    assert r.C[0] > 0 and r.C[1] < 0 and r.C[2] < 0
