"""The oracle's overflow rule (reading R3): a transition cube that lists more
than 14 dielectric blocks is halved until it lists at most 14.  Any
conductor-free cube centred at the walk's point is a valid transition domain
(Sec. II-A), so the rule changes the walks' paths but not the estimator's
expectation.

Pinned on the two-plate structure with its high-k cube cut into 32 touching
blocks of the same material (the same permittivity everywhere): cubes near the
gap overflow and are halved, the walks differ from those of the uncut
structure, and both estimates agree with each other and with the independent
whole-structure finite-difference solve."""
import numpy as np

from oracle import oracle as O
from paper_2507_09730_gb300 import workloads as W

N_WALKS = 200_000


def test_overflow_halving_keeps_the_estimate():
    O.build()
    s0 = W.tiny_two_plate()
    s32 = W.split_blocks(s0, (4, 4, 2))
    a = O.frw_run(s0, 0, N_WALKS, N=8, seed=0, request=21, records=True)
    b = O.frw_run(s32, 0, N_WALKS, N=8, seed=0, request=21, records=True)
    assert a.stats[10] == 0                       # one block: never more than 14
    assert b.stats[10] > 0                        # 32 blocks: cubes near the gap were halved
    # halving changes paths: more hops, and some walks differ
    assert b.stats[0] > a.stats[0]
    assert (a.hops != b.hops).any()
    for k in range(3):
        sig = np.hypot(a.stderr[k], b.stderr[k])
        assert abs(a.C[k] - b.C[k]) <= 3.0 * sig, (k, a.C[k], b.C[k], sig)


def test_overflow_structure_matches_whole_structure_fdm(two_plate_fdm):
    """The cut structure has the uncut one's permittivity in every grid cell, so
    the same whole-structure solve is its reference."""
    s0, (c1, _), c2 = two_plate_fdm
    s32 = W.split_blocks(s0, (4, 4, 2))
    from tests import fdm_reference as F
    r = O.frw_run(s32, 0, N_WALKS, N=8, seed=0, request=22, records=False)
    assert r.stats[10] > 0
    for k in range(2):
        tol = 3.0 * r.stderr[k] + abs(c1[k] - c2[k])
        assert abs(r.C[k] - c2[k]) <= tol, (k, r.C[k], c2[k], tol)
    # the cut changes nothing the solve can see (a coarse row, computed again)
    np.testing.assert_allclose(F.capacitance_row(s32, 0, 0.05), c1, rtol=1e-9, atol=0)
