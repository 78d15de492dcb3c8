"""Permittivity voxel maps (Sec. III-A: permittivity constant per voxel) as a
structure input: the oracle's expansion of a map into dielectric boxes against
the definition cell by cell, and walks on a map that reproduces a block
structure equal to that structure's walks."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2507_09730_gb300 import workloads as W

NONE = O.VOXEL_NONE


def _edges(lo, hi, n):
    return [float(hi) if i == n else float(lo) + ((float(hi) - float(lo)) * i) / n for i in range(n + 1)]


@pytest.mark.parametrize("dims,fill,seed", [((5, 4, 3), 0.5, 1), ((8, 8, 8), 0.9, 2), ((1, 1, 6), 1.0, 3),
                                            ((7, 3, 9), 0.2, 4), ((6, 6, 2), 0.0, 5)])
def test_voxel_boxes_cover_every_cell_once(dims, fill, seed):
    rng = np.random.default_rng(seed)
    # few materials and runs of equal cells, so that merging happens
    vm = np.where(rng.random(dims) < fill, rng.integers(0, 2, dims), NONE).astype(np.uint8)
    lo, hi = np.array([0.0, -1.0, 0.5]), np.array([4.0, 2.0, 1.7])
    blo, bhi, bm = O.voxel_blocks(lo, hi, vm)
    e = [_edges(lo[a], hi[a], dims[a]) for a in range(3)]
    cover = np.zeros(dims, int)
    mat = np.full(dims, NONE, int)
    for b in range(bm.shape[0]):
        # every box face is a cell edge of the map
        idx = [(e[a].index(blo[b, a]), e[a].index(bhi[b, a])) for a in range(3)]
        sl = tuple(slice(i0, i1) for i0, i1 in idx)
        cover[sl] += 1
        mat[sl] = bm[b]
    assert ((cover == 1) == (vm != NONE)).all() and (cover <= 1).all()
    assert (mat[vm != NONE] == vm[vm != NONE]).all()
    # boxes ordered by their first cell; no two boxes that could be one along z
    first = [tuple(e[a].index(blo[b, a]) for a in range(3)) for b in range(bm.shape[0])]
    assert first == sorted(first)
    if fill == 0.0:
        assert bm.shape[0] == 0


def test_voxel_map_of_a_block_gives_the_block_structure_walks():
    """The two-plate structure's high-k cube given as 2 x 2 x 2 cells of a 20^3 map
    loads as the same single block, so every walk is the same."""
    s0, sv = W.tiny_two_plate(), W.voxel_two_plate()
    blo, bhi, bm = O.voxel_blocks(sv.domain_lo, sv.domain_hi, sv.voxel_mat)
    np.testing.assert_array_equal(blo, s0.block_lo)
    np.testing.assert_array_equal(bhi, s0.block_hi)
    np.testing.assert_array_equal(bm, s0.block_mat)
    a = O.frw_run(s0, 0, 2000, N=8, seed=0, request=31)
    b = O.frw_run(sv, 0, 2000, N=8, seed=0, request=31)
    for f in ("k", "hops", "steps", "branch", "omega"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))


def test_blocks_lie_on_top_of_the_voxel_map():
    """Material at points of the voxel interconnect: the last block containing the
    point, else its voxel cell's material, else the background (brute force over
    the map), against the oracle's box list with its later-wins rule."""
    s = W.voxel_interconnect(0)
    blo, bhi, bm = O.structure_blocks(s)
    nv = int((s.voxel_mat != NONE).sum())
    assert bm.shape[0] >= s.n_blocks + 1 and bm.shape[0] <= s.n_blocks + nv
    rng = np.random.default_rng(9)
    dims = s.voxel_mat.shape
    e = [np.array(_edges(s.domain_lo[a], s.domain_hi[a], dims[a])) for a in range(3)]
    for p in rng.uniform(s.domain_lo, s.domain_hi, (3000, 3)):
        want = s.background
        cell = tuple(int(np.searchsorted(e[a], p[a], side="right") - 1) for a in range(3))
        if s.voxel_mat[cell] != NONE:
            want = int(s.voxel_mat[cell])
        for b in range(s.n_blocks):
            if (s.block_lo[b] <= p).all() and (p < s.block_hi[b]).all():
                want = int(s.block_mat[b])
        got = s.background
        for b in range(bm.shape[0]):
            if (blo[b] <= p).all() and (p < bhi[b]).all():
                got = int(bm[b])
        assert got == want, (p, got, want)
