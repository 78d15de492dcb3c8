"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module only *generates* inputs (box lists, permittivity tables, random cube
descriptions); it holds none of the method's arithmetic.  Every generator is a
pure function of its seed (numpy ``default_rng``), so the GPU path and the CPU
oracle see bit-identical inputs.

Geometry is in micrometres; permittivities are relative (the vacuum permittivity
is applied by the solver).  A structure is

* a grounded domain box (its walls are the ground electrode, conductor index
  ``n_cond``),
* ``n_cond`` disjoint axis-aligned conductor boxes (one box per conductor),
* a background material and an ordered list of axis-aligned dielectric blocks;
  where blocks overlap, the later block wins.

This is the structure the FRW algorithm takes as input (paper, Algorithm 1:
"a 3-D structure of conductors and dielectrics").  The synthetic families stand
in for the paper's proprietary RT1-RT8 / Case 1-2 layouts (Sec. IV, Fig. 5):
conformal 10 nm shells, layout-dependent-effect (LDE) blocks and high-k blocks.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Structure",
    "CubeSet",
    "tiny_two_plate",
    "l_shape_pair",
    "split_conductor",
    "split_blocks",
    "voxel_two_plate",
    "voxel_interconnect",
    "interconnect",
    "batched_family",
    "serving_pool",
    "random_cubes",
    "CONFIG1_EPS",
]


@dataclass
class Structure:
    """Conductor boxes + background + ordered dielectric blocks (see module doc).
    A conductor is one box, or (``cond_id`` given: the conductor of each box) the
    union of several boxes; only single-box conductors can be masters."""

    name: str
    domain_lo: np.ndarray            # (3,) float64
    domain_hi: np.ndarray            # (3,) float64
    cond_lo: np.ndarray              # (n_boxes, 3) float64
    cond_hi: np.ndarray              # (n_boxes, 3) float64
    eps: np.ndarray                  # (n_mat,) float64, relative permittivity per material
    background: int                  # material id of the background dielectric
    block_lo: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    block_hi: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    block_mat: np.ndarray = field(default_factory=lambda: np.zeros((0,), np.int32))
    masters: tuple = (0,)            # conductors the workload extracts rows for
    cond_id: np.ndarray | None = None   # (n_boxes,) int32 conductor of each box; None: box k = conductor k
    # permittivity voxel map over the domain, shape (nx, ny, nz) uint8 (x slowest):
    # cell (i, j, k) has material voxel_mat[i, j, k], 255 = none (background); the
    # blocks lie on top of it
    voxel_mat: np.ndarray | None = None

    def __post_init__(self):
        self.domain_lo = np.ascontiguousarray(self.domain_lo, np.float64).reshape(3)
        self.domain_hi = np.ascontiguousarray(self.domain_hi, np.float64).reshape(3)
        self.cond_lo = np.ascontiguousarray(self.cond_lo, np.float64).reshape(-1, 3)
        self.cond_hi = np.ascontiguousarray(self.cond_hi, np.float64).reshape(-1, 3)
        self.eps = np.ascontiguousarray(self.eps, np.float64).reshape(-1)
        self.block_lo = np.ascontiguousarray(self.block_lo, np.float64).reshape(-1, 3)
        self.block_hi = np.ascontiguousarray(self.block_hi, np.float64).reshape(-1, 3)
        self.block_mat = np.ascontiguousarray(self.block_mat, np.int32).reshape(-1)
        if self.cond_id is not None:
            self.cond_id = np.ascontiguousarray(self.cond_id, np.int32).reshape(-1)
        if self.voxel_mat is not None:
            self.voxel_mat = np.ascontiguousarray(self.voxel_mat, np.uint8)
            assert self.voxel_mat.ndim == 3

    @property
    def n_boxes(self) -> int:
        return int(self.cond_lo.shape[0])

    @property
    def n_cond(self) -> int:
        return self.n_boxes if self.cond_id is None else int(self.cond_id.max()) + 1

    def boxes_of(self, k: int) -> np.ndarray:
        """Indices of conductor k's boxes."""
        return np.array([k]) if self.cond_id is None else np.flatnonzero(self.cond_id == k)

    @property
    def n_blocks(self) -> int:
        return int(self.block_lo.shape[0])

    @property
    def n_mat(self) -> int:
        return int(self.eps.shape[0])

    def scaled_eps(self, factor: float) -> "Structure":
        """Same geometry with every permittivity multiplied by ``factor``."""
        return Structure(self.name + f"*eps{factor:g}", self.domain_lo, self.domain_hi,
                         self.cond_lo, self.cond_hi, self.eps * factor, self.background,
                         self.block_lo, self.block_hi, self.block_mat, self.masters, self.cond_id, self.voxel_mat)


# ---------------------------------------------------------------------------
# Workload 0: two 1.0 x 0.2 x 1.0 um plates, 0.3 um gap, high-k cube across the gap
# ---------------------------------------------------------------------------
def tiny_two_plate() -> Structure:
    """Grounded 4x4x4 um box, two plates with a 0.3 um gap along y, background
    eps 3.9 and one eps-25 cube of 0.4 um straddling the gap.  Mirror-symmetric
    about y = 2 (so C11 = C22 and C12 = C21 in expectation)."""
    return Structure(
        name="tiny_two_plate",
        domain_lo=[0.0, 0.0, 0.0], domain_hi=[4.0, 4.0, 4.0],
        cond_lo=[[1.5, 1.65, 1.5], [1.5, 2.15, 1.5]],
        cond_hi=[[2.5, 1.85, 2.5], [2.5, 2.35, 2.5]],
        eps=[3.9, 25.0], background=0,
        block_lo=[[1.8, 1.8, 1.8]], block_hi=[[2.2, 2.2, 2.2]], block_mat=[1],
        masters=(0, 1),
    )


def l_shape_pair() -> Structure:
    """The two-plate structure with the second conductor an L: its plate plus a
    0.2 um leg along +y at the high-x end, touching the plate (two boxes, one
    conductor).  Every face lies on the 0.05 um grid."""
    s = tiny_two_plate()
    return Structure(
        name="l_shape_pair", domain_lo=s.domain_lo, domain_hi=s.domain_hi,
        cond_lo=[[1.5, 1.65, 1.5], [1.5, 2.15, 1.5], [2.3, 2.35, 1.5]],
        cond_hi=[[2.5, 1.85, 2.5], [2.5, 2.35, 2.5], [2.5, 2.95, 2.5]],
        eps=s.eps, background=s.background, block_lo=s.block_lo, block_hi=s.block_hi, block_mat=s.block_mat,
        masters=(0,), cond_id=[0, 1, 1],
    )


def split_conductor(s: Structure, k: int, pieces: int, axis: int = 0) -> Structure:
    """The same structure with single-box conductor k cut into `pieces` touching
    boxes along `axis` (the same conductor, the same union)."""
    (kb,) = s.boxes_of(k)
    ids = np.arange(s.n_boxes) if s.cond_id is None else s.cond_id
    lo, hi = s.cond_lo[kb], s.cond_hi[kb]
    cuts = np.linspace(lo[axis], hi[axis], pieces + 1)
    blo, bhi, cid = [], [], []
    for b in range(s.n_boxes):
        if b != kb:
            blo.append(s.cond_lo[b]); bhi.append(s.cond_hi[b]); cid.append(int(ids[b]))
            continue
        for p in range(pieces):
            l, h = lo.copy(), hi.copy()
            l[axis], h[axis] = cuts[p], cuts[p + 1]
            blo.append(l); bhi.append(h); cid.append(k)
    return Structure(s.name + f"+split{k}x{pieces}", s.domain_lo, s.domain_hi, np.array(blo), np.array(bhi),
                     s.eps, s.background, s.block_lo, s.block_hi, s.block_mat, s.masters, np.array(cid))


def split_blocks(s: Structure, pieces=(4, 4, 2)) -> Structure:
    """The same structure with every dielectric block cut into
    pieces[0] x pieces[1] x pieces[2] touching blocks of its material (the same
    union, so the same permittivity everywhere).  With 4 x 4 x 2 the two-plate
    structure's high-k cube becomes 32 blocks with every face on the 0.05 um grid,
    so transition cubes near the gap list more than 14 blocks."""
    blo, bhi, bm = [], [], []
    for b in range(s.n_blocks):
        lo, hi = s.block_lo[b], s.block_hi[b]
        cuts = [np.linspace(lo[a], hi[a], pieces[a] + 1) for a in range(3)]
        for i in range(pieces[0]):
            for j in range(pieces[1]):
                for k in range(pieces[2]):
                    ix = (i, j, k)
                    blo.append([cuts[a][ix[a]] for a in range(3)])
                    bhi.append([cuts[a][ix[a] + 1] for a in range(3)])
                    bm.append(int(s.block_mat[b]))
    return Structure(s.name + "+split_blocks" + "x".join(map(str, pieces)), s.domain_lo, s.domain_hi,
                     s.cond_lo, s.cond_hi, s.eps, s.background, np.array(blo), np.array(bhi),
                     np.array(bm, np.int32), s.masters, s.cond_id)


VOXEL_NONE = 255


def voxel_two_plate() -> Structure:
    """The two-plate structure with its high-k cube given as a permittivity voxel
    map instead of a block: 20^3 cells of 0.2 um over the 4 um domain, cells 9-10
    on every axis ([1.8, 2.2] um) of the high-k material, the rest none
    (background).  The same permittivity everywhere as tiny_two_plate()."""
    s = tiny_two_plate()
    vm = np.full((20, 20, 20), VOXEL_NONE, np.uint8)
    vm[9:11, 9:11, 9:11] = 1
    return Structure("voxel_two_plate", s.domain_lo, s.domain_hi, s.cond_lo, s.cond_hi, s.eps, s.background,
                     masters=s.masters, voxel_mat=vm)


def voxel_interconnect(seed: int = 0, dims=(10, 10, 4), fill: float = 0.3) -> Structure:
    """The interconnect structure with a random permittivity voxel map under its
    shells and LDE blocks: each cell of a dims grid over the domain is, with
    probability `fill`, one of two extra dielectrics (eps 3.2 or 4.1), else none.
    The blocks stay on top of the map."""
    s = interconnect(seed)
    rng = np.random.default_rng(np.random.SeedSequence([7, seed, *dims]))
    n0 = s.n_mat
    eps = np.concatenate([s.eps, [3.2, 4.1]])
    vm = np.where(rng.random(dims) < fill, rng.integers(n0, n0 + 2, dims), VOXEL_NONE).astype(np.uint8)
    return Structure(f"voxel_interconnect{seed}", s.domain_lo, s.domain_hi, s.cond_lo, s.cond_hi, eps, s.background,
                     s.block_lo, s.block_hi, s.block_mat, s.masters, s.cond_id, vm)


# ---------------------------------------------------------------------------
# Workload 2: three metal layers of parallel / crossing wires with shells + LDE
# ---------------------------------------------------------------------------
_ILD, _SHELL, _LDE = 0, 1, 2


def _place_across(rng, n, span_lo, span_hi, wmin=0.05, wmax=0.2, smin=0.05):
    widths = rng.uniform(wmin, wmax, n)
    slack = (span_hi - span_lo) - widths.sum() - smin * (n - 1)
    assert slack > 0.0
    parts = rng.dirichlet(np.ones(n + 1)) * slack
    lo = np.empty(n)
    x = span_lo + parts[0]
    for i in range(n):
        lo[i] = x
        x += widths[i] + smin + parts[i + 1]
    return lo, lo + widths


def _stack(rng, name, lateral, layers, wires_per_layer, n_lde, zsize, length_margin=0.5,
           shell=0.01, lde_side=(0.1, 0.6)):
    """Wires along alternating axes on each layer, each with a conformal shell."""
    c_lo, c_hi, b_lo, b_hi, b_mat = [], [], [], [], []
    for li, (z0, z1) in enumerate(layers):
        along = 0 if li % 2 == 0 else 1
        across = 1 - along
        lo, hi = _place_across(rng, wires_per_layer, length_margin, lateral - length_margin)
        for a, b in zip(lo, hi):
            wl = np.zeros(3)
            wh = np.zeros(3)
            wl[along], wh[along] = length_margin, lateral - length_margin
            wl[across], wh[across] = a, b
            wl[2], wh[2] = z0, z1
            c_lo.append(wl)
            c_hi.append(wh)
    # LDE blocks first (lower priority), then the conformal shells on top.
    dom_hi = np.array([lateral, lateral, zsize])
    for _ in range(n_lde):
        side = rng.uniform(lde_side[0], lde_side[1], 3)
        side[2] = min(side[2], 0.5 * zsize)
        lo = rng.uniform(0.0, 1.0, 3) * (dom_hi - side)
        b_lo.append(lo)
        b_hi.append(lo + side)
        b_mat.append(_LDE)
    for wl, wh in zip(c_lo, c_hi):
        b_lo.append(wl - shell)
        b_hi.append(wh + shell)
        b_mat.append(_SHELL)
    return c_lo, c_hi, b_lo, b_hi, b_mat, dom_hi


def interconnect(seed: int = 0) -> Structure:
    """4 x 4 x 1.6 um grounded box; M1 (z 0.20-0.30, along x), M2 (z 0.50-0.62,
    along y), M3 (z 0.85-1.00, along x); 8 wires per layer of widths U[0.05, 0.2],
    spacing >= 0.05, length 3.0; a 10 nm eps-7.0 shell around every wire in an
    eps-2.7 ILD; 12 eps-5 LDE blocks with sides U[0.1, 0.6].  Masters: the fourth
    wire of each layer."""
    rng = np.random.default_rng(np.random.SeedSequence([2, seed]))
    layers = [(0.20, 0.30), (0.50, 0.62), (0.85, 1.00)]
    c_lo, c_hi, b_lo, b_hi, b_mat, dom_hi = _stack(rng, "interconnect", 4.0, layers, 8, 12, 1.6)
    return Structure(
        name=f"interconnect_s{seed}", domain_lo=[0, 0, 0], domain_hi=dom_hi,
        cond_lo=c_lo, cond_hi=c_hi, eps=[2.7, 7.0, 5.0], background=_ILD,
        block_lo=b_lo, block_hi=b_hi, block_mat=b_mat, masters=(3, 11, 19),
    )


def _family_member(rng, idx: int, n_cond: int) -> Structure:
    n_layers = int(rng.integers(2, 7))
    n_layers = max(1, min(n_layers, n_cond))
    per = [n_cond // n_layers + (1 if i < n_cond % n_layers else 0) for i in range(n_layers)]
    wires_max = max(per)
    density = rng.uniform(0.6, 1.0)
    lateral = max(2.0, (wires_max * 0.3) / density + 1.0)
    pitch = 0.35
    layers = []
    for li in range(n_layers):
        z0 = 0.2 + li * pitch
        layers.append((z0, z0 + rng.uniform(0.10, 0.15)))
    zsize = layers[-1][1] + 0.6
    c_lo, c_hi, b_lo, b_hi, b_mat = [], [], [], [], []
    for li, (z0, z1) in enumerate(layers):
        sub = _stack(rng, "", lateral, [(z0, z1)], per[li], 0, zsize)
        # _stack always lays layer 0 along x; alternate by swapping x / y on odd layers
        for wl, wh in zip(sub[0], sub[1]):
            if li % 2 == 1:
                wl = wl[[1, 0, 2]]
                wh = wh[[1, 0, 2]]
            c_lo.append(wl)
            c_hi.append(wh)
    dom_hi = np.array([lateral, lateral, zsize])
    n_lde = int(rng.integers(4, 16))
    for _ in range(n_lde):
        side = rng.uniform(0.1, 0.6, 3)
        side[2] = min(side[2], 0.5 * zsize)
        lo = rng.uniform(0.0, 1.0, 3) * (dom_hi - side)
        b_lo.append(lo)
        b_hi.append(lo + side)
        b_mat.append(_LDE)
    for wl, wh in zip(c_lo, c_hi):
        b_lo.append(wl - 0.01)
        b_hi.append(wh + 0.01)
        b_mat.append(_SHELL)
    return Structure(
        name=f"family_{idx}_n{n_cond}", domain_lo=[0, 0, 0], domain_hi=dom_hi,
        cond_lo=c_lo, cond_hi=c_hi, eps=[2.7, 7.0, 5.0], background=_ILD,
        block_lo=b_lo, block_hi=b_hi, block_mat=b_mat,
        masters=tuple(range(n_cond)),
    )


def batched_family(n_structures: int = 64, seed: int = 0, n_min: int = 2, n_max: int = 200):
    """Structures generated like :func:`interconnect` with 2-6 layers, conductor
    counts log-uniform in [n_min, n_max] and random wire density."""
    rng = np.random.default_rng(np.random.SeedSequence([3, seed]))
    out = []
    for i in range(n_structures):
        n = int(round(np.exp(rng.uniform(np.log(n_min), np.log(n_max)))))
        out.append(_family_member(rng, i, max(n_min, min(n_max, n))))
    return out


def serving_pool(n_structures: int = 32, seed: int = 0):
    """Pool of request structures with 4-200 conductors (see :func:`batched_family`)."""
    return batched_family(n_structures, seed=1000 + seed, n_min=4, n_max=200)


@dataclass
class Request:
    t: float            # arrival time (s from the start)
    structure: int      # index into the pool
    master: int
    sigma: float        # relative 1-sigma target


def serving_requests(pool, rate: float = 200.0, duration: float = 60.0, seed: int = 0,
                     sigma_lo: float = 0.005, sigma_hi: float = 0.02):
    """Poisson arrivals of mean `rate` per second over `duration` seconds; each
    request draws a structure of the pool, a master among its conductors and a
    1-sigma target uniform in [sigma_lo, sigma_hi]."""
    rng = np.random.default_rng(np.random.SeedSequence([4, seed]))
    out, t = [], 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            return out
        k = int(rng.integers(0, len(pool)))
        out.append(Request(t, k, int(rng.integers(0, pool[k].n_cond)), float(rng.uniform(sigma_lo, sigma_hi))))


# ---------------------------------------------------------------------------
# Workload 1: random transition cubes given directly as integer voxel ranges
# ---------------------------------------------------------------------------
CONFIG1_EPS = np.array([2.5, 3.9, 7.0, 25.0])


@dataclass
class CubeSet:
    """``n`` lattice cubes of edge ``N``.  Cube c has background material
    ``bg[c]`` and ``nblk[c]`` blocks; block b covers voxels
    ``ranges[c, b, 2a] <= i_a < ranges[c, b, 2a+1]`` on axis a and has material
    ``mat[c, b]``; later blocks win."""

    N: int
    bg: np.ndarray        # (n,) int32
    nblk: np.ndarray      # (n,) int32
    ranges: np.ndarray    # (n, kmax, 6) int32
    mat: np.ndarray       # (n, kmax) int32
    eps: np.ndarray       # (n_mat,) float64

    @property
    def n(self) -> int:
        return int(self.bg.shape[0])


def random_cubes(n_cubes: int, N: int = 16, seed: int = 0, kmin: int = 2, kmax: int = 6,
                 eps=CONFIG1_EPS) -> CubeSet:
    """Per cube: a background and ``kmin..kmax`` random axis-aligned sub-blocks with
    integer voxel ranges uniform in [0, N], each with a material drawn from ``eps``."""
    rng = np.random.default_rng(np.random.SeedSequence([1, seed, N]))
    n_mat = len(eps)
    bg = rng.integers(0, n_mat, n_cubes).astype(np.int32)
    nblk = rng.integers(kmin, kmax + 1, n_cubes).astype(np.int32)
    ranges = np.zeros((n_cubes, kmax, 6), np.int32)
    mat = np.zeros((n_cubes, kmax), np.int32)
    for c in range(n_cubes):
        for b in range(nblk[c]):
            for a in range(3):
                lo = int(rng.integers(0, N))
                hi = int(rng.integers(lo + 1, N + 1))
                ranges[c, b, 2 * a], ranges[c, b, 2 * a + 1] = lo, hi
            mat[c, b] = int(rng.integers(0, n_mat))
    return CubeSet(N, bg, nblk, ranges, mat, np.asarray(eps, np.float64))
