"""Python face of the CPU oracle (test infrastructure).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the library.  It shares no
code with the CUDA path.

Two independent routes to the same quantities live here:

* ``liborc`` (``frw_oracle.c``): the step-by-step method (Philox, explicit
  lattices, MicroWalk of Algorithm 3, conjugate-gradient FD solves of Eq. 4-8,
  the FRW driver of Algorithm 1).
* :func:`absorption_exact`: the absorbing Markov chain of Eq. 9 built from the
  jump law and solved directly with a sparse LU (scipy), giving the exit
  distribution e_c^T B (Theorem 1) and E(tau) of Eq. 11.  It does not use the FD
  symmetric form at all, so it pins the C code's solves from the other side.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "frw_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")

KIND_SGF, KIND_FLUX_PAR, KIND_FLUX_PERP, KIND_SGF_HOM, KIND_FLUX_HOM = range(5)
BOUNDARY = 15
EPS0 = 8.8541878128e-3  # fF / um


def build(force: bool = False) -> str:
    """Compile the oracle (plain gcc, no FMA contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.POINTER
        d, i, u32, u64, u8 = (ctypes.c_double, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64,
                              ctypes.c_uint8)
        L.orc_philox4x32_10.argtypes = [P(u32), P(u32), P(u32)]
        L.orc_w_table.argtypes = [P(d), i, P(u32)]
        L.orc_microwalk.argtypes = [i, P(u8), P(d), i, u64, u64, u64, u32, P(ctypes.c_int32), P(u64)]
        L.orc_microwalk_many.argtypes = [i, P(u8), P(d), i, u64, u64, u64, u64, P(ctypes.c_int32),
                                         P(u64)]
        L.orc_lattice_from_ranges.argtypes = [i, i, i, P(ctypes.c_int32), P(ctypes.c_int32), P(u8)]
        L.orc_fd_solve.argtypes = [i, P(d), P(d), P(d)]
        L.orc_fd_solve.restype = i
        L.orc_sgf.argtypes = [i, P(d), P(d)]
        L.orc_sgf.restype = i
        L.orc_flux.argtypes = [i, P(d), i, P(d)]
        L.orc_flux.restype = i
        L.orc_expected_steps.argtypes = [i, P(d)]
        L.orc_expected_steps.restype = d
        L.orc_table.argtypes = [i, i, i, i, P(u8), P(d), P(u32), P(u8), P(d)]
        L.orc_panel_node.argtypes = [i, i, i, i, i, P(ctypes.c_int32)]
        L.orc_microwalk_e.argtypes = [i, P(u8), P(ctypes.c_int16), P(d), i, u64, u64, u64, u32,
                                      P(ctypes.c_int32), P(u64)]
        L.orc_microwalk_e.restype = i
        L.orc_microwalk_e_many.argtypes = [i, P(u8), P(ctypes.c_int16), P(d), i, u64, u64, u64, u64, u32,
                                           P(ctypes.c_int32), P(ctypes.c_int32), P(u64)]
        L.orc_frw_run.argtypes = ([P(d), P(d), i, P(d), P(d), P(ctypes.c_int32), i, i, P(d), P(d), P(ctypes.c_int32), i,
                                   P(d), i, i, u64, u64, i, i, d, i, i, i, i, u64, u64, d, u64,
                                   P(d), P(d), P(u64), P(d), P(ctypes.c_int32), P(u32), P(u64),
                                   P(ctypes.c_int32), P(u64)])
        L.orc_frw_run.restype = i
        L.orc_fdm_transitions.argtypes = [i, P(u8), P(d), i, P(u32), P(ctypes.c_int32)]
        _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


# ---------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    """Philox4x32-10 block (Salmon et al., SC'11)."""
    c = np.asarray(ctr, np.uint32)
    k = np.asarray(key, np.uint32)
    o = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32), _p(o, ctypes.c_uint32))
    return o


def w_table(eps):
    """Quantised alpha table W[v][i] of Eq. 6 (16 x 16, row = current material)."""
    e = np.ascontiguousarray(eps, np.float64)
    W = np.zeros((16, 16), np.uint32)
    lib().orc_w_table(_p(e, ctypes.c_double), len(e), _p(W, ctypes.c_uint32))
    return W


def microwalk_many(N, lat, eps, seed, request, walk0, n):
    """``n`` MicroWalks (walk ids walk0.., hop 0) -> (exit nodes (n, 3), steps (n,))."""
    L = np.ascontiguousarray(lat, np.uint8).reshape(-1)
    e = np.ascontiguousarray(eps, np.float64)
    nodes = np.zeros((int(n), 3), np.int32)
    steps = np.zeros(int(n), np.uint64)
    lib().orc_microwalk_many(N, _p(L, ctypes.c_uint8), _p(e, ctypes.c_double), len(e), int(seed),
                             int(request), int(walk0), int(n), _p(nodes, ctypes.c_int32),
                             _p(steps, ctypes.c_uint64))
    return nodes, steps


def node_to_panel(N, nodes):
    """Exit nodes (one coordinate -1 or N) -> natural panel index f*N^2 + u*N + v."""
    nodes = np.asarray(nodes).reshape(-1, 3)
    out = np.empty(len(nodes), np.int64)
    for a in range(3):
        o = [b for b in range(3) if b != a]
        for side, val in ((0, -1), (1, N)):
            m = nodes[:, a] == val
            out[m] = ((2 * a + side) * N + nodes[m, o[0]]) * N + nodes[m, o[1]]
    return out


def lattice_from_ranges(N, bg, ranges, mats):
    r = np.ascontiguousarray(ranges, np.int32).reshape(-1, 6)
    m = np.ascontiguousarray(mats, np.int32).reshape(-1)
    lat = np.zeros(N * N * N, np.uint8)
    lib().orc_lattice_from_ranges(N, int(bg), len(m), _p(r, ctypes.c_int32), _p(m, ctypes.c_int32),
                                  _p(lat, ctypes.c_uint8))
    return lat.reshape(N, N, N)


def microwalk(N, lat, eps, seed, request, walk, hop=0):
    """One MicroWalk (Algorithm 3) on an explicit lattice -> (exit node, steps)."""
    L = np.ascontiguousarray(lat, np.uint8).reshape(-1)
    e = np.ascontiguousarray(eps, np.float64)
    node = np.zeros(3, np.int32)
    steps = np.zeros(1, np.uint64)
    lib().orc_microwalk(N, _p(L, ctypes.c_uint8), _p(e, ctypes.c_double), len(e), int(seed),
                        int(request), int(walk), int(hop), _p(node, ctypes.c_int32),
                        _p(steps, ctypes.c_uint64))
    return node, int(steps[0])


def sgf(N, eps_lattice):
    """Discrete SGF of Eq. 8 by CG on the symmetric FD system; faces in natural
    order (face 2a+side, (u, v) on the other axes in increasing order)."""
    e = np.ascontiguousarray(eps_lattice, np.float64).reshape(-1)
    P = np.zeros(6 * N * N)
    it = lib().orc_sgf(N, _p(e, ctypes.c_double), _p(P, ctypes.c_double))
    assert it > 0, "CG did not converge"
    return P.reshape(6, N, N)


def flux(N, eps_lattice, axis):
    """First-cube flux kernel (times h) along +axis, natural face order."""
    e = np.ascontiguousarray(eps_lattice, np.float64).reshape(-1)
    F = np.zeros(6 * N * N)
    it = lib().orc_flux(N, _p(e, ctypes.c_double), int(axis), _p(F, ctypes.c_double))
    assert it > 0, "CG did not converge"
    return F.reshape(6, N, N)


def fd_solve(N, eps_lattice, rhs):
    e = np.ascontiguousarray(eps_lattice, np.float64).reshape(-1)
    b = np.ascontiguousarray(rhs, np.float64).reshape(-1)
    y = np.zeros_like(b)
    it = lib().orc_fd_solve(N, _p(e, ctypes.c_double), _p(b, ctypes.c_double), _p(y, ctypes.c_double))
    assert it > 0
    return y.reshape(N, N, N)


def expected_steps(N, eps_lattice):
    """E(tau) of Eq. 11 via the FD solve."""
    e = np.ascontiguousarray(eps_lattice, np.float64).reshape(-1)
    return float(lib().orc_expected_steps(N, _p(e, ctypes.c_double)))


def table(N, kind, axis, naxis, profile, eps):
    """Canonical-order sampling table: (thresholds u32[6N^2], negative-sign flags, total)."""
    prof = np.zeros(64, np.uint8)
    if profile is not None:
        prof[:N] = np.asarray(profile, np.uint8)
    e = np.ascontiguousarray(eps, np.float64)
    thr = np.zeros(6 * N * N, np.uint32)
    neg = np.zeros(6 * N * N, np.uint8)
    tot = np.zeros(1)
    lib().orc_table(N, kind, axis, naxis, _p(prof, ctypes.c_uint8), _p(e, ctypes.c_double),
                    _p(thr, ctypes.c_uint32), _p(neg, ctypes.c_uint8), _p(tot, ctypes.c_double))
    return thr, neg, float(tot[0])


def panel_node(N, kind, axis, naxis, n):
    node = np.zeros(3, np.int32)
    lib().orc_panel_node(N, kind, axis, naxis, int(n), _p(node, ctypes.c_int32))
    return node


# ---------------------------------------------------------------------------
# Permittivity voxel map of a structure -> dielectric boxes.  The map's cells
# partition the domain uniformly (cell i of axis a spans [e(i), e(i + 1)) with
# e(i) = lo + ((hi - lo) * i) / n and e(n) = hi); every cell with a material is
# covered by exactly one box: maximal runs of one material along z, runs of equal
# extent and material merged over consecutive y, rectangles merged over
# consecutive x, boxes ordered by their first cell.  They lie below the blocks.
VOXEL_NONE = 255


def voxel_blocks(domain_lo, domain_hi, vm):
    vm = np.asarray(vm, np.uint8)
    nx, ny, nz = vm.shape
    boxes = []                       # [i0, i1, j0, j1, k0, k1, m]
    last_x = {}                      # (j0, j1, k0, k1, m) -> box extended at the previous x
    for i in range(nx):
        rects = []                   # [j0, j1, k0, k1, m]
        last_y = {}                  # (k0, k1, m) -> rect
        for j in range(ny):
            col = [int(v) for v in vm[i, j]]
            k = 0
            while k < nz:
                m = col[k]
                k1 = k + 1
                while k1 < nz and col[k1] == m:
                    k1 += 1
                if m != VOXEL_NONE:
                    r = last_y.get((k, k1, m))
                    if r is not None and r[1] == j:
                        r[1] = j + 1
                    else:
                        r = [j, j + 1, k, k1, m]
                        last_y[(k, k1, m)] = r
                        rects.append(r)
                k = k1
        for r in rects:
            b = last_x.get(tuple(r))
            if b is not None and b[1] == i:
                b[1] = i + 1
            else:
                b = [i, i + 1] + r
                last_x[tuple(r)] = b
                boxes.append(b)
    boxes.sort(key=lambda b: (b[0], b[2], b[4]))
    lo, hi = np.asarray(domain_lo, np.float64), np.asarray(domain_hi, np.float64)

    def e(a, i, n):
        return float(hi[a]) if i == n else float(lo[a]) + ((float(hi[a]) - float(lo[a])) * float(i)) / float(n)

    blo = np.array([[e(0, b[0], nx), e(1, b[2], ny), e(2, b[4], nz)] for b in boxes]).reshape(-1, 3)
    bhi = np.array([[e(0, b[1], nx), e(1, b[3], ny), e(2, b[5], nz)] for b in boxes]).reshape(-1, 3)
    return blo, bhi, np.array([b[6] for b in boxes], np.int32)


def structure_blocks(s):
    """The structure's dielectric boxes in priority order: its voxel map's boxes
    (if any), then its blocks."""
    if getattr(s, "voxel_mat", None) is None:
        return s.block_lo, s.block_hi, s.block_mat
    vlo, vhi, vm = voxel_blocks(s.domain_lo, s.domain_hi, s.voxel_mat)
    return (np.ascontiguousarray(np.concatenate([vlo, s.block_lo.reshape(-1, 3)])),
            np.ascontiguousarray(np.concatenate([vhi, s.block_hi.reshape(-1, 3)])),
            np.ascontiguousarray(np.concatenate([vm, s.block_mat.astype(np.int32)])))


# ---------------------------------------------------------------------------
@dataclass
class RunResult:
    S1: np.ndarray
    S2: np.ndarray
    n: int
    omega: np.ndarray
    k: np.ndarray
    hops: np.ndarray
    steps: np.ndarray
    branch: np.ndarray
    stats: np.ndarray
    n_tables: int

    @property
    def C(self):
        return self.S1 / self.n

    @property
    def stderr(self):
        n = self.n
        v = (self.S2 - self.S1 ** 2 / n) / (n * (n - 1.0))
        return np.sqrt(np.maximum(v, 0.0))


def frw_run(s, master, n_walks, N=8, seed=0, request=0, hybrid=1, first_mode=0, gauss_frac=0.5,
            max_hops=100000, walk_begin=0, sigma_target=0.0, batch=16384, records=True, mwe=0, fdm=False):
    """Run walks ``walk_begin .. walk_begin + n_walks - 1`` of Algorithm 1 for
    ``master`` on structure ``s`` (a :class:`workloads.Structure`).  ``fdm``: the
    non-stratified transitions solve the cube's FD system (Algorithm 2, FRW-FDM)
    instead of running MicroWalk; they are counted in ``stats[4]``."""
    L = lib()
    nc = s.n_cond
    cid = None if s.cond_id is None else np.ascontiguousarray(s.cond_id, np.int32)
    if cid is not None and int((cid == master).sum()) != 1:
        raise ValueError("the master must be a single box (its Gaussian surface)")
    S1 = np.zeros(nc + 1)
    S2 = np.zeros(nc + 1)
    used = np.zeros(1, np.uint64)
    stats = np.zeros(11, np.uint64)
    n = int(n_walks)
    if records:
        om, kk, hp, st, br = (np.zeros(n), np.zeros(n, np.int32), np.zeros(n, np.uint32),
                              np.zeros(n, np.uint64), np.zeros(n, np.int32))
        rp = (_p(om, ctypes.c_double), _p(kk, ctypes.c_int32), _p(hp, ctypes.c_uint32),
              _p(st, ctypes.c_uint64), _p(br, ctypes.c_int32))
    else:
        om = kk = hp = st = br = None
        rp = (None,) * 5
    blo, bhi, bmat = structure_blocks(s)
    blo = np.ascontiguousarray(blo, np.float64)
    bhi = np.ascontiguousarray(bhi, np.float64)
    bmat = np.ascontiguousarray(bmat, np.int32)
    ntab = L.orc_frw_run(
        _p(s.domain_lo, ctypes.c_double), _p(s.domain_hi, ctypes.c_double), s.n_boxes,
        _p(s.cond_lo, ctypes.c_double), _p(s.cond_hi, ctypes.c_double), None if cid is None else _p(cid, ctypes.c_int32), nc,
        int(bmat.shape[0]),
        _p(blo, ctypes.c_double), _p(bhi, ctypes.c_double), _p(bmat, ctypes.c_int32), s.n_mat, _p(s.eps, ctypes.c_double), int(s.background),
        int(N), int(seed), int(request), int(hybrid), int(first_mode), float(gauss_frac),
        int(max_hops), int(mwe), int(bool(fdm)), int(master), int(walk_begin), n, float(sigma_target), int(batch),
        _p(S1, ctypes.c_double), _p(S2, ctypes.c_double), _p(used, ctypes.c_uint64), *rp,
        _p(stats, ctypes.c_uint64))
    u = int(used[0])
    if records:
        om, kk, hp, st, br = om[:u], kk[:u], hp[:u], st[:u], br[:u]
    return RunResult(S1, S2, u, om, kk, hp, st, br, stats, ntab)


def fdm_transitions(N, lat, eps, u):
    """FD-based transitions (Algorithm 2) of one lattice of material ids: the
    boundary node sampled from the SGF of Eq. 8 for each 32-bit word of ``u``."""
    lat = np.ascontiguousarray(lat, np.uint8).reshape(-1)
    e = np.ascontiguousarray(eps, np.float64)
    u = np.ascontiguousarray(u, np.uint32)
    nodes = np.zeros((u.size, 3), np.int32)
    lib().orc_fdm_transitions(int(N), _p(lat, ctypes.c_uint8), _p(e, ctypes.c_double), int(u.size),
                              _p(u, ctypes.c_uint32), _p(nodes, ctypes.c_int32))
    return nodes


def microwalk_e(N, lat, cond, eps, seed, request, walk, hop=1):
    """One MicroWalk-E walk (reading R8 of frw_oracle.c) on an explicit lattice with
    conductor nodes (cond >= 0).  -> (conductor reached or -1, exit node, steps)."""
    lat = np.ascontiguousarray(lat, np.uint8).ravel()
    cond = np.ascontiguousarray(cond, np.int16).ravel()
    e = np.ascontiguousarray(eps, np.float64)
    node = np.zeros(3, np.int32)
    st = np.zeros(1, np.uint64)
    c = lib().orc_microwalk_e(int(N), _p(lat, ctypes.c_uint8), _p(cond, ctypes.c_int16), _p(e, ctypes.c_double),
                              len(e), int(seed), int(request), int(walk), int(hop), _p(node, ctypes.c_int32),
                              _p(st, ctypes.c_uint64))
    return int(c), node, int(st[0])


def microwalk_e_many(N, lat, cond, eps, seed, request, walk0, n, hop=0):
    """n MicroWalk-E walks (walk ids walk0.., the given hop) -> (conductor reached or
    -1, exit nodes (n, 3), steps)."""
    lat = np.ascontiguousarray(lat, np.uint8).ravel()
    cond = np.ascontiguousarray(cond, np.int16).ravel()
    e = np.ascontiguousarray(eps, np.float64)
    co = np.zeros(n, np.int32)
    nodes = np.zeros((n, 3), np.int32)
    st = np.zeros(n, np.uint64)
    lib().orc_microwalk_e_many(int(N), _p(lat, ctypes.c_uint8), _p(cond, ctypes.c_int16), _p(e, ctypes.c_double),
                               len(e), int(seed), int(request), int(walk0), int(n), int(hop), _p(co, ctypes.c_int32),
                               _p(nodes, ctypes.c_int32), _p(st, ctypes.c_uint64))
    return co, nodes, st


# ---------------------------------------------------------------------------
def absorption_exact(N, lat, eps, quantised=True):
    """Exit distribution and expected length of MicroWalk from the absorbing chain
    (Eq. 9, Theorem 1, Eq. 11), solved with a sparse direct LU.

    The chain's one-step law is the jump law of Eq. 6: from interior node v the
    probability of neighbour i is alpha_i / sum(alpha).  With ``quantised`` the
    implemented 32-bit law is used instead: P(k) = (ceil(p_k 2^32 / S) -
    ceil(p_{k-1} 2^32 / S)) / 2^32 with p the prefix sums of the integer weights.

    Returns (P[6, N, N] in natural face order, E(tau))."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl

    lat = np.asarray(lat).reshape(N, N, N)
    eps = np.asarray(eps, np.float64)
    n = N ** 3
    W = w_table(eps).astype(np.float64) if quantised else None

    def idx(i, j, k):
        return (i * N + j) * N + k

    def panel(a, side, x):
        o = [b for b in range(3) if b != a]
        return ((2 * a + side) * N + x[o[0]]) * N + x[o[1]]

    rows, cols, vals = [], [], []
    brow, bcol, bval = [], [], []
    for i in range(N):
        for j in range(N):
            for k in range(N):
                v = idx(i, j, k)
                mv = int(lat[i, j, k])
                wts, dests = [], []
                for kk in range(6):
                    a, d = kk >> 1, (1 if kk & 1 else -1)
                    x = [i, j, k]
                    x[a] += d
                    if x[a] < 0 or x[a] >= N:
                        w = W[mv, BOUNDARY] if quantised else 1.0
                        dests.append(("b", panel(a, 0 if x[a] < 0 else 1, x)))
                    else:
                        mi = int(lat[x[0], x[1], x[2]])
                        w = W[mv, mi] if quantised else eps[mi] / (eps[mi] + eps[mv])
                        dests.append(("i", idx(*x)))
                    wts.append(w)
                wts = np.asarray(wts)
                if quantised:
                    S = int(wts.sum())
                    pre = np.cumsum(wts.astype(np.int64))
                    ce = [-(-int(p) * 2 ** 32 // S) for p in pre]
                    prob = np.diff(np.concatenate([[0], ce])) / 2.0 ** 32
                else:
                    prob = wts / wts.sum()
                rows.append(v)
                cols.append(v)
                vals.append(1.0)
                for (kind, dst), pr in zip(dests, prob):
                    if kind == "i":
                        rows.append(v)
                        cols.append(dst)
                        vals.append(-pr)
                    else:
                        brow.append(v)
                        bcol.append(dst)
                        bval.append(pr)
    A = sp.csc_matrix((vals, (rows, cols)), shape=(n, n))
    B = sp.csr_matrix((bval, (brow, bcol)), shape=(n, 6 * N * N))
    ec = np.zeros(n)
    for i in (N // 2 - 1, N // 2):
        for j in (N // 2 - 1, N // 2):
            for k in (N // 2 - 1, N // 2):
                ec[idx(i, j, k)] = 0.125
    lu = spl.splu(A.T.tocsc())
    y = lu.solve(ec)           # y^T = e_c^T (I - Q_TT)^{-1}
    P = B.T @ y
    Etau = float(y.sum())
    return P.reshape(6, N, N), Etau


def absorption_exact_e(N, lat, cond, eps):
    """MicroWalk-E's exact absorbing chain (reading R8): dielectric voxels are the
    transient states; a step leaves the lattice (boundary panel) or lands on a
    conductor voxel (absorbed there), both with weight alpha = 1; the quantised
    32-bit law as in :func:`absorption_exact`.

    Returns (P[6, N, N] exit probabilities per boundary panel, Q[c] absorption
    probability per conductor id, E(tau))."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl

    lat = np.asarray(lat).reshape(N, N, N)
    cond = np.asarray(cond).reshape(N, N, N)
    W = w_table(np.asarray(eps, np.float64)).astype(np.int64)
    diel = cond < 0
    ids = -np.ones((N, N, N), np.int64)
    ids[diel] = np.arange(int(diel.sum()))
    n = int(diel.sum())
    nc = int(cond.max()) + 1 if (cond >= 0).any() else 0

    def panel(a, side, x):
        o = [b for b in range(3) if b != a]
        return ((2 * a + side) * N + x[o[0]]) * N + x[o[1]]

    rows, cols, vals = [], [], []
    brow, bcol, bval = [], [], []
    crow, ccol, cval = [], [], []
    for i in range(N):
        for j in range(N):
            for k in range(N):
                if not diel[i, j, k]:
                    continue
                v = int(ids[i, j, k])
                mv = int(lat[i, j, k])
                wts, dests = [], []
                for kk in range(6):
                    a, d = kk >> 1, (1 if kk & 1 else -1)
                    x = [i, j, k]
                    x[a] += d
                    if x[a] < 0 or x[a] >= N:
                        wts.append(W[mv, BOUNDARY])
                        dests.append(("b", panel(a, 0 if x[a] < 0 else 1, x)))
                    elif cond[x[0], x[1], x[2]] >= 0:
                        wts.append(W[mv, BOUNDARY])
                        dests.append(("c", int(cond[x[0], x[1], x[2]])))
                    else:
                        wts.append(W[mv, int(lat[x[0], x[1], x[2]])])
                        dests.append(("i", int(ids[x[0], x[1], x[2]])))
                S = int(sum(wts))
                pre = np.cumsum(np.asarray(wts, np.int64))
                ce = [-(-int(p) * 2 ** 32 // S) for p in pre]
                prob = np.diff(np.concatenate([[0], ce])) / 2.0 ** 32
                rows.append(v)
                cols.append(v)
                vals.append(1.0)
                for (kind, dst), pr in zip(dests, prob):
                    if kind == "i":
                        rows.append(v)
                        cols.append(dst)
                        vals.append(-pr)
                    elif kind == "b":
                        brow.append(v)
                        bcol.append(dst)
                        bval.append(pr)
                    else:
                        crow.append(v)
                        ccol.append(dst)
                        cval.append(pr)
    A = sp.csc_matrix((vals, (rows, cols)), shape=(n, n))
    B = sp.csr_matrix((bval, (brow, bcol)), shape=(n, 6 * N * N))
    Cm = sp.csr_matrix((cval, (crow, ccol)), shape=(n, max(nc, 1)))
    ec = np.zeros(n)
    for i in (N // 2 - 1, N // 2):
        for j in (N // 2 - 1, N // 2):
            for k in (N // 2 - 1, N // 2):
                ec[ids[i, j, k]] += 0.125
    y = spl.splu(A.T.tocsc()).solve(ec)
    return (B.T @ y).reshape(6, N, N), np.asarray(Cm.T @ y).ravel()[:nc], float(y.sum())
