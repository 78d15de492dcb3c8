"""Whole-structure finite-difference capacitance solver: an independent check of
the random-walk estimator (test infrastructure only).

It solves Laplace's equation with piecewise-constant permittivity (Eq. 1) on a
uniform cell-centred grid over the whole domain, with the interface rule of the
paper's difference schemes (Eq. 4 and Eq. 5): between two cells of permittivity
eps_p and eps_q the face coupling is 2 eps_p eps_q / (eps_p + eps_q) (the two
half-cells in series), and between a cell and a boundary face (a conductor
surface or a grounded wall, both on cell faces) it is 2 eps_p.  The master
conductor is held at 1 V and every other conductor and the walls at 0 V; the
charge on conductor k is eps0 times the flux leaving its surface (Gauss's law,
Sec. II-A), which is C_{master,k}.

Plain numpy / scipy: a sparse matrix and a Jacobi-preconditioned conjugate
gradient solve, nothing shared with the random-walk code.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as sla

EPS0 = 8.8541878128e-3   # vacuum permittivity in fF/um


def capacitance_row(s, master: int, h: float, rtol: float = 1e-11, energy: bool = False):
    """C_{master,k} for k = 0..n_cond-1 (fF) on a grid of spacing h (um).

    Every box face of the structure must lie on a grid plane, and no two
    conductors may touch (both are checked).  With ``energy`` also returns
    eps0 * sum over faces of coupling * h * (potential jump)^2, the discrete
    field energy times 2, which equals C_{master,master} at 1 V."""
    lo = np.asarray(s.domain_lo, float)
    hi = np.asarray(s.domain_hi, float)
    n = np.rint((hi - lo) / h).astype(int)
    if not np.allclose(n * h, hi - lo):
        raise ValueError("the domain is not a whole number of cells")
    for boxes in (s.cond_lo, s.cond_hi, s.block_lo, s.block_hi):
        for b in np.asarray(boxes, float).reshape(-1, 3):
            t = (b - lo) / h
            if not np.allclose(t, np.rint(t)):
                raise ValueError("a box face is not on a grid plane")
    centres = [lo[a] + (np.arange(n[a]) + 0.5) * h for a in range(3)]
    P = np.meshgrid(*centres, indexing="ij")

    def inside(blo, bhi):
        m = np.ones(P[0].shape, bool)
        for a in range(3):
            m &= (P[a] >= blo[a]) & (P[a] < bhi[a])
        return m

    eps = np.full(P[0].shape, float(s.eps[s.background]))
    for b in range(s.n_blocks):                     # later blocks win
        eps[inside(s.block_lo[b], s.block_hi[b])] = s.eps[s.block_mat[b]]
    cond = np.full(P[0].shape, -1)
    cid = np.arange(s.n_boxes) if s.cond_id is None else s.cond_id
    for b in range(s.n_boxes):                  # a conductor is the union of its boxes
        cond[inside(s.cond_lo[b], s.cond_hi[b])] = cid[b]
    free = cond < 0
    idx = np.full(P[0].shape, -1)
    idx[free] = np.arange(int(free.sum()))
    nu = int(free.sum())
    v = np.zeros(s.n_cond)
    v[master] = 1.0

    diag = np.zeros(nu)
    rhs = np.zeros(nu)
    rows, cols, vals = [], [], []

    def pairs(a):
        sp_ = [slice(None)] * 3
        sq_ = [slice(None)] * 3
        sp_[a] = slice(0, n[a] - 1)
        sq_[a] = slice(1, n[a])
        return tuple(sp_), tuple(sq_)

    for a in range(3):
        p, q = pairs(a)
        ep, eq = eps[p], eps[q]
        cp, cq = cond[p], cond[q]
        ip, iq = idx[p], idx[q]
        if ((cp >= 0) & (cq >= 0) & (cp != cq)).any():
            raise ValueError("two conductors touch")
        m = (cp < 0) & (cq < 0)                     # cell - cell (Eq. 4)
        g = 2.0 * ep[m] * eq[m] / (ep[m] + eq[m])
        np.add.at(diag, ip[m], g)
        np.add.at(diag, iq[m], g)
        rows += [ip[m], iq[m]]
        cols += [iq[m], ip[m]]
        vals += [-g, -g]
        for fm, fi, fe, ck in (((cp < 0) & (cq >= 0), ip, ep, cq), ((cq < 0) & (cp >= 0), iq, eq, cp)):
            g = 2.0 * fe[fm]                        # cell - conductor face (Eq. 5)
            np.add.at(diag, fi[fm], g)
            np.add.at(rhs, fi[fm], g * v[ck[fm]])
        for side in (0, n[a] - 1):                  # cell - grounded wall (Eq. 5)
            sl = [slice(None)] * 3
            sl[a] = side
            c, e, i = cond[tuple(sl)], eps[tuple(sl)], idx[tuple(sl)]
            if (c >= 0).any():
                raise ValueError("a conductor touches a wall")
            np.add.at(diag, i, 2.0 * e)

    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(nu, nu))
    A = A + sp.diags(diag)
    phi, info = sla.cg(A, rhs, rtol=rtol, maxiter=100000, M=sp.diags(1.0 / diag))
    if info != 0:
        raise RuntimeError("conjugate gradient did not converge")
    full = np.zeros(P[0].shape)
    full[free] = phi
    for k in range(s.n_cond):
        full[cond == k] = v[k]

    Q = np.zeros(s.n_cond)
    U = 0.0
    for a in range(3):
        p, q = pairs(a)
        cp, cq = cond[p], cond[q]
        ep, eq = eps[p], eps[q]
        fp, fq = full[p], full[q]
        m = (cp < 0) & (cq < 0)
        U += float(np.sum(2.0 * ep[m] * eq[m] / (ep[m] + eq[m]) * h * (fp[m] - fq[m]) ** 2))
        m = (cp < 0) != (cq < 0)
        e_free = np.where(cp < 0, ep, eq)[m]
        U += float(np.sum(2.0 * e_free * h * (fp[m] - fq[m]) ** 2))
        for side in (0, n[a] - 1):
            sl = [slice(None)] * 3
            sl[a] = side
            U += float(np.sum(2.0 * eps[tuple(sl)] * h * full[tuple(sl)] ** 2))
        m = (cp >= 0) & (cq < 0)
        np.add.at(Q, cp[m], 2.0 * eq[m] * h * (fp[m] - fq[m]))
        m = (cq >= 0) & (cp < 0)
        np.add.at(Q, cq[m], 2.0 * ep[m] * h * (fq[m] - fp[m]))
    if energy:
        return EPS0 * Q, EPS0 * U
    return EPS0 * Q
