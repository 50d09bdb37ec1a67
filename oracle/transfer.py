"""Inter-grid transfer operators between levels l-1 (coarse) and l (fine).

Oracle (test infrastructure only).

* d-linear prolongation for 3:1 refinement: the coarse nodal function is
  evaluated at the fine vertices (Sec. 2.2, Sec. 3.2 "P is d-linear").
* BoxMG operator-dependent prolongation (Sec. 2.4): identity on c-points,
  solutions of the collapsed (lumped along the face normal) stencil equations
  on gamma-points, and of the full stencil equations on f-points; one solve
  per coarse cell and per coarse vertex e (the characteristic vector).
* Restriction R = P^T (no scaling, Ritz-Galerkin consistency, Sec. 2.2).
* Injection I: a coarse vertex takes the value of the coinciding fine vertex
  (FAS, Sec. 2.3).
* Galerkin coarse operator A_{l-1} = R A_l P (Sec. 2.2).

A coarse cell E (lower corner at fine index 3E) owns the (3+1)^d fine vertices
of its closure, local coordinates l in {0,1,2,3}^d.  The "closure weights"
W[E, l, e] are the values of P e on those vertices for the 2^d corners e of E.
Fine vertices are stored once: vertex i belongs to the coarse cell
I = min(floor(i/3), n_c - 1) (per axis) and keeps its 2^d weights towards the
corners of that cell ("vertex weights", shape (n_f+1,)*d + (2^d,)).

Dirichlet boundary (a reading of Sec. 2.1, boundary vertices carry no test
function and no unknown): weights of fine boundary vertices and weights towards
coarse boundary vertices are zero; BoxMG treats boundary points as known
zeros.
"""
from __future__ import annotations

import itertools

import numpy as np

from .fem import LevelOperator, corners, offsets


def closure_points(d: int):
    return list(itertools.product(range(4), repeat=d))


def _cell_index(n_c: int, d: int):
    return np.indices((n_c,) * d)


def _mask_boundary(W: np.ndarray, n_c: int) -> np.ndarray:
    """Zero weights of fine boundary vertices and towards coarse boundary vertices."""
    d = W.ndim - 2
    ci = _cell_index(n_c, d)
    for k, l in enumerate(closure_points(d)):
        fb = np.zeros((n_c,) * d, dtype=bool)
        for a in range(d):
            if l[a] == 0:
                fb |= ci[a] == 0
            elif l[a] == 3:
                fb |= ci[a] == n_c - 1
        W[..., k, :][fb] = 0.0
    for ie, e in enumerate(corners(d)):
        cb = np.zeros((n_c,) * d, dtype=bool)
        for a in range(d):
            cb |= (ci[a] + e[a] == 0) | (ci[a] + e[a] == n_c)
        W[..., ie][cb] = 0.0
    return W


def dlinear_closure_weights(d: int, n_c: int) -> np.ndarray:
    """W[E, l, e] = prod_k (l_k/3 if e_k else 1 - l_k/3): the coarse d-linear
    hat of corner e evaluated at the fine vertex 3E + l."""
    pts = closure_points(d)
    cs = corners(d)
    w = np.zeros((len(pts), len(cs)))
    for k, l in enumerate(pts):
        for ie, e in enumerate(cs):
            val = 1.0
            for a in range(d):
                val *= l[a] / 3.0 if e[a] else 1.0 - l[a] / 3.0
            w[k, ie] = val
    W = np.broadcast_to(w, (n_c,) * d + w.shape).copy()
    return _mask_boundary(W, n_c)


def boxmg_closure_weights(stencils: np.ndarray, n_c: int) -> np.ndarray:
    """BoxMG prolongation (Sec. 2.4) for 3:1 coarsening.

    ``stencils`` are the assembled 3^d stencils of the fine level (shape
    (3 n_c + 1,)*d + (3^d,)).  For every coarse cell and corner e:
      1. c-points: 1 at the corner e, 0 at the other corners;
      2. gamma-points on sub-faces with |F| free directions, |F| = 1 .. d-1 in
         increasing order (edges, then faces in 3-D): the stencil is lumped
         along the normal directions and A~ P e = 0 is solved on the 2^|F|
         points of the sub-face with its rim (already known) as data;
      3. f-points (|F| = d): A P e = 0 on the 2^d interior points.
    Sub-faces on the domain boundary hold zeros.
    """
    d = stencils.ndim - 1
    pts = closure_points(d)
    pidx = {l: k for k, l in enumerate(pts)}
    offs = offsets(d)
    oidx = {o: s for s, o in enumerate(offs)}
    cshape = (n_c,) * d
    ci = _cell_index(n_c, d)
    Sc = np.empty(cshape + (len(pts), len(offs)))
    for k, l in enumerate(pts):
        Sc[..., k, :] = stencils[tuple(slice(lk, lk + 3 * n_c, 3) for lk in l)]
    cs = corners(d)
    W = np.zeros(cshape + (len(pts), len(cs)))
    for ie, e in enumerate(cs):
        v = np.zeros(cshape + (len(pts),))
        v[..., pidx[tuple(3 * ek for ek in e)]] = 1.0
        for nfree in range(1, d + 1):
            for F in itertools.combinations(range(d), nfree):
                B = [a for a in range(d) if a not in F]
                for fixed in itertools.product((0, 3), repeat=len(B)):
                    unk = []
                    for free in itertools.product((1, 2), repeat=nfree):
                        l = [0] * d
                        for a, val in zip(F, free):
                            l[a] = val
                        for a, val in zip(B, fixed):
                            l[a] = val
                        unk.append(tuple(l))
                    m = len(unk)
                    M = np.zeros(cshape + (m, m))
                    rhs = np.zeros(cshape + (m,))
                    for p, lp in enumerate(unk):
                        for oF in itertools.product((-1, 0, 1), repeat=nfree):
                            coef = np.zeros(cshape)
                            for oB in itertools.product((-1, 0, 1), repeat=len(B)):
                                o = [0] * d
                                for a, val in zip(F, oF):
                                    o[a] = val
                                for a, val in zip(B, oB):
                                    o[a] = val
                                coef = coef + Sc[..., pidx[lp], oidx[tuple(o)]]
                            q = list(lp)
                            for a, val in zip(F, oF):
                                q[a] += val
                            q = tuple(q)
                            if q in unk:
                                M[..., p, unk.index(q)] += coef
                            else:
                                rhs[..., p] -= coef * v[..., pidx[q]]
                    on_bnd = np.zeros(cshape, dtype=bool)
                    for a, val in zip(B, fixed):
                        on_bnd |= (ci[a] == 0) if val == 0 else (ci[a] == n_c - 1)
                    M[on_bnd] = np.eye(m)
                    rhs[on_bnd] = 0.0
                    sol = np.linalg.solve(M, rhs[..., None])[..., 0]
                    for p, lp in enumerate(unk):
                        v[..., pidx[lp]] = sol[..., p]
        W[..., ie] = v
    return _mask_boundary(W, n_c)


def vertex_weights(W: np.ndarray, n_c: int) -> np.ndarray:
    """Per-fine-vertex storage of P: weights towards the corners of the owning
    coarse cell I = min(floor(i/3), n_c-1)."""
    d = W.ndim - 2
    n_f = 3 * n_c
    Pv = np.zeros((n_f + 1,) * d + (2 ** d,))
    for k, l in enumerate(closure_points(d)):
        vsl, csl = [], []
        for a in range(d):
            if l[a] < 3:
                vsl.append(slice(l[a], l[a] + 3 * n_c, 3))
                csl.append(slice(None))
            else:
                vsl.append(slice(n_f, n_f + 1))
                csl.append(slice(n_c - 1, n_c))
        Pv[tuple(vsl)] = W[tuple(csl) + (k,)]
    return Pv


def _owner(n_f: int, n_c: int) -> np.ndarray:
    return np.minimum(np.arange(n_f + 1) // 3, n_c - 1)


def prolong(Pv: np.ndarray, uc: np.ndarray) -> np.ndarray:
    """u_f = P u_c: u_f[i] = sum_e Pv[i, e] u_c[I(i) + e]."""
    d = uc.ndim
    n_c = uc.shape[0] - 1
    n_f = 3 * n_c
    own = _owner(n_f, n_c)
    uf = np.zeros((n_f + 1,) * d)
    for ie, e in enumerate(corners(d)):
        uf += Pv[..., ie] * uc[np.ix_(*[own + e[a] for a in range(d)])]
    return uf


def restrict(Pv: np.ndarray, rf: np.ndarray) -> np.ndarray:
    """r_c = P^T r_f: every fine vertex adds Pv[i, e] r_f[i] to u_c[I(i) + e]."""
    d = rf.ndim
    n_f = rf.shape[0] - 1
    n_c = n_f // 3
    own = _owner(n_f, n_c)
    shape_c = (n_c + 1,) * d
    rc = np.zeros(int(np.prod(shape_c)))
    for ie, e in enumerate(corners(d)):
        tgt = np.ravel_multi_index(np.ix_(*[own + e[a] for a in range(d)]), shape_c)
        tgt = np.broadcast_to(tgt, rf.shape)
        rc += np.bincount(tgt.ravel(), weights=(Pv[..., ie] * rf).ravel(),
                          minlength=rc.size)
    return rc.reshape(shape_c)


def inject(uf: np.ndarray) -> np.ndarray:
    """u_c = I u_f: the coarse vertex J takes the fine value at 3J."""
    return uf[tuple(slice(None, None, 3) for _ in range(uf.ndim))].copy()


def galerkin(op: LevelOperator, W: np.ndarray, n_c: int) -> LevelOperator:
    """A_{l-1} = P^T A_l P, formed cell by cell.

    Every fine vertex in the closure of coarse cell E has weights only towards
    the corners of E (d-linear: tensor-product hat; BoxMG: gamma-points only
    see the corners of their sub-face), so the coarse element matrix is
    K_E = sum over the 3^d children c of E of P_c^T K_c P_c, with P_c[b, e] =
    W[E, k_c + b, e] for the child at local offset k_c.  Boundary rows and
    columns of P are zero, so the assembled coarse operator equals the
    interior block of R A P."""
    d = op.d
    pts = closure_points(d)
    pidx = {l: k for k, l in enumerate(pts)}
    cs = corners(d)
    Kc = np.zeros((n_c,) * d + (len(cs), len(cs)))
    for k in itertools.product(range(3), repeat=d):
        sl = tuple(slice(ka, ka + 3 * n_c, 3) for ka in k)
        if op.Kc is not None:
            Kk = op.Kc[sl]
        else:
            Kk = op.eps[sl][..., None, None] * op.Kref
        rows = [pidx[tuple(ka + ba for ka, ba in zip(k, b))] for b in cs]
        Pk = W[..., rows, :]
        Kc += np.einsum("...be,...bc,...cf->...ef", Pk, Kk, Pk, optimize=True)
    return LevelOperator(d, n_c, Kc=Kc)
