"""d-linear finite elements on one level of a regular 3:1 spacetree.

Oracle (test infrastructure only).  Follows the discretisation of Section 2.1
of the paper: every vertex surrounded by 2^d cells of its level carries a
d-linear "pagoda" shape function; testing against shape functions of the same
level gives compact 3^d stencils; boundary vertices carry no test function
(Dirichlet data, here zero).  The PDE is -div(eps grad u) = f (Eq. 1) with eps
constant per fine cell.

Conventions: vertex arrays have shape (n+1,)*d (last axis = x), cell arrays
shape (n,)*d.  A cell corner is a tuple b in {0,1}^d in numpy-axis order; the
list ``corners(d)`` is ordered with the last axis running fastest, so that the
flat corner index is sum_j b_j 2^j with j = 0 for x.  Stencil offsets
``offsets(d)`` in {-1,0,1}^d are ordered the same way (flat index
sum_j (o_j+1) 3^j, centre = (3^d-1)/2).
"""
from __future__ import annotations

import itertools

import numpy as np


def corners(d: int):
    return list(itertools.product((0, 1), repeat=d))


def offsets(d: int, radius: int = 1):
    return list(itertools.product(range(-radius, radius + 1), repeat=d))


def reference_element_matrix(d: int) -> np.ndarray:
    """K_ref[a, b] = integral over the unit cell of grad(phi_a) . grad(phi_b)
    for the d-linear shape functions phi_b(xi) = prod_k (b_k xi_k + (1-b_k)(1-xi_k)).

    The integrand is a polynomial of degree <= 2 in every variable, so 2-point
    Gauss-Legendre quadrature per dimension is exact.  On a cell of width h the
    matrix scales to h^(d-2) K_ref (Sec. 2.1: d-linear FEM on a Cartesian cell).
    """
    g, w = np.polynomial.legendre.leggauss(2)
    g = 0.5 * (g + 1.0)
    w = 0.5 * w
    cs = corners(d)
    K = np.zeros((len(cs), len(cs)))
    for q in itertools.product(range(2), repeat=d):
        xi = [g[qi] for qi in q]
        wq = np.prod([w[qi] for qi in q])
        grads = []
        for b in cs:
            gb = []
            for k in range(d):
                comp = 1.0 if b[k] else -1.0
                for m in range(d):
                    if m != k:
                        comp *= xi[m] if b[m] else 1.0 - xi[m]
                gb.append(comp)
            grads.append(np.array(gb))
        for a in range(len(cs)):
            for bb in range(len(cs)):
                K[a, bb] += wq * grads[a].dot(grads[bb])
    return K


def _vslice(b, n):
    """Slices that pick, for every cell, its corner vertex ``cell + b``."""
    return tuple(slice(bk, bk + n) for bk in b)


def zero_boundary(a: np.ndarray) -> np.ndarray:
    for ax in range(a.ndim):
        idx = [slice(None)] * a.ndim
        idx[ax] = 0
        a[tuple(idx)] = 0.0
        idx[ax] = -1
        a[tuple(idx)] = 0.0
    return a


def interior(a: np.ndarray) -> np.ndarray:
    return a[tuple(slice(1, -1) for _ in range(a.ndim))]


class LevelOperator:
    """The stiffness operator of one level, stored element-wise.

    Either ``eps`` (per-cell scalar, fine level: K_e = eps_e h^(d-2) K_ref) or
    ``Kc`` (per-cell 2^d x 2^d matrices, Galerkin coarse levels).  The operator
    is applied matrix-free by accumulating element-wise mat-vecs into the
    vertices (Sec. 4.2 of the paper); only interior rows are kept.
    """

    def __init__(self, d: int, n: int, eps=None, Kc=None):
        self.d, self.n = d, n
        self.h = 1.0 / n
        self.eps = eps
        self.Kc = Kc
        if (eps is None) == (Kc is None):
            raise ValueError("exactly one of eps, Kc")
        self.Kref = reference_element_matrix(d) * self.h ** (d - 2)

    @staticmethod
    def from_eps(d: int, n: int, eps, eps_is_scalar: bool):
        e = np.asarray(eps, dtype=np.float64)
        if eps_is_scalar:
            e = np.full((n,) * d, float(e.reshape(-1)[0]))
        if e.shape != (n,) * d:
            raise ValueError(f"eps must have shape {(n,) * d}")
        return LevelOperator(d, n, eps=e)

    def cell_matrix(self, a: int, b: int) -> np.ndarray:
        """Entry (a, b) of every cell's element matrix, as a cell array."""
        if self.Kc is not None:
            return self.Kc[..., a, b]
        return self.eps * self.Kref[a, b]

    def element_matrices(self) -> np.ndarray:
        if self.Kc is not None:
            return self.Kc
        return self.eps[..., None, None] * self.Kref

    def apply(self, u: np.ndarray) -> np.ndarray:
        """(A u) at every vertex; boundary rows are set to zero."""
        cs = corners(self.d)
        out = np.zeros_like(u)
        for ia, a in enumerate(cs):
            sa = _vslice(a, self.n)
            for ib, b in enumerate(cs):
                out[sa] += self.cell_matrix(ia, ib) * u[_vslice(b, self.n)]
        return zero_boundary(out)

    def stencils(self) -> np.ndarray:
        """Assembled 3^d stencil of every vertex, shape (n+1,)*d + (3^d,).

        Entry o of vertex i is A[i, i+o] = sum over the cells e that contain both
        i (as corner a) and i+o (as corner a+o) of K_e[a, a+o].  Rows of boundary
        vertices contain the partial sums of their existing cells.
        """
        d, n = self.d, self.n
        cs = corners(d)
        cidx = {c: k for k, c in enumerate(cs)}
        offs = offsets(d)
        st = np.zeros((n + 1,) * d + (len(offs),))
        for ia, a in enumerate(cs):
            sa = _vslice(a, n)
            for so, o in enumerate(offs):
                b = tuple(ak + ok for ak, ok in zip(a, o))
                if b not in cidx:
                    continue
                st[sa + (so,)] += self.cell_matrix(ia, cidx[b])
        return st

    def diagonal(self) -> np.ndarray:
        cs = corners(self.d)
        dg = np.zeros((self.n + 1,) * self.d)
        for ia, a in enumerate(cs):
            dg[_vslice(a, self.n)] += self.cell_matrix(ia, ia)
        return dg


def load_vector(f: np.ndarray, h: float, d: int) -> np.ndarray:
    """Lumped load b_i = h^d f(x_i) at interior vertices, zero on the boundary.

    The paper does not state its right-hand side discretisation; this is the
    lumped-mass reading (exact row sums of the d-linear mass matrix)."""
    b = (h ** d) * np.asarray(f, dtype=np.float64).copy()
    return zero_boundary(b)
