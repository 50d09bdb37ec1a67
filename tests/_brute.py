"""Brute-force dense constructions used to pin the oracle on tiny grids.

These build the finite-element matrices from the *global* hat functions
phi_i(x) = prod_k max(0, 1 - |x_k - x_ik| / h) and Gauss quadrature over every
cell, and the d-linear prolongation by evaluating the coarse hats at the fine
vertices.  They use no element matrix, stencil or weight table of the oracle,
so agreement with the oracle is evidence from a second route.
"""
from __future__ import annotations

import itertools

import numpy as np


def vertex_positions(d: int, n: int) -> np.ndarray:
    """(N_all, d) positions of all vertices, C order (last axis fastest)."""
    g = np.meshgrid(*([np.arange(n + 1) / n] * d), indexing="ij")
    return np.stack([x.ravel() for x in g], axis=1)


def interior_mask(d: int, n: int) -> np.ndarray:
    idx = np.indices((n + 1,) * d).reshape(d, -1).T
    return np.all((idx > 0) & (idx < n), axis=1)


def hat_and_grad(pos: np.ndarray, x: np.ndarray, h: float):
    """Values and gradients of all global hats (rows of pos) at point x."""
    t = (x[None, :] - pos) / h
    psi = np.maximum(0.0, 1.0 - np.abs(t))
    dpsi = np.where(np.abs(t) < 1.0, -np.sign(t), 0.0) / h
    val = np.prod(psi, axis=1)
    d = pos.shape[1]
    grad = np.empty_like(pos)
    for k in range(d):
        others = np.prod(np.delete(psi, k, axis=1), axis=1) if d > 1 else 1.0
        grad[:, k] = dpsi[:, k] * others
    return val, grad


def stiffness_dense(d: int, n: int, eps_cells) -> np.ndarray:
    """A[i, j] = sum_cells eps_c int_c grad phi_i . grad phi_j over ALL vertices
    (boundary rows included); 2-point Gauss per direction is exact here."""
    h = 1.0 / n
    pos = vertex_positions(d, n)
    eps = np.broadcast_to(np.asarray(eps_cells, dtype=float), (n,) * d)
    g, w = np.polynomial.legendre.leggauss(2)
    g = 0.5 * (g + 1.0)
    w = 0.5 * w
    A = np.zeros((len(pos), len(pos)))
    for cell in itertools.product(range(n), repeat=d):
        for q in itertools.product(range(2), repeat=d):
            x = (np.array(cell) + np.array([g[k] for k in q])) * h
            wq = np.prod([w[k] for k in q]) * h ** d
            _, grad = hat_and_grad(pos, x, h)
            nz = np.nonzero(np.any(grad != 0.0, axis=1))[0]
            G = grad[nz]
            A[np.ix_(nz, nz)] += eps[cell] * wq * (G @ G.T)
    return A


def dlinear_prolongation_dense(d: int, n_c: int) -> np.ndarray:
    """P[i, J] = phi^coarse_J(x_i) over all fine/coarse vertices."""
    n_f = 3 * n_c
    pf = vertex_positions(d, n_f)
    pc = vertex_positions(d, n_c)
    H = 1.0 / n_c
    t = np.abs(pf[:, None, :] - pc[None, :, :]) / H
    return np.prod(np.maximum(0.0, 1.0 - t), axis=2)


def interior_block(M: np.ndarray, rows_mask, cols_mask) -> np.ndarray:
    return M[np.ix_(rows_mask, cols_mask)]


# ---------------------------------------------------------------------------
# adaptive trees: the nodal space over the leaf cells, from the global hats

def leaf_cells(tree):
    """(level, cell index tuple) of every leaf cell of a tree given by its
    per-level ``exists`` / ``refined`` flags."""
    out = []
    for l in range(1, tree.L + 1):
        leaf = tree.exists[l] & ~tree.refined[l]
        out += [(l, tuple(c)) for c in np.argwhere(leaf)]
    return out


def hats_and_grads(pos: np.ndarray, widths: np.ndarray, x: np.ndarray):
    """Values and gradients at x of the hats centred at pos (rows) with the
    given widths (one per row)."""
    t = (x[None, :] - pos) / widths[:, None]
    psi = np.maximum(0.0, 1.0 - np.abs(t))
    dpsi = np.where(np.abs(t) < 1.0, -np.sign(t), 0.0) / widths[:, None]
    d = pos.shape[1]
    grad = np.empty_like(pos)
    for k in range(d):
        others = np.prod(np.delete(psi, k, axis=1), axis=1) if d > 1 else 1.0
        grad[:, k] = dpsi[:, k] * others
    return np.prod(psi, axis=1), grad


def adaptive_system_dense(tree, eps_fine, f_fn, pos: np.ndarray, widths: np.ndarray):
    """A[i, j] = sum over leaf cells c of eps_c int_c grad phi_i . grad phi_j and
    the lumped load b_i = sum_c |c| / 2^d sum_{corners x} f(x) phi_i(x), for the
    hats phi_i of the given positions and widths (positions in [0,1]^d, array
    axis order).  eps of a leaf cell: the mean of the fine cells it covers.
    2-point Gauss per direction is exact: every hat is d-linear on every leaf
    cell."""
    d = tree.d
    g, w = np.polynomial.legendre.leggauss(2)
    g = 0.5 * (g + 1.0)
    w = 0.5 * w
    A = np.zeros((len(pos), len(pos)))
    b = np.zeros(len(pos))
    for l, cell in leaf_cells(tree):
        h = 1.0 / 3 ** l
        s = 3 ** (tree.L - l)
        e = float(np.mean(eps_fine[tuple(slice(s * c, s * c + s) for c in cell)])) \
            if np.ndim(eps_fine) else float(eps_fine)
        lo = np.array(cell) * h
        for q in itertools.product(range(2), repeat=d):
            x = lo + np.array([g[k] for k in q]) * h
            wq = np.prod([w[k] for k in q]) * h ** d
            _, grad = hats_and_grads(pos, widths, x)
            nz = np.nonzero(np.any(grad != 0.0, axis=1))[0]
            G = grad[nz]
            A[np.ix_(nz, nz)] += e * wq * (G @ G.T)
        for corner in itertools.product((0, 1), repeat=d):
            x = lo + np.array(corner) * h
            val, _ = hats_and_grads(pos, widths, x)
            b += (h ** d / 2 ** d) * f_fn(x) * val
    return A, b
