"""The additive cycles on an adaptive 3:1 spacetree (regular or ragged levels).

Oracle (test infrastructure only).  Follows Sec. 2.1 of the paper: cells of
level l are cut into 3^d children where the tree refines; a vertex of level l
that is surrounded by 2^d cells of its level carries a d-linear pagoda, the
others are hanging (or boundary) vertices and carry no test function.  The
shape functions of all levels form a hierarchical generating system over the
adaptive grid; the nodal space over the adaptive grid (the composite space
V_h) consists of the functions that are continuous and d-linear on every leaf
cell, and the pagoda of every level's active vertex lies in it.

Every function is held by its values at the leaf nodes (all corners of leaf
cells, hanging positions included), so
  * the bilinear form is the sum of the leaf cells' element matrices,
    a(u, v) = v^T K u (Sec. 2.1: eps_c h^(d-2) K_ref per cell);
  * the load is lumped per leaf cell (the reading of the regular oracle:
    every corner of a cell of width h takes h^d / 2^d f(x));
  * the level-l pagodas are the columns of Phi_l (their values at the leaf
    nodes), and the residual that level l sees is r_l = Phi_l^T (b - K u),
    the residual of the composite problem tested with level l's shape
    functions.  On a fully refined tree Phi_l = P^(L-l) and r_l = R^(L-l) r_L
    (Alg. 1).  fas_level_residuals restates the level-wise FAS/HTMG form of
    Eq. 4 on the spacetree (injection, hierarchical values, Galerkin element
    matrices, cell by cell); the tests check that both give the same r_l.
The level operator of level l is A_l = Phi_l^T K Phi_l (Ritz-Galerkin over
the generating system, Sec. 2.2) and M_l = diag(A_l).

The cycle is Eq. 9 on the generating system: every level takes a damped
Jacobi step on its residual, the damping equation of level l-1 takes the
smoothed restriction of level l's residual (Eq. 8), and
  u += sum_l Phi_l c_l - sum_{l >= 2} Phi_{l-1} c~_{l-1}.

Readings for the adaptive tree (the paper leaves them open):
  * the smoothed restriction's window on level l covers only the level's
    active vertices: residuals at hanging or absent positions count as zero;
  * the exact R~ of level l is omega Phi_{l-1}^T K Phi_l M_l^-1 r_l (R A_l
    with A_l and R taken over the generating system);
  * eps of a leaf cell coarser than the given fine eps is the mean of the
    fine cells it covers;
  * the residual norm of Eq. 10 runs over the vertices of the nodal space
    (every free position once, on the finest level where it is active), with
    h_i the spacing of that level.
"""
from __future__ import annotations

import dataclasses
import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import cycle as rc
from .fem import corners, reference_element_matrix

OMEGA = rc.OMEGA
OMEGA_TILDE = rc.OMEGA_TILDE


# --------------------------------------------------------------------------
# the tree
# --------------------------------------------------------------------------

@dataclasses.dataclass
class AdaptiveTree:
    """Spacetree of depth L: exists[l] marks the level-l cells that exist,
    refined[l] those that are cut into 3^d children (none on level L).  Level
    1 always exists in full (l_min = 1)."""
    d: int
    L: int
    exists: dict
    refined: dict

    @property
    def N(self) -> int:
        return 3 ** self.L


def tree_from_refinement(d: int, L: int, refine) -> AdaptiveTree:
    """Builds a tree top-down: refine(l, centres, h) -> bool array tells, for
    the existing level-l cells with the given centres (shape (..., d), last
    axis = x), which are cut (l < L)."""
    exists, refined = {}, {}
    exists[1] = np.ones((3,) * d, dtype=bool)
    for l in range(1, L + 1):
        n = 3 ** l
        h = 1.0 / n
        if l == L:
            refined[l] = np.zeros((n,) * d, dtype=bool)
            break
        idx = np.indices((n,) * d)
        # centres with the last array axis as the x coordinate
        centres = np.stack([(idx[d - 1 - k] + 0.5) * h for k in range(d)], axis=-1)
        want = np.asarray(refine(l, centres, h), dtype=bool)
        refined[l] = exists[l] & want
        child = refined[l]
        for ax in range(d):
            child = np.repeat(child, 3, axis=ax)
        exists[l + 1] = child
    return AdaptiveTree(d, L, exists, refined)


def regular_tree(d: int, L: int) -> AdaptiveTree:
    return tree_from_refinement(d, L, lambda l, c, h: np.ones(c.shape[:-1], dtype=bool))


# --------------------------------------------------------------------------
# the discrete system over the leaf nodes
# --------------------------------------------------------------------------

@dataclasses.dataclass
class AdaptiveSystem:
    tree: AdaptiveTree
    node_id: np.ndarray     # (N+1)^d: leaf node id at every fine-index position, -1 if none
    coords: np.ndarray      # (n_nodes, d) fine indices of the leaf nodes (array-axis order)
    boundary: np.ndarray    # (n_nodes,) bool
    K: sp.csr_matrix        # leaf stiffness
    b: np.ndarray           # lumped load at the leaf nodes
    Phi: dict               # l -> (n_nodes, n_active_l) pagodas of level l's active vertices
    PhiB: dict              # l -> (n_nodes, n_b) truncated pagodas of level l's boundary vertices
    bnd: dict               # l -> (n_b, d) those boundary vertices (level-l indices)
    active: dict            # l -> (n_active_l, d) level-l vertex indices of the active vertices
    active_grid: dict       # l -> (3^l+1)^d int: column of Phi_l, -1 if not active
    diag: dict              # l -> diag(Phi_l^T K Phi_l)
    S_trunc: np.ndarray     # truncated smoothed restriction stencil (5^d)
    eps: object = None      # the inputs: eps (scalar or per fine cell), f at fine positions
    f: np.ndarray = None

    @property
    def d(self) -> int:
        return self.tree.d

    @property
    def L(self) -> int:
        return self.tree.L


def _leaf_cells(tree: AdaptiveTree):
    """(level, cell index array (m, d)) of every leaf cell."""
    out = []
    for l in range(1, tree.L + 1):
        leaf = tree.exists[l] & ~tree.refined[l]
        out.append((l, np.argwhere(leaf)))
    return out


def _leaf_eps(eps, tree: AdaptiveTree, l: int, cells: np.ndarray) -> np.ndarray:
    if np.ndim(eps) == 0 or np.size(eps) == 1:
        return np.full(len(cells), float(np.ravel(eps)[0]))
    s = 3 ** (tree.L - l)
    out = np.empty(len(cells))
    for i, c in enumerate(cells):
        sl = tuple(slice(s * ck, s * ck + s) for ck in c)
        out[i] = eps[sl].mean()
    return out


def build_system(tree: AdaptiveTree, eps, f) -> AdaptiveSystem:
    """Leaf nodes, leaf stiffness and load, and every level's pagodas.

    eps: scalar or per fine cell (shape (N,)*d); f: values at the fine-index
    positions (shape (N+1,)*d)."""
    d, L, N = tree.d, tree.L, tree.N
    cs = np.array(corners(d))                      # corner offsets, array-axis order
    Kref = reference_element_matrix(d)
    leaves = _leaf_cells(tree)
    # leaf nodes
    present = np.zeros((N + 1,) * d, dtype=bool)
    for l, cells in leaves:
        s = 3 ** (L - l)
        for b in cs:
            pos = s * (cells + b)
            present[tuple(pos.T)] = True
    node_id = -np.ones((N + 1,) * d, dtype=np.int64)
    coords = np.argwhere(present)
    node_id[tuple(coords.T)] = np.arange(len(coords))
    boundary = np.any((coords == 0) | (coords == N), axis=1)
    # stiffness and lumped load
    rows, cols, vals = [], [], []
    b = np.zeros(len(coords))
    for l, cells in leaves:
        if len(cells) == 0:
            continue
        s = 3 ** (L - l)
        h = 1.0 / 3 ** l
        e = _leaf_eps(eps, tree, l, cells)
        ids = np.stack([node_id[tuple((s * (cells + bb)).T)] for bb in cs], axis=1)
        scale = e * h ** (d - 2)
        for a in range(len(cs)):
            for bb in range(len(cs)):
                rows.append(ids[:, a])
                cols.append(ids[:, bb])
                vals.append(scale * Kref[a, bb])
            np.add.at(b, ids[:, a], (h ** d / 2 ** d) * f[tuple(coords[ids[:, a]].T)])
    K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(len(coords),) * 2)
    # active vertices and their pagodas at the leaf nodes
    Phi, active, active_grid, diag, PhiB, bnd = {}, {}, {}, {}, {}, {}

    def pagodas(verts, s):
        # values of the pagodas of width s (fine units) centred at the level
        # vertices verts, at the leaf nodes (truncated to the domain): a leaf
        # node p lies in the level cell floor(p / s), and only that cell's 2^d
        # corners v have pagodas that reach it, with the value
        # prod_k (1 - |p_k - s v_k| / s)
        n = N // s
        col = -np.ones((n + 1,) * d, dtype=np.int64)
        col[tuple(verts.T)] = np.arange(len(verts))
        cell = np.minimum(coords // s, n - 1)
        r_, c_, v_ = [], [], []
        for bb in cs:
            v = cell + bb
            w = np.prod(1.0 - np.abs(coords - s * v) / s, axis=1)
            j = col[tuple(v.T)]
            ok = (j >= 0) & (w > 0.0)
            r_.append(np.nonzero(ok)[0])
            c_.append(j[ok])
            v_.append(w[ok])
        return sp.csr_matrix((np.concatenate(v_), (np.concatenate(r_), np.concatenate(c_))),
                             shape=(len(coords), len(verts)))

    for l in range(1, L + 1):
        n = 3 ** l
        s = 3 ** (L - l)
        # vertex j is surrounded by the cells j - 1 + b, b in {0,1}^d; cells
        # outside the domain count as present for boundary vertices
        pad = np.zeros((n + 2,) * d, dtype=bool)
        pad[tuple(slice(1, n + 1) for _ in range(d))] = tree.exists[l]
        padb = np.ones((n + 2,) * d, dtype=bool)
        padb[tuple(slice(1, n + 1) for _ in range(d))] = tree.exists[l]
        surrounded = np.ones((n + 1,) * d, dtype=bool)
        surrounded_b = np.ones((n + 1,) * d, dtype=bool)
        for bb in cs:
            sl = tuple(slice(bk, bk + n + 1) for bk in bb)
            surrounded &= pad[sl]
            surrounded_b &= padb[sl]
        inner = np.zeros((n + 1,) * d, dtype=bool)
        inner[tuple(slice(1, n) for _ in range(d))] = True
        act = np.argwhere(surrounded & inner)
        grid = -np.ones((n + 1,) * d, dtype=np.int64)
        grid[tuple(act.T)] = np.arange(len(act))
        Ph = pagodas(act, s)
        Phi[l], active[l], active_grid[l] = Ph, act, grid
        diag[l] = np.asarray((Ph.multiply(K @ Ph)).sum(axis=0)).ravel()
        bv = np.argwhere(surrounded_b & ~inner)
        PhiB[l], bnd[l] = pagodas(bv, s), bv
    S = rc.truncate_stencil(rc.smoothed_prolongation_stencil(d))
    return AdaptiveSystem(tree, node_id, coords, boundary, K, b, Phi, PhiB, bnd, active,
                          active_grid, diag, S, eps, f)


# --------------------------------------------------------------------------
# residuals, the composite problem, the cycle
# --------------------------------------------------------------------------

def free_vertices(sys_: AdaptiveSystem):
    """The vertices of the nodal space over the adaptive grid: every position
    that is an active vertex of some level, on the finest such level.
    Returns (levels, columns): level l and column of Phi_l of each."""
    finest = -np.ones(len(sys_.coords), dtype=np.int64)
    col = -np.ones(len(sys_.coords), dtype=np.int64)
    for l in range(1, sys_.L + 1):
        s = 3 ** (sys_.L - l)
        ids = sys_.node_id[tuple((s * sys_.active[l]).T)]
        finest[ids] = l
        col[ids] = np.arange(len(ids))
    sel = np.nonzero(finest >= 0)[0]
    return finest[sel], col[sel], sel


def composite_basis(sys_: AdaptiveSystem) -> sp.csr_matrix:
    """Columns: the pagoda of every free position on its finest level."""
    lev, col, _ = free_vertices(sys_)
    blocks = [sys_.Phi[l][:, col[lev == l]] for l in range(1, sys_.L + 1) if np.any(lev == l)]
    return sp.hstack(blocks).tocsr()


def residual(sys_: AdaptiveSystem, u: np.ndarray) -> np.ndarray:
    """b - K u at the leaf nodes (Dirichlet nodes included; nothing tests them)."""
    return sys_.b - sys_.K @ u


def level_residuals(sys_: AdaptiveSystem, u: np.ndarray, lmin: int = 1) -> dict:
    rr = residual(sys_, u)
    return {l: sys_.Phi[l].T @ rr for l in range(lmin, sys_.L + 1)}


def residual_norm(sys_: AdaptiveSystem, u: np.ndarray) -> float:
    """Eq. 10 over the vertices of the nodal space, h_i of their level."""
    rr = residual(sys_, u)
    lev, col, _ = free_vertices(sys_)
    acc = 0.0
    for l in range(1, sys_.L + 1):
        m = lev == l
        if not np.any(m):
            continue
        r_l = sys_.Phi[l].T @ rr
        acc += float(np.sum((3.0 ** -l) ** sys_.d * r_l[col[m]] ** 2))
    return float(np.sqrt(acc))


def _to_grid(sys_: AdaptiveSystem, l: int, x: np.ndarray) -> np.ndarray:
    g = np.zeros((3 ** l + 1,) * sys_.d)
    g[tuple(sys_.active[l].T)] = x
    return g


def smoothed_restriction(sys_: AdaptiveSystem, l: int, r_l: np.ndarray, omega: float,
                         mode: str = "truncated") -> np.ndarray:
    """b~_{l-1} on the active vertices of level l-1 (Eq. 8)."""
    if mode == "truncated":
        g = rc.apply_stencil_at_coarse(sys_.S_trunc, _to_grid(sys_, l, r_l))
        return omega * g[tuple(sys_.active[l - 1].T)]
    if mode == "exact":
        y = sys_.K @ (sys_.Phi[l] @ (r_l / sys_.diag[l]))
        return omega * (sys_.Phi[l - 1].T @ y)
    raise ValueError(mode)


def inject(sys_: AdaptiveSystem, l: int, x_l: np.ndarray) -> np.ndarray:
    """I: values of level l at the active vertices of level l-1 (the level-l
    vertex at the same position; zero where it is not active)."""
    g = _to_grid(sys_, l, x_l)
    return g[tuple((3 * sys_.active[l - 1]).T)]


def cycle(sys_: AdaptiveSystem, u: np.ndarray, variant: str = "jac", rtilde: str = "truncated",
          omega: float = OMEGA, omega_tilde: float = OMEGA_TILDE, omega_exp: float = 0.5,
          lmin: int = 1, return_parts: bool = False):
    """One additive cycle (Eq. 9 on the generating system) over levels lmin..L.

    jac: u += sum_l Phi_l c_l - sum_{l>lmin} Phi_{l-1} c~_{l-1}, c~_{l-1} =
         omega~ M_{l-1}^-1 R~ r_l;  pi: c~ of level l is P I c_l, so
         u += sum_l Phi_l c_l - sum_{l>lmin} Phi_{l-1} I c_l;  additive / exp:
         Eq. 2 with omega_add = 1 / omega_exp^(L-l) (the global depth L)."""
    L = sys_.L
    r = level_residuals(sys_, u, lmin)
    c = {l: omega * r[l] / sys_.diag[l] for l in range(lmin, L + 1)}
    du = np.zeros_like(u)
    for l in range(lmin, L + 1):
        scale = omega_exp ** (L - l) if variant == "exp" else 1.0
        du += scale * (sys_.Phi[l] @ c[l])
    parts = {"r": r, "c": c}
    if variant == "jac":
        bt, ct = {}, {}
        for l in range(lmin + 1, L + 1):
            bt[l - 1] = smoothed_restriction(sys_, l, r[l], omega, rtilde)
            ct[l - 1] = omega_tilde * bt[l - 1] / sys_.diag[l - 1]
            du -= sys_.Phi[l - 1] @ ct[l - 1]
        parts["bt"], parts["ct"] = bt, ct
    elif variant == "pi":
        for l in range(lmin + 1, L + 1):
            du -= sys_.Phi[l - 1] @ inject(sys_, l, c[l])
    elif variant not in ("additive", "exp"):
        raise ValueError(variant)
    u_new = u + du
    if return_parts:
        return u_new, parts
    return u_new


def solve(sys_: AdaptiveSystem, u0=None, tol: float = 1e-8, max_cycles: int = 2000, **kw):
    """Cycles until ||r||_h / ||r_0||_h <= tol (Eq. 10); returns (u, history)."""
    u = np.zeros(len(sys_.coords)) if u0 is None else u0.copy()
    r0 = residual_norm(sys_, u)
    hist = [1.0]
    for _ in range(max_cycles):
        u = cycle(sys_, u, **kw)
        rel = residual_norm(sys_, u) / r0 if r0 > 0 else 0.0
        hist.append(rel)
        if not np.isfinite(rel) or rel > 1e6 or rel <= tol:
            break
    return u, np.array(hist)


def dirichlet_lift(sys_: AdaptiveSystem, g: np.ndarray) -> np.ndarray:
    """A function of the adaptive grid's space (continuous, d-linear on every
    leaf cell) that takes the Dirichlet values g at the boundary vertices:
    a combination of the truncated pagodas of the boundary vertices, each
    position on the finest level where it is a boundary vertex surrounded by
    its level's cells.  Boundary nodes that hang take the interpolated value
    (g there is not used)."""
    # finest level on which each boundary node is a surrounded boundary vertex
    finest = -np.ones(len(sys_.coords), dtype=np.int64)
    col = -np.ones(len(sys_.coords), dtype=np.int64)
    for l in range(1, sys_.L + 1):
        s = 3 ** (sys_.L - l)
        ids = sys_.node_id[tuple((s * sys_.bnd[l]).T)]
        finest[ids] = l
        col[ids] = np.arange(len(ids))
    # the pagodas are hierarchical, not nodal: a coarse one is non-zero at
    # finer positions, a fine one vanishes at every coarser position and at
    # the other vertices of its level.  So the levels are set from the
    # coarsest down, each with the part of g the coarser pagodas have not
    # produced there yet.
    u = np.zeros(len(sys_.coords))
    for l in range(1, sys_.L + 1):
        ids = np.nonzero(finest == l)[0]
        if len(ids) == 0:
            continue
        u = u + sys_.PhiB[l][:, col[ids]] @ (g[ids] - u[ids])
    return u


def direct_solution(sys_: AdaptiveSystem, g=None) -> np.ndarray:
    """The solution of the composite problem: find u in V_h (with Dirichlet
    values g at the boundary vertices, zero if None) such that a(u, phi) =
    (f, phi) for every basis function phi of the nodal space."""
    B = composite_basis(sys_)
    uD = np.zeros(len(sys_.coords)) if g is None else dirichlet_lift(sys_, g)
    rhs = B.T @ (sys_.b - sys_.K @ uD)
    A = (B.T @ sys_.K @ B).tocsc()
    x = spla.spsolve(A, rhs)
    return uD + B @ x


def sample(sys_: AdaptiveSystem, fn) -> np.ndarray:
    """fn(x) at the leaf nodes; x has the last array axis as the x coordinate."""
    pts = sys_.coords[:, ::-1] / sys_.tree.N
    return fn(pts)


# --------------------------------------------------------------------------
# the level-wise FAS/HTMG form (Eq. 4) on the spacetree
# --------------------------------------------------------------------------

def _closure_weights(d: int) -> np.ndarray:
    """d-linear weights W[p, e] of the 4^d closure points p of a coarse cell
    (local coordinates 0..3, last axis fastest) towards its corners e."""
    pts = list(itertools.product(range(4), repeat=d))
    cs = corners(d)
    W = np.zeros((len(pts), len(cs)))
    for i, p in enumerate(pts):
        for k, e in enumerate(cs):
            W[i, k] = np.prod([pj / 3.0 if ej else 1.0 - pj / 3.0 for pj, ej in zip(p, e)])
    return W


def fas_level_residuals(sys_: AdaptiveSystem, u: np.ndarray, return_diag: bool = False):
    """Level residuals r_l = b_l - A_l u_l at the active vertices of every
    level, computed cell by cell in the FAS/HTMG form of Eq. 4:

      u_l = I u_{l+1}: every level holds the function's values at its
        vertices (correction vertices the injection of the finer level,
        hanging ones the interpolation of their coarse cell);
      a leaf cell contributes its load and its element matrix
        eps h^(d-2) K_ref; a refined cell contributes the Galerkin element
        matrix K_E = sum_c W_c^T K_c W_c of its 3^d children and the
        right-hand side b_E = sum_c W_c^T (b_c - K_c u^_c) with the
        hierarchical values u^_c = u_c - W_c u_E of the children
        (R r^_{l+1} with r^ = b - A u^, u^ = (id - P I) u);
      r_l(v) = sum over the level-l cells E at v of (b_E - K_E u_E)(v).

    With Galerkin element matrices this equals the residual of the composite
    problem tested with level l's shape functions; the tests check that.
    return_diag also returns every level's diagonal sum_E K_E(v, v) at the
    active vertices (M_l of the Jacobi steps)."""
    tree = sys_.tree
    d, L, N = tree.d, tree.L, tree.N
    cs = np.array(corners(d))
    nc = len(cs)
    Kref = reference_element_matrix(d)
    W = _closure_weights(d)
    kids = np.array(list(itertools.product(range(3), repeat=d)))
    # closure point index of every child corner: child kc, corner b -> kc + b
    cp = np.array([[np.ravel_multi_index(tuple(kc + b), (4,) * d) for b in cs] for kc in kids])
    Kc, bc = {}, {}           # per level: element matrices and right-hand sides of the cells
    uvals = {}
    for l in range(L, 0, -1):
        n = 3 ** l
        s = 3 ** (L - l)
        h = 1.0 / n
        ex = tree.exists[l]
        K_l = np.zeros((n,) * d + (nc, nc))
        b_l = np.zeros((n,) * d + (nc,))
        # values of the function at every level-l vertex position
        grid = np.indices((n + 1,) * d).reshape(d, -1).T
        uvals[l] = np.full((n + 1,) * d, np.nan)
        ok = np.zeros((n + 1,) * d, dtype=bool)
        for bb in cs:
            cells = np.argwhere(ex)
            ok[tuple((cells + bb).T)] = True
        pos = grid[ok.reshape(-1)]
        uvals[l][tuple(pos.T)] = evaluate(sys_, u, s * pos)
        leaf = ex & ~tree.refined[l]
        cells = np.argwhere(leaf)
        if len(cells):
            e = _leaf_eps(sys_.eps, tree, l, cells)
            K_l[tuple(cells.T)] = (e * h ** (d - 2))[:, None, None] * Kref
            fv = np.stack([sys_.f[tuple((s * (cells + bb)).T)] for bb in cs], axis=1)
            b_l[tuple(cells.T)] = (h ** d / 2 ** d) * fv
        ref = np.argwhere(tree.refined[l]) if l < L else np.zeros((0, d), dtype=int)
        for E in ref:
            KE = np.zeros((nc, nc))
            bE = np.zeros(nc)
            uE = np.array([uvals[l][tuple(E + bb)] for bb in cs])
            for ci, kc in enumerate(kids):
                child = tuple(3 * E + kc)
                Wc = W[cp[ci]]                          # child's corners x coarse corners
                Kk = Kc[l + 1][child]
                uc = np.array([uvals[l + 1][tuple(3 * E + kc + bb)] for bb in cs])
                uhat = uc - Wc @ uE
                KE += Wc.T @ Kk @ Wc
                bE += Wc.T @ (bc[l + 1][child] - Kk @ uhat)
            K_l[tuple(E)] = KE
            b_l[tuple(E)] = bE
        Kc[l], bc[l] = K_l, b_l
    out, diag = {}, {}
    for l in range(1, L + 1):
        n = 3 ** l
        r = np.zeros((n + 1,) * d)
        dg = np.zeros((n + 1,) * d)
        cells = np.argwhere(tree.exists[l])
        uE = np.stack([uvals[l][tuple((cells + bb).T)] for bb in cs], axis=1)
        KE = Kc[l][tuple(cells.T)]
        contrib = bc[l][tuple(cells.T)] - np.einsum("mab,mb->ma", KE, uE)
        for k, bb in enumerate(cs):
            np.add.at(r, tuple((cells + bb).T), contrib[:, k])
            np.add.at(dg, tuple((cells + bb).T), KE[:, k, k])
        out[l] = r[tuple(sys_.active[l].T)]
        diag[l] = dg[tuple(sys_.active[l].T)]
    return (out, diag) if return_diag else out


# --------------------------------------------------------------------------
# dynamic refinement
# --------------------------------------------------------------------------

def evaluate(sys_: AdaptiveSystem, u: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """The function of the adaptive grid's space with leaf-node values u at
    fine-index positions pts (shape (m, d), array-axis order, integers in
    0..N of sys_'s tree): d-linear interpolation inside the leaf cell that
    contains each point."""
    tree = sys_.tree
    d, L = tree.d, tree.L
    out = np.full(len(pts), np.nan)
    todo = np.ones(len(pts), dtype=bool)
    cs = np.array(corners(d))
    for l in range(1, L + 1):
        s = 3 ** (L - l)
        n = 3 ** l
        cell = np.minimum(pts // s, n - 1)             # the level-l cell holding the point
        leaf = tree.exists[l][tuple(cell.T)] & ~tree.refined[l][tuple(cell.T)]
        sel = todo & leaf
        if not np.any(sel):
            continue
        c = cell[sel]
        t = (pts[sel] - s * c) / s                      # local coordinates in [0, 1]
        val = np.zeros(int(sel.sum()))
        for b in cs:
            w = np.prod(np.where(b == 1, t, 1.0 - t), axis=1)
            val += w * u[sys_.node_id[tuple((s * (c + b)).T)]]
        out[sel] = val
        todo &= ~sel
    return out


def from_vertex_values(sys_: AdaptiveSystem, v: np.ndarray) -> np.ndarray:
    """The function of the adaptive grid's space that takes the values v at
    the vertices of the nodal space and at the boundary vertices; hanging
    nodes get the d-linear interpolation of their coarse cell (v there is not
    used).  Built level by level from the coarsest: the pagodas of one level
    vanish at the other vertices of that level and at every coarser
    position, so each level adds what the coarser ones left over."""
    u = dirichlet_lift(sys_, v)
    lev, col, sel = free_vertices(sys_)
    for l in range(1, sys_.L + 1):
        m = lev == l
        if not np.any(m):
            continue
        coef = v[sel[m]] - u[sel[m]]
        u = u + sys_.Phi[l][:, col[m]] @ coef
    return u


def transfer(old: AdaptiveSystem, u_old: np.ndarray, new: AdaptiveSystem) -> np.ndarray:
    """The iterate on a changed tree: the vertices of the new tree take the
    value of the old function at their position, i.e. new vertices are
    d-linear interpolations of the old grid (Sec. 5: new and hanging vertices
    are initialised by d-linear interpolation); vertices that hang in the new
    tree take the interpolation of their new coarse cell; removed vertices
    drop out."""
    if old.tree.L != new.tree.L or old.tree.d != new.tree.d:
        raise ValueError("the trees must have the same depth and dimension")
    return from_vertex_values(new, evaluate(old, u_old, new.coords))


def band_tree(d: int, L: int, L_base: int, centre, radius: float, width: float) -> AdaptiveTree:
    """Depth L_base everywhere and L within `width` of the circle (sphere) of
    the given radius about `centre` (x first): the shape of the adaptive
    workload (depth 8 within 0.05 of the circle r = 0.3 about the centre,
    depth 3 elsewhere).  A cell is refined when it reaches within width of the
    circle, with its half-diagonal as the margin."""
    ctr = np.asarray(centre, dtype=float)

    def ref(l, c, h):
        if l < L_base:
            return np.ones(c.shape[:-1], dtype=bool)
        r = np.sqrt(((c - ctr) ** 2).sum(-1))
        return np.abs(r - radius) <= width + 0.5 * np.sqrt(d) * h

    return tree_from_refinement(d, L, ref)


def moving_band_solve(d: int, L: int, L_base: int, eps, f_fn, centre, radius: float,
                      width: float, shift: float, every: int, moves: int, tol: float = 1e-8,
                      max_cycles: int = 2000, **kw):
    """Cycles on a tree whose refined band moves by `shift` along x after every
    `every` cycles, `moves` times, then stays; the iterate is carried over by
    transfer() at each move.  f_fn(x) gives f at points (m, d), x first.
    Returns (system of the last tree, u, list of (cycle, relative residual
    on the current tree))."""
    ctr = np.array(centre, dtype=float)
    N = 3 ** L
    idx = np.indices((N + 1,) * d).reshape(d, -1).T
    f = f_fn(idx[:, ::-1] / N).reshape((N + 1,) * d)

    def system(c):
        return build_system(band_tree(d, L, L_base, c, radius, width), eps, f)

    S = system(ctr)
    u = np.zeros(len(S.coords))
    r0 = residual_norm(S, u)
    hist = [(0, 1.0)]
    k = 0
    for m in range(moves + 1):
        steps = every if m < moves else max_cycles - k
        for _ in range(steps):
            u = cycle(S, u, **kw)
            k += 1
            rel = residual_norm(S, u) / r0
            hist.append((k, rel))
            if m == moves and (rel <= tol or not np.isfinite(rel)):
                return S, u, hist
        if m < moves:
            ctr = ctr + np.array([shift] + [0.0] * (d - 1))
            S_new = system(ctr)
            u = transfer(S, u, S_new)
            S = S_new
    return S, u, hist


# --------------------------------------------------------------------------
# the adaptive runs of Sec. 5: refinement at the boundary and by derivatives
# --------------------------------------------------------------------------

def refine_cells(tree: AdaptiveTree, l: int, cells: np.ndarray) -> AdaptiveTree:
    """A copy of the tree with the given existing leaf cells of level l < L
    cut into their 3^d children."""
    d, L = tree.d, tree.L
    exists = {k: v.copy() for k, v in tree.exists.items()}
    refined = {k: v.copy() for k, v in tree.refined.items()}
    for k in range(1, L + 1):
        exists.setdefault(k, np.zeros((3 ** k,) * d, dtype=bool))
    if len(cells):
        refined[l][tuple(cells.T)] = True
        for c in cells:
            exists[l + 1][tuple(slice(3 * ck, 3 * ck + 3) for ck in c)] = True
    return AdaptiveTree(d, L, exists, refined)


def coarse_tree(d: int, L: int, depth: int) -> AdaptiveTree:
    """Regular up to level `depth`, no cells below: the start of the runs
    (Sec. 5 starts from a two-grid scheme, depth 2)."""
    T = tree_from_refinement(d, L, lambda l, c, h: np.full(c.shape[:-1], l < depth))
    return T


def second_derivative_indicator(sys_: AdaptiveSystem, u: np.ndarray):
    """Largest absolute second difference along the coordinate axes at every
    vertex of the nodal space, on the spacing of its level (Sec. 5: absolute
    second derivatives along both axes in every unknown).  Returns (levels,
    level indices (m, d), values)."""
    lev, col, sel = free_vertices(sys_)
    L, N = sys_.L, sys_.tree.N
    vals = np.zeros(len(sel))
    vidx = np.zeros((len(sel), sys_.d), dtype=np.int64)
    for l in range(1, L + 1):
        m = lev == l
        if not np.any(m):
            continue
        v = sys_.active[l][col[m]]
        vidx[m] = v
        s = 3 ** (L - l)
        h = 1.0 / 3 ** l
        centre = u[sel[m]]
        best = np.zeros(int(m.sum()))
        for k in range(sys_.d):
            e = np.zeros(sys_.d, dtype=np.int64)
            e[k] = s
            up = evaluate(sys_, u, np.minimum(s * v + e, N))
            dn = evaluate(sys_, u, np.maximum(s * v - e, 0))
            best = np.maximum(best, np.abs(up - 2.0 * centre + dn) / h ** 2)
        vals[m] = best
    return lev, vidx, vals


def _top_fraction(vals: np.ndarray, fraction: float, bins: int = 64) -> np.ndarray:
    """Indices of (approximately) the largest `fraction` of vals, by a bin
    sort over [0, max]: the highest bins are taken while they fit the share
    (at least the top bin)."""
    if len(vals) == 0 or vals.max() <= 0.0:
        return np.zeros(0, dtype=np.int64)
    edges = np.linspace(0.0, vals.max(), bins + 1)
    which = np.minimum(np.searchsorted(edges, vals, side="right") - 1, bins - 1)
    target = fraction * len(vals)
    taken = np.zeros(len(vals), dtype=bool)
    count = 0
    for b in range(bins - 1, -1, -1):
        in_bin = which == b
        n_b = int(in_bin.sum())
        if count > 0 and count + n_b > target:
            break
        taken |= in_bin
        count += n_b
    return np.nonzero(taken)[0]


def amr_step(sys_: AdaptiveSystem, u: np.ndarray, lmax: int, fraction: float = 0.1,
             bottom: bool = True) -> AdaptiveTree:
    """One refinement of Sec. 5's runs: the leaf cells along the bottom
    boundary x_2 = 0 (where u = 1 is prescribed), and the leaf cells around
    the vertices with the (about) `fraction` largest second derivatives,
    unless they are on level lmax already."""
    tree = sys_.tree
    d = tree.d
    ax2 = d - 2                                   # array axis of x_2
    new = tree
    to_refine = {l: set() for l in range(1, lmax)}
    for l in range(1, lmax):
        leaf = tree.exists[l] & ~tree.refined[l]
        if bottom:
            sl = [slice(None)] * d
            sl[ax2] = 0
            cells = np.argwhere(leaf[tuple(sl)])
            for c in cells:
                full = list(c)
                full.insert(ax2, 0)
                to_refine[l].add(tuple(full))
    lev, vidx, vals = second_derivative_indicator(sys_, u)
    for i in _top_fraction(vals, fraction):
        l = int(lev[i])
        if l >= lmax:
            continue
        leaf = tree.exists[l] & ~tree.refined[l]
        for bb in corners(d):
            c = vidx[i] - 1 + np.array(bb)
            if np.all(c >= 0) and np.all(c < 3 ** l) and leaf[tuple(c)]:
                to_refine[l].add(tuple(int(x) for x in c))
    for l in range(1, lmax):
        if to_refine[l]:
            new = refine_cells(new, l, np.array(sorted(to_refine[l])))
    return new


def amr_solve(d: int, lmax: int, g_fn, f_fn=None, eps=1.0, start_depth: int = 2,
              every: int = 2, tol: float = 1e-8, max_cycles: int = 400, **kw):
    """Sec. 5's adaptive runs: start from a regular depth-`start_depth` tree,
    refine (amr_step) after every `every` cycles, carry the iterate over by
    d-linear interpolation, cycle until the normalised residual on the
    current tree reaches tol once the tree has stopped changing.

    Returns (system, u, history of (cycle, normalised residual, dof updates
    so far)): the cost counts every level's active vertices per cycle (the
    paper's "dof updates plus updates on coarser levels")."""
    N = 3 ** lmax
    idx = np.indices((N + 1,) * d).reshape(d, -1).T
    pts = idx[:, ::-1] / N
    f = (f_fn(pts) if f_fn else np.zeros(len(pts))).reshape((N + 1,) * d)

    def system(tree):
        return build_system(tree, eps, f)

    S = system(coarse_tree(d, lmax, start_depth))
    u = from_vertex_values(S, sample(S, g_fn))
    r0 = residual_norm(S, u)
    updates = 0
    hist = [(0, 1.0, 0)]
    changed = True
    for k in range(1, max_cycles + 1):
        u = cycle(S, u, **kw)
        updates += sum(len(S.active[l]) for l in range(1, lmax + 1))
        rel = residual_norm(S, u) / r0
        hist.append((k, rel, updates))
        if not np.isfinite(rel) or rel > 1e6:
            break
        if not changed and rel <= tol:
            break
        if k % every == 0:
            T = amr_step(S, u, lmax)
            changed = any(not np.array_equal(T.exists[l], S.tree.exists[l])
                          for l in range(1, lmax + 1))
            if changed:
                S_new = system(T)
                u = transfer(S, u, S_new)
                # the boundary values of new boundary vertices come from g
                g = sample(S_new, g_fn)
                v = evaluate(S_new, u, S_new.coords)
                v[S_new.boundary] = g[S_new.boundary]
                u = from_vertex_values(S_new, v)
                S = S_new
    return S, u, hist
