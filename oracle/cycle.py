"""The additive multigrid cycles of the paper on a regular 3:1 spacetree.

Oracle (test infrastructure only).  Levels are numbered as in the paper
(Sec. 2.1): l = 1 is the coarsest level holding unknowns (l_min = 1), l = L the
finest (l_max); level l has 3^l cells per dimension.

Implemented, each in the paper's order and notation:

* ``cycle``  with ``variant``:
    - "jac"       adAFAC-Jac, Algorithm 1 / Eq. 9: every level restricts the
                  fine residual (b_l = R^{L-l} r_L), the auxiliary right-hand
                  side b~_{l-1} = R~ r_l, one damped Jacobi step on the
                  correction and on the damping equation, and the update
                  u += sum_l P^{L-l} c_l - sum_{l>=2} P^{L-l+1} c~_{l-1};
    - "pi"        adAFAC-PI, Algorithm 2: the damping of level l is
                  c~_l = P I c_l and u += sum_l P^{L-l} c_l - sum_{l>=2} P^{L-l} c~_l;
    - "additive"  plain additive multigrid, Eq. 2 with omega_add = 1;
    - "exp"       Eq. 2 with exponential damping omega_add(l) = w^(L-l).
* ``form``: "cs" (correction scheme, residuals restricted directly) or "fas"
  (FAS/HTMG, Eq. 4: injected coarse solutions u_l = I u_{l+1}, hierarchical
  u^_{l+1} = u_{l+1} - P u_l, coarse right-hand sides
  b_l = R (b_{l+1} - A_{l+1} u^_{l+1}) and residuals r_l = b_l - A_l u_l).
* ``rtilde``: "truncated" (Sec. 3.2 option 1: the smoothed operator
  M^{-1} A_{eps=1} P for d-linear P, transposed, cut to the 5^d support of P,
  scaled by omega; M~ = M) or "exact" (R~ = omega R A_l M_l^{-1} with the
  level's own operator).
* ``residual_norm``: Eq. 10, ||r||_h^2 = sum_i h^d r_i^2 over the fine dofs.

Readings of passages the paper leaves open are listed in the module-level
constants below and in the design notes of the repository.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import fem, transfer
from .fem import LevelOperator, corners, interior, offsets, zero_boundary

OMEGA = 0.6          # Jacobi damping of the paper's runs (Sec. 5)
OMEGA_TILDE = 0.6    # reading: the damping equation uses the same omega


@dataclasses.dataclass
class Level:
    l: int
    n: int
    op: LevelOperator
    diag: np.ndarray
    Pv: np.ndarray | None = None      # prolongation from level l-1 (vertex weights)
    W: np.ndarray | None = None       # closure weights of P (coarse cells of l-1)


@dataclasses.dataclass
class Hierarchy:
    d: int
    L: int
    levels: dict          # l -> Level
    b: np.ndarray         # fine load vector
    S_full: np.ndarray    # M^{-1} A_{eps=1} P, 7^d, centred on a coarse vertex
    S_trunc: np.ndarray   # its 5^d truncation

    @property
    def fine(self) -> Level:
        return self.levels[self.L]


def smoothed_prolongation_stencil(d: int) -> np.ndarray:
    """The smoothed operator M^{-1} A_{eps=1} P (Sec. 3.2) for d-linear P with
    3:1 coarsening, as a 7^d array centred on a coarse vertex: column J of
    D^{-1} A P restricted to the fine vertices 3J + o, o in [-3, 3]^d.

    Evaluated on a level with 15 cells per dimension around the interior coarse
    vertex J = (2, ..., 2), whose 7^d neighbourhood contains no boundary vertex.
    It does not depend on the mesh width (A and D scale alike)."""
    n_c = 5
    n_f = 3 * n_c
    op = LevelOperator.from_eps(d, n_f, [1.0], True)
    W = transfer.dlinear_closure_weights(d, n_c)
    Pv = transfer.vertex_weights(W, n_c)
    e = np.zeros((n_c + 1,) * d)
    e[(2,) * d] = 1.0
    w = op.apply(transfer.prolong(Pv, e))
    dg = op.diagonal()
    w = np.where(dg != 0, w / np.where(dg != 0, dg, 1.0), 0.0)
    return w[tuple(slice(3, 10) for _ in range(d))].copy()


def truncate_stencil(S_full: np.ndarray) -> np.ndarray:
    """Keep the 5^d support of d-linear P, dropping the outer ring (Sec. 3.2
    option 1: the small negative entries by which the support grows)."""
    return S_full[tuple(slice(1, 6) for _ in range(S_full.ndim))].copy()


def coarse_eps(eps: np.ndarray) -> np.ndarray:
    """eps of the level-(l-1) cells: the arithmetic mean of their 3^d children
    (the reading of rediscretisation with a varying parameter; every coarse
    cell covers the same number of fine cells)."""
    d = eps.ndim
    n_c = eps.shape[0] // 3
    shape = []
    for _ in range(d):
        shape += [n_c, 3]
    return eps.reshape(shape).mean(axis=tuple(range(1, 2 * d, 2)))


def build_hierarchy(d: int, L: int, eps, eps_is_scalar: bool, f,
                    transfer_kind: str = "dlinear", coarse_op: str = "galerkin") -> Hierarchy:
    """Fine operator from eps, then for l = L .. 2: P_l (d-linear or BoxMG from
    the level-l stencils), the coarse operator A_{l-1} -- Galerkin
    P_l^T A_l P_l (Sec. 2.2) or rediscretised from the averaged eps -- and
    the diagonals."""
    if L < 1:
        raise ValueError("depth must be >= 1")
    n = 3 ** L
    op = LevelOperator.from_eps(d, n, eps, eps_is_scalar)
    levels = {L: Level(L, n, op, op.diagonal())}
    for l in range(L, 1, -1):
        fine = levels[l]
        n_c = fine.n // 3
        if transfer_kind == "dlinear":
            W = transfer.dlinear_closure_weights(d, n_c)
        elif transfer_kind == "boxmg":
            W = transfer.boxmg_closure_weights(fine.op.stencils(), n_c)
        else:
            raise ValueError(transfer_kind)
        fine.W = W
        fine.Pv = transfer.vertex_weights(W, n_c)
        if coarse_op == "galerkin":
            cop = transfer.galerkin(fine.op, W, n_c)
        elif coarse_op == "rediscretised":
            cop = LevelOperator.from_eps(d, n_c, coarse_eps(fine.op.eps), False)
        else:
            raise ValueError(coarse_op)
        levels[l - 1] = Level(l - 1, n_c, cop, cop.diagonal())
    b = fem.load_vector(f, 1.0 / n, d)
    S_full = smoothed_prolongation_stencil(d)
    return Hierarchy(d, L, levels, b, S_full, truncate_stencil(S_full))


# --------------------------------------------------------------------------
# level-wise building blocks
# --------------------------------------------------------------------------

def residual(H: Hierarchy, l: int, u: np.ndarray, b: np.ndarray) -> np.ndarray:
    """r = b - A_l u at the interior vertices of level l."""
    return zero_boundary(b - H.levels[l].op.apply(u))


def jacobi_correction(H: Hierarchy, l: int, rhs: np.ndarray, omega: float) -> np.ndarray:
    """One damped Jacobi step from a zero initial guess: omega diag(A_l)^{-1} rhs."""
    dg = H.levels[l].diag
    out = np.zeros_like(rhs)
    I = tuple(slice(1, -1) for _ in range(rhs.ndim))
    out[I] = omega * rhs[I] / dg[I]
    return out


def R(H: Hierarchy, l: int, r: np.ndarray) -> np.ndarray:
    """Restriction from level l to l-1 (R = P_l^T)."""
    return zero_boundary(transfer.restrict(H.levels[l].Pv, r))


def P(H: Hierarchy, l: int, c: np.ndarray) -> np.ndarray:
    """Prolongation from level l-1 to l."""
    return zero_boundary(transfer.prolong(H.levels[l].Pv, c))


def P_pow(H: Hierarchy, l_from: int, l_to: int, c: np.ndarray) -> np.ndarray:
    """P^{l_to - l_from}: repeated prolongation from level l_from to l_to."""
    for l in range(l_from + 1, l_to + 1):
        c = P(H, l, c)
    return c


def apply_stencil_at_coarse(S: np.ndarray, r: np.ndarray) -> np.ndarray:
    """(S^T r)[J] = sum_o S[o] r[3J + o] for the interior coarse vertices J;
    S is a (2k+1)^d array centred on the coarse vertex."""
    d = r.ndim
    n_f = r.shape[0] - 1
    n_c = n_f // 3
    k = (S.shape[0] - 1) // 2
    out = np.zeros((n_c + 1,) * d)
    I = tuple(slice(1, n_c) for _ in range(d))
    for o in offsets(d, k):
        s = S[tuple(oi + k for oi in o)]
        if s == 0.0:
            continue
        sl = tuple(slice(3 + oi, 3 * (n_c - 1) + oi + 1, 3) for oi in o)
        out[I] += s * r[sl]
    return out


def Rtilde(H: Hierarchy, l: int, r: np.ndarray, omega: float, mode: str) -> np.ndarray:
    """Smoothed restriction from level l to l-1 (Sec. 3.2, Eq. 8).

    truncated: omega * (truncated M^{-1} A_{eps=1} P)^T r
    exact:     omega * R A_l M_l^{-1} r"""
    if mode == "truncated":
        return omega * apply_stencil_at_coarse(H.S_trunc, r)
    if mode == "exact":
        dg = H.levels[l].diag
        x = np.zeros_like(r)
        I = tuple(slice(1, -1) for _ in range(r.ndim))
        x[I] = r[I] / dg[I]
        return omega * R(H, l, H.levels[l].op.apply(x))
    raise ValueError(mode)


def residual_norm(H: Hierarchy, r: np.ndarray) -> float:
    """Eq. 10: ||r||_h = sqrt(sum_i h_i^d r_i^2); on a regular tree every fine
    dof has h_i = 3^-L."""
    h = 1.0 / H.fine.n
    return float(np.sqrt(np.sum(h ** H.d * interior(r) ** 2)))


def max_residual(r: np.ndarray) -> float:
    return float(np.max(np.abs(interior(r))))


# --------------------------------------------------------------------------
# the cycle
# --------------------------------------------------------------------------

def level_residuals(H: Hierarchy, u: np.ndarray, form: str):
    """Residual r_l of every level for the current fine iterate u.

    cs : r_L = b - A_L u, r_l = R r_{l+1}          (b_l = R^{L-l} r_L, Alg. 1)
    fas: u_l = I u_{l+1}; u^_{l+1} = u_{l+1} - P u_l;
         b_l = R (b_{l+1} - A_{l+1} u^_{l+1});  r_l = b_l - A_l u_l  (Eq. 4)
    """
    L = H.L
    r = {L: residual(H, L, u, H.b)}
    if form == "cs":
        for l in range(L - 1, 0, -1):
            r[l] = R(H, l + 1, r[l + 1])
        return r
    if form != "fas":
        raise ValueError(form)
    ul = {L: u}
    for l in range(L - 1, 0, -1):
        ul[l] = zero_boundary(transfer.inject(ul[l + 1]))
    bl = {L: H.b}
    for l in range(L - 1, 0, -1):
        uhat = zero_boundary(ul[l + 1] - P(H, l + 1, ul[l]))
        rhat = zero_boundary(bl[l + 1] - H.levels[l + 1].op.apply(uhat))
        bl[l] = R(H, l + 1, rhat)
        r[l] = residual(H, l, ul[l], bl[l])
    return r


def cycle(H: Hierarchy, u: np.ndarray, variant: str = "jac", form: str = "cs",
          rtilde: str = "truncated", omega: float = OMEGA,
          omega_tilde: float = OMEGA_TILDE, omega_exp: float = 0.5,
          return_parts: bool = False, lmin: int = 1):
    """One additive cycle over the levels lmin .. L; returns the new fine
    iterate (and the level data).

    Reading of Alg. 1's final update (its printed sum starts one level too
    coarse and counts c_{l_min} twice): u += sum_{l=lmin}^{L} P^{L-l} c_l
    - sum_{l=lmin+1}^{L} P^{L-l+1} c~_{l-1}, which is Eq. 9 with
    M^{-1}_{l_min-1} = 0 (no damping below the coarsest level).  Alg. 2 is read
    the same way.  lmin > 1 drops the coarser levels (Sec. 5 adds correction
    levels one by one below a fixed finest level)."""
    L = H.L
    if not 1 <= lmin <= L:
        raise ValueError("lmin must be in 1 .. L")
    r = level_residuals(H, u, form)
    c = {l: jacobi_correction(H, l, r[l], omega) for l in range(lmin, L + 1)}
    du = np.zeros_like(u)
    parts = {"r": r, "c": c}
    if variant in ("jac", "additive", "exp"):
        for l in range(lmin, L + 1):
            scale = omega_exp ** (L - l) if variant == "exp" else 1.0
            du += scale * P_pow(H, l, L, c[l])
    if variant == "jac":
        bt, ct = {}, {}
        for l in range(lmin + 1, L + 1):
            bt[l - 1] = Rtilde(H, l, r[l], omega, rtilde)
            ct[l - 1] = jacobi_correction(H, l - 1, bt[l - 1], omega_tilde)
            du -= P_pow(H, l - 1, L, ct[l - 1])
        parts["bt"], parts["ct"] = bt, ct
    elif variant == "pi":
        ct = {}
        for l in range(lmin, L + 1):
            du += P_pow(H, l, L, c[l])
        for l in range(lmin + 1, L + 1):
            ct[l] = P(H, l, zero_boundary(transfer.inject(c[l])))
            du -= P_pow(H, l, L, ct[l])
        parts["ct"] = ct
    elif variant not in ("additive", "exp"):
        raise ValueError(variant)
    # boundary vertices carry Dirichlet data, not unknowns (Sec. 2.1): the
    # update acts on the interior and the iterate keeps its boundary values
    u_new = u + zero_boundary(du)
    if return_parts:
        return u_new, parts
    return u_new


def with_boundary(g: np.ndarray) -> np.ndarray:
    """Initial iterate for Dirichlet data g: g on the boundary, 0 inside (the
    setups of Sec. 5 prescribe u = 1 on x_2 = 0 and u = 0 elsewhere on the
    boundary)."""
    return g - zero_boundary(np.array(g, dtype=np.float64))


def solve(H: Hierarchy, u0=None, tol: float = 1e-8, max_cycles: int = 500,
          **kw):
    """Cycles until ||r_n||_h / ||r_0||_h <= tol.  Returns (u, history) where
    history[n] is the normalised residual of iterate n (history[0] = 1).  The
    boundary entries of u0 are the Dirichlet values (zero by default)."""
    u = np.zeros_like(H.b) if u0 is None else u0.copy()
    r0 = residual_norm(H, residual(H, H.L, u, H.b))
    hist = [1.0]
    for _ in range(max_cycles):
        u = cycle(H, u, **kw)
        rel = residual_norm(H, residual(H, H.L, u, H.b)) / r0
        hist.append(rel)
        if rel <= tol or not np.isfinite(rel) or rel > 1e6:
            break
    return u, hist
