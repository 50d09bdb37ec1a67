"""Seeded synthetic inputs for the adAFAC solver.

This module only *generates inputs*: the per-cell material parameter eps, the
right-hand side f sampled at the vertices, the manufactured exact solution and
random initial guesses.  It contains none of the solver's arithmetic (no
stencils, transfer operators, residuals or cycles), so that both the CPU oracle
and the CUDA path can draw the very same inputs from it.

Grid convention shared by every consumer of these arrays
---------------------------------------------------------
A regular spacetree of depth L in d dimensions (3:1 refinement per dimension,
Section 2.1 of the paper) has n = 3**L cells per dimension, mesh width
h = 1/n and (n+1)**d vertices on the unit cube.  Vertex arrays are C-ordered
numpy arrays of shape (n+1,)*d whose *last* axis is x (the fastest running
index), then y, then z.  Cell arrays have shape (n,)*d with the same order;
cell (i_z, i_y, i_x) spans the vertices i .. i+1 along every axis.

Workloads (the problem set-ups of the paper's Section 5 scaled to the
configurations this library is measured on):

* ``poisson2d_d4``  -Laplace u = f on the unit square, depth 4, eps = 1,
  f = 2 pi^2 sin(pi x) sin(pi y)  (exact u = sin(pi x) sin(pi y)).
* ``jump2d_d6``     -div(eps grad u) = 1, depth 6, eps constant on blocks of
  27 x 27 fine cells, each block 1 or 1e-3 with probability 1/2 (seed 1903).
* ``poisson3d_d5``  -Laplace u = f on the unit cube, depth 5, eps = 1,
  f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z).

Random numbers come from numpy's PCG64 bit generator with the stated seed.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Workload",
    "WORKLOADS",
    "get",
    "vertex_coords",
    "manufactured_solution",
    "manufactured_rhs",
    "constant_rhs",
    "eps_random_blocks",
    "random_vertex_field",
]


def vertex_coords(dim: int, depth: int):
    """Coordinates of all vertices: a list of ``dim`` arrays of shape (n+1,)*dim.

    Entry k of the list is the coordinate along numpy axis k (axis dim-1 is x).
    """
    n = 3 ** depth
    x1 = np.arange(n + 1, dtype=np.float64) / n
    return np.meshgrid(*([x1] * dim), indexing="ij")


def manufactured_solution(dim: int, depth: int) -> np.ndarray:
    """u(x) = prod_k sin(pi x_k) sampled at every vertex (zero on the boundary)."""
    u = np.ones((3 ** depth + 1,) * dim)
    for xk in vertex_coords(dim, depth):
        u = u * np.sin(np.pi * xk)
    # sin(pi) is 1.2e-16 in floating point; the boundary is exactly zero.
    _zero_boundary(u)
    return u


def manufactured_rhs(dim: int, depth: int) -> np.ndarray:
    """f = dim * pi^2 * prod_k sin(pi x_k) (so that -Laplace u = f for the
    manufactured solution), sampled at every vertex including the boundary."""
    return dim * math.pi ** 2 * manufactured_solution(dim, depth)


def constant_rhs(dim: int, depth: int, value: float = 1.0) -> np.ndarray:
    return np.full((3 ** depth + 1,) * dim, float(value))


def eps_random_blocks(dim: int, depth: int, block_cells: int, low: float,
                      seed: int) -> np.ndarray:
    """Per-cell eps: blocks of ``block_cells``**dim fine cells, each block 1 or
    ``low`` with probability 1/2, drawn from PCG64(seed) in C order over blocks."""
    n = 3 ** depth
    if n % block_cells:
        raise ValueError("block size must divide the number of cells per dimension")
    nb = n // block_cells
    rng = np.random.Generator(np.random.PCG64(seed))
    coin = rng.integers(0, 2, size=(nb,) * dim)
    blocks = np.where(coin == 1, float(low), 1.0)
    eps = blocks
    for ax in range(dim):
        eps = np.repeat(eps, block_cells, axis=ax)
    return np.ascontiguousarray(eps)


def random_vertex_field(dim: int, depth: int, seed: int) -> np.ndarray:
    """Uniform(-1, 1) values at interior vertices, zero on the boundary; used as
    an arbitrary initial guess when iterates are compared."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.uniform(-1.0, 1.0, size=(3 ** depth + 1,) * dim)
    _zero_boundary(u)
    return u


def _zero_boundary(a: np.ndarray) -> None:
    for ax in range(a.ndim):
        idx = [slice(None)] * a.ndim
        idx[ax] = 0
        a[tuple(idx)] = 0.0
        idx[ax] = -1
        a[tuple(idx)] = 0.0


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    dim: int
    depth: int
    eps_kind: str                 # "scalar" or "blocks"
    eps_value: float = 1.0        # scalar eps
    eps_low: float = 1e-3         # low value of the random blocks
    block_cells: int = 27
    seed: int = 1903
    rhs_kind: str = "manufactured"  # or "constant"
    transfer: str = "dlinear"       # "dlinear" or "boxmg"

    @property
    def n(self) -> int:
        return 3 ** self.depth

    def eps(self):
        """Returns (eps_array, is_scalar)."""
        if self.eps_kind == "scalar":
            return np.array([self.eps_value], dtype=np.float64), True
        return eps_random_blocks(self.dim, self.depth, self.block_cells,
                                 self.eps_low, self.seed), False

    def f(self) -> np.ndarray:
        if self.rhs_kind == "manufactured":
            return manufactured_rhs(self.dim, self.depth)
        return constant_rhs(self.dim, self.depth, 1.0)

    def exact(self):
        if self.rhs_kind == "manufactured" and self.eps_kind == "scalar" \
                and self.eps_value == 1.0:
            return manufactured_solution(self.dim, self.depth)
        return None

    def level_dofs(self):
        """Interior vertex count (3^l - 1)^d of every level l = 1..L."""
        return [(3 ** l - 1) ** self.dim for l in range(1, self.depth + 1)]

    def with_depth(self, depth: int) -> "Workload":
        return dataclasses.replace(self, name=f"{self.name}@{depth}", depth=depth)


WORKLOADS = {
    "poisson2d_d4": Workload("poisson2d_d4", 2, 4, "scalar"),
    "jump2d_d6": Workload("jump2d_d6", 2, 6, "blocks", eps_low=1e-3,
                          block_cells=27, seed=1903, rhs_kind="constant",
                          transfer="boxmg"),
    "poisson3d_d5": Workload("poisson3d_d5", 3, 5, "scalar"),
    # the largest request of the serving mix: 3-D depth 5, eps on blocks of
    # level-3 cells (9^3 fine cells), each 1 or 1e-2; f = 1; BoxMG + Galerkin
    "jump3d_d5": Workload("jump3d_d5", 3, 5, "blocks", eps_low=1e-2,
                          block_cells=9, seed=1903, rhs_kind="constant",
                          transfer="boxmg"),
}


def get(name: str) -> Workload:
    return WORKLOADS[name]


@dataclasses.dataclass(frozen=True)
class ServingRequest:
    """One solve of the serving stream: its tree, material and right-hand
    side, and its arrival time on a unit-rate Poisson clock (multiply by the
    mean inter-arrival time of the offered load)."""
    index: int
    dim: int
    depth: int
    eps: np.ndarray
    f: np.ndarray
    arrival: float


def serving_requests(count: int, seed: int = 1903, low: float = 1e-2):
    """The serving mix: 80 % 2-D solves with depth uniform in 3..6, 20 % 3-D
    with depth uniform in 3..5; eps on blocks of level-min(3, depth-1) cells,
    each block 1 or ``low`` with probability 1/2; f = 1; exponential
    inter-arrival times of mean 1.  Request i draws from PCG64(seed) (shape and
    arrival) and PCG64(seed + 1 + i) (its eps blocks)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for i in range(count):
        three_d = rng.uniform() < 0.2
        dim = 3 if three_d else 2
        depth = int(rng.integers(3, 6)) if three_d else int(rng.integers(3, 7))
        t += float(rng.exponential(1.0))
        block = 3 ** (depth - min(3, depth - 1))
        eps = eps_random_blocks(dim, depth, block, low, seed + 1 + i)
        out.append(ServingRequest(i, dim, depth, eps, constant_rhs(dim, depth), t))
    return out


# ---------------------------------------------------------------------------
# The setups of the paper's Sec. 5: f = 0, u = 1 on x_2 = 0 and u = 0 on the
# rest of the boundary, eps = 1 or 10^-k / 10^k in one of three geometries.
# Coordinates: x_1 is the last array axis (x), x_2 the one before (y); the
# 3-D variants extend the 2-D geometry uniformly along z.

def _cell_centres(dim: int, depth: int):
    n = 3 ** depth
    c1 = (np.arange(n) + 0.5) / n
    return np.meshgrid(*([c1] * dim), indexing="ij")


def bottom_boundary(dim: int, depth: int) -> np.ndarray:
    """Dirichlet values: 1 at the vertices with x_2 = 0, 0 elsewhere."""
    g = np.zeros((3 ** depth + 1,) * dim)
    idx = [slice(None)] * dim
    idx[dim - 2] = 0
    g[tuple(idx)] = 1.0
    return g


def eps_halves(dim: int, depth: int, low: float) -> np.ndarray:
    """eps = 1 for x_1 < 1/2, ``low`` for x_1 >= 1/2 (by cell centre; the split
    does not coincide with the 3:1 mesh lines)."""
    c = _cell_centres(dim, depth)
    return np.where(c[dim - 1] < 0.5, 1.0, float(low))


def eps_needle(dim: int, depth: int, high: float) -> np.ndarray:
    """A line of width 0.02 with eps = ``high`` in eps = 1: the cells whose
    centre lies within 0.01 of x_1 = 1/2 and below x_2 = 1/2 (the line starts
    at the boundary x_2 = 0 and ends half-way into the domain)."""
    c = _cell_centres(dim, depth)
    inside = (np.abs(c[dim - 1] - 0.5) < 0.01) & (c[dim - 2] < 0.5)
    return np.where(inside, float(high), 1.0)


def eps_checkerboard(dim: int, depth: int, low: float) -> np.ndarray:
    """Four regions separated by the lines x_2 = 5 x_1 - 2.5 and
    x_2 = 0.2 x_1 + 0.5, eps = 1 and ``low`` in checkerboard fashion."""
    c = _cell_centres(dim, depth)
    x1, x2 = c[dim - 1], c[dim - 2]
    s = (x2 - 5.0 * x1 + 2.5) * (x2 - 0.2 * x1 - 0.5)
    return np.where(s > 0, 1.0, float(low))
