"""Pins of the adaptive-tree oracle (oracle/adaptive.py).

* On a fully refined tree the generating-system cycle is the regular
  oracle's cycle, for every variant and both smoothed restrictions.
* On adaptive trees with hanging vertices, the composite problem it solves
  equals the one assembled from the global hat functions by quadrature over
  the leaf cells (tests/_brute.py), and the cycles converge to its solution.
* Linear boundary data with f = 0 give the linear function at every leaf
  node, hanging ones included: the space reproduces linears.
* Iterates stay in the space of the adaptive grid: values at hanging nodes
  are the interpolation of the surrounding vertices.
"""
import itertools

import numpy as np
import pytest

import workloads as wl
from oracle import adaptive as ad
from oracle import cycle as oc

from . import _brute


def _band_tree(d, L):
    # refine a band around the circle r = 0.3 about the centre (the shape of
    # the adaptive workload), coarser far from it
    def ref(l, c, h):
        r = np.sqrt(((c - 0.5) ** 2).sum(-1))
        return np.abs(r - 0.3) <= 0.05 + h
    return ad.tree_from_refinement(d, L, ref)


def _corner_tree(d, L):
    return ad.tree_from_refinement(d, L, lambda l, c, h: np.all(c < 0.4, axis=-1))


@pytest.mark.parametrize("d,L", [(2, 3), (3, 2)])
@pytest.mark.parametrize("variant,rtilde", [("jac", "truncated"), ("jac", "exact"),
                                            ("additive", "truncated"), ("pi", "truncated"),
                                            ("exp", "truncated")])
def test_fully_refined_tree_is_the_regular_cycle(d, L, variant, rtilde):
    N = 3 ** L
    eps = np.random.default_rng(5).uniform(0.05, 2.0, size=(N,) * d)
    f = wl.manufactured_rhs(d, L)
    S = ad.build_system(ad.regular_tree(d, L), eps, f)
    H = oc.build_hierarchy(d, L, eps, False, f, "dlinear")
    u0g = wl.random_vertex_field(d, L, 11)
    u0 = u0g[tuple(S.coords.T)]
    ua = ad.cycle(S, u0, variant=variant, rtilde=rtilde, omega_exp=0.7)
    ur = oc.cycle(H, u0g, variant=variant, rtilde=rtilde, omega_exp=0.7)
    assert np.abs(ua - ur[tuple(S.coords.T)]).max() <= 1e-13 * np.abs(ur).max()
    assert ad.residual_norm(S, u0) == pytest.approx(
        oc.residual_norm(H, oc.residual(H, L, u0g, H.b)), rel=1e-13)


def _active_vertices_by_hand(T):
    """Every level's vertices surrounded by 2^d existing cells of their level
    (interior ones), found vertex by vertex from the tree's flags."""
    d = T.d
    out = []
    for l in range(1, T.L + 1):
        n = 3 ** l
        for v in itertools.product(range(1, n), repeat=d):
            if all(T.exists[l][tuple(vk - 1 + bk for vk, bk in zip(v, b))]
                   for b in itertools.product((0, 1), repeat=d)):
                out.append((l, v))
    return out


@pytest.mark.parametrize("tree", ["corner", "band"])
def test_composite_problem_equals_the_hat_function_assembly(tree):
    # second route: all shape functions of the generating system (every
    # level's active vertices, found by hand), global hats, quadrature on the
    # leaf cells, a least-squares solve of the singular system; its function
    # must equal the oracle's solution at every leaf node, hanging ones too
    d, L = 2, 3
    T = _corner_tree(d, L) if tree == "corner" else _band_tree(d, L)
    N = 3 ** L
    eps = np.random.default_rng(3).uniform(0.2, 3.0, size=(N,) * d)
    f = wl.manufactured_rhs(d, L)
    S = ad.build_system(T, eps, f)
    u = ad.direct_solution(S)
    gen = _active_vertices_by_hand(T)
    pos = np.array([np.array(v) / 3 ** l for l, v in gen])
    widths = np.array([3.0 ** -l for l, _ in gen])
    f_fn = lambda x: f[tuple(np.rint(x * N).astype(int))]
    A, b = _brute.adaptive_system_dense(T, eps, f_fn, pos, widths)
    x, *_ = np.linalg.lstsq(A, b, rcond=1e-13)
    vals = np.array([_brute.hats_and_grads(pos, widths, p / N)[0] @ x for p in S.coords])
    assert np.abs(u - vals).max() <= 1e-9 * np.abs(vals).max()
    lev, col, sel = ad.free_vertices(S)
    assert len(sel) < len(S.coords) - S.boundary.sum()  # the tree has hanging nodes


@pytest.mark.parametrize("d,L,tree", [(2, 4, "band"), (2, 3, "corner"), (3, 3, "corner")])
@pytest.mark.parametrize("variant", ["jac", "additive", "pi"])
def test_cycles_converge_to_the_composite_solution(d, L, tree, variant):
    T = _corner_tree(d, L) if tree == "corner" else _band_tree(d, L)
    S = ad.build_system(T, 1.0, wl.constant_rhs(d, L))
    ud = ad.direct_solution(S)
    u, hist = ad.solve(S, tol=1e-11, max_cycles=1000, variant=variant)
    assert hist[-1] <= 1e-11
    assert np.abs(u - ud).max() <= 1e-8 * np.abs(ud).max()


@pytest.mark.parametrize("tree", ["corner", "band"])
def test_linear_boundary_data_give_the_linear_solution(tree):
    d, L = 2, 4
    T = _corner_tree(d, L) if tree == "corner" else _band_tree(d, L)
    S = ad.build_system(T, 1.0, np.zeros((3 ** L + 1,) * d))
    g = ad.sample(S, lambda x: 1.0 + 2.0 * x[:, 0] - 3.0 * x[:, 1])
    assert np.abs(ad.dirichlet_lift(S, g) - g)[S.boundary].max() <= 1e-14
    assert np.abs(ad.direct_solution(S, g) - g).max() <= 1e-12
    u, hist = ad.solve(S, u0=ad.dirichlet_lift(S, g), tol=1e-12, max_cycles=1000)
    assert np.abs(u - g).max() <= 1e-10


def test_iterates_stay_in_the_space_of_the_adaptive_grid():
    d, L = 2, 3
    S = ad.build_system(_corner_tree(d, L), 1.0, wl.manufactured_rhs(d, L))
    B = ad.composite_basis(S).toarray()
    u = B @ np.random.default_rng(1).standard_normal(B.shape[1])
    for _ in range(3):
        u = ad.cycle(S, u)
    # u is a combination of the nodal space's basis functions: hanging nodes
    # carry the interpolated values
    x, *_ = np.linalg.lstsq(B, u, rcond=None)
    assert np.abs(B @ x - u).max() <= 1e-12 * np.abs(u).max()
    lev, col, sel = ad.free_vertices(S)
    hanging = np.setdiff1d(np.nonzero(~S.boundary)[0], sel)
    assert len(hanging) > 0


# ---------------------------------------------------------------------------
# dynamic refinement: the band moves, vertices are interpolated

def test_vertex_values_rebuild_any_function_of_the_space():
    d, L = 2, 4
    S = ad.build_system(_band_tree(d, L), 1.0, wl.constant_rhs(d, L))
    B = ad.composite_basis(S)
    u = B @ np.random.default_rng(2).standard_normal(B.shape[1])
    assert np.abs(ad.from_vertex_values(S, u) - u).max() <= 1e-13 * np.abs(u).max()


def test_transfer_to_a_finer_tree_keeps_the_function():
    d, L = 2, 4
    coarse = ad.build_system(ad.band_tree(d, L, 2, (0.5, 0.5), 0.3, 0.03), 1.0,
                             wl.constant_rhs(d, L))
    fine = ad.build_system(ad.band_tree(d, L, 2, (0.5, 0.5), 0.3, 0.12), 1.0,
                           wl.constant_rhs(d, L))
    assert len(fine.coords) > len(coarse.coords)
    B = ad.composite_basis(coarse)
    u = B @ np.random.default_rng(4).standard_normal(B.shape[1])
    v = ad.transfer(coarse, u, fine)
    # the finer tree represents the coarse tree's function exactly
    assert np.abs(ad.evaluate(fine, v, coarse.coords) - u).max() <= 1e-13 * np.abs(u).max()


def test_transfer_of_a_linear_function_is_exact_both_ways():
    d, L = 2, 4
    a = ad.build_system(ad.band_tree(d, L, 2, (0.5, 0.5), 0.3, 0.05), 1.0, wl.constant_rhs(d, L))
    b = ad.build_system(ad.band_tree(d, L, 2, (0.6, 0.5), 0.3, 0.05), 1.0, wl.constant_rhs(d, L))
    lin = lambda x: 0.5 - 1.5 * x[:, 0] + 2.0 * x[:, 1]
    ua = ad.sample(a, lin)
    assert np.abs(ad.transfer(a, ua, b) - ad.sample(b, lin)).max() <= 1e-13
    assert np.abs(ad.transfer(b, ad.sample(b, lin), a) - ua).max() <= 1e-13


def test_a_band_that_does_not_move_is_the_static_solve():
    d, L = 2, 4
    one = lambda x: np.ones(len(x))
    S, u, hist = ad.moving_band_solve(d, L, 2, 1.0, one, (0.5, 0.5), 0.3, 0.05, 0.0, 5, 3,
                                      tol=1e-9)
    Ss = ad.build_system(ad.band_tree(d, L, 2, (0.5, 0.5), 0.3, 0.05), 1.0, wl.constant_rhs(d, L))
    us, hs = ad.solve(Ss, tol=1e-9)
    # the same cycles; re-building the iterate at each (empty) move only
    # rounds it (1e-16 of the values)
    assert len(hist) == len(hs)
    np.testing.assert_allclose([h for _, h in hist], hs, rtol=0, atol=1e-13)
    assert np.abs(u - us).max() <= 1e-12 * np.abs(us).max()


def test_moving_band_converges_to_the_last_trees_solution():
    d, L = 2, 4
    one = lambda x: np.ones(len(x))
    S, u, hist = ad.moving_band_solve(d, L, 2, 1.0, one, (0.5, 0.5), 0.3, 0.05, 0.05, 5, 4,
                                      tol=1e-9)
    assert hist[-1][1] <= 1e-9
    ud = ad.direct_solution(S)
    assert np.abs(u - ud).max() <= 1e-7 * np.abs(ud).max()
    # the band moved: the last tree differs from the first
    first = ad.band_tree(d, L, 2, (0.5, 0.5), 0.3, 0.05)
    assert not np.array_equal(first.exists[L], S.tree.exists[L])


@pytest.mark.parametrize("d,L,tree", [(2, 3, "corner"), (2, 4, "band"), (3, 3, "corner"),
                                      (2, 3, "regular")])
def test_level_wise_fas_htmg_gives_the_tested_residuals(d, L, tree):
    # Eq. 4 on the spacetree, cell by cell (injection, hierarchical values,
    # Galerkin element matrices of refined cells) against the composite
    # residual tested with every level's pagodas
    T = {"corner": _corner_tree, "band": _band_tree,
         "regular": lambda d, L: ad.regular_tree(d, L)}[tree](d, L)
    N = 3 ** L
    eps = np.random.default_rng(3).uniform(0.2, 3.0, size=(N,) * d)
    S = ad.build_system(T, eps, wl.manufactured_rhs(d, L))
    B = ad.composite_basis(S)
    u = B @ np.random.default_rng(1).standard_normal(B.shape[1])
    rf, dg = ad.fas_level_residuals(S, u, return_diag=True)
    rg = ad.level_residuals(S, u)
    for l in rg:
        assert np.abs(rf[l] - rg[l]).max() <= 1e-13 * np.abs(rg[l]).max(), l
        # the Jacobi diagonal from the cells' Galerkin element matrices
        assert np.abs(dg[l] - S.diag[l]).max() <= 1e-13 * S.diag[l].max(), l


# ---------------------------------------------------------------------------
# the adaptive runs of Sec. 5

def test_second_derivative_indicator_is_exact_for_quadratics():
    d, L = 2, 3
    S = ad.build_system(_corner_tree(d, L), 1.0, wl.constant_rhs(d, L))
    lin = ad.from_vertex_values(S, ad.sample(S, lambda x: 2.0 * x[:, 0] - x[:, 1]))
    assert np.abs(ad.second_derivative_indicator(S, lin)[2]).max() <= 1e-9
    # u = x^2 - 3 y^2 (nodal values): central second differences give 2 and 6
    quad = ad.from_vertex_values(S, ad.sample(S, lambda x: x[:, 0] ** 2 - 3.0 * x[:, 1] ** 2))
    lev, vidx, vals = ad.second_derivative_indicator(S, quad)
    # vertices whose axis neighbours are vertices of the nodal space on their
    # own level (away from hanging nodes) see the exact values
    interior = np.all((vidx >= 1) & (vidx <= 3 ** lev[:, None] - 1), axis=1)
    assert np.isclose(np.median(vals[interior]), 6.0, rtol=1e-9)


def test_top_fraction_takes_the_largest_values():
    v = np.random.default_rng(0).exponential(size=5000)
    sel = ad._top_fraction(v, 0.1)
    assert 0.05 * len(v) <= len(sel) <= 0.1 * len(v)
    rest = np.setdiff1d(np.arange(len(v)), sel)
    assert v[sel].min() >= v[rest].max() - v.max() / 64    # within one bin


def test_amr_run_refines_the_bottom_and_converges_to_the_composite_solution():
    d, lmax = 2, 4
    bottom = lambda x: (x[:, 1] == 0).astype(float)
    S, u, hist = ad.amr_solve(d, lmax, bottom, tol=1e-8, max_cycles=300)
    assert hist[-1][1] <= 1e-8
    # every cell along x_2 = 0 reaches the finest level
    assert np.all(S.tree.exists[lmax][0, :])
    # the tree is adaptive, not regular
    assert not np.all(S.tree.exists[lmax])
    ud = ad.direct_solution(S, ad.sample(S, bottom))
    assert np.abs(u - ud).max() <= 1e-7
    # the cost counts every level's active vertices per cycle
    assert hist[-1][2] == pytest.approx(sum(h[2] - p[2] for h, p in zip(hist[1:], hist[:-1])))


def test_adafac_jac_converges_on_an_adaptive_run_across_a_strong_material_jump():
    # Sec. 5.2: with d-linear transfers adAFAC-Jac converges for every jump
    # eps = 10^-k tested; here the halves setup, eps = 1e-7 right of x_1 = 1/2
    d, lmax = 2, 5
    bottom = lambda x: (x[:, 1] == 0).astype(float)
    eps = wl.eps_halves(d, lmax, 1e-7)
    S, u, hist = ad.amr_solve(d, lmax, bottom, eps=eps, tol=1e-8, max_cycles=400, variant="jac")
    assert hist[-1][1] <= 1e-8
    ud = ad.direct_solution(S, ad.sample(S, bottom))
    assert np.abs(u - ud).max() <= 1e-6
