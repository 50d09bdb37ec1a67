"""Pins of the oracle's cycles (Alg. 1, Alg. 2, Eq. 2, Eq. 4, Eq. 9, Eq. 10)."""
import itertools
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spl

import workloads as wl
from oracle import cycle, fem, transfer
from tests import _brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "smoothed_prolongation_2d.txt")


def _golden():
    return np.loadtxt(GOLDEN, comments="#")


def test_smoothed_stencil_matches_the_printed_one():
    # Sec. 3.2 prints M^{-1} A_{eps=1} P (d = 2) to three or four digits
    S = cycle.smoothed_prolongation_stencil(2)
    G = _golden()
    assert G.shape == (7, 7)
    for v, g in zip(S.ravel(), G.ravel()):
        text = f"{g:.10g}"
        digits = len(text.split(".")[1]) if "." in text else 0
        assert abs(v - g) <= 0.6 * 10.0 ** (-max(digits, 3)) + 1e-12, (v, g)


def test_truncated_stencil_facts_2d():
    S = cycle.smoothed_prolongation_stencil(2)
    T = cycle.truncate_stencil(S)
    ring = S.copy()
    ring[1:6, 1:6] = 0.0
    assert ring.max() <= 1e-15                       # dropped entries are <= 0
    assert T.min() >= -1e-15
    nz = np.argwhere(np.abs(T) > 1e-14)
    assert len(nz) == 9                              # a plus: centre, +-1, +-2
    assert all((i == 2) or (j == 2) for i, j in nz)
    assert T[2, 2] == pytest.approx(4 / 9)
    assert T[2, 1] == pytest.approx(1 / 6) and T[0, 2] == pytest.approx(1 / 12)
    assert T.sum() == pytest.approx(13 / 9)


def test_truncated_stencil_facts_3d():
    S = cycle.smoothed_prolongation_stencil(3)
    T = cycle.truncate_stencil(S)
    ring = S.copy()
    ring[1:6, 1:6, 1:6] = 0.0
    assert ring.max() <= 1e-15
    assert T.min() >= -1e-15
    assert int(np.sum(np.abs(T) > 1e-14)) == 61
    assert T[2, 2, 2] == pytest.approx(16 / 27)
    assert T.sum() == pytest.approx(169 / 27)
    # full smoothed operator: zero sum (A annihilates constants away from the
    # boundary), symmetric under axis permutations and reflections
    assert abs(S.sum()) < 1e-13
    np.testing.assert_allclose(S, S.transpose(1, 0, 2), atol=1e-15)
    np.testing.assert_allclose(S, S[::-1], atol=1e-15)


@pytest.mark.parametrize("d,variant", [(2, "jac"), (2, "additive"), (2, "pi"), (3, "jac")])
def test_single_level_is_damped_jacobi(d, variant):
    # L = l_min = 1: no coarser level, the cycle is one damped Jacobi step;
    # diag(A) = 8 eps / 3 (2-D) or 32 h eps / 12 (3-D) for constant eps
    eps = 2.0
    n = 3
    f = np.random.default_rng(0).standard_normal((n + 1,) * d)
    H = cycle.build_hierarchy(d, 1, [eps], True, f)
    u = fem.zero_boundary(np.random.default_rng(1).standard_normal((n + 1,) * d))
    got = cycle.cycle(H, u, variant=variant)
    dg = 8 * eps / 3 if d == 2 else 32 * eps / (12 * n)
    want = u + 0.6 * (H.b - H.fine.op.apply(u)) / dg
    fem.zero_boundary(want)
    np.testing.assert_allclose(got, want, atol=1e-14)


def _dense_hierarchy(d, L, eps):
    """A_l, P_l, D_l as dense interior matrices, from global hats and quadrature."""
    A = {}
    Pm = {}
    n = 3 ** L
    Afull = _brute.stiffness_dense(d, n, eps)
    fin = _brute.interior_mask(d, n)
    A[L] = Afull[np.ix_(fin, fin)]
    for l in range(L, 1, -1):
        n_c = 3 ** (l - 1)
        Pd = _brute.dlinear_prolongation_dense(d, n_c)
        Pm[l] = Pd[np.ix_(_brute.interior_mask(d, 3 * n_c), _brute.interior_mask(d, n_c))]
        A[l - 1] = Pm[l].T @ A[l] @ Pm[l]
    D = {l: np.diag(np.diag(A[l])) for l in A}
    return A, Pm, D


def _injection_dense(d, n_c):
    n_f = 3 * n_c
    cin = [J for J in itertools.product(range(1, n_c), repeat=d)]
    fin = [i for i in itertools.product(range(1, n_f), repeat=d)]
    fpos = {i: k for k, i in enumerate(fin)}
    I = np.zeros((len(cin), len(fin)))
    for k, J in enumerate(cin):
        I[k, fpos[tuple(3 * j for j in J)]] = 1.0
    return I


def _rtilde_truncated_2d_dense(n_c):
    """R~ from the closed-form entries of the printed stencil's 5x5 core:
    4/9 at the coarse vertex, 1/6 and 1/12 at distance 1 and 2 along the axes."""
    n_f = 3 * n_c
    cin = [J for J in itertools.product(range(1, n_c), repeat=2)]
    fin = [i for i in itertools.product(range(1, n_f), repeat=2)]
    fpos = {i: k for k, i in enumerate(fin)}
    w = {0: 4 / 9, 1: 1 / 6, 2: 1 / 12}
    Rt = np.zeros((len(cin), len(fin)))
    for k, J in enumerate(cin):
        c = (3 * J[0], 3 * J[1])
        for t in range(-2, 3):
            for p in ((c[0] + t, c[1]), (c[0], c[1] + t)):
                if p in fpos:
                    Rt[k, fpos[p]] = w[abs(t)]
    return Rt


def _rtilde_truncated_dense(d, n_c):
    """R~ / omega from brute-force matrices of the eps = 1 problem on the level
    of n_f = 3 n_c cells: S = D^-1 A P (A from the global hats, P from the
    coarse hats evaluated at the fine vertices), kept where the fine vertex
    lies within two fine cells of 3J in every direction (the 5^d support of
    P), and transposed: row J restricts the fine residual to coarse vertex J."""
    n_f = 3 * n_c
    fin = _brute.interior_mask(d, n_f)
    cin = _brute.interior_mask(d, n_c)
    A = _brute.stiffness_dense(d, n_f, 1.0)[np.ix_(fin, fin)]
    P = _brute.dlinear_prolongation_dense(d, n_c)[np.ix_(fin, cin)]
    S = (A @ P) / np.diag(A)[:, None]
    fpos = np.indices((n_f + 1,) * d).reshape(d, -1).T[fin]
    cpos = np.indices((n_c + 1,) * d).reshape(d, -1).T[cin]
    dist = np.abs(fpos[:, None, :] - 3 * cpos[None, :, :]).max(axis=2)
    S[dist > 2] = 0.0
    return S.T


@pytest.mark.parametrize("d,L,variant,rtilde,lmin", [
    (2, 2, "jac", "truncated", 1), (2, 3, "jac", "truncated", 1), (2, 3, "jac", "exact", 1),
    (2, 3, "additive", "truncated", 1), (2, 3, "pi", "truncated", 1),
    (2, 3, "exp", "truncated", 1), (3, 2, "jac", "exact", 1), (3, 2, "pi", "exact", 1),
    (3, 2, "jac", "truncated", 1),
    (2, 3, "jac", "truncated", 2), (2, 3, "pi", "truncated", 2), (2, 3, "jac", "exact", 3)])
def test_cycle_equals_dense_restatement_of_eq9(d, L, variant, rtilde, lmin):
    rng = np.random.default_rng(12)
    n = 3 ** L
    eps = rng.uniform(0.2, 3.0, size=(n,) * d)
    f = rng.standard_normal((n + 1,) * d)
    H = cycle.build_hierarchy(d, L, eps, False, f)
    u = fem.zero_boundary(rng.standard_normal((n + 1,) * d))
    got = fem.interior(cycle.cycle(H, u, variant=variant, rtilde=rtilde, omega_exp=0.7,
                                   lmin=lmin)).ravel()

    A, Pm, D = _dense_hierarchy(d, L, eps)
    w = wt = 0.6
    b = fem.interior(H.b).ravel()
    ui = fem.interior(u).ravel()
    r = b - A[L] @ ui

    def Pchain(l):          # prolongation from level l to L
        M = np.eye(A[L].shape[0])
        for m in range(L, l, -1):
            M = M @ Pm[m]
        return M

    M = np.zeros((A[L].shape[0], A[L].shape[0]))
    for l in range(lmin, L + 1):
        scale = 0.7 ** (L - l) if variant == "exp" else 1.0
        M += scale * Pchain(l) @ (w * np.linalg.inv(D[l])) @ Pchain(l).T
    if variant == "jac":
        for l in range(lmin + 1, L + 1):
            if rtilde == "exact":
                Rt = w * Pm[l].T @ A[l] @ np.linalg.inv(D[l])
            elif d == 2:
                Rt = w * _rtilde_truncated_2d_dense(3 ** (l - 1))
            else:
                Rt = w * _rtilde_truncated_dense(d, 3 ** (l - 1))
            M -= Pchain(l - 1) @ (wt * np.linalg.inv(D[l - 1])) @ Rt @ Pchain(l).T
    if variant == "pi":
        for l in range(lmin + 1, L + 1):
            PI = Pm[l] @ _injection_dense(d, 3 ** (l - 1))
            M -= Pchain(l) @ PI @ (w * np.linalg.inv(D[l])) @ Pchain(l).T
    want = ui + M @ r
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-12 * np.abs(want).max())


@pytest.mark.parametrize("transfer_kind", ["dlinear", "boxmg"])
def test_fas_form_equals_correction_scheme(transfer_kind):
    # with Galerkin operators, b_l - A_l I u = R r_{l+1} exactly (Eq. 4)
    w = wl.get("jump2d_d6").with_depth(4)
    eps, sc = w.eps()
    H = cycle.build_hierarchy(2, 4, eps, sc, w.f(), transfer_kind)
    u = wl.random_vertex_field(2, 4, 7)
    for variant in ("jac", "pi", "additive"):
        a = cycle.cycle(H, u, variant=variant, form="cs")
        b = cycle.cycle(H, u, variant=variant, form="fas")
        np.testing.assert_allclose(a, b, atol=1e-12 * np.abs(a).max())


@pytest.mark.parametrize("d,L,transfer_kind", [(2, 3, "boxmg"), (2, 3, "dlinear"), (3, 2, "boxmg")])
def test_all_variants_converge_to_the_direct_solution(d, L, transfer_kind):
    rng = np.random.default_rng(21)
    n = 3 ** L
    eps = rng.choice([1.0, 1e-2], size=(n,) * d)
    f = np.ones((n + 1,) * d)
    H = cycle.build_hierarchy(d, L, eps, False, f, transfer_kind)
    Afull = _brute.stiffness_dense(d, n, eps)
    fin = _brute.interior_mask(d, n)
    x = np.linalg.solve(Afull[np.ix_(fin, fin)], fem.interior(H.b).ravel())
    for variant in ("jac", "pi", "additive"):
        u, hist = cycle.solve(H, variant=variant, tol=1e-13, max_cycles=2000)
        assert hist[-1] <= 1e-13
        np.testing.assert_allclose(fem.interior(u).ravel(), x, rtol=1e-9,
                                   atol=1e-10 * np.abs(x).max())


def test_manufactured_solution_error_is_second_order():
    errs = {}
    for d, depths in ((2, (3, 4, 5)), (3, (2, 3))):
        for L in depths:
            w = wl.Workload("m", d, L, "scalar")
            H = cycle.build_hierarchy(d, L, *w.eps(), w.f())
            u, hist = cycle.solve(H, tol=1e-10, max_cycles=400)
            errs[d, L] = np.abs(u - wl.manufactured_solution(d, L)).max()
    for d, L in ((2, 3), (2, 4), (3, 2)):
        ratio = errs[d, L] / errs[d, L + 1]
        assert 8.0 < ratio < 10.0, (d, L, ratio)


def test_residual_norm_eq10():
    H = cycle.build_hierarchy(2, 2, [1.0], True, np.zeros((10, 10)))
    r = np.zeros((10, 10))
    r[1:-1, 1:-1] = 2.0
    assert cycle.residual_norm(H, r) == pytest.approx(np.sqrt(64 * 4 / 81))
    assert cycle.max_residual(r) == 2.0


def _lambda_max(H, variant):
    L, d = H.L, H.d
    n = 3 ** L
    N = (n - 1) ** d
    I = tuple(slice(1, -1) for _ in range(d))
    b_saved = H.b.copy()
    H.b[:] = 0.0

    def BA(x):
        u = np.zeros((n + 1,) * d)
        u[I] = x.reshape((n - 1,) * d)
        return (u - cycle.cycle(H, u, variant=variant))[I].ravel()

    op = spl.LinearOperator((N, N), matvec=BA)
    lam = spl.eigs(op, k=1, which="LM", return_eigenvectors=False, maxiter=5000)
    H.b[:] = b_saved
    return float(np.abs(lam).max())


def test_plain_additive_overshoot_grows_with_the_number_of_levels():
    # Sec. 2.2 / 5.1: summing all levels' corrections overshoots more the more
    # levels there are (lambda_max of the preconditioned operator B A grows
    # towards 2, where the iteration stops converging); adAFAC's damping keeps
    # lambda_max lower, adAFAC-PI keeps it below one
    lam = {}
    for L in (2, 3, 4):
        H = cycle.build_hierarchy(2, L, [1.0], True, np.zeros((3 ** L + 1,) * 2))
        for v in ("additive", "jac", "pi"):
            lam[v, L] = _lambda_max(H, v)
    assert lam["additive", 2] < lam["additive", 3] < lam["additive", 4]
    assert lam["additive", 4] > 1.5
    for L in (3, 4):
        assert lam["jac", L] < lam["additive", L] - 0.2
        assert lam["pi", L] < 1.0


# ---------------------------------------------------------------------------
# non-zero Dirichlet data (the setups of Sec. 5: u = 1 on x_2 = 0)

@pytest.mark.parametrize("d,L,transfer_kind", [(2, 3, "dlinear"), (2, 3, "boxmg"), (3, 2, "dlinear")])
def test_linear_boundary_data_give_the_linear_solution(d, L, transfer_kind):
    # d-linear elements contain the linear functions and, for constant eps and
    # f = 0, A applied to a linear function vanishes at interior vertices:
    # the discrete solution is the linear function itself
    n = 3 ** L
    coords = np.meshgrid(*([np.arange(n + 1) / n] * d), indexing="ij")
    lin = 0.3 + sum((k + 1) * 0.7 * c for k, c in enumerate(coords))
    H = cycle.build_hierarchy(d, L, [2.5], True, np.zeros((n + 1,) * d), transfer_kind)
    for variant in ("jac", "pi", "additive"):
        u, hist = cycle.solve(H, cycle.with_boundary(lin), variant=variant, tol=1e-13,
                              max_cycles=3000)
        assert hist[-1] <= 1e-13
        np.testing.assert_allclose(u, lin, rtol=0, atol=1e-10)


@pytest.mark.parametrize("d,L,transfer_kind", [(2, 3, "boxmg"), (3, 2, "boxmg")])
def test_boundary_data_match_a_lifted_direct_solve(d, L, transfer_kind):
    # u_I = A_II^-1 (b_I - A_IB g_B) with the brute-force stiffness matrix
    rng = np.random.default_rng(5)
    n = 3 ** L
    eps = rng.choice([1.0, 1e-3], size=(n,) * d)
    g = np.zeros((n + 1,) * d)
    g[0] = 1.0  # u = 1 on the face x_2 = 0 (first array axis), 0 elsewhere
    f = np.ones((n + 1,) * d)
    H = cycle.build_hierarchy(d, L, eps, False, f, transfer_kind)
    Afull = _brute.stiffness_dense(d, n, eps)
    fin = _brute.interior_mask(d, n)
    gb = cycle.with_boundary(g).ravel()
    rhs = fem.interior(H.b).ravel() - Afull[np.ix_(fin, ~fin)] @ gb[~fin]
    x = np.linalg.solve(Afull[np.ix_(fin, fin)], rhs)
    u, hist = cycle.solve(H, cycle.with_boundary(g), variant="jac", tol=1e-13, max_cycles=3000)
    assert hist[-1] <= 1e-13
    np.testing.assert_allclose(fem.interior(u).ravel(), x, rtol=1e-9, atol=1e-10)
    np.testing.assert_array_equal(u - fem.zero_boundary(u.copy()), cycle.with_boundary(g))


# ---------------------------------------------------------------------------
# rediscretised coarse operators

def test_rediscretised_levels_are_the_fem_operator_of_the_averaged_eps():
    d, L = 2, 3
    rng = np.random.default_rng(9)
    eps = rng.choice([1.0, 1e-2, 5.0], size=(3 ** L,) * d)
    H = cycle.build_hierarchy(d, L, eps, False, np.ones((3 ** L + 1,) * d), "boxmg",
                              coarse_op="rediscretised")
    e = eps
    for l in range(L - 1, 0, -1):
        n_c = 3 ** l
        avg = np.zeros((n_c,) * d)
        for i in range(n_c):
            for j in range(n_c):
                avg[i, j] = e[3 * i:3 * i + 3, 3 * j:3 * j + 3].sum() / 9.0
        A = _brute.stiffness_dense(d, n_c, avg)
        fin = _brute.interior_mask(d, n_c)
        lv = H.levels[l]
        Ad = np.stack([fem.interior(lv.op.apply(v.reshape((n_c + 1,) * d))).ravel()
                       for v in np.eye((n_c + 1) ** d)[fin]], axis=1)
        np.testing.assert_allclose(Ad, A[np.ix_(fin, fin)], rtol=1e-12, atol=1e-14)
        e = avg


@pytest.mark.parametrize("d", [2, 3])
def test_rediscretised_equals_galerkin_when_eps_is_constant_on_coarse_cells(d):
    # d-linear P and eps constant on every level-1 cell: each coarse
    # rediscretisation is the Galerkin operator (the identity behind Sec. 2.2)
    L = 3 if d == 2 else 2
    rng = np.random.default_rng(4)
    block = rng.choice([1.0, 0.1, 3.0], size=(3,) * d)
    eps = block
    for ax in range(d):
        eps = np.repeat(eps, 3 ** (L - 1), axis=ax)
    f = np.ones((3 ** L + 1,) * d)
    Hg = cycle.build_hierarchy(d, L, eps, False, f, "dlinear")
    Hr = cycle.build_hierarchy(d, L, eps, False, f, "dlinear", coarse_op="rediscretised")
    for l in range(1, L):
        n_c = 3 ** l
        fin = _brute.interior_mask(d, n_c)
        units = np.eye((n_c + 1) ** d)[fin]

        def dense(op):
            return np.stack([fem.interior(op.apply(v.reshape((n_c + 1,) * d))).ravel()
                             for v in units], axis=1)

        np.testing.assert_allclose(dense(Hr.levels[l].op), dense(Hg.levels[l].op),
                                   rtol=1e-12, atol=1e-13)


def _vcycle(H, l, u, b, nu=2, w=0.6):
    """A multiplicative V(nu, nu)-cycle with damped Jacobi smoothing on the
    same hierarchy (the textbook scheme, for comparison only): pre-smoothing,
    coarse correction P (cycle on R r), post-smoothing; exact solve on level 1."""
    lev = H.levels[l]
    d = H.d

    def jacobi(u):
        r = fem.zero_boundary(b - lev.op.apply(u))
        return u + cycle.jacobi_correction(H, l, r, w)

    if l == 1:
        n = lev.n
        N = (n + 1) ** d
        M = np.zeros((N, N))
        for k in range(N):
            e = np.zeros(N)
            e[k] = 1.0
            M[:, k] = lev.op.apply(e.reshape((n + 1,) * d)).ravel()
        inn = _brute.interior_mask(d, n)
        x = np.zeros(N)
        x[inn] = np.linalg.solve(M[np.ix_(inn, inn)], b.ravel()[inn])
        return x.reshape(b.shape)
    for _ in range(nu):
        u = jacobi(u)
    rc = cycle.R(H, l, fem.zero_boundary(b - lev.op.apply(u)))
    u = u + cycle.P(H, l, _vcycle(H, l - 1, np.zeros_like(rc), rc, nu, w))
    for _ in range(nu):
        u = jacobi(u)
    return u


def _cycles_to(H, step, tol=1e-8, cap=2000):
    u = np.zeros_like(H.b)
    r0 = cycle.residual_norm(H, cycle.residual(H, H.L, u, H.b))
    for c in range(1, cap + 1):
        u = step(u)
        if cycle.residual_norm(H, cycle.residual(H, H.L, u, H.b)) / r0 <= tol:
            return c
    return cap


def test_slow_convergence_on_fine_blocks_is_a_property_of_the_geometric_hierarchy():
    # Sec. 2.4 and Sec. 5: BoxMG transfers restore the Poisson convergence for
    # jumps that the coarse levels can represent, and no cycle on the same
    # hierarchy does better when the blocks are finer than the coarse cells.
    # 2-D depth 3, f = 1, eps in {1, 1e-2}; counts to 1e-8 from u = 0.
    d, L, n = 2, 3, 27
    f = wl.constant_rhs(d, L)

    def counts(eps, kind):
        H = cycle.build_hierarchy(d, L, eps, False, f, kind)
        return (_cycles_to(H, lambda u: cycle.cycle(H, u, variant="jac")),
                _cycles_to(H, lambda u: _vcycle(H, L, u, H.b), cap=400))

    jac0, v0 = counts(np.ones((n, n)), "dlinear")
    rng = np.random.Generator(np.random.PCG64(1903))
    cols = np.broadcast_to(np.repeat(rng.choice([1.0, 1e-2], size=9), 3)[:, None], (n, n))
    # eps varying along x in columns of 3 cells: BoxMG interpolation is the
    # exact 1-D one, d-linear is not
    jb, vb = counts(cols.copy(), "boxmg")
    jd, vd = counts(cols.copy(), "dlinear")
    assert jb <= 1.15 * jac0 and vb <= 1.2 * v0, (jb, vb, jac0, v0)
    assert jd >= 2 * jac0 and vd >= 2 * v0, (jd, vd)
    # random blocks of level-1 cells: every level resolves them
    for kind in ("dlinear", "boxmg"):
        j, _ = counts(wl.eps_random_blocks(d, L, 9, 1e-2, 1903), kind)
        assert j <= 1.3 * jac0, (kind, j, jac0)
    # random blocks of level-2 cells, finer than the level-1 cells: the
    # multiplicative cycle slows by the same factor as adAFAC-Jac, so the
    # slowdown belongs to the coarse spaces, not to the additive method
    j, v = counts(wl.eps_random_blocks(d, L, 3, 1e-2, 1903), "boxmg")
    assert j >= 4 * jac0 and v >= 4 * v0, (j, v, jac0, v0)
    assert abs((j / jac0) / (v / v0) - 1.0) <= 0.3, (j / jac0, v / v0)
