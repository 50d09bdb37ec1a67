"""Pins of the oracle's transfer operators and Galerkin coarse operators
(Sec. 2.2, 2.4)."""
import itertools

import numpy as np
import pytest

from oracle import fem, transfer
from tests import _brute


def _P_dense_from_oracle(Pv, d, n_c):
    """Columns P e_J of the oracle's prolongation for every interior coarse J."""
    cols = []
    for J in itertools.product(range(1, n_c), repeat=d):
        e = np.zeros((n_c + 1,) * d)
        e[J] = 1.0
        cols.append(transfer.prolong(Pv, e).ravel())
    return np.array(cols).T


@pytest.mark.parametrize("d,n_c", [(2, 3), (2, 9), (3, 3)])
def test_dlinear_P_equals_coarse_hats(d, n_c):
    # P e_J must be the coarse d-linear hat of J sampled at the fine vertices
    Pv = transfer.vertex_weights(transfer.dlinear_closure_weights(d, n_c), n_c)
    got = _P_dense_from_oracle(Pv, d, n_c)
    Pd = _brute.dlinear_prolongation_dense(d, n_c)
    fine_in = _brute.interior_mask(d, 3 * n_c)
    coarse_in = _brute.interior_mask(d, n_c)
    want = Pd[:, coarse_in].copy()
    want[~fine_in] = 0.0
    np.testing.assert_allclose(got, want, atol=1e-15)


def test_dlinear_P_reproduces_constants_away_from_boundary():
    d, n_c = 2, 9
    Pv = transfer.vertex_weights(transfer.dlinear_closure_weights(d, n_c), n_c)
    ones = np.zeros((n_c + 1,) * d)
    ones[1:-1, 1:-1] = 1.0
    pf = transfer.prolong(Pv, ones)
    np.testing.assert_allclose(pf[3:-3, 3:-3], 1.0, atol=1e-15)


@pytest.mark.parametrize("kind", ["dlinear", "boxmg"])
def test_restriction_is_transpose(kind):
    rng = np.random.default_rng(3)
    d, n_c = 2, 9
    n_f = 3 * n_c
    if kind == "dlinear":
        W = transfer.dlinear_closure_weights(d, n_c)
    else:
        eps = rng.uniform(1e-2, 1.0, size=(n_f, n_f))
        W = transfer.boxmg_closure_weights(
            fem.LevelOperator.from_eps(d, n_f, eps, False).stencils(), n_c)
    Pv = transfer.vertex_weights(W, n_c)
    r = fem.zero_boundary(rng.standard_normal((n_f + 1,) * d))
    v = fem.zero_boundary(rng.standard_normal((n_c + 1,) * d))
    lhs = np.vdot(transfer.restrict(Pv, r), v)
    rhs = np.vdot(r, transfer.prolong(Pv, v))
    assert lhs == pytest.approx(rhs, rel=1e-13)


@pytest.mark.parametrize("d,L,eps", [(2, 2, 1.0), (2, 3, 7.0), (3, 2, 0.3)])
def test_boxmg_equals_dlinear_for_constant_eps(d, L, eps):
    # Sec. 5.1: for Poisson BoxMG yields the geometric (d-linear) transfers
    n_f = 3 ** L
    op = fem.LevelOperator.from_eps(d, n_f, [eps], True)
    Wb = transfer.boxmg_closure_weights(op.stencils(), n_f // 3)
    Wd = transfer.dlinear_closure_weights(d, n_f // 3)
    np.testing.assert_allclose(Wb, Wd, atol=1e-14)


def test_boxmg_gamma_points_for_eps_varying_along_x():
    # eps depends on x only: the stencil collapsed along y is the 1-D flux
    # operator [-eps_l, eps_l + eps_r, -eps_r], whose discrete harmonic
    # interpolant is linear in the resistance sum_j 1/eps_j
    rng = np.random.default_rng(11)
    d, n_f = 2, 27
    n_c = 9
    col = rng.uniform(1e-3, 1.0, size=n_f)
    eps = np.broadcast_to(col[None, :], (n_f, n_f)).copy()
    W = transfer.boxmg_closure_weights(
        fem.LevelOperator.from_eps(d, n_f, eps, False).stencils(), n_c)
    pidx = {l: k for k, l in enumerate(transfer.closure_points(2))}
    cidx = {c: k for k, c in enumerate(fem.corners(2))}
    for Ey in range(1, n_c - 1):          # interior horizontal coarse lines
        for Ex in range(1, n_c - 1):
            res = 1.0 / col[3 * Ex:3 * Ex + 3]
            for lx in (1, 2):
                want_left = res[lx:].sum() / res.sum()
                # fine point (y = 3 Ey, x = 3 Ex + lx): local (0, lx) of cell (Ey, Ex)
                got_left = W[Ey, Ex, pidx[(0, lx)], cidx[(0, 0)]]
                got_right = W[Ey, Ex, pidx[(0, lx)], cidx[(0, 1)]]
                assert got_left == pytest.approx(want_left, rel=1e-12)
                assert got_right == pytest.approx(1.0 - want_left, rel=1e-12)


def test_boxmg_3d_points_for_eps_varying_along_x():
    # 3-D, eps depends on x only.  gamma points on coarse edges along x: the
    # stencil collapsed along y and z is again the 1-D flux operator, so the
    # weights are linear in the resistance.  gamma points on coarse faces
    # normal to x: collapsed along x the operator in (y, z) has constant
    # coefficients, so the weights are the bilinear ones.
    rng = np.random.default_rng(12)
    d, n_f, n_c = 3, 9, 3
    col = rng.uniform(1e-3, 1.0, size=n_f)
    eps = np.broadcast_to(col[None, None, :], (n_f,) * 3).copy()
    W = transfer.boxmg_closure_weights(
        fem.LevelOperator.from_eps(d, n_f, eps, False).stencils(), n_c)
    pidx = {l: k for k, l in enumerate(transfer.closure_points(3))}
    cidx = {c: k for k, c in enumerate(fem.corners(3))}
    Ex = 1                                  # both edge ends interior
    res = 1.0 / col[3 * Ex:3 * Ex + 3]
    for Ez in (1, 2):
        for Ey in (1, 2):
            for lx in (1, 2):
                want = res[lx:].sum() / res.sum()
                w0 = W[Ez, Ey, Ex, pidx[(0, 0, lx)], cidx[(0, 0, 0)]]
                w1 = W[Ez, Ey, Ex, pidx[(0, 0, lx)], cidx[(0, 0, 1)]]
                assert w0 == pytest.approx(want, rel=1e-12)
                assert w1 == pytest.approx(1.0 - want, rel=1e-12)
    # the face x = 3 Ex of the interior cell (1, 1, 1), all of whose corners
    # are interior vertices
    for ly in (1, 2):
        for lz in (1, 2):
            w = W[1, 1, 1, pidx[(lz, ly, 0)], cidx[(0, 0, 0)]]
            assert w == pytest.approx((1 - ly / 3) * (1 - lz / 3), rel=1e-12)


@pytest.mark.parametrize("d,L", [(2, 3), (3, 2)])
def test_boxmg_fpoint_equations_hold(d, L):
    # the defining property: (A P e)_f = 0 at every f-point, checked with the
    # element-wise operator (a different route than the stencil solves)
    rng = np.random.default_rng(2)
    n_f = 3 ** L
    n_c = n_f // 3
    eps = rng.choice([1.0, 1e-3], size=(n_f,) * d)
    op = fem.LevelOperator.from_eps(d, n_f, eps, False)
    Pv = transfer.vertex_weights(transfer.boxmg_closure_weights(op.stencils(), n_c), n_c)
    fmask = np.ones((n_f + 1,) * d, dtype=bool)
    for ax in range(d):
        idx = np.arange(n_f + 1) % 3 == 0
        shape = [1] * d
        shape[ax] = n_f + 1
        fmask &= ~idx.reshape(shape)
    for J in itertools.product(range(1, n_c), repeat=d):
        e = np.zeros((n_c + 1,) * d)
        e[J] = 1.0
        w = op.apply(transfer.prolong(Pv, e))
        assert np.abs(w[fmask]).max() < 1e-13 * max(1.0, np.abs(w).max())


def _dense_from_apply(apply, d, n):
    cols = []
    for J in itertools.product(range(1, n), repeat=d):
        e = np.zeros((n + 1,) * d)
        e[J] = 1.0
        cols.append(fem.interior(apply(e)).ravel())
    return np.array(cols).T


@pytest.mark.parametrize("kind,d,L", [("dlinear", 2, 2), ("boxmg", 2, 2),
                                      ("boxmg", 2, 3), ("boxmg", 3, 2)])
def test_galerkin_equals_dense_RAP(kind, d, L):
    rng = np.random.default_rng(4)
    n_f = 3 ** L
    n_c = n_f // 3
    eps = rng.uniform(1e-3, 1.0, size=(n_f,) * d)
    op = fem.LevelOperator.from_eps(d, n_f, eps, False)
    if kind == "dlinear":
        W = transfer.dlinear_closure_weights(d, n_c)
    else:
        W = transfer.boxmg_closure_weights(op.stencils(), n_c)
    Pv = transfer.vertex_weights(W, n_c)
    cop = transfer.galerkin(op, W, n_c)
    # brute-force dense stiffness and the oracle's P as a dense matrix
    Afull = _brute.stiffness_dense(d, n_f, eps)
    fin = _brute.interior_mask(d, n_f)
    A = Afull[np.ix_(fin, fin)]
    Pm = _P_dense_from_oracle(Pv, d, n_c)[fin]
    want = Pm.T @ A @ Pm
    got = _dense_from_apply(cop.apply, d, n_c)
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-13 * np.abs(want).max())


@pytest.mark.parametrize("d", [2, 3])
def test_galerkin_equals_rediscretisation_for_cellwise_constant_eps(d):
    # d-linear P is exact for the coarse FE space: R A P = coarse FE stiffness
    # when eps is constant on every coarse cell
    rng = np.random.default_rng(8)
    n_c = 3
    n_f = 9
    eps_c = rng.uniform(0.1, 2.0, size=(n_c,) * d)
    eps_f = eps_c
    for ax in range(d):
        eps_f = np.repeat(eps_f, 3, axis=ax)
    op = fem.LevelOperator.from_eps(d, n_f, eps_f, False)
    cop = transfer.galerkin(op, transfer.dlinear_closure_weights(d, n_c), n_c)
    ref = fem.LevelOperator.from_eps(d, n_c, eps_c, False)
    np.testing.assert_allclose(_dense_from_apply(cop.apply, d, n_c),
                               _dense_from_apply(ref.apply, d, n_c), atol=1e-14)


def test_galerkin_boxmg_properties():
    rng = np.random.default_rng(9)
    d, n_f = 2, 27
    n_c = 9
    eps = rng.choice([1.0, 1e-3], size=(n_f, n_f))
    op = fem.LevelOperator.from_eps(d, n_f, eps, False)
    cop = transfer.galerkin(op, transfer.boxmg_closure_weights(op.stencils(), n_c), n_c)
    M = _dense_from_apply(cop.apply, d, n_c)
    np.testing.assert_allclose(M, M.T, atol=1e-14 * np.abs(M).max())
    assert np.all(np.diag(M) > 0)
    st = cop.stencils()
    # interior rows (all neighbours interior) sum to zero: constants lie in the
    # kernel of the Neumann-free interior operator
    assert np.abs(st[2:-2, 2:-2].sum(axis=-1)).max() < 1e-13 * np.abs(st).max()
