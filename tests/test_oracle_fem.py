"""Pins of the oracle's finite-element layer (Eq. 1, Sec. 2.1)."""
import itertools

import numpy as np
import pytest

from oracle import fem
from tests import _brute


def _hamming(a, b):
    return sum(x != y for x, y in zip(a, b))


def test_reference_element_matrix_2d_closed_form():
    # bilinear element: 2/3 on the diagonal, -1/6 along an edge, -1/3 across
    K = fem.reference_element_matrix(2)
    cs = fem.corners(2)
    want = {0: 2 / 3, 1: -1 / 6, 2: -1 / 3}
    for i, a in enumerate(cs):
        for j, b in enumerate(cs):
            assert K[i, j] == pytest.approx(want[_hamming(a, b)], abs=1e-15)


def test_reference_element_matrix_3d_closed_form():
    # trilinear element: 1/3 diagonal, 0 along an edge, -1/12 across a face
    # diagonal and across the body diagonal
    K = fem.reference_element_matrix(3)
    cs = fem.corners(3)
    want = {0: 1 / 3, 1: 0.0, 2: -1 / 12, 3: -1 / 12}
    for i, a in enumerate(cs):
        for j, b in enumerate(cs):
            assert K[i, j] == pytest.approx(want[_hamming(a, b)], abs=1e-15)


@pytest.mark.parametrize("eps", [1.0, 3.5])
def test_assembled_stencil_2d(eps):
    # constant eps: eps/3 * [-1 -1 -1; -1 8 -1; -1 -1 -1], independent of h
    op = fem.LevelOperator.from_eps(2, 9, [eps], True)
    st = op.stencils()[4, 4].reshape(3, 3)
    want = eps / 3.0 * np.array([[-1, -1, -1], [-1, 8, -1], [-1, -1, -1]])
    np.testing.assert_allclose(st, want, atol=1e-14)


@pytest.mark.parametrize("n", [3, 9, 27])
def test_assembled_stencil_3d(n):
    # constant eps = 1: h/12 * (32 centre, 0 face, -2 edge, -1 corner neighbours)
    op = fem.LevelOperator.from_eps(3, n, [1.0], True)
    c = n // 2
    st = op.stencils()[c, c, c].reshape(3, 3, 3)
    h = 1.0 / n
    for o in itertools.product((-1, 0, 1), repeat=3):
        nz = sum(abs(x) for x in o)
        want = h / 12 * {0: 32, 1: 0, 2: -2, 3: -1}[nz]
        assert st[tuple(x + 1 for x in o)] == pytest.approx(want, abs=1e-15)


@pytest.mark.parametrize("d,n", [(2, 3), (2, 9), (3, 3)])
def test_operator_matches_global_quadrature(d, n):
    # A u from element-wise accumulation == dense stiffness matrix assembled
    # from global hat functions (brute force), for random per-cell eps
    rng = np.random.default_rng(5)
    eps = rng.uniform(0.1, 10.0, size=(n,) * d)
    A = _brute.stiffness_dense(d, n, eps)
    inner = _brute.interior_mask(d, n)
    u = rng.standard_normal((n + 1,) * d)
    fem.zero_boundary(u)
    op = fem.LevelOperator.from_eps(d, n, eps, False)
    got = op.apply(u).ravel()[inner]
    want = (A @ u.ravel())[inner]
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(op.diagonal().ravel()[inner], np.diag(A)[inner],
                               rtol=1e-13)


def test_operator_symmetric_and_zero_row_sums():
    rng = np.random.default_rng(1)
    d, n = 2, 27
    eps = rng.uniform(1e-3, 1.0, size=(n, n))
    op = fem.LevelOperator.from_eps(d, n, eps, False)
    u, v = rng.standard_normal((2, n + 1, n + 1))
    fem.zero_boundary(u)
    fem.zero_boundary(v)
    assert np.vdot(op.apply(u), v) == pytest.approx(np.vdot(u, op.apply(v)), rel=1e-12)
    ones = np.ones((n + 1, n + 1))
    # rows of vertices whose neighbourhood excludes the boundary sum to zero
    assert np.abs(op.apply(ones)[2:-2, 2:-2]).max() < 1e-13


def test_load_vector():
    f = np.arange(100.0).reshape(10, 10)
    b = fem.load_vector(f, 1.0 / 9, 2)
    assert b[3, 4] == pytest.approx(f[3, 4] / 81)
    assert b[0, 4] == 0.0 and b[9, 9] == 0.0
