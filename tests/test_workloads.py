"""The seeded input generators shared by the oracle, the tests and the bench
(workloads/): shapes, value sets and reproducibility of the configurations
and of the serving stream."""
import numpy as np
import pytest

import workloads as wl


@pytest.mark.parametrize("name", sorted(wl.WORKLOADS))
def test_configurations_have_the_stated_shapes(name):
    w = wl.get(name)
    eps, sc = w.eps()
    N = 3 ** w.depth
    assert w.f().shape == (N + 1,) * w.dim
    if sc:
        assert eps.shape == (1,) and eps[0] > 0
    else:
        assert eps.shape == (N,) * w.dim
        assert set(np.unique(eps)) <= {1.0, w.eps_low}
        # constant on blocks of block_cells^d fine cells
        b = w.block_cells
        blocks = eps.reshape(*sum(((N // b, b) for _ in range(w.dim)), ()))
        axes = tuple(range(1, 2 * w.dim, 2))
        assert np.all(blocks.max(axis=axes) == blocks.min(axis=axes))
    assert len(w.level_dofs()) == w.depth and w.level_dofs()[-1] == (N - 1) ** w.dim


def test_random_blocks_are_reproducible_and_seed_dependent():
    a = wl.eps_random_blocks(2, 4, 9, 1e-3, 1903)
    b = wl.eps_random_blocks(2, 4, 9, 1e-3, 1903)
    c = wl.eps_random_blocks(2, 4, 9, 1e-3, 1904)
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, c)


def test_serving_stream_mix_and_arrivals():
    reqs = wl.serving_requests(400, seed=1903)
    dims = np.array([r.dim for r in reqs])
    assert 0.7 < np.mean(dims == 2) < 0.9          # 80 % 2-D
    for r in reqs:
        lo, hi = (3, 6) if r.dim == 2 else (3, 5)
        assert lo <= r.depth <= hi
        assert set(np.unique(r.eps)) <= {1.0, 1e-2}
        assert r.f.shape == (3 ** r.depth + 1,) * r.dim
    t = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(t) > 0)
    assert 0.8 < np.mean(np.diff(t)) < 1.2           # unit-rate Poisson clock
    again = wl.serving_requests(400, seed=1903)
    assert all(np.array_equal(a.eps, b.eps) and a.arrival == b.arrival
               for a, b in zip(reqs, again))


def test_manufactured_rhs_matches_its_solution():
    # f = d pi^2 prod sin(pi x_i) for u = prod sin(pi x_i)
    for d, L in ((2, 3), (3, 2)):
        u = wl.manufactured_solution(d, L)
        f = wl.manufactured_rhs(d, L)
        np.testing.assert_allclose(f, d * np.pi ** 2 * u, rtol=1e-14, atol=1e-14)
