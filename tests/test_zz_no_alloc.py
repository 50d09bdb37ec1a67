"""adafac_residual_norm_static: the residual norm sqrt(h^d sum_i r_i^2) of
r = b - A u, computed with the library's fixed device scratch array instead of
a workspace, for callers that cannot allocate device memory.  It must agree
with the oracle's norm and with the handle's own residual norm on the same u
and b, call after call, ignore b's boundary ring, and reject trees larger than
its scratch without launching.

This file is named so that pytest collects it last: the check also covers a
process in which every other test has already run."""
import ctypes

import numpy as np
import pytest

import workloads as wl
from oracle import cycle as oc
from oracle import fem
from paper_1903_10367_gb300 import adafac


def test_trees_beyond_the_scratch_are_rejected_before_any_launch():
    lib = adafac.load()
    fake = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    # (3^6 + 1)^3 = 389 M vertices > 4096 * 16384
    assert lib.adafac_residual_norm_static(3, 6, 1.0, fake, fake, fake, None) == 1
    assert lib.adafac_residual_norm_static(4, 2, 1.0, fake, fake, fake, None) == 1
    assert lib.adafac_residual_norm_static(2, 3, -1.0, fake, fake, fake, None) == 1
    assert lib.adafac_residual_norm_static(2, 3, 1.0, None, fake, fake, None) == 1


def _oracle_norm(d, L, eps, u, b):
    """The oracle's residual norm of u against b: the fine operator from eps
    and the norm over the interior vertices."""
    n = 3 ** L
    op = fem.LevelOperator.from_eps(d, n, [eps], True)
    H = oc.Hierarchy(d, L, {L: oc.Level(L, n, op, op.diagonal())}, b, None, None)
    return oc.residual_norm(H, oc.residual(H, L, u, b))


def _static_norms(d, L, eps, u, b, calls=2):
    torch = pytest.importorskip("torch")
    ud = torch.from_numpy(np.ascontiguousarray(u).reshape(-1)).cuda()
    bd = torch.from_numpy(np.ascontiguousarray(b).reshape(-1)).cuda()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    got = []
    for _ in range(calls):
        out.fill_(-1.0)
        adafac.residual_norm_static(d, L, eps, ud, bd, out)
        torch.cuda.synchronize()
        got.append(out.item())
    return got


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


@pytest.mark.gpu
@pytest.mark.parametrize("d,L,eps", [(2, 4, 1.0), (2, 5, 2.5), (3, 3, 1.0), (3, 4, 0.7)])
def test_static_scratch_norm_equals_the_handle_and_oracle_norms_on_consecutive_calls(d, L, eps):
    _cuda()
    f = wl.manufactured_rhs(d, L)
    S = adafac.Solver(d, L, eps, f, adafac.default_options())
    S.cycle(3)
    _, ab = S.residual_norm()
    u = np.ascontiguousarray(S.solution())
    S.close()
    b = fem.load_vector(f, 1.0 / 3 ** L, d)
    want = _oracle_norm(d, L, eps, u, b)
    assert ab == pytest.approx(want, rel=1e-12)
    for got in _static_norms(d, L, eps, u, b):
        assert got == pytest.approx(want, rel=1e-12)
        assert got == pytest.approx(ab, rel=1e-12)


@pytest.mark.gpu
@pytest.mark.parametrize("d,L,eps,seed", [(3, 5, 1.3, 4), (2, 6, 0.9, 5), (3, 2, 1.0, 6)])
def test_static_scratch_norm_of_random_fields_ignores_the_ring_of_b(d, L, eps, seed):
    # random u with non-zero Dirichlet values on its ring (they enter the
    # stencil of the vertices next to the boundary) and random b whose ring is
    # then overwritten with garbage: the norm equals the oracle's on the same
    # u and the interior of b.  3-D depth 5 uses 888 of the 4096 partial sums,
    # and none of the sizes is a multiple of a block's 16384 vertices.
    _cuda()
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (3 ** L + 1,) * d
    u = rng.uniform(-1.0, 1.0, size=shape)
    b = rng.uniform(-1.0, 1.0, size=shape) * (1.0 / 3 ** L) ** d
    want = _oracle_norm(d, L, eps, u, b)
    ring = b - fem.zero_boundary(b.copy())
    b_bad = fem.zero_boundary(b.copy()) + np.where(ring != 0.0, 1e30, 0.0)
    b_bad[(0,) * d] = np.nan
    for got in _static_norms(d, L, eps, u, b_bad):
        assert got == pytest.approx(want, rel=1e-12)
