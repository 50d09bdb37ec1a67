"""The fused 3-D sweeps (uniform operator, d-linear transfers, mixed
precision) against the level-by-level kernels and the FP64 oracle.

Both GPU paths compute the same FP32 cycles on the correction equation with
FP64 refinement; they differ only in summation order, so their iterates agree
to FP32 rounding (checked at 2e-5 relative, well above the ~1e-6 observed
spread and far below any algorithmic difference, which would show up at
O(1e-2)).  Mathematically the refined iteration equals the FP64 iteration, so
the oracle's FP64 iterates bound both to the same tolerance.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import cycle as oc
from oracle import fem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1903_10367_gb300 import adafac  # noqa: E402

FP32_RTOL = 2e-5


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _solver(L, path, **opt):
    o = adafac.default_options(precision="mixed", path=path, **opt)
    return adafac.Solver(3, L, 1.0, wl.manufactured_rhs(3, L), o)


@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("variant", ["jac", "additive", "exp"])
@pytest.mark.parametrize("k", [1, 2, 5])
def test_fused_equals_levelwise_and_oracle(L, variant, k):
    n_cycles = 2 * k + 1
    a = _solver(L, "auto", variant=variant, inner_cycles=k, omega_exp=0.7)
    b = _solver(L, "levelwise", variant=variant, inner_cycles=k, omega_exp=0.7)
    a.cycle(n_cycles)
    b.cycle(n_cycles)
    ua, ub = a.solution(), b.solution()
    assert _rel(ua, ub) < FP32_RTOL
    H = oc.build_hierarchy(3, L, [1.0], True, wl.manufactured_rhs(3, L))
    u = np.zeros_like(H.b)
    for _ in range(n_cycles):
        u = oc.cycle(H, u, variant=variant, omega_exp=0.7)
    assert _rel(ua, u) < FP32_RTOL
    if L >= 3:
        # level L-1 vectors of the last cycle come from the fused restriction
        for f in ("r", "bt", "g"):
            fa, fb = a.field(f, L - 1), b.field(f, L - 1)
            assert _rel(fa, fb) < 1e-4, f
    a.close()
    b.close()


@pytest.fixture(scope="module")
def depth5_steps():
    """Two FP64 oracle cycles of the 3-D depth-5 workload (243^3 cells) from a
    random initial iterate, with the level vectors of each cycle."""
    f = wl.get("poisson3d_d5").f()
    H = oc.build_hierarchy(3, 5, np.array([1.0]), True, f)
    u0 = wl.random_vertex_field(3, 5, 23)
    steps = {}
    u = u0
    for k in (1, 2):
        u, parts = oc.cycle(H, u, return_parts=True)
        steps[k] = (u - u0, parts)
    return f, u0, steps


@pytest.mark.parametrize("k", [1, 2])
def test_fused_step_at_depth5_matches_the_oracle_step_by_step(depth5_steps, k):
    # At depth 5 the fused sweeps run with all their tile seams and slab
    # boundaries between full tiles: the up-pass has 4 x 10 tiles of 20 x 8
    # coarse columns (the restriction and damping windows of coarse columns
    # 20 and 21 straddle a seam) in 11 slabs along z, and its blocks skip the
    # boundary masks (their residual regions stay inside the interior); the
    # down-pass has 4 x 11 tiles of 64 x 22 fine columns in 13 slabs, three
    # of the four x-tiles storing without masks.  Depths 2 to 4 take the
    # masked paths.  One refinement step of k FP32 cycles
    # from a random iterate must give the correction of k FP64 oracle cycles,
    # and the level vectors of the step's last cycle those of the oracle's
    # k-th cycle: r_l, b~_l = omega S~^T r_{l+1} and g_l = c_l - c~_l.
    f, u0, steps = depth5_steps
    want, parts = steps[k]
    S = adafac.Solver(3, 5, 1.0, f, adafac.default_options(precision="mixed", inner_cycles=k))
    S.set_solution(u0)
    S.cycle(k)
    got = S.solution() - u0
    fields = {(name, l): S.field(name, l) for l in range(1, 5) for name in ("r", "bt", "g")}
    S.close()
    assert _rel(got, want) < FP32_RTOL
    for l in range(1, 5):
        g_want = parts["c"][l] - parts["ct"][l]
        for name, w in (("r", parts["r"][l]), ("bt", parts["bt"][l]), ("g", g_want)):
            a = fields[(name, l)].reshape(w.shape)
            assert _rel(a, w) < FP32_RTOL, (name, l, _rel(a, w))


def test_fused_counts_cycles_and_converges_like_levelwise():
    res = {}
    for path in ("auto", "levelwise"):
        S = _solver(4, path)
        res[path] = S.solve(1e-8, 1000)
        S.close()
    assert res["auto"][0] == res["levelwise"][0]
    assert res["auto"][1] <= 1e-8


def test_fused_reset_and_repeated_solves_are_reproducible():
    S = _solver(3, "auto", inner_cycles=5)
    c1, r1 = S.solve(1e-8, 500)
    u1 = S.solution()
    S.reset()
    c2, r2 = S.solve(1e-8, 500)
    assert (c1, r1) == (c2, r2)
    assert np.array_equal(u1, S.solution())
    S.close()


def test_full_size_poisson3d_d5_mixed_fused():
    # the 3-D depth-5 workload (243^3 cells, 14.2M unknowns) through the fused
    # path; the oracle evaluates the FP64 residual of the GPU solution
    w = wl.get("poisson3d_d5")
    S = adafac.Solver(3, 5, 1.0, w.f(), adafac.default_options(precision="mixed"))
    cycles, rel = S.solve(1e-8, 500)
    u = S.solution()
    S.close()
    assert rel <= 1e-8
    op = fem.LevelOperator.from_eps(3, 243, [1.0], True)
    b = fem.load_vector(w.f(), 1.0 / 243, 3)
    r = fem.zero_boundary(b - op.apply(u))
    assert np.sqrt(np.sum(r ** 2)) / np.sqrt(np.sum(b ** 2)) <= 1.01e-8
    # O(h^2) error of the manufactured solution against the depth-4 solve
    err5 = np.abs(u - wl.manufactured_solution(3, 5)).max()
    w4 = w.with_depth(4)
    S4 = adafac.Solver(3, 4, 1.0, w4.f(), adafac.default_options(precision="mixed"))
    S4.solve(1e-10, 500)
    err4 = np.abs(S4.solution() - wl.manufactured_solution(3, 4)).max()
    S4.close()
    assert 8.0 < err4 / err5 < 10.0


@pytest.mark.parametrize("scale", [2.0 ** 60, 2.0 ** -60])
def test_fused_solve_is_exactly_scale_invariant(scale):
    # the problem is linear: scaling f by a power of two scales every FP32 and
    # FP64 value of the iteration by the same power, and the fixed-point
    # refinement residual follows the magnitude of u -- the iterates must be
    # the exactly scaled ones, with the same cycle count
    f = wl.manufactured_rhs(3, 3)
    o = adafac.default_options(precision="mixed", inner_cycles=5)
    res = []
    for s in (1.0, scale):
        S = adafac.Solver(3, 3, 1.0, f * s, o)
        c, rel = S.solve(1e-8, 500)
        res.append((c, rel, S.solution()))
        S.close()
    assert res[0][0] == res[1][0]
    assert res[0][1] == pytest.approx(res[1][1], rel=1e-12)
    assert np.array_equal(res[0][2] * scale, res[1][2])


def test_fused_refinement_residual_matches_the_oracle():
    # the fixed-point refinement residual: its norm (recorded in the history
    # when the next refinement step starts) equals the oracle's FP64 residual
    # norm of the same iterate; the per-thread sums are FP32, hence 1e-6
    L = 4
    f = wl.manufactured_rhs(3, L)
    S = adafac.Solver(3, L, 1.0, f, adafac.default_options(precision="mixed", inner_cycles=4))
    S.cycle(4)
    u4 = S.solution()
    S.cycle(4)
    h = S.history()
    S.close()
    H = oc.build_hierarchy(3, L, [1.0], True, f)
    r0 = oc.residual_norm(H, H.b)
    r4 = oc.residual_norm(H, oc.residual(H, L, u4, H.b))
    assert h[0] == pytest.approx(1.0, rel=1e-6)
    assert h[1] == pytest.approx(r4 / r0, rel=1e-6)


def test_maximum_size_poisson3d_d6_mixed_fused():
    # the largest tree of the suite: depth 6 (729^3 cells, 389 M vertices,
    # about 34 GiB of workspace).  Sampled residuals use the oracle's assembled
    # stencil (taken on a 3^3 grid and scaled by h, as the 3-D d-linear
    # stiffness is proportional to h); their mean square estimates the
    # normalised residual of Eq. 10, which must be at the tolerance.  The
    # O(h^2) error against the depth-5 solve fixes the discretisation.
    w6 = wl.get("poisson3d_d5").with_depth(6)
    f6 = w6.f()
    S = adafac.Solver(3, 6, 1.0, f6, adafac.default_options(precision="mixed"))
    cycles, rel = S.solve(1e-8, 500)
    u = S.solution()
    S.close()
    assert rel <= 1e-8
    n = 729
    st = fem.LevelOperator.from_eps(3, 3, [1.0], True).stencils()[1, 1, 1] * (3.0 / n)
    rng = np.random.Generator(np.random.PCG64(7))
    idx = rng.integers(1, n, size=(200000, 3))
    b = (1.0 / n) ** 3 * f6[idx[:, 0], idx[:, 1], idx[:, 2]]
    Au = np.zeros(len(idx))
    for s, o in enumerate(fem.offsets(3)):
        Au += st[s] * u[idx[:, 0] + o[0], idx[:, 1] + o[1], idx[:, 2] + o[2]]
    est = np.sqrt(np.mean((b - Au) ** 2) / np.mean(b ** 2))
    assert est <= 1.5e-8, est
    err6 = np.abs(u - wl.manufactured_solution(3, 6)).max()
    del u
    S5 = adafac.Solver(3, 5, 1.0, w6.with_depth(5).f(), adafac.default_options(precision="mixed"))
    S5.solve(1e-10, 500)
    err5 = np.abs(S5.solution() - wl.manufactured_solution(3, 5)).max()
    S5.close()
    assert 8.0 < err5 / err6 < 10.0


@pytest.mark.parametrize("L,lmin", [(4, 2), (4, 3), (3, 2)])
def test_fused_with_fewer_levels_equals_levelwise_and_oracle(L, lmin):
    a = _solver(L, "auto", inner_cycles=3, lmin=lmin)
    b = _solver(L, "levelwise", inner_cycles=3, lmin=lmin)
    a.cycle(7)
    b.cycle(7)
    ua, ub = a.solution(), b.solution()
    assert _rel(ua, ub) < FP32_RTOL
    H = oc.build_hierarchy(3, L, [1.0], True, wl.manufactured_rhs(3, L))
    u = np.zeros_like(H.b)
    for _ in range(7):
        u = oc.cycle(H, u, lmin=lmin)
    assert _rel(ua, u) < FP32_RTOL
    a.close()
    b.close()
