"""Parity of the adaptive-tree cycles (adafac_adaptive_*) with the oracle on
static spacetrees with hanging vertices (oracle/adaptive.py, Sec. 2.1, 2.3 and
Eq. 9 on the generating system).

Both sides compute the same FP64 sums in other orders: the iterates, the level
vectors and the Eq. 10 norm agree to 1e-10 relative, the FP64 parity bar."""
import numpy as np
import pytest

import workloads as wl
from oracle import adaptive as ad
from oracle import cycle as oc

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1903_10367_gb300 import adafac  # noqa: E402

RTOL = 1e-10


def _band_tree(d, L):
    # a band around the circle r = 0.3 about the centre (the adaptive
    # workload's shape), coarse elsewhere
    def ref(l, c, h):
        r = np.sqrt(((c - 0.5) ** 2).sum(-1))
        return np.abs(r - 0.3) <= 0.05 + h
    return ad.tree_from_refinement(d, L, ref)


def _corner_tree(d, L):
    return ad.tree_from_refinement(d, L, lambda l, c, h: np.all(c < 0.4, axis=-1))


TREES = {"band": _band_tree, "corner": _corner_tree,
         "regular": lambda d, L: ad.regular_tree(d, L)}


def _close(got, want, what, rtol=RTOL, scale=0.0):
    # relative to the larger of the result's magnitude and `scale`, the
    # magnitude of the values it is summed from (a sum that cancels to
    # rounding noise is compared with its inputs)
    err = np.abs(got - want).max() / max(np.abs(want).max(), scale, 1e-300)
    assert err <= rtol, f"{what}: relative max error {err:.3e}"


def _problem(tree, d, L, eps_kind="random", seed=3):
    T = TREES[tree](d, L)
    N = 3 ** L
    eps = 1.0 if eps_kind == "scalar" else np.random.default_rng(seed).uniform(0.2, 3.0,
                                                                              size=(N,) * d)
    f = wl.manufactured_rhs(d, L)
    S = ad.build_system(T, eps, f)
    return T, eps, f, S


def _gpu(T, eps, f, **opt):
    o = adafac.default_options(precision="fp64", **opt)
    return adafac.AdaptiveSolver(T.d, T.L, [T.refined[l] for l in range(1, T.L)], eps, f, o)


def _start(S, seed=11):
    # a random iterate at the leaf nodes, zero on the boundary
    u = np.random.default_rng(seed).uniform(-1.0, 1.0, size=len(S.coords))
    u[S.boundary] = 0.0
    return u


CASES = [("band", 2, 3), ("band", 2, 4), ("corner", 2, 4), ("corner", 3, 2), ("band", 3, 3)]


@pytest.mark.parametrize("tree,d,L", CASES)
def test_setup_matches_the_oracle_system(tree, d, L):
    T, eps, f, S = _problem(tree, d, L)
    G = _gpu(T, eps, f)
    N = 3 ** L
    assert np.array_equal(G.nodes(), np.ravel_multi_index(S.coords.T, (N + 1,) * d))
    for l in range(1, L + 1):
        act = G.level("active", l).astype(np.int64)
        n = 3 ** l
        assert np.array_equal(act, np.ravel_multi_index(S.active[l].T, (n + 1,) * d)), l
        _close(G.level("invdiag", l), 1.0 / S.diag[l], f"1/M_{l}", 1e-12)
    rel, ab = G.residual_norm()
    assert rel == 1.0
    assert ab == pytest.approx(ad.residual_norm(S, np.zeros(len(S.coords))), rel=1e-12)
    G.close()


@pytest.mark.parametrize("tree,d,L", CASES)
@pytest.mark.parametrize("variant,rtilde", [("jac", "truncated"), ("jac", "exact"),
                                            ("additive", "truncated"), ("pi", "truncated"),
                                            ("exp", "truncated")])
def test_cycles_match_the_oracle(tree, d, L, variant, rtilde):
    T, eps, f, S = _problem(tree, d, L)
    u0 = _start(S)
    G = _gpu(T, eps, f, variant=variant, rtilde=rtilde, omega_exp=0.7)
    G.set_solution(u0)
    u = u0
    for k in range(3):
        u, parts = ad.cycle(S, u, variant=variant, rtilde=rtilde, omega_exp=0.7,
                            return_parts=True)
        G.cycle(1)
        got = G.solution()
        _close(got, u, f"iterate after cycle {k + 1}")
        if k == 0:
            # the level vectors of the first cycle
            for l in range(1, L + 1):
                _close(G.level("r", l), parts["r"][l], f"r_{l}")
            if variant == "jac":
                for l in range(1, L):
                    _close(G.level("bt", l), parts["bt"][l], f"b~_{l}",
                           scale=np.abs(parts["r"][l + 1]).max())
    rel, ab = G.residual_norm()
    assert ab == pytest.approx(ad.residual_norm(S, u), rel=RTOL)
    G.close()


@pytest.mark.parametrize("lmin", [2, 3])
def test_fewer_levels_match_the_oracle(lmin):
    T, eps, f, S = _problem("band", 2, 4)
    u0 = _start(S)
    G = _gpu(T, eps, f, lmin=lmin)
    G.set_solution(u0)
    u = u0
    for _ in range(2):
        u = ad.cycle(S, u, lmin=lmin)
    G.cycle(2)
    _close(G.solution(), u, f"iterate, lmin {lmin}")
    G.close()


def test_fully_refined_tree_equals_the_regular_gpu_path():
    # on the fully refined tree the generating system is the regular
    # hierarchy: the adaptive kernels and the regular FP64 kernels give the
    # same iterates
    d, L = 2, 4
    N = 3 ** L
    eps = np.random.default_rng(5).uniform(0.05, 2.0, size=(N,) * d)
    f = wl.manufactured_rhs(d, L)
    T = ad.regular_tree(d, L)
    G = _gpu(T, eps, f)
    R = adafac.Solver(d, L, eps, f, adafac.default_options(precision="fp64"))
    G.cycle(4)
    R.cycle(4)
    _close(G.solution(), R.solution().reshape(-1)[G.nodes()], "adaptive vs regular")
    G.close()
    R.close()


@pytest.mark.parametrize("tree,d,L,eps_kind", [("band", 2, 4, "random"), ("corner", 3, 3, "scalar")])
def test_solve_reaches_the_composite_solution(tree, d, L, eps_kind):
    T, eps, f, S = _problem(tree, d, L, eps_kind)
    G = _gpu(T, eps, f)
    cycles, rel = G.solve(1e-10, 2000)
    assert rel <= 1e-10
    ug = G.solution()
    # the oracle's own Eq. 10 norm of the GPU solution's residual
    r0 = ad.residual_norm(S, np.zeros(len(S.coords)))
    assert ad.residual_norm(S, ug) / r0 <= 1.01e-10
    # the error is bounded by the condition number (about 1e3 here) times
    # the relative residual
    _close(ug, ad.direct_solution(S), "converged iterate vs direct solve", 1e-6)
    # the oracle takes the same number of cycles to the same tolerance
    _, hist = ad.solve(S, tol=1e-10, max_cycles=2000)
    assert abs((len(hist) - 1) - cycles) <= 1
    G.close()


def _flags(T):
    return [T.refined[l] for l in range(1, T.L)]


def test_transfer_between_trees_matches_the_oracle():
    # the band moves by 0.1 along x: new vertices take the old function's
    # value, hanging ones the interpolation of their new coarse cell
    d, L = 2, 4
    f = wl.constant_rhs(d, L)
    Ta = ad.band_tree(d, L, 2, (0.5, 0.5), 0.3, 0.05)
    Tb = ad.band_tree(d, L, 2, (0.6, 0.5), 0.3, 0.05)
    Sa, Sb = ad.build_system(Ta, 1.0, f), ad.build_system(Tb, 1.0, f)
    o = adafac.default_options(precision="fp64")
    A = adafac.AdaptiveSolver(d, L, _flags(Ta), 1.0, f, o)
    B = adafac.AdaptiveSolver(d, L, _flags(Tb), 1.0, f, o)
    A.cycle(4)
    ua = A.solution()
    B.transfer_from(A)
    _close(B.solution(), ad.transfer(Sa, ua, Sb), "transferred iterate")
    # the reference of the normalised residual moves with the iterate
    rel, ab = B.residual_norm()
    assert rel == pytest.approx(ab / ad.residual_norm(Sa, np.zeros(len(Sa.coords))), rel=1e-12)
    A.close()
    B.close()


def test_moving_band_solve_matches_the_oracle():
    # the survey's adaptive workload on a small tree: depth 2 everywhere,
    # depth 4 within 0.05 of the circle r = 0.3, the band moving +x by 0.05
    # after every 5 cycles, 4 times, then cycles to 1e-9
    d, L, every, moves, shift = 2, 4, 5, 4, 0.05
    one = lambda x: np.ones(len(x))
    S, u_or, hist = ad.moving_band_solve(d, L, 2, 1.0, one, (0.5, 0.5), 0.3, 0.05, shift,
                                         every, moves, tol=1e-9)
    f = np.ones((3 ** L + 1,) * d)
    o = adafac.default_options(precision="fp64")
    ctr = np.array([0.5, 0.5])
    G = adafac.AdaptiveSolver(d, L, _flags(ad.band_tree(d, L, 2, ctr, 0.3, 0.05)), 1.0, f, o)
    rels = [1.0]
    for m in range(moves):
        for _ in range(every):
            G.cycle(1)
            rels.append(G.residual_norm()[0])
        ctr = ctr + np.array([shift, 0.0])
        N = adafac.AdaptiveSolver(d, L, _flags(ad.band_tree(d, L, 2, ctr, 0.3, 0.05)), 1.0, f, o)
        N.transfer_from(G)
        G.close()
        G = N
    while rels[-1] > 1e-9 and len(rels) < 2000:
        G.cycle(1)
        rels.append(G.residual_norm()[0])
    assert len(rels) == len(hist)
    np.testing.assert_allclose(rels, [h for _, h in hist], rtol=1e-8, atol=1e-14)
    _close(G.solution(), u_or, "iterate on the last tree")
    G.close()


@pytest.mark.parametrize("tree,d,L", [("band", 2, 4), ("corner", 3, 3), ("band", 3, 3)])
@pytest.mark.parametrize("variant", ["jac", "additive", "pi", "exp"])
def test_brick_and_csr_engines_give_the_same_iterates(tree, d, L, variant):
    # the brick engine (per-level grids; the default) and the CSR engine
    # (pagoda matrices; path "generic") compute the same cycles in other
    # summation orders
    T, eps, f, S = _problem(tree, d, L)
    u0 = _start(S)
    out = {}
    for path in ("auto", "generic"):
        o = adafac.default_options(precision="fp64", variant=variant, omega_exp=0.7, path=path)
        G = adafac.AdaptiveSolver(T.d, T.L, [T.refined[l] for l in range(1, T.L)], eps, f, o)
        G.set_solution(u0)
        G.cycle(3)
        out[path] = (G.solution(), G.residual_norm(),
                     [G.level("g", l) for l in range(1, L + 1)])
        G.close()
    _close(out["auto"][0], out["generic"][0], "brick vs CSR iterate", 1e-12)
    assert out["auto"][1][1] == pytest.approx(out["generic"][1][1], rel=1e-12)
    for l in range(L):
        _close(out["auto"][2][l], out["generic"][2][l], f"g_{l + 1}", 1e-12,
               scale=np.abs(out["generic"][2][l]).max() + 1e-300)


FP32_RTOL = 5e-5


@pytest.mark.parametrize("tree,d,L", [("band", 2, 4), ("corner", 2, 4), ("band", 3, 3)])
@pytest.mark.parametrize("variant", ["jac", "additive", "pi"])
@pytest.mark.parametrize("k", [1, 3])
def test_mixed_refinement_step_matches_the_oracle(tree, d, L, variant, k):
    # one refinement step of k FP32 cycles on the correction equation equals
    # k FP64 oracle cycles (the cycle is linear in the residual) up to FP32
    # rounding: 5e-5 of the correction's largest entry (the bound of the
    # regular path's mixed tests: 6e-8 per operation, eps ratios to 15,
    # k <= 3 cycles over several levels)
    T, eps, f, S = _problem(tree, d, L)
    u0 = _start(S)
    u = u0
    for _ in range(k):
        u = ad.cycle(S, u, variant=variant)
    o = adafac.default_options(precision="mixed", variant=variant, inner_cycles=k)
    G = adafac.AdaptiveSolver(T.d, T.L, [T.refined[l] for l in range(1, T.L)], eps, f, o)
    G.set_solution(u0)
    G.cycle(k)
    got = G.solution() - u0
    G.close()
    _close(got, u - u0, "mixed step correction", FP32_RTOL)


@pytest.mark.parametrize("tree,d,L", [("band", 2, 4), ("corner", 3, 3)])
def test_mixed_solve_meets_the_oracle_residual(tree, d, L):
    T, eps, f, S = _problem(tree, d, L)
    o = adafac.default_options(precision="mixed")
    G = adafac.AdaptiveSolver(T.d, T.L, [T.refined[l] for l in range(1, T.L)], eps, f, o)
    cycles, rel = G.solve(1e-8, 5000)
    assert rel <= 1e-8
    ug = G.solution()
    r0 = ad.residual_norm(S, np.zeros(len(S.coords)))
    assert ad.residual_norm(S, ug) / r0 <= 1.01e-8
    # the FP64 engine needs the same cycles, up to one refinement step
    G64 = _gpu(T, eps, f)
    c64, _ = G64.solve(1e-8, 5000)
    assert abs(c64 - cycles) <= o.inner_cycles
    G.close()
    G64.close()


def test_mixed_is_refused_on_the_sparse_matrix_engine():
    T, eps, f, S = _problem("band", 2, 3)
    for opt in (dict(path="generic"), dict(rtilde="exact")):
        o = adafac.default_options(precision="mixed", **opt)
        with pytest.raises(adafac.AdafacError):
            adafac.AdaptiveSolver(T.d, T.L, [T.refined[l] for l in range(1, T.L)], eps, f, o)
