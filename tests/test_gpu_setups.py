"""The setups of the paper's Sec. 5 on regular trees: non-zero Dirichlet data
(u = 1 on x_2 = 0), f = 0, eps = 1 or 10^-k / 10^k in the halves, needle and
checkerboard geometries.  GPU against the oracle, and the stability
observations that hold on regular trees."""
import numpy as np
import pytest

import workloads as wl
from oracle import cycle as oc

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1903_10367_gb300 import adafac  # noqa: E402

RTOL = 1e-10


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _setup(name, L):
    return {"halves": wl.eps_halves(2, L, 1e-7),
            "checker": wl.eps_checkerboard(2, L, 1e-5),
            "needle": wl.eps_needle(2, L, 10.0)}[name]


@pytest.mark.parametrize("name,transfer,variant", [
    ("checker", "boxmg", "jac"), ("halves", "dlinear", "jac"), ("needle", "boxmg", "pi"),
    ("halves", "boxmg", "additive")])
def test_one_cycle_with_dirichlet_data_matches_oracle(name, transfer, variant):
    L = 4
    n = 3 ** L
    eps = _setup(name, L)
    g = wl.bottom_boundary(2, L)
    f = np.zeros((n + 1,) * 2)
    S = adafac.Solver(2, L, eps, f, adafac.default_options(transfer=transfer, variant=variant))
    S.set_boundary(g)
    u0 = wl.random_vertex_field(2, L, 3)
    S.set_solution(u0)
    S.cycle(1)
    H = oc.build_hierarchy(2, L, eps, False, f, transfer)
    start = u0 + oc.with_boundary(g)
    u1 = oc.cycle(H, start, variant=variant)
    assert _rel(S.solution(), u1) < RTOL
    S.cycle(2)
    u3 = oc.cycle(H, oc.cycle(H, u1, variant=variant), variant=variant)
    assert _rel(S.solution(), u3) < RTOL
    S.close()


@pytest.mark.parametrize("d,L,prec,transfer", [(2, 4, "fp64", "dlinear"), (2, 4, "mixed", "boxmg"),
                                               (3, 3, "mixed", "dlinear"), (3, 3, "fp64", "boxmg")])
def test_linear_boundary_data_give_the_linear_solution(d, L, prec, transfer):
    # constant eps, f = 0: the d-linear FEM reproduces linear functions
    # exactly (3-D mixed d-linear runs the fused path)
    n = 3 ** L
    coords = np.meshgrid(*([np.arange(n + 1) / n] * d), indexing="ij")
    lin = 0.3 + sum((k + 1) * 0.7 * c for k, c in enumerate(coords))
    S = adafac.Solver(d, L, 2.5, np.zeros((n + 1,) * d),
                      adafac.default_options(transfer=transfer, precision=prec))
    S.set_boundary(lin)
    c, rel = S.solve(1e-11, 3000)
    u = S.solution()
    assert rel <= 1e-11
    assert np.abs(u - lin).max() <= 1e-8
    # reset keeps the Dirichlet values
    S.reset()
    assert np.array_equal(S.solution(), oc.with_boundary(lin))
    S.close()


@pytest.mark.parametrize("name,transfer,variant", [
    ("halves", "dlinear", "jac"), ("halves", "boxmg", "additive"), ("checker", "boxmg", "jac"),
    ("needle", "dlinear", "jac")])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_paper_setups_converge_to_the_oracle_solution(name, transfer, variant, prec):
    L = 4
    n = 3 ** L
    eps = _setup(name, L)
    g = wl.bottom_boundary(2, L)
    f = np.zeros((n + 1,) * 2)
    S = adafac.Solver(2, L, eps, f, adafac.default_options(transfer=transfer, variant=variant,
                                                           precision=prec))
    S.set_boundary(g)
    c, rel = S.solve(1e-10, 5000)
    u = S.solution()
    S.close()
    H = oc.build_hierarchy(2, L, eps, False, f, transfer)
    # the oracle's FP64 residual of the GPU solution is at the tolerance
    r0 = oc.residual_norm(H, oc.residual(H, L, oc.with_boundary(g), H.b))
    assert oc.residual_norm(H, oc.residual(H, L, u, H.b)) / r0 <= 1.05e-10
    # and the solution is the oracle's, up to the conditioning of the jump
    # (eps contrasts of 1e5 .. 1e7 amplify a 1e-10 residual)
    u_ref, hist = oc.solve(H, oc.with_boundary(g), variant=variant, tol=1e-12, max_cycles=5000)
    assert hist[-1] <= 1e-12
    assert _rel(u, u_ref) < 1e-4


def test_stability_on_regular_trees_halves_jump():
    # Sec. 5, eps jump of seven orders across x_1 = 1/2 (not a mesh line):
    # with d-linear transfers plain additive multigrid is unstable, the
    # additive damping of adAFAC-Jac makes it converge, and BoxMG transfers
    # stabilise every variant
    L = 5
    n = 3 ** L
    eps = wl.eps_halves(2, L, 1e-7)
    g = wl.bottom_boundary(2, L)
    f = np.zeros((n + 1,) * 2)

    def run(transfer, variant):
        S = adafac.Solver(2, L, eps, f, adafac.default_options(transfer=transfer,
                                                               variant=variant))
        S.set_boundary(g)
        try:
            c, rel = S.solve(1e-8, 3000)
            return c
        except adafac.AdafacError as e:
            assert e.status == 3  # DIVERGED
            return None
        finally:
            S.close()

    assert run("dlinear", "additive") is None
    c_jac = run("dlinear", "jac")
    assert c_jac is not None
    for variant in ("additive", "jac", "pi"):
        c = run("boxmg", variant)
        assert c is not None and c < c_jac


def test_oscillations_grow_with_the_number_of_correction_levels():
    # Sec. 5, regular level 6, eps jump of seven orders across x_1 = 1/2: the
    # sample point next to (1/2, 1/2), normalised by the converged value,
    # oscillates when correction levels are added below the finest (l_min
    # lowered) with d-linear transfers and plain additive multigrid; the
    # additive damping of adAFAC-Jac shrinks the oscillations by orders of
    # magnitude, and BoxMG transfers remove them
    L = 6
    n = 3 ** L
    eps = wl.eps_halves(2, L, 1e-7)
    g = wl.bottom_boundary(2, L)
    f = np.zeros((n + 1,) * 2)
    sy, sx = n // 2, n // 2 + 1
    S = adafac.Solver(2, L, eps, f, adafac.default_options(transfer="boxmg"))
    S.set_boundary(g)
    S.solve(1e-12, 20000)
    ref = S.solution()[sy, sx]
    S.close()

    def amplitude(transfer, variant, lmin, cycles=80):
        S = adafac.Solver(2, L, eps, f, adafac.default_options(transfer=transfer,
                                                               variant=variant, lmin=lmin))
        S.set_boundary(g)
        t = []
        for _ in range(cycles):
            S.cycle(1)
            t.append(S.solution()[sy, sx] / ref)
        S.close()
        t = np.array(t)
        return max(t.max() - 1.0, 0.0) + max(-t.min(), 0.0)

    add = {lmin: amplitude("dlinear", "additive", lmin) for lmin in (3, 2, 1)}
    assert add[3] < 0.01 < add[2] < add[1]
    assert add[1] > 1000.0
    assert amplitude("dlinear", "jac", 1) < 1e-2 * add[1]
    assert amplitude("boxmg", "additive", 1) < 0.1
