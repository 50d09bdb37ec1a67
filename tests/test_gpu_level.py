"""Parity of the grid-shaped level kernels of the mixed-precision cycles
(varying eps, BoxMG transfers, adAFAC-PI, exponential damping, fewer levels)
with the CPU FP64 oracle and with the library's generic per-level kernels.
The cases span coarse grids on both sides of the size below which the
restriction takes the warp-per-vertex kernel (2-D depth <= 4, 3-D depth <= 3
at level L-1) and the thread-per-vertex one (2-D depth >= 5, 3-D depth >= 4).

One refinement step of k FP32 cycles from an iterate u0 computes the same
correction as k FP64 cycles of the oracle (the cycle is linear in the
residual), up to FP32 rounding: the corrections agree to 5e-5 of their
largest entry, and the two GPU kernel sets agree with each other to the same
bound.  The bound: FP32 rounds each operation to 6e-8 relative; a cycle
sums each level's window with coefficient ratios up to 1e2 (the eps jumps
of the cases), which amplifies rounding relative to the result by up to
about that ratio, over k <= 3 cycles and several levels: ~6e-8 * 1e2 * 3 *
3 ~ 5e-5.  Measured errors are 2e-6 .. 1e-5.  Converged solutions meet the 1e-8 tolerance in the oracle's own FP64
residual.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import cycle as oc

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1903_10367_gb300 import adafac  # noqa: E402

FP32_RTOL = 5e-5


def _eps(d, L, kind, seed=5):
    n = 3 ** L
    if kind == "scalar":
        return 1.0
    if kind == "blocks":
        return wl.eps_random_blocks(d, L, 3 ** max(L - 3, 0) if L > 1 else 1, 1e-2, 1903)
    return np.random.default_rng(seed).uniform(0.05, 2.0, size=(n,) * d)


def _close(got, want, rtol, what):
    scale = max(np.abs(want).max(), 1e-300)
    err = np.abs(got - want).max() / scale
    assert err <= rtol, f"{what}: relative max error {err:.3e} > {rtol:.1e}"


def _oracle_kw(opt):
    return dict(lmin=opt.get("lmin", 1), variant=opt.get("variant", "jac"),
                rtilde=opt.get("rtilde", "truncated"), omega_exp=opt.get("omega_exp", 0.5))


CASES = [
    (3, 3, "random", "boxmg", dict(variant="jac")),
    (3, 3, "random", "dlinear", dict(variant="jac")),
    (3, 3, "scalar", "boxmg", dict(variant="additive")),
    (3, 4, "blocks", "boxmg", dict(variant="jac")),
    (3, 3, "random", "boxmg", dict(variant="pi")),
    (3, 3, "random", "dlinear", dict(variant="exp", omega_exp=0.7)),
    (3, 3, "random", "boxmg", dict(variant="jac", lmin=2)),
    (3, 2, "random", "boxmg", dict(variant="jac", rtilde="exact")),
    (3, 1, "random", "boxmg", dict(variant="jac")),
    (3, 4, "random", "dlinear", dict(variant="pi")),
    (2, 5, "blocks", "boxmg", dict(variant="jac")),
    (2, 5, "random", "boxmg", dict(variant="additive")),
    (2, 5, "random", "dlinear", dict(variant="exp", omega_exp=0.7)),
    (2, 5, "blocks", "boxmg", dict(variant="jac", lmin=3)),
    (2, 5, "random", "boxmg", dict(variant="pi")),
    (2, 4, "blocks", "boxmg", dict(variant="jac")),
    (2, 5, "random", "dlinear", dict(variant="pi")),
    (2, 4, "scalar", "boxmg", dict(variant="additive")),
    (2, 3, "random", "boxmg", dict(variant="jac", lmin=2)),
    (2, 4, "random", "dlinear", dict(variant="exp", omega_exp=0.7)),
    (2, 1, "random", "dlinear", dict(variant="jac")),
]


@pytest.mark.parametrize("d,L,eps_kind,transfer,opt", CASES)
@pytest.mark.parametrize("k", [1, 3])
def test_refinement_step_matches_oracle_and_generic_kernels(d, L, eps_kind, transfer, opt, k):
    eps = _eps(d, L, eps_kind)
    f = wl.manufactured_rhs(d, L)
    sc = np.isscalar(eps)
    H = oc.build_hierarchy(d, L, np.array([eps]) if sc else eps, sc, f, transfer)
    u0 = wl.random_vertex_field(d, L, 11)
    u = u0
    for _ in range(k):
        u = oc.cycle(H, u, **_oracle_kw(opt))
    want = u - u0
    got = {}
    for path in ("auto", "generic"):
        o = adafac.default_options(transfer=transfer, precision="mixed", path=path, **opt)
        S = adafac.Solver(d, L, eps, f, o)
        S.set_solution(u0)
        S.cycle(k)
        got[path] = S.solution() - u0
        fields = {}
        if L >= 2 and opt.get("lmin", 1) < L:
            fields["r"] = S.field("r", L - 1)
            fields["g"] = S.field("g", L - 1)
        got[path + "_fields"] = fields
        S.close()
    _close(got["auto"], want, FP32_RTOL, "grid kernels vs oracle")
    _close(got["generic"], want, FP32_RTOL, "generic kernels vs oracle")
    _close(got["auto"], got["generic"], FP32_RTOL, "grid vs generic kernels")
    for name, a in got["auto_fields"].items():
        _close(a, got["generic_fields"][name], FP32_RTOL, f"level L-1 {name}")


@pytest.mark.parametrize("d,L,eps_kind,transfer", [
    (3, 4, "blocks", "boxmg"), (3, 3, "random", "dlinear"), (2, 5, "blocks", "boxmg")])
def test_mixed_solve_meets_the_oracle_residual(d, L, eps_kind, transfer):
    eps = _eps(d, L, eps_kind)
    f = wl.constant_rhs(d, L)
    H = oc.build_hierarchy(d, L, eps, False, f, transfer)
    S = adafac.Solver(d, L, eps, f, adafac.default_options(transfer=transfer, precision="mixed"))
    cycles, rel = S.solve(1e-8, 5000)
    assert rel <= 1e-8
    ug = S.solution()
    r0 = oc.residual_norm(H, H.b)
    r = oc.residual_norm(H, oc.residual(H, L, ug, H.b))
    assert r / r0 <= 1.01e-8, r / r0
    # the generic kernels need the same number of refinement steps
    Sg = adafac.Solver(d, L, eps, f, adafac.default_options(transfer=transfer, precision="mixed",
                                                            path="generic"))
    cg, _ = Sg.solve(1e-8, 5000)
    inner = adafac.default_options().inner_cycles
    assert abs(cg - cycles) <= inner
    S.close()
    Sg.close()


def test_refinement_norms_match_the_oracle_residual_norms():
    # the grid-shaped FP64 refinement residual reports the Eq. 10 norm of the
    # oracle's residual of the same iterate
    d, L = 3, 3
    eps = _eps(d, L, "random")
    f = wl.manufactured_rhs(d, L)
    H = oc.build_hierarchy(d, L, eps, False, f, "boxmg")
    S = adafac.Solver(d, L, eps, f, adafac.default_options(transfer="boxmg", precision="mixed",
                                                           inner_cycles=4))
    S.cycle(8)  # two refinement steps: norms of u0 = 0 and of the first step's iterate
    hist = S.history()
    assert len(hist) == 2
    S2 = adafac.Solver(d, L, eps, f, adafac.default_options(transfer="boxmg", precision="mixed",
                                                            inner_cycles=4))
    S2.cycle(4)
    u1 = S2.solution()
    r0 = oc.residual_norm(H, H.b)
    r1 = oc.residual_norm(H, oc.residual(H, L, u1, H.b))
    assert hist[0] == pytest.approx(1.0, rel=1e-14)
    assert hist[1] == pytest.approx(r1 / r0, rel=1e-10)
    S.close()
    S2.close()
