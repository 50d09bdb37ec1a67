"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

FP64 mode: setup arrays (BoxMG P, Galerkin stencils, inverse diagonals) and
per-cycle iterates and level vectors agree with the oracle to 1e-10 relative
(the stated FP64 parity bar; both sides compute the same sums in different
orders, so they differ by rounding only, ~1e-14).  MIXED mode: the converged
iterate's FP64 residual, evaluated by the oracle, meets the 1e-8 relative
tolerance and the solution agrees with the oracle's.
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

RTOL = 1e-10


def _case(d, L, eps_kind="scalar", transfer="dlinear", seed=5, rhs="manufactured"):
    n = 3 ** L
    if eps_kind == "scalar":
        eps, sc = np.array([1.0]), True
    elif eps_kind == "blocks":
        bc = 27 if n >= 27 else 3
        eps, sc = wl.eps_random_blocks(d, L, bc, 1e-3, 1903), False
    else:
        eps = np.random.default_rng(seed).uniform(0.05, 2.0, size=(n,) * d)
        sc = False
    f = wl.manufactured_rhs(d, L) if rhs == "manufactured" else wl.constant_rhs(d, L)
    return eps, sc, f


def _pair(d, L, eps_kind="scalar", transfer="dlinear", **opt):
    eps, sc, f = _case(d, L, eps_kind, transfer)
    H = oc.build_hierarchy(d, L, eps, sc, f, transfer, coarse_op=opt.get("coarse_op", "galerkin"))
    o = adafac.default_options(transfer=transfer, **opt)
    S = adafac.Solver(d, L, float(eps[0]) if sc else eps, f, o)
    return H, S


def _close(got, want, rtol=RTOL, what=""):
    scale = max(np.abs(want).max(), 1e-300)
    err = np.abs(got - want).max() / scale
    assert err <= rtol, f"{what}: relative max error {err:.3e} > {rtol:.1e}"


# ---------------------------------------------------------------------------
# setup

@pytest.mark.parametrize("d,L,eps_kind", [(2, 4, "blocks"), (2, 3, "random"), (3, 3, "random")])
def test_boxmg_and_galerkin_setup_match_oracle(d, L, eps_kind):
    H, S = _pair(d, L, eps_kind, "boxmg")
    I = tuple(slice(1, -1) for _ in range(d))
    for l in range(L, 1, -1):
        P = S.field("P", l)
        for c in range(2 ** d):
            _close(P[c], H.levels[l].Pv[..., c], 1e-12, f"P level {l} corner {c}")
    for l in range(1, L):
        st = S.field("stencil", l)
        want = H.levels[l].op.stencils()
        for s in range(3 ** d):
            _close(st[s][I], want[..., s][I], 1e-12, f"stencil level {l} entry {s}")
    for l in range(1, L + 1):
        inv = S.field("invdiag", l)
        _close(inv[I], 1.0 / H.levels[l].diag[I], 1e-12, f"invdiag level {l}")
    S.close()


@pytest.mark.parametrize("d,L,eps_kind,transfer", [(2, 4, "blocks", "boxmg"), (3, 3, "random", "dlinear")])
def test_rediscretised_coarse_operators_match_oracle(d, L, eps_kind, transfer):
    H, S = _pair(d, L, eps_kind, transfer, coarse_op="rediscretised")
    I = tuple(slice(1, -1) for _ in range(d))
    for l in range(1, L):
        st = S.field("stencil", l)
        want = H.levels[l].op.stencils()
        # relative to the largest entry: the face entries of the 3-D d-linear
        # element are zero (the oracle's carry rounding noise)
        scale = np.abs(want[I]).max()
        for s in range(3 ** d):
            err = np.abs(st[s][I] - want[..., s][I]).max() / scale
            assert err <= 1e-12, f"stencil level {l} entry {s}: {err:.3e}"
        _close(S.field("invdiag", l)[I], 1.0 / H.levels[l].diag[I], 1e-12, f"invdiag level {l}")
    S.close()


def test_uniform_levels_match_galerkin_for_constant_eps():
    # scalar eps with d-linear transfers keeps every level's stencil uniform;
    # the oracle forms R A P explicitly
    H, S = _pair(3, 3, "scalar", "dlinear")
    I = tuple(slice(1, -1) for _ in range(3))
    for l in range(1, 4):
        _close(S.field("invdiag", l)[I], 1.0 / H.levels[l].diag[I], 1e-13, f"level {l}")
    S.close()


# ---------------------------------------------------------------------------
# one cycle from an arbitrary iterate, every level vector

CASES = [
    (2, 4, "scalar", "dlinear", dict(variant="jac")),
    (2, 4, "scalar", "dlinear", dict(variant="additive")),
    (2, 4, "scalar", "dlinear", dict(variant="pi")),
    (2, 4, "scalar", "dlinear", dict(variant="exp", omega_exp=0.7)),
    (2, 4, "blocks", "dlinear", dict(variant="jac", rtilde="exact")),
    (2, 4, "blocks", "boxmg", dict(variant="jac")),
    (2, 4, "blocks", "boxmg", dict(variant="jac", form="fas")),
    (2, 4, "blocks", "boxmg", dict(variant="pi", form="fas")),
    (2, 1, "scalar", "dlinear", dict(variant="jac")),
    (3, 1, "scalar", "dlinear", dict(variant="jac")),
    (3, 1, "random", "boxmg", dict(variant="additive")),
    (2, 2, "random", "boxmg", dict(variant="jac")),
    (3, 3, "scalar", "dlinear", dict(variant="jac")),
    (3, 3, "random", "boxmg", dict(variant="jac")),
    (3, 3, "random", "dlinear", dict(variant="pi", form="fas")),
    (3, 2, "random", "boxmg", dict(variant="jac", rtilde="exact")),
    (2, 4, "blocks", "boxmg", dict(variant="jac", coarse_op="rediscretised")),
    (2, 3, "random", "dlinear", dict(variant="pi", coarse_op="rediscretised")),
    (3, 3, "random", "boxmg", dict(variant="jac", coarse_op="rediscretised")),
    (2, 4, "blocks", "boxmg", dict(variant="jac", lmin=2)),
    (2, 4, "scalar", "dlinear", dict(variant="pi", lmin=3)),
    (2, 4, "scalar", "dlinear", dict(variant="additive", lmin=4)),
    (3, 3, "random", "dlinear", dict(variant="jac", lmin=2)),
]


def _oracle_kw(opt):
    return dict(lmin=opt.get("lmin", 1), variant=opt.get("variant", "jac"), form=opt.get("form", "cs"),
                rtilde=opt.get("rtilde", "truncated"), omega_exp=opt.get("omega_exp", 0.5))


@pytest.mark.parametrize("d,L,eps_kind,transfer,opt", CASES)
def test_one_cycle_matches_oracle(d, L, eps_kind, transfer, opt):
    H, S = _pair(d, L, eps_kind, transfer, **opt)
    u0 = wl.random_vertex_field(d, L, 11)
    S.set_solution(u0)
    S.cycle(1)
    u1, parts = oc.cycle(H, u0, return_parts=True, **_oracle_kw(opt))
    _close(S.solution(), u1, RTOL, "u after one cycle")
    lmin = opt.get("lmin", 1)
    for l in range(lmin, L + 1):
        _close(S.field("r", l), parts["r"][l], RTOL, f"r level {l}")
    if opt.get("variant", "jac") == "jac":
        for l in range(lmin, L):
            _close(S.field("bt", l), parts["bt"][l], RTOL, f"b~ level {l}")
            want_g = parts["c"][l] - parts["ct"][l]
            _close(S.field("g", l), want_g, RTOL, f"g level {l}")
    S.close()


@pytest.mark.parametrize("d,L,eps_kind,transfer", [(2, 5, "blocks", "boxmg"), (3, 3, "scalar", "dlinear")])
def test_five_cycles_iterates_match_oracle(d, L, eps_kind, transfer):
    H, S = _pair(d, L, eps_kind, transfer)
    u = np.zeros_like(H.b)
    for k in range(5):
        S.cycle(1)
        u = oc.cycle(H, u)
        _close(S.solution(), u, RTOL, f"iterate {k + 1}")
    S.close()


def test_solve_history_matches_oracle_poisson2d_d4():
    # the configuration of the paper's consistency study: plain additive and
    # adAFAC-Jac to 1e-8 (Sec. 5.1)
    for variant in ("jac", "additive"):
        H, S = _pair(2, 4, "scalar", "dlinear", variant=variant)
        u, hist = oc.solve(H, tol=1e-8, variant=variant)
        cycles, rel = S.solve(1e-8, 500)
        assert cycles == len(hist) - 1
        gh = S.history()
        np.testing.assert_allclose(gh[:len(hist)], hist, rtol=1e-8, atol=1e-14)
        _close(S.solution(), u, RTOL, f"{variant} converged iterate")
        S.close()


def test_full_size_jump2d_d6_boxmg_fp64_iterates():
    # the 2-D depth-6 workload at full size: 729^2 cells, random 27x27 blocks
    w = wl.get("jump2d_d6")
    eps, sc = w.eps()
    H = oc.build_hierarchy(2, 6, eps, sc, w.f(), "boxmg")
    S = adafac.Solver(2, 6, eps, w.f(), adafac.default_options(transfer="boxmg"))
    u = np.zeros_like(H.b)
    for k in range(3):
        S.cycle(1)
        u = oc.cycle(H, u)
    _close(S.solution(), u, RTOL, "depth-6 iterate 3")
    S.close()


# ---------------------------------------------------------------------------
# mixed precision: FP32 cycles on the correction equation, FP64 refinement

@pytest.mark.parametrize("d,L,eps_kind,transfer", [
    (2, 4, "scalar", "dlinear"), (2, 5, "blocks", "boxmg"), (3, 3, "scalar", "dlinear"),
    (3, 3, "random", "boxmg")])
def test_mixed_converges_to_oracle_solution(d, L, eps_kind, transfer):
    H, S = _pair(d, L, eps_kind, transfer, precision="mixed")
    cycles, rel = S.solve(1e-8, 2000)
    assert rel <= 1e-8
    ug = S.solution()
    r0 = oc.residual_norm(H, H.b)
    r = oc.residual_norm(H, oc.residual(H, L, ug, H.b))
    assert r / r0 <= 1.01e-8, r / r0
    u_ref, _ = oc.solve(H, tol=1e-11, max_cycles=3000)
    _close(ug, u_ref, 1e-5, "mixed solution vs oracle")
    S.close()


def test_mixed_matches_fp64_cycle_count_within_a_few_cycles():
    eps, sc, f = _case(2, 5, "blocks")
    res = {}
    for prec in ("fp64", "mixed"):
        S = adafac.Solver(2, 5, eps, f, adafac.default_options(transfer="boxmg", precision=prec))
        res[prec] = S.solve(1e-8, 2000)[0]
        S.close()
    assert res["mixed"] <= res["fp64"] + 2 * adafac.default_options().inner_cycles


# ---------------------------------------------------------------------------
# control, errors, state

def test_residual_norm_query_and_reset():
    H, S = _pair(2, 3, "scalar", "dlinear")
    rel, ab = S.residual_norm()
    assert rel == pytest.approx(1.0)
    assert ab == pytest.approx(oc.residual_norm(H, H.b), rel=1e-12)
    S.cycle(3)
    u = np.zeros_like(H.b)
    for _ in range(3):
        u = oc.cycle(H, u)
    want = oc.residual_norm(H, oc.residual(H, 3, u, H.b)) / oc.residual_norm(H, H.b)
    assert S.residual_norm()[0] == pytest.approx(want, rel=1e-9)
    S.reset()
    assert np.abs(S.solution()).max() == 0.0
    S.close()


def test_nan_input_is_reported_as_divergence():
    d, L = 2, 3
    f = wl.manufactured_rhs(d, L)
    f[5, 5] = np.nan
    S = adafac.Solver(d, L, 1.0, f)
    with pytest.raises(adafac.AdafacError) as ei:
        S.solve(1e-8, 50)
    assert ei.value.status == 3
    # the context stays usable
    S2 = adafac.Solver(d, L, 1.0, wl.manufactured_rhs(d, L))
    assert S2.solve(1e-8, 200)[1] <= 1e-8
    S.close()
    S2.close()


def test_not_converged_status_and_launch_count():
    S = adafac.Solver(2, 3, 1.0, wl.manufactured_rhs(2, 3))
    with pytest.raises(adafac.AdafacError) as ei:
        S.solve(1e-12, 3)
    assert ei.value.status == 6
    assert S.launch_count() > 0
    S.close()


def test_device_inputs_equal_host_inputs():
    eps, sc, f = _case(2, 4, "blocks")
    a = adafac.Solver(2, 4, eps, f, adafac.default_options(transfer="boxmg"))
    b = adafac.Solver(2, 4, torch.from_numpy(eps).cuda(), torch.from_numpy(f).cuda(),
                      adafac.default_options(transfer="boxmg"))
    a.cycle(4)
    b.cycle(4)
    assert np.array_equal(a.solution(), b.solution())
    a.close()
    b.close()
