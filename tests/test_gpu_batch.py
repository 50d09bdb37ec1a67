"""The batched path (ADAFAC_PATH_BATCHED, csrc/batch.cu): a whole refinement
step of the mixed-precision solve -- FP64 residual and Eq. 10 norm, k FP32
cycles of Algorithm 1, u += e -- in one launch, a cluster of CTAs per
instance, cluster barriers between the steps of the cycle.

* One refinement step of k FP32 cycles from an iterate u0 computes the
  correction of k FP64 oracle cycles (the cycle is linear in the residual) to
  the FP32 bound of the level path's tests, 5e-5 of its largest entry
  (FP32 rounding 6e-8, coefficient ratios up to 1e2, k <= 3 cycles, several
  levels).  The cases span every cluster size the size rule picks (1 .. 16
  CTAs), one and several units per CTA, and the degenerate trees (depth 1,
  lmin = L).
* The vertex arithmetic and the norm partials do not depend on the cluster
  size or on the other instances of a launch: iterates repeat bit for bit
  for every cluster size and inside the request server's shared launches.
* Converged solves meet the tolerance in the oracle's own FP64 residual.
"""
import time

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


def _opts(transfer, **kw):
    return adafac.default_options(transfer=transfer, precision="mixed", path="batched", **kw)


CASES = [
    # d, L, eps, transfer, options        (fine vertices -> CTAs per instance)
    (2, 1, "random", "dlinear", dict(variant="jac")),                   # 16 -> 1, on chip
    (2, 3, "random", "boxmg", dict(variant="jac")),                     # 784 -> 1, on chip
    (2, 3, "random", "boxmg", dict(variant="jac", lmin=3)),             # no coarse level
    (2, 4, "blocks", "boxmg", dict(variant="jac")),                     # 6724 -> 1, on chip
    (2, 4, "random", "dlinear", dict(variant="exp", omega_exp=0.7)),
    (2, 4, "scalar", "boxmg", dict(variant="additive")),
    (2, 5, "blocks", "boxmg", dict(variant="jac")),                     # 59536 -> 16
    (2, 5, "random", "boxmg", dict(variant="pi")),
    (2, 5, "random", "dlinear", dict(variant="pi")),
    (2, 5, "blocks", "boxmg", dict(variant="jac", lmin=3)),
    (2, 6, "blocks", "boxmg", dict(variant="jac")),                     # 532900: 65 units / CTA
    (3, 1, "random", "boxmg", dict(variant="jac")),                     # 64 -> 1
    (3, 2, "random", "boxmg", dict(variant="jac")),                     # 1000 -> 1, on chip
    (3, 3, "random", "boxmg", dict(variant="jac")),                     # 21952 -> 8
    (3, 3, "random", "dlinear", dict(variant="jac")),
    (3, 3, "scalar", "boxmg", dict(variant="additive")),
    (3, 3, "random", "boxmg", dict(variant="pi")),
    (3, 3, "random", "dlinear", dict(variant="exp", omega_exp=0.7)),
    (3, 3, "random", "boxmg", dict(variant="jac", lmin=2)),
    (3, 4, "blocks", "boxmg", dict(variant="jac")),                     # 571787 -> 16
]


@pytest.mark.parametrize("d,L,eps_kind,transfer,opt", CASES)
@pytest.mark.parametrize("k", [1, 3])
def test_batched_step_matches_the_oracle_and_the_level_path(d, L, eps_kind, transfer, opt, k):
    if L >= 6 and k > 1:
        pytest.skip("one cycle suffices at this size")
    eps = _eps(d, L, eps_kind)
    f = wl.manufactured_rhs(d, L)
    sc = np.isscalar(eps)
    H = oc.build_hierarchy(d, L, np.array([eps]) if sc else eps, sc, f, transfer)
    u0 = wl.random_vertex_field(d, L, 11)
    u = u0
    for _ in range(k):
        u = oc.cycle(H, u, lmin=opt.get("lmin", 1), variant=opt.get("variant", "jac"),
                     omega_exp=opt.get("omega_exp", 0.5))
    want = u - u0
    got, fields = {}, {}
    for path in ("batched", "levelwise"):
        o = adafac.default_options(transfer=transfer, precision="mixed", path=path, **opt)
        S = adafac.Solver(d, L, eps, f, o)
        S.set_solution(u0)
        S.cycle(k)
        got[path] = S.solution() - u0
        if L >= 2 and opt.get("lmin", 1) < L:
            fields[path] = {name: S.field(name, L - 1) for name in ("r", "bt", "g")}
        S.close()
    _close(got["batched"], want, FP32_RTOL, "batched step vs oracle")
    _close(got["batched"], got["levelwise"], FP32_RTOL, "batched vs level path")
    for name in fields.get("batched", {}):
        _close(fields["batched"][name], fields["levelwise"][name], FP32_RTOL,
               f"level L-1 {name}")


def test_batched_step_with_dirichlet_data_matches_the_oracle():
    d, L = 2, 4
    n = 3 ** L
    eps = wl.eps_checkerboard(2, L, 1e-5)
    g = wl.bottom_boundary(2, L)
    f = np.zeros((n + 1,) * 2)
    S = adafac.Solver(d, L, eps, f, _opts("boxmg", inner_cycles=2))
    S.set_boundary(g)
    u0 = wl.random_vertex_field(2, L, 3)
    S.set_solution(u0)
    S.cycle(2)
    H = oc.build_hierarchy(2, L, eps, False, f, "boxmg")
    start = u0 + oc.with_boundary(g)
    want = oc.cycle(H, oc.cycle(H, start))
    _close(S.solution() - start, want - start, FP32_RTOL, "batched step with Dirichlet data")
    S.close()


@pytest.mark.parametrize("d,L,eps_kind,transfer", [(2, 5, "blocks", "boxmg"),
                                                   (3, 3, "random", "dlinear"),
                                                   (2, 4, "blocks", "boxmg")])
def test_every_cluster_size_gives_the_same_iterates(d, L, eps_kind, transfer):
    # one CTA holds the vectors of the 2-D depth-4 grid in shared memory, the
    # larger clusters keep them in device memory: the same iterates
    eps = _eps(d, L, eps_kind)
    f = wl.constant_rhs(d, L)
    results = []
    sizes = [1, 2, 4, 8, 16]
    for ctas in sizes:
        S = adafac.Solver(d, L, eps, f, _opts(transfer, inner_cycles=8))
        if ctas > 8:
            try:
                S.set_batch_cluster(ctas)
            except adafac.AdafacError:
                S.close()
                continue  # the device places clusters of at most 8
        else:
            S.set_batch_cluster(ctas)
        assert S.batch_cluster() == ctas
        S.cycle(24)
        results.append((ctas, S.solution(), S.history()))
        S.close()
    assert len(results) >= 4
    _, u_ref, h_ref = results[0]
    for ctas, u, h in results[1:]:
        assert np.array_equal(u, u_ref), ctas
        assert np.array_equal(h, h_ref), ctas


def test_cluster_size_rule_and_its_checks():
    S = adafac.Solver(2, 3, 1.0, wl.constant_rhs(2, 3), _opts("dlinear"))
    assert S.batch_cluster() == 1
    for bad in (0, 3, 32):
        with pytest.raises(adafac.AdafacError):
            S.set_batch_cluster(bad)
    S.close()
    S = adafac.Solver(2, 5, 1.0, wl.constant_rhs(2, 5), _opts("dlinear"))
    assert S.batch_cluster() in (8, 16)
    S.close()
    # AUTO takes the batched path on the smallest grids only
    A = adafac.Solver(2, 3, 1.0, wl.constant_rhs(2, 3), adafac.default_options(precision="mixed"))
    assert A.batch_cluster() == 1
    A.close()
    L = adafac.Solver(2, 4, 1.0, wl.constant_rhs(2, 4),
                      adafac.default_options(precision="mixed"))
    with pytest.raises(adafac.AdafacError):
        L.batch_cluster()
    L.close()


@pytest.mark.parametrize("opt", [dict(precision="fp64", path="batched"),
                                 dict(precision="mixed", path="batched", rtilde="exact")])
def test_configurations_the_batched_path_does_not_cover_are_refused(opt):
    with pytest.raises(adafac.AdafacError) as e:
        adafac.workspace_size(2, 3, adafac.default_options(**opt))
    assert e.value.status == 1 and "BATCHED" in str(e.value)


@pytest.mark.parametrize("d,L,eps_kind,transfer", [(2, 5, "blocks", "boxmg"),
                                                   (3, 3, "random", "dlinear"),
                                                   (2, 3, "blocks", "boxmg")])
def test_batched_solve_meets_the_oracle_residual(d, L, eps_kind, transfer):
    eps = _eps(d, L, eps_kind)
    f = wl.constant_rhs(d, L)
    H = oc.build_hierarchy(d, L, eps, False, f, transfer)
    S = adafac.Solver(d, L, eps, f, _opts(transfer))
    cycles, rel = S.solve(1e-8, 5000)
    assert rel <= 1e-8
    ug = S.solution()
    r0 = oc.residual_norm(H, H.b)
    r = oc.residual_norm(H, oc.residual(H, L, ug, H.b))
    assert r / r0 <= 1.01e-8, r / r0
    # the level path needs the same number of refinement steps, give or take one
    Sl = adafac.Solver(d, L, eps, f, adafac.default_options(transfer=transfer, precision="mixed"))
    cl, _ = Sl.solve(1e-8, 5000)
    assert abs(cl - cycles) <= adafac.default_options().inner_cycles
    S.close()
    Sl.close()


def test_refinement_norms_match_the_oracle_residual_norms():
    d, L = 3, 3
    eps = _eps(d, L, "random")
    f = wl.manufactured_rhs(d, L)
    H = oc.build_hierarchy(d, L, eps, False, f, "boxmg")
    S = adafac.Solver(d, L, eps, f, _opts("boxmg", inner_cycles=4))
    S.cycle(8)
    hist = S.history()
    assert len(hist) == 2
    S2 = adafac.Solver(d, L, eps, f, _opts("boxmg", inner_cycles=4))
    S2.cycle(4)
    u1 = S2.solution()
    r0 = oc.residual_norm(H, H.b)
    r1 = oc.residual_norm(H, oc.residual(H, L, u1, H.b))
    assert hist[0] == pytest.approx(1.0, rel=1e-14)
    assert hist[1] == pytest.approx(r1 / r0, rel=1e-10)
    # the explicit query evaluates the same norm with the level kernels
    rel, _ = S2.residual_norm()
    assert rel == pytest.approx(r1 / r0, rel=1e-10)
    S.close()
    S2.close()


def _server_mix():
    """Batched requests of several launch groups (two of them with more than
    one request), one on the level path and one in FP64."""
    out = []
    spec = [(2, 3, "batched"), (2, 3, "batched"), (2, 4, "batched"), (2, 5, "batched"),
            (2, 5, "batched"), (3, 2, "batched"), (3, 3, "batched"), (2, 4, "levelwise"),
            (2, 3, "fp64")]
    for i, (d, L, path) in enumerate(spec):
        eps = wl.eps_random_blocks(d, L, 3 ** max(L - 3, 0), 1e-2, seed=1903 + i)
        f = wl.constant_rhs(d, L)
        if path == "fp64":
            opts = adafac.default_options(transfer="boxmg")
        else:
            opts = adafac.default_options(transfer="boxmg", precision="mixed", path=path)
        out.append((d, L, eps, f, opts))
    return out


def test_server_results_equal_the_same_solves_alone_bit_for_bit():
    cases = _server_mix()
    alone = []
    for d, L, eps, f, opts in cases:
        S = adafac.Solver(d, L, eps, f, opts)
        c, _ = S.solve(1e-8, 3000)
        alone.append((c, S.solution()))
        S.close()
    srv = adafac.Server(4 << 30, n_streams=8, max_running=16)
    tickets = [srv.submit(d, L, eps, f, opts) for (d, L, eps, f, opts) in cases]
    t0 = time.time()
    while not all(srv.poll(t)["state"] in ("done", "failed") for t in tickets):
        assert time.time() - t0 < 120.0, "server did not finish"
        time.sleep(0.002)
    for (d, L, eps, f, opts), (c_alone, u_alone), t in zip(cases, alone, tickets):
        info = srv.poll(t)
        assert info["state"] == "done" and info["status"] == 0, info
        assert info["rel"] <= 1e-8
        assert info["cycles"] == c_alone
        u = srv.fetch(t)
        if opts.path == adafac.PATH["batched"]:
            assert np.array_equal(u, u_alone), (d, L)
        else:
            assert np.abs(u - u_alone).max() <= 1e-12 * max(np.abs(u_alone).max(), 1e-300)
    assert srv.stats() == (0, 0, 0)
    srv.close()


def test_server_runs_many_batched_requests_of_one_group_together():
    # more requests of one launch group than fit into one launch
    d, L = 2, 3
    opts = _opts("boxmg")
    eps = [wl.eps_random_blocks(d, L, 1, 1e-2, seed=7 + i) for i in range(80)]
    f = wl.constant_rhs(d, L)
    srv = adafac.Server(4 << 30, n_streams=4, max_running=80)
    tickets = [srv.submit(d, L, e, f, opts) for e in eps]
    t0 = time.time()
    while not all(srv.poll(t)["state"] in ("done", "failed") for t in tickets):
        assert time.time() - t0 < 120.0, "server did not finish"
        time.sleep(0.002)
    for e, t in zip(eps[:5], tickets[:5]):
        S = adafac.Solver(d, L, e, f, opts)
        c, _ = S.solve(1e-8, 3000)
        info = srv.poll(t)
        assert info["state"] == "done" and info["cycles"] == c
        assert np.array_equal(srv.fetch(t), S.solution())
        S.close()
    for t in tickets[5:]:
        assert srv.poll(t)["state"] == "done"
        srv.fetch(t)
    srv.close()
