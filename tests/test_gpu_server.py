"""The request server (adafac_server_*): every solve delivered by the
continuous-batching loop equals the same solve run alone through a handle,
requests are admitted by device-memory footprint, and requests that can never
fit are refused."""
import time

import numpy as np
import pytest

import workloads as wl
from paper_1903_10367_gb300 import adafac

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)


def _mix():
    """Solves of several shapes: 2-D random-block eps with BoxMG, 3-D constant
    eps (the fused path), FP64 and mixed precision."""
    out = []
    for i, (d, L, prec) in enumerate([(2, 3, "mixed"), (2, 4, "mixed"), (2, 5, "mixed"),
                                      (3, 3, "mixed"), (3, 4, "mixed"), (2, 4, "fp64"),
                                      (3, 3, "fp64"), (2, 3, "fp64")]):
        if d == 2:
            eps = wl.eps_random_blocks(2, L, 3 ** max(L - 3, 0), 1e-2, seed=1903 + i)
            f = wl.constant_rhs(2, L)
            opts = adafac.default_options(transfer="boxmg", precision=prec)
        else:
            eps = 1.0
            f = wl.manufactured_rhs(3, L)
            opts = adafac.default_options(precision=prec)
        out.append((d, L, eps, f, opts))
    return out


def _alone(d, L, eps, f, opts):
    S = adafac.Solver(d, L, eps, f, opts)
    c, rel = S.solve(1e-8, 2000)
    u = S.solution()
    S.close()
    return c, u


def _wait(srv, tickets, timeout=120.0):
    t0 = time.time()
    while time.time() - t0 < timeout:
        if all(srv.poll(t)["state"] in ("done", "failed") for t in tickets):
            return
        time.sleep(0.002)
    raise AssertionError("server did not finish")


def test_each_result_is_the_same_alone_and_in_the_mix():
    cases = _mix()
    alone = [_alone(*c) for c in cases]
    srv = adafac.Server(4 << 30, n_streams=8, max_running=16)
    tickets = [srv.submit(d, L, eps, f, opts) for (d, L, eps, f, opts) in cases]
    _wait(srv, tickets)
    for (c_alone, u_alone), t in zip(alone, tickets):
        info = srv.poll(t)
        assert info["state"] == "done" and info["status"] == 0
        assert info["rel"] <= 1e-8
        assert info["cycles"] == c_alone
        assert info["latency_ms"] >= info["queue_ms"] >= 0.0
        u = srv.fetch(t)
        scale = max(np.abs(u_alone).max(), 1e-300)
        assert np.abs(u - u_alone).max() / scale <= 1e-12
    assert srv.stats() == (0, 0, 0)
    srv.close()


def test_admission_by_memory_runs_everything_within_the_budget():
    # four solves of which only one fits into the pool at a time
    opts = adafac.default_options(precision="mixed")
    need = adafac.workspace_size(3, 4, opts)
    budget = int(need * 1.5)
    srv = adafac.Server(budget, n_streams=4, max_running=8)
    f = wl.manufactured_rhs(3, 4)
    tickets = [srv.submit(3, 4, 1.0, f * (k + 1), opts) for k in range(4)]
    peak = 0
    t0 = time.time()
    while time.time() - t0 < 120.0:
        p, r, b = srv.stats()
        peak = max(peak, b)
        assert b <= budget and r <= 1
        if p == 0 and r == 0:
            break
        time.sleep(0.0005)
    infos = [srv.poll(t) for t in tickets]
    for t, info in zip(tickets, infos):
        assert info["state"] == "done", info
        srv.fetch(t)
    assert peak >= need
    # each later request waited for the previous one to leave the pool
    assert sum(i["queue_ms"] > 0.5 for i in infos) >= 3
    srv.close()


def test_a_request_larger_than_the_pool_is_refused():
    srv = adafac.Server(1 << 20, n_streams=1, max_running=2)
    with pytest.raises(adafac.AdafacError) as e:
        srv.submit(3, 5, 1.0, None, adafac.default_options(precision="mixed"))
    assert e.value.status == 2  # OOM
    with pytest.raises(adafac.AdafacError):
        srv.poll(12345)
    srv.close()
