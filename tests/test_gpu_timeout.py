"""The bounded waits of the fused 3-D sweeps give up without faulting the GPU.

With the poll limit set to 0 every wait for a staged plane gives up before
its first poll.  No copy hangs and no address is wrong: the test only makes
the bound run out.  The contract: the solve returns TIMEOUT naming where
the first wait gave up, the sweeps store nothing (the iterate is bitwise
the one from before the call), and the handle, once reset with the default
limit, and a fresh handle both solve normally."""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1903_10367_gb300 import adafac  # noqa: E402

DEFAULT_POLLS = 1 << 22


def _solver(L):
    o = adafac.default_options(precision="mixed", inner_cycles=4)
    return adafac.Solver(3, L, 1.0, wl.manufactured_rhs(3, L), o)


@pytest.mark.parametrize("L", [3, 4])
def test_a_wait_that_runs_out_reports_timeout_and_keeps_the_iterate(L):
    S = _solver(L)
    S.cycle(4)                       # one good refinement step
    u_before = S.solution().copy()
    S.set_wait_limit(0)
    with pytest.raises(adafac.AdafacError) as ei:
        S.solve(1e-8, 40)
    assert ei.value.status == 4      # ADAFAC_ERR_TIMEOUT
    assert "bounded device-side wait gave up" in str(ei.value)
    assert "mode" in str(ei.value) and "block" in str(ei.value)
    assert np.array_equal(S.solution(), u_before)
    # the handle itself recovers after a reset with the default limit
    S.set_wait_limit(DEFAULT_POLLS)
    S.reset()
    cycles, rel = S.solve(1e-8, 500)
    assert rel <= 1e-8
    S.close()
    F = _solver(L)
    c2, rel2 = F.solve(1e-8, 500)
    F.close()
    assert rel2 <= 1e-8 and c2 == cycles


def test_negative_limits_are_refused():
    S = _solver(2)
    with pytest.raises(adafac.AdafacError) as ei:
        S.set_wait_limit(-1)
    assert ei.value.status == 1
    S.close()
