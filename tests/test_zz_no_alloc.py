"""adafac_residual_norm_static: the Eq. 10 residual norm computed with the
library's fixed device scratch array instead of a workspace.  It must agree
with the handle's own residual norm (adafac_residual_norm) on the same u and b,
call after call, and reject trees larger than its scratch without launching.

This file is named so that pytest collects it last: the check also covers a
process in which every other test has already run."""
import ctypes

import numpy as np
import pytest

import workloads as wl
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


@pytest.mark.gpu
@pytest.mark.parametrize("d,L,eps", [(2, 4, 1.0), (2, 5, 2.5), (3, 3, 1.0), (3, 4, 0.7)])
def test_static_scratch_norm_equals_the_handle_norm_on_consecutive_calls(d, L, eps):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    f = wl.manufactured_rhs(d, L)
    S = adafac.Solver(d, L, eps, f, adafac.default_options())
    S.cycle(3)
    _, ab = S.residual_norm()
    u = torch.from_numpy(np.ascontiguousarray(S.solution()).reshape(-1)).cuda()
    b = torch.from_numpy(fem.load_vector(f, 1.0 / 3 ** L, d).reshape(-1)).cuda()
    S.close()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(-1.0)
        adafac.residual_norm_static(d, L, eps, u, b, out)
        torch.cuda.synchronize()
        assert out.item() == pytest.approx(ab, rel=1e-12)
