"""The autotuner of launch shapes (adafac_autotune).

Every candidate shape computes the same values, so a tuned solve must repeat
the untuned one bit for bit: the same cycle count, the same residual history
and the same iterate.  A second handle of the same problem shape takes the
stored choice without timing.
"""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1903_10367_gb300 import adafac  # noqa: E402


def _solve(d, L, eps, f, opts, tune):
    S = adafac.Solver(d, L, eps, f, opts)
    rec = S.autotune(3) if tune else None
    cycles, rel = S.solve(1e-8, 5000)
    out = (cycles, S.history(), S.solution())
    S.close()
    return out, rec


CASES = [
    # fused 3-D sweeps: Poisson, scalar eps, d-linear
    (3, 4, "scalar", "dlinear", 1),
    # grid-shaped level kernels: varying eps, BoxMG, 3-D and 2-D
    (3, 4, "blocks", "boxmg", 2),
    (2, 5, "blocks", "boxmg", 2),
]


@pytest.mark.parametrize("d,L,eps_kind,transfer,path", CASES)
def test_tuned_solve_repeats_the_untuned_one_bit_for_bit(d, L, eps_kind, transfer, path):
    eps = 1.0 if eps_kind == "scalar" else wl.eps_random_blocks(d, L, 3 ** (L - 3), 1e-2, 1903)
    f = wl.manufactured_rhs(d, L)
    opts = adafac.default_options(transfer=transfer, precision="mixed")
    (c0, h0, u0), _ = _solve(d, L, eps, f, opts, False)
    (c1, h1, u1), rec = _solve(d, L, eps, f, opts, True)
    assert rec["path"] == path
    assert rec["candidates"] > 2
    assert 0.0 < rec["us_tuned"] <= rec["us_default"]
    if path == 1:
        # slab counts along z: at most one per interior coarse / fine plane
        assert 1 <= rec["sweep_nz"] <= 3 ** (L - 1) - 1
        assert 1 <= rec["sweep_nz_down"] <= 3 ** L - 1
    else:
        assert rec["res_bx"] * rec["res_by"] in (128, 256) and rec["res_bx"] % 32 == 0
        assert rec["upd_bx"] * rec["upd_by"] in (128, 256) and rec["upd_bx"] % 32 == 0
    assert c1 == c0
    np.testing.assert_array_equal(h1, h0)
    np.testing.assert_array_equal(u1, u0)
    # the same shape again: the stored choice, no timing
    (c2, h2, u2), rec2 = _solve(d, L, eps, f, opts, True)
    assert rec2["cached"] == 1
    for k in ("path", "sweep_nz", "sweep_nz_down", "res_bx", "res_by", "res_zr", "upd_bx", "upd_by"):
        assert rec2[k] == rec[k]
    assert c2 == c0
    np.testing.assert_array_equal(u2, u0)


def test_nothing_to_tune_in_fp64():
    S = adafac.Solver(2, 4, 1.0, wl.manufactured_rhs(2, 4), adafac.default_options())
    rec = S.autotune(2)
    assert rec["path"] == 0 and rec["candidates"] == 0
    S.close()
