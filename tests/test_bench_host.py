"""Host-side pieces of bench.py: the byte accounting of the roofline, the L2
flush rule, the kernel fingerprint and the entry points the bench line needs."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import workloads as wl  # noqa: E402


def test_entry_points_exist():
    for name in ("bench_ours", "bench_reference", "run_serving", "run_oracle_sample",
                 "kernel_source_hash", "main"):
        assert callable(getattr(bench, name)), name


def test_algorithmic_bytes_of_the_fine_kernels():
    w = wl.get("poisson3d_d5")
    N = 242 ** 3
    assert bench._algorithmic_bytes("fine_down", w, "mixed", True) == 12 * N
    assert bench._algorithmic_bytes("fine_up", w, "mixed", True) == 8 * N
    assert bench._algorithmic_bytes("refine", w, "mixed", True) == 20 * N


def test_l2_flush_only_for_small_workloads():
    assert not bench._needs_flush(wl.get("poisson3d_d5"), "mixed")
    assert bench._needs_flush(wl.get("poisson2d_d4"), "fp64")


def test_kernel_fingerprint_is_stable():
    assert bench.kernel_source_hash() == bench.kernel_source_hash()
    assert len(bench.kernel_source_hash()) == 16
