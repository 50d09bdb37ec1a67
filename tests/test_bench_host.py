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


def test_algorithmic_bytes_of_the_level_kernels_count_structural_nonzeros():
    # BoxMG weights that are not zero by structure: (5/3)^3 per fine vertex
    w = wl.get("jump3d_d5")
    N = 242 ** 3
    p_b = (5.0 / 3.0) ** 3 * 4
    assert bench._algorithmic_bytes("fine_update", w, "mixed", False) == round((12 + p_b + 4) * N)
    assert bench._algorithmic_bytes("fine_restrict", w, "mixed", False) == round((4 + p_b) * N)
    assert bench._algorithmic_bytes("fine_residual", w, "mixed", False) == 16 * N


def test_traffic_lookup_checks_sources_and_reports_the_capture_shape():
    w = wl.get("poisson3d_d5")
    good = bench.kernel_source_hash(bench.TRAFFIC_SOURCES["poisson3d_d5"])
    table = {"poisson3d_d5": {"source_hash": good, "launch_shape": {"sweep_nz": 9, "sweep_nz_down": 9},
                              "bytes": {"fine_up": 123}}}
    assert bench._traffic_from_profile("fine_up", w, table=table) == (123, {"sweep_nz": 9, "sweep_nz_down": 9})
    assert bench._traffic_from_profile("fine_down", w, table=table)[0] is None
    stale = {"poisson3d_d5": dict(table["poisson3d_d5"], source_hash="0" * 16)}
    assert bench._traffic_from_profile("fine_up", w, table=stale) == (None, None)
    assert bench._shape_differs({"sweep_nz": 9, "sweep_nz_down": 9}, {"sweep_nz": 8, "sweep_nz_down": 8})
    assert not bench._shape_differs({"sweep_nz": 9, "sweep_nz_down": 9}, {"sweep_nz": 9, "sweep_nz_down": 9, "path": 1})
    assert not bench._shape_differs(None, {"sweep_nz": 8})


def test_committed_traffic_table_matches_the_current_kernel_sources():
    # the committed ncu figures describe the kernels in this tree
    for name in ("poisson3d_d5", "jump3d_d5"):
        w = wl.get(name)
        kinds = {"poisson3d_d5": "fine_up", "jump3d_d5": "fine_restrict"}
        traffic, _ = bench._traffic_from_profile(kinds[name], w)
        assert traffic and traffic > 0, name
