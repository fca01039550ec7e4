"""bench.py's closing summary object and its relative-error helper (no GPU):
the summary repeats the headline figures of every form under flat keys so a
truncated tail of the JSON line still shows them."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_relative_error_helper():
    import bench
    assert bench.rel(1.1, 1.0) == abs(1.1 - 1.0) / 1.0
    assert bench.rel(2e-4, 1e-4, scale=0.05) == abs(2e-4 - 1e-4) / 0.05
    assert bench.rel(1.0, 0.0) is None


def test_summary_collects_the_forms():
    import bench
    flux = {"kernel": "k_flux_update_mixed", "frac": 0.34, "avg_launch_ms": 0.37}
    qg = {"kernel": "k_qgrad_mixed", "frac": 0.74, "other": flux}
    err = {"converged_10k": {"cl_rel_err": 7e-6, "cd_rel_err": 1.6e-6, "cp_max_abs_err": 2.6e-6},
           "bench_cloud_after_timed_steps": {"residual_at_fp64_state": {"rel_l2": 1.5e-5}, "cd_rel_err": 8e-8}}
    forms = {"fp64": {"value": 6.3e7, "ms_per_step": 39.7},
             "mixed": {"value": 7.8e8, "ms_per_step": 3.2, "roofline": qg, "error": err},
             "mixed_speedup_vs_fp64": 12.4, "batched": {"value": 8.1e8, "speedup_vs_sequential": 1.75},
             "batched_speedup_vs_fp64": 12.9, "mixed_10m": {"value": 8.6e8}}
    line = {"value": 6.3e7, "edge_iterations_per_s": 5.1e8, "roofline": {"frac": 0.845, "hbm_frac": 0.031},
            "cpu_baseline": {"value": 4.1e5, "cores": 16}}
    s = bench.summary_of(line, forms)
    assert s["value"] == 6.3e7 and abs(s["rdp_s"] - 1 / 6.3e7) < 1e-20
    assert s["roofline_frac"] == 0.845 and s["roofline_hbm_frac"] == 0.031
    assert s["mixed_flux_hbm_frac"] == 0.34 and s["mixed_qgrad_hbm_frac"] == 0.74
    assert s["mixed_flux_ms_per_launch"] == 0.37
    assert s["mixed_converged_cd_rel_err"] == 1.6e-6 and s["mixed_residual_rel_l2_err"] == 1.5e-5
    assert s["mixed_speedup_vs_fp64"] == 12.4 and s["batched_speedup_vs_sequential"] == 1.75
    assert s["mixed_10m_value"] == 8.6e8 and s["cpu_baseline_cores"] == 16
