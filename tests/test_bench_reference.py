"""bench.py's reference arm (`--impl reference`) on the CPU: the oracle times
whole iterations of its solver loop on the configured cloud, on every host
core, and rank 0 prints the JSON line of the contract. Checked here on the
10k-point cloud; no GPU is involved."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _args(**kw):
    a = {"workload": "naca0012_10k", "shuffle": 1, "mach": 1.2, "aoa": 0.0, "order": 2, "inner": 3,
         "limiter": 1.0, "scheme": "rk4", "steps": 2, "warmup": 1, "cfl": 0.2, "ref_extra": False}
    a.update(kw)
    return type("A", (), a)()


def test_reference_line_follows_the_contract(capsys):
    import bench
    assert bench.run_reference(_args(), 0, 1) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["unit"] == bench.UNIT and line["metric"] == bench.METRIC
    assert line["value"] > 0.0 and line["higher_is_better"] is True and line["dtype"] == "f64"
    assert line["config"]["workload"] == "naca0012_10k" and line["config"]["scheme"] == "rk4"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert cb["nproc"] >= cb["cores"] and cb["cpu_model"]
    # measured, not extrapolated: the steps' time is the line's step time
    assert abs(line["value"] - line["config"]["points"] * 1e3 / line["ms_per_step"]) <= 1e-9 * line["value"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_steps_are_oracle_iterations():
    """One timed step is one iteration of the oracle's solver loop: W + K
    steps from the start state give the oracle's own state after W + K
    iterations, with either thread count."""
    import bench
    import oracle
    from paper_2403_13287_gb300.cloudgen import naca0012_cloud, smooth_state
    c = naca0012_cloud(40, 12, seed=2)
    m = oracle.split_stencils(c)
    args = _args()
    U0 = smooth_state(c, args.mach, args.aoa, amp=0.05, seed=7)
    ref, _ = oracle.solve(c, m, U0, 3, order=2, inner=3, scheme=1, cfl=args.cfl, mach=args.mach,
                          aoa_deg=args.aoa, limiter=args.limiter)
    for threads in (1, 3):
        times, U = bench.oracle_iterations(c, m, U0, args, 3, threads)
        assert len(times) == 3 and np.array_equal(U, ref)
    oracle.set_threads(1)
