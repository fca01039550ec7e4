"""bench.py's reference arm (`--impl reference`) on the CPU: the oracle times
a bounded sample of the workload, the points of the first 1/8 of the grid
rays, and rank 0 prints the JSON line of the contract. Checked here on the
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
         "limiter": 1.0, "scheme": "rk4", "steps": 1, "warmup": 0}
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
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_wedge_sample_keeps_every_evaluated_stencil_whole():
    """A point of the sample that keeps a residual of its own (not far field)
    has all its neighbours in the sample, the same points as in the whole
    cloud, in the same order; points cut from a neighbour become far field."""
    import bench
    from paper_2403_13287_gb300.cloudgen import CLOUDS, naca0012_cloud
    for shuffled in (False, True):
        c = naca0012_cloud(*CLOUDS["naca0012_10k"], shuffle=shuffled)
        sub, pts = bench.wedge_sample(c, shuffled)
        assert sub["n"] == len(pts) and np.all(np.diff(pts) > 0)
        assert (c["L"] + 1) * (c["W"] // 8) == sub["n"]
        off, idx, soff, sidx = c["nbr_offsets"], c["nbr_idx"], sub["nbr_offsets"], sub["nbr_idx"]
        kept = 0
        for k, p in enumerate(pts):
            full = idx[off[p]:off[p + 1]]
            mine = pts[sidx[soff[k]:soff[k + 1]]]
            if sub["flags"][k] != 2:
                assert np.array_equal(mine, full)
                assert sub["flags"][k] == c["flags"][p]
                kept += 1
            else:
                assert c["flags"][p] == 2 or len(mine) < len(full)
        assert kept > 0.8 * sub["n"]
