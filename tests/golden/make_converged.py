"""Write tests/golden/converged_*.json: converged Cl, Cd and residue history of
the FP64 CPU oracle on small seeded clouds (calls only the oracle and the
input generator). Run from the repository root:

    python tests/golden/make_converged.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2403_13287_gb300.cloudgen import naca0012_cloud  # noqa: E402

CASES = [
    # name, W, L, seed, order, scheme, mach, aoa, limiter, cfl, iterations
    ("naca0012_96x56_m085_a1_rk4_lim1", 96, 56, 11, 2, 1, 0.85, 1.0, 1.0, 0.2, 1500),
    ("naca0012_128x77_m063_a2_rk4_nolim", 128, 77, 11, 2, 1, 0.63, 2.0, 0.0, 0.2, 1000),
]


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    for name, W, L, seed, order, scheme, mach, aoa, lim, cfl, iters in CASES:
        t = time.time()
        c = naca0012_cloud(W, L, seed=seed)
        m = oracle.split_stencils(c)
        U = oracle.freestream_state(c["n"], mach, aoa)
        U, hist = oracle.solve(c, m, U, iters, order=order, inner=3, scheme=scheme, cfl=cfl,
                               mach=mach, aoa_deg=aoa, limiter=lim)
        cl, cd, cp = oracle.forces(c, U, mach, aoa)
        out = {
            "source": "FP64 CPU oracle (oracle/lskum_oracle.c, orc_solve) run by "
                      "tests/golden/make_converged.py; inputs from cloudgen.naca0012_cloud",
            "cloud": {"W": W, "L": L, "seed": seed},
            "order": order, "inner": 3, "scheme": scheme, "mach": mach, "aoa_deg": aoa,
            "limiter_K": lim, "cfl": cfl, "iterations": iters,
            "cl": cl, "cd": cd, "cp": cp.tolist(),
            "residue_first": hist[1], "residue_last": hist[-1],
            "residue_every_100": hist[::100].tolist(),
            "seconds": time.time() - t,
        }
        with open(os.path.join(here, "converged_%s.json" % name), "w") as f:
            json.dump(out, f, indent=1)
        print(name, "cl %.10f cd %.10f residue %.3e -> %.3e (%.0f s)" % (cl, cd, hist[1], hist[-1], out["seconds"]),
              flush=True)


if __name__ == "__main__":
    main()
