"""Write the stored oracle results under tests/golden/ (calls only the FP64
CPU oracle and the input generator). Run from the repository root:

    python tests/golden/make_converged.py [name ...]

converged_*.json: solves run until the residue has fallen by the stated
factor from its largest value (the convergence criterion of these goldens:
a drop of at least 1e-8, i.e. eight decades, and Cl, Cd unchanged to 1e-7
of the larger over the last 1000 iterations); Cl, Cd, wall Cp and the
residue history.
run_*.json: a fixed number of iterations of a larger cloud with the whole
residue history (the 160k-point transonic workload, 2000 iterations).

The oracle runs on all host cores (its OpenMP build, bitwise the serial one).
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

# name: (W, L, seed, order, scheme, mach, aoa, limiter K, cfl, iterations, kind)
CASES = {
    "converged_naca0012_128x77_m120_a0_rk4_lim1": (128, 77, 11, 2, 1, 1.2, 0.0, 1.0, 1.5, 12000, "converged"),
    "converged_naca0012_128x77_m063_a2_rk4_o1": (128, 77, 11, 1, 1, 0.63, 2.0, 0.0, 1.0, 10000, "converged"),
    "converged_naca0012_128x77_m085_a1_rk4_o1": (128, 77, 11, 1, 1, 0.85, 1.0, 0.0, 1.0, 36000, "converged"),
    "run_naca0012_160k_m085_a1_rk4_lim1": (512, 311, 2403_13287, 2, 1, 0.85, 1.0, 1.0, 0.2, 2000, "run"),
}


def main(names):
    here = os.path.dirname(os.path.abspath(__file__))
    threads = oracle.set_threads(os.cpu_count() or 1)
    for name in names:
        W, L, seed, order, scheme, mach, aoa, lim, cfl, iters, kind = CASES[name]
        t = time.time()
        c = naca0012_cloud(W, L, seed=seed)
        m = oracle.split_stencils(c)
        U = oracle.freestream_state(c["n"], mach, aoa)
        chunk = 1000 if kind == "converged" else iters
        hist, forces = [], []
        for _ in range(iters // chunk):
            U, h = oracle.solve(c, m, U, chunk, order=order, inner=3, scheme=scheme, cfl=cfl,
                                mach=mach, aoa_deg=aoa, limiter=lim)
            hist.append(h)
            forces.append(oracle.forces(c, U, mach, aoa)[:2])
        hist = np.concatenate(hist)
        cl, cd, cp = oracle.forces(c, U, mach, aoa)
        out = {
            "source": "FP64 CPU oracle (oracle/lskum_oracle.c, orc_solve) run by "
                      "tests/golden/make_converged.py; inputs from cloudgen.naca0012_cloud",
            "cloud": {"W": W, "L": L, "seed": seed, "n": int(c["n"])},
            "order": order, "inner": 3, "scheme": scheme, "mach": mach, "aoa_deg": aoa,
            "limiter_K": lim, "cfl": cfl, "iterations": iters,
            "cl": cl, "cd": cd, "cp": cp.tolist(),
            "residue_first": float(hist[1]), "residue_max": float(hist.max()),
            "residue_last": float(hist[-1]), "residue_drop": float(hist[-1] / hist.max()),
            "seconds": time.time() - t, "oracle_threads": threads,
        }
        if kind == "converged":
            out["residue_every_100"] = hist[::100].tolist()
            out["forces_every_1000"] = [list(f) for f in forces]
            if len(forces) >= 2:
                out["force_change_last_1000"] = [abs(forces[-1][0] - forces[-2][0]),
                                                 abs(forces[-1][1] - forces[-2][1])]
        else:
            out["residue_history"] = hist.tolist()
        with open(os.path.join(here, "%s.json" % name), "w") as f:
            json.dump(out, f, indent=1)
        print(name, "cl %.10f cd %.10f residue %.3e -> %.3e (drop %.1e, %.0f s)" % (
            cl, cd, hist.max(), hist[-1], hist[-1] / hist.max(), out["seconds"]), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(CASES))
