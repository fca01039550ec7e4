"""Converged flow physics on the GPU, and its approach under refinement
(needs a GPU).

The FP64 CUDA path reproduces the oracle's converged goldens to 1e-8
(test_gpu_converged.py), so the physics checks the oracle passes on its
10k-point goldens (test_oracle_converged_physics.py) hold here too. This file
runs them again on the GPU's own converged solutions, and adds what the
oracle cannot afford on the CPU: the same solves on a cloud twice as fine in
each direction (40k points). Refinement must move the solution toward the
physics:
* M 1.2, alpha 0 (second order, K = 1): the leading-edge pressure rises
  toward the pitot pressure, and the wave drag grows toward its fine-grid
  value of about 0.1, from below;
* M 0.63, alpha 2 (first order): the discretisation drag shrinks and the
  lift grows toward the thin-airfoil value 2 pi alpha / sqrt(1 - M^2).
"""
import numpy as np
import pytest

from paper_2403_13287_gb300.cloudgen import naca0012_cloud

pytestmark = pytest.mark.gpu

GAMMA = 1.4


def pitot_cp(M, g=GAMMA):
    p02_p1 = (((g + 1) ** 2 * M * M / (4 * g * M * M - 2 * (g - 1))) ** (g / (g - 1))
              * (1 - g + 2 * g * M * M) / (g + 1))
    return (p02_p1 - 1) / (0.5 * g * M * M)


def isentropic_stagnation_cp(M, g=GAMMA):
    return ((1 + 0.5 * (g - 1) * M * M) ** (g / (g - 1)) - 1) / (0.5 * g * M * M)


def _converged(W, L, order, mach, aoa, lim, cfl, iters):
    from paper_2403_13287_gb300.lskum import Solver
    c = naca0012_cloud(W, L, seed=11)
    s = Solver(c, order=order, inner_iters=3, time_scheme=1, cfl=cfl, mach=mach, aoa_deg=aoa, limiter_K=lim,
               precision=0, reorder=1)
    h = s.step(iters)
    cl, cd, cp = s.forces()
    s.close()
    assert h[-1] <= 1e-8 * h.max(), "not converged"
    wo = c["wall_order"]
    return cl, cd, cp, c["x"][wo], c["y"][wo]


@pytest.fixture(scope="module")
def supersonic():
    return [_converged(128, 77, 2, 1.2, 0.0, 1.0, 1.5, 12000), _converged(256, 154, 2, 1.2, 0.0, 1.0, 1.0, 30000)]


@pytest.fixture(scope="module")
def subsonic():
    return [_converged(128, 77, 1, 0.63, 2.0, 0.0, 1.0, 10000), _converged(256, 154, 1, 0.63, 2.0, 0.0, 1.0, 30000)]


def test_supersonic_physics_and_refinement(supersonic):
    le_cp, cds = [], []
    for cl, cd, cp, xw, yw in supersonic:
        W = len(cp)
        le = W // 2
        assert 0.0 < cp[le] < pitot_cp(1.2)
        for side in (np.arange(le - 1, 0, -1), np.arange(le + 1, W)):
            keep = side[(xw[side] > 0.005) & (xw[side] < 0.9)]
            assert np.all(np.diff(cp[keep]) <= 1e-9)
        assert 0.03 < cd < 0.12 and abs(cl) <= 2e-2 * cd
        le_cp.append(cp[(xw < 0.01)].max())
        cds.append(cd)
    print("M 1.2: nose Cp %s (pitot %.4f), Cd %s" % (le_cp, pitot_cp(1.2), cds))
    assert le_cp[1] > le_cp[0]
    assert cds[1] > cds[0]


def test_subsonic_physics_and_refinement(subsonic):
    cls, cds = [], []
    for cl, cd, cp, xw, yw in subsonic:
        W = len(cp)
        upper = np.zeros(W, dtype=bool)
        upper[1:W // 2] = True
        lower = np.zeros(W, dtype=bool)
        lower[W // 2 + 1:] = True
        front = xw < 0.1
        k = np.argmax(np.where(front, cp, -np.inf))
        assert cp[k] <= isentropic_stagnation_cp(0.63) + 1e-3 and yw[k] <= 0.0
        ku = np.argmin(np.where(upper, cp, np.inf))
        assert cp[ku] < cp[lower].min() and xw[ku] < 0.25
        cls.append(cl)
        cds.append(cd)
    cl_pg = 2 * np.pi * np.radians(2.0) / np.sqrt(1 - 0.63 ** 2)
    print("M 0.63: Cl %s (thin airfoil %.4f), Cd %s" % (cls, cl_pg, cds))
    assert abs(cds[1]) < abs(cds[0])
    assert abs(cls[1] - cl_pg) < abs(cls[0] - cl_pg)
