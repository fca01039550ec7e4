"""The 2.5M-point workload in the configuration bench.py times (needs a GPU).

Second order, 3 inner iterations, Venkatakrishnan limiter K = 1, M 1.2,
alpha 0, the cloud presented in shuffled order and renumbered in Morton
order; FP64 and the mixed form (autotuned launch shapes). The oracle cannot
evaluate all 2.5M points in a test, so it evaluates sampled points one by
one: a point's residual depends on q within five stencil rings (the
neighbours' q~ need their q-derivatives after the first-order pass and three
Jacobi inner passes, each reaching one ring further), so the oracle runs on
that 5-ring sub-cloud with the sample point's own flag and every other point
far field (no residual of its own), and the outermost ring given stencils
that only need to be non-degenerate (their derivatives never reach the
sample point). That this sampling is exact is checked without a GPU on the
10k-point cloud. Tolerances as for the small clouds: 1e-12 S (FP64), 3e-5 S
(mixed); one forward-Euler iteration checks the fused update at the samples.
"""
import numpy as np
import pytest

import oracle
from paper_2403_13287_gb300.cloudgen import CLOUDS, naca0012_cloud, smooth_state

MACH, AOA, LIM, RINGS = 1.2, 0.0, 1.0, 5


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.fixture(scope="module")
def full():
    W, L = CLOUDS["naca0012_2p5m"]
    c = naca0012_cloud(W, L, shuffle=True)
    U = smooth_state(c, MACH, AOA, amp=0.05, seed=7)
    rng = np.random.default_rng(2024)
    flags = c["flags"]
    samples = np.concatenate([rng.choice(np.nonzero(flags == 0)[0], 160, replace=False),
                              rng.choice(np.nonzero(flags == 1)[0], 32, replace=False)])
    return c, U, samples


def _sub_cloud(c, p):
    """The RINGS-ring neighbourhood of point p as a cloud of its own
    (index 0 = p), and the map to global indices."""
    off, idx = c["nbr_offsets"], c["nbr_idx"]
    ring = {int(p): 0}
    frontier = [int(p)]
    for r in range(1, RINGS + 1):
        nxt = []
        for q in frontier:
            for j in idx[off[q]:off[q + 1]]:
                j = int(j)
                if j not in ring:
                    ring[j] = r
                    nxt.append(j)
        frontier = nxt
    glob = np.array(sorted(ring, key=lambda j: (ring[j], j)), dtype=np.int64)
    loc = {int(g): k for k, g in enumerate(glob)}
    rows = []
    for g in glob:
        full_row = [loc[int(j)] for j in idx[off[g]:off[g + 1]] if int(j) in loc]
        if ring[int(g)] < RINGS:
            assert len(full_row) == off[g + 1] - off[g]
            rows.append(full_row)
        else:
            # outermost ring: any non-degenerate stencil (its derivatives do not reach p)
            d2 = (c["x"][glob] - c["x"][g]) ** 2 + (c["y"][glob] - c["y"][g]) ** 2
            d2[loc[int(g)]] = np.inf
            rows.append([int(k) for k in np.argsort(d2, kind="stable")[:8]])
    sub_off = np.zeros(len(glob) + 1, np.int32)
    sub_off[1:] = np.cumsum([len(r) for r in rows])
    flags = np.full(len(glob), 2, np.int32)
    flags[0] = c["flags"][p]
    sub = {"n": len(glob), "x": c["x"][glob], "y": c["y"][glob], "nx": c["nx"][glob], "ny": c["ny"][glob],
           "flags": flags, "nbr_offsets": sub_off, "nbr_idx": np.array([j for r in rows for j in r], np.int32),
           "wall_order": np.zeros(0, np.int32)}
    return sub, glob


def _oracle_at(c, U, samples):
    R = np.zeros((4, len(samples)))
    S = np.zeros((4, len(samples)))
    dt = np.zeros(len(samples))
    for k, p in enumerate(samples):
        sub, glob = _sub_cloud(c, p)
        m = oracle.split_stencils(sub)
        Rs, Ss = oracle.residual(sub, m, U[:, glob], order=2, inner=3, want_scale=True, limiter=LIM)
        R[:, k], S[:, k] = Rs[:, 0], Ss[:, 0]
        dt[k] = oracle.timestep(sub, U[:, glob], 0.2)[0]
    return R, S, dt


@pytest.fixture(scope="module")
def reference(full):
    c, U, samples = full
    return _oracle_at(c, U, samples)


def test_sampled_oracle_equals_the_whole_cloud_oracle():
    """No GPU: on the 10k-point cloud (shuffled, walls included) the 5-ring
    sub-cloud evaluation gives the whole-cloud oracle's residual, scale and
    time step at the sampled points bit for bit."""
    c = naca0012_cloud(*CLOUDS["naca0012_10k"], shuffle=True)
    U = smooth_state(c, MACH, AOA, amp=0.05, seed=7)
    Rf, Sf = oracle.residual(c, oracle.split_stencils(c), U, order=2, inner=3, want_scale=True, limiter=LIM)
    dtf = oracle.timestep(c, U, 0.2)
    rng = np.random.default_rng(1)
    samples = np.concatenate([rng.choice(np.nonzero(c["flags"] == 0)[0], 60, replace=False),
                              np.nonzero(c["flags"] == 1)[0][:20]])
    R, S, dt = _oracle_at(c, U, samples)
    assert np.array_equal(R, Rf[:, samples]) and np.array_equal(S, Sf[:, samples])
    assert np.array_equal(dt, dtf[samples])


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [0, 1])
def test_full_size_residual_at_sampled_points(full, reference, precision):
    from paper_2403_13287_gb300.lskum import Solver
    c, U, samples = full
    Ro, S, _ = reference
    s = Solver(c, order=2, inner_iters=3, time_scheme=1, cfl=0.2, mach=MACH, aoa_deg=AOA, limiter_K=LIM,
               precision=precision, reorder=1)
    if precision == 1:
        s.autotune()
    R = s.residual(_dev(U)).cpu().numpy()[:, samples]
    tol = 1e-12 if precision == 0 else 3e-5
    assert np.all(np.abs(R - Ro) <= tol * S), np.max(np.abs(R - Ro) / S)
    assert np.all(np.abs(Ro).max(axis=0) > 0.0)
    s.close()


@pytest.mark.gpu
def test_full_size_update_at_sampled_points(full, reference):
    """One forward-Euler iteration: U - dt R at the samples (wall points
    then lose their normal momentum)."""
    from paper_2403_13287_gb300.lskum import Solver
    c, U, samples = full
    Ro, S, dt = reference
    s = Solver(c, order=2, inner_iters=3, time_scheme=0, cfl=0.2, mach=MACH, aoa_deg=AOA, limiter_K=LIM,
               reorder=1)
    s.set_state(U)
    s.step(1)
    U1 = s.get_state()[:, samples]
    want = U[:, samples] - dt * Ro
    wall = c["flags"][samples] == 1
    nx, ny = c["nx"][samples], c["ny"][samples]
    mn = want[1] * nx + want[2] * ny
    want[1, wall] -= (mn * nx)[wall]
    want[2, wall] -= (mn * ny)[wall]
    scale = np.abs(U[:, samples]) + dt * S
    assert np.all(np.abs(U1 - want) <= 1e-12 * scale), np.max(np.abs(U1 - want) / scale)
    s.close()
