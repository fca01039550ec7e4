"""Mixed-precision form (precision = 1) against the FP64 CPU oracle (needs a GPU).

The form evaluates q, grad q and the split fluxes in FP32 and keeps U, the
RK accumulation, the residue and ill-conditioned least-squares closures in
FP64. Tolerances follow from FP32 rounding (unit roundoff 6e-8): each flux
and each perturbation dG carries a relative error of a few ulp of |G|
amplified by the exp of the q -> rho map and by the stencil weights, so the
residual is compared against the same summand scale S as the FP64 tests,
|R_mixed - R_oracle| <= 3e-5 S (500 ulp of S), and q-derivatives against
their summand scale at 2e-5. A formula error shows up at O(S).
"""
import numpy as np
import pytest

import oracle
from paper_2403_13287_gb300.cloudgen import naca0012_cloud

pytestmark = pytest.mark.gpu

GAMMA = 1.4


def _solver(cloud, **kw):
    from paper_2403_13287_gb300.lskum import Solver
    return Solver(cloud, precision=1, **kw)


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _perturbed_state(cloud, mach, aoa, amp=0.05, seed=0):
    rng = np.random.default_rng(seed)
    x, y = cloud["x"], cloud["y"]
    k = rng.uniform(1.0, 3.0, 4)
    ph = rng.uniform(0, 2 * np.pi, 4)
    a = np.radians(aoa)
    rho = 1.0 + amp * np.sin(k[0] * x + ph[0]) * np.cos(k[1] * y + ph[1])
    u = mach * np.cos(a) + amp * np.cos(k[2] * y + ph[2])
    v = mach * np.sin(a) + amp * np.sin(k[3] * x + ph[3])
    p = 1.0 / GAMMA * (1.0 + amp * np.cos(k[1] * x - k[0] * y))
    U = np.stack([rho, rho * u, rho * v, p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v)])
    U[:, cloud["flags"] == 2] = oracle.freestream(mach, aoa)[:, None]
    wall = cloud["flags"] == 1
    mn = U[1, wall] * cloud["nx"][wall] + U[2, wall] * cloud["ny"][wall]
    U[1, wall] -= mn * cloud["nx"][wall]
    U[2, wall] -= mn * cloud["ny"][wall]
    return np.ascontiguousarray(U)


@pytest.fixture(scope="module")
def small():
    return naca0012_cloud(130, 24, seed=11)


@pytest.mark.parametrize("order,limiter", [(1, 0.0), (2, 0.0), (2, 1.0)])
@pytest.mark.parametrize("reorder", [0, 1])
def test_mixed_residual_matches_oracle(small, order, limiter, reorder):
    U = _perturbed_state(small, 0.85, 1.0, seed=2)
    s = _solver(small, order=order, inner_iters=3, reorder=reorder, limiter_K=limiter)
    R = s.residual(_dev(U)).cpu().numpy()
    Ro, S = oracle.residual(small, oracle.split_stencils(small), U, order=order, inner=3,
                            want_scale=True, limiter=limiter)
    err = np.abs(R - Ro) / np.maximum(S, 1e-300)
    assert np.all(np.abs(R - Ro) <= 3e-5 * S), err.max()
    # and the form is not trivially equal to the FP64 one: FP32 rounding shows
    assert err.max() > 1e-12


@pytest.mark.parametrize("inner", [0, 1, 2, 3])
@pytest.mark.parametrize("limiter", [0.0, 1.0])
def test_mixed_q_derivatives_match_oracle(small, inner, limiter):
    U = _perturbed_state(small, 0.63, 2.0, seed=1)
    s = _solver(small, order=2, inner_iters=inner, limiter_K=limiter)
    qx, qy = s.q_derivatives(_dev(U))
    qx, qy = qx.cpu().numpy(), qy.cpu().numpy()
    q = oracle.q_variables(U)
    ox, oy = oracle.q_derivatives(small, q, inner=inner)
    if limiter:
        ox, oy = oracle.limit_gradients(small, q, ox, oy, limiter)
    off, idx = small["nbr_offsets"], small["nbr_idx"]
    rows = np.repeat(np.arange(small["n"]), np.diff(off))
    d = np.hypot(small["x"][idx] - small["x"][rows], small["y"][idx] - small["y"][rows])
    # q itself is stored in FP32, so each difference q_i - q_0 carries an
    # absolute error of order eps32 (|q_i| + |q_0|), amplified by 1/|d| in the
    # least-squares weights: the summand scale includes |q_i| + |q_0|
    S = np.zeros_like(q)
    for k in range(4):
        term = (np.abs(q[k, idx]) + np.abs(q[k, rows])
                + 0.5 * d * (np.hypot(ox[k, idx], oy[k, idx]) + np.hypot(ox[k, rows], oy[k, rows]))) / d
        S[k] = np.bincount(rows, weights=term, minlength=small["n"]) / np.diff(off)
    assert np.all(np.abs(qx - ox) <= 2e-5 * S)
    assert np.all(np.abs(qy - oy) <= 2e-5 * S)


@pytest.fixture(scope="module")
def closure_cloud():
    """A small cloud with FP64-closure points (least-squares closures that
    FP32 would get wrong): the most irregular of a few jittered clouds."""
    best, best_n = None, 0
    for W, L, seed, jitter in ((130, 24, 11, 0.1), (160, 40, 5, 0.25), (96, 56, 3, 0.35), (120, 40, 7, 0.45)):
        from paper_2403_13287_gb300.lskum import LskumError
        c = naca0012_cloud(W, L, seed=seed, jitter=jitter, shuffle=True)
        try:
            s = _solver(c, order=2)
        except LskumError:                  # a singular stencil: not a usable cloud
            continue
        n64 = s.mixed_fp64_points()
        s.close()
        if n64 > best_n:
            best, best_n = c, n64
    assert best_n > 0, "no candidate cloud has FP64-closure points"
    return best


@pytest.mark.parametrize("variant", [7, 22, 23])
@pytest.mark.parametrize("order,limiter", [(1, 0.0), (2, 1.0)])
def test_pipelined_shapes_residual_matches_oracle(closure_cloud, variant, order, limiter):
    """The software-pipelined flux loop (shapes 7, 22, 23). In the plain
    boundary mode it takes the neighbour rows by cp.async into shared memory,
    where the point's own row and its FP64-closure sums also wait; on a
    shuffled cloud with FP64-closure points it meets the mixed form's bar."""
    c = closure_cloud
    U = _perturbed_state(c, 0.85, 1.0, seed=5)
    s = _solver(c, order=order, inner_iters=3, reorder=1, limiter_K=limiter)
    assert s.mixed_fp64_points() > 0
    s.set_tuning(variant, 0)
    R = s.residual(_dev(U)).cpu().numpy()
    s.close()
    Ro, S = oracle.residual(c, oracle.split_stencils(c), U, order=order, inner=3, want_scale=True,
                            limiter=limiter)
    err = np.abs(R - Ro) / np.maximum(S, 1e-300)
    assert np.all(np.abs(R - Ro) <= 3e-5 * S), err.max()


def test_fp64_context_has_no_fp64_closure_points(small):
    from paper_2403_13287_gb300.lskum import Solver
    s = Solver(small, precision=0)
    assert s.mixed_fp64_points() == 0
    s.close()


def test_mixed_freestream_is_exactly_preserved():
    c = naca0012_cloud(320, 30)
    s = _solver(c, order=2, mach=1.2, aoa_deg=0.0, limiter_K=1.0)
    assert np.all(s.residual().cpu().numpy() == 0.0)


def test_mixed_short_trajectory_tracks_oracle(small):
    mach, aoa, lim = 0.85, 1.0, 1.0
    U0 = oracle.freestream_state(small["n"], mach, aoa)
    Uo, ho = oracle.solve(small, oracle.split_stencils(small), U0, 30, order=2, inner=3, scheme=1,
                          cfl=0.2, mach=mach, aoa_deg=aoa, limiter=lim)
    s = _solver(small, order=2, inner_iters=3, time_scheme=1, cfl=0.2, mach=mach, aoa_deg=aoa,
                limiter_K=lim)
    h = s.step(30)
    U = s.get_state()
    assert np.max(np.abs(U - Uo) / (np.abs(Uo) + 1e-3)) < 1e-4
    assert np.allclose(h, ho, rtol=1e-3, atol=1e-9)
