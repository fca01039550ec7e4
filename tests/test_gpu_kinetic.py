"""The kinetic boundary mode of the CUDA path against the oracle (needs a GPU).

Wall and far-field points see the mirror images of their neighbours across
their tangent lines (reflected gas at the wall, the free stream outside), and
take the interior formulas on that augmented stencil; far-field points are
updated instead of held. Tolerances as for the plain mode: the FP64 residual
within 1e-12 of the oracle's summand scale S, q-derivatives within 2e-12 of
the least-squares summand scale (the images add as many terms again at
boundary points), trajectories 1e-10 relative; the mixed form within 3e-5 S.
"""
import numpy as np
import pytest

import oracle
from paper_2403_13287_gb300.cloudgen import naca0012_cloud

pytestmark = pytest.mark.gpu

GAMMA = 1.4


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _solver(cloud, **kw):
    from paper_2403_13287_gb300.lskum import Solver
    kw.setdefault("boundary", 1)
    return Solver(cloud, **kw)


def _state(cloud, mach, aoa, amp=0.05, seed=0):
    """A smooth seeded perturbation of the free stream everywhere, far-field
    points included (they are not held in this mode); no normal momentum at
    the wall."""
    rng = np.random.default_rng(seed)
    x, y = cloud["x"], cloud["y"]
    k = rng.uniform(0.5, 2.0, 4)
    ph = rng.uniform(0, 2 * np.pi, 4)
    a = np.radians(aoa)
    rho = 1.0 + amp * np.sin(k[0] * x + ph[0]) * np.cos(k[1] * y + ph[1])
    u = mach * np.cos(a) + amp * np.cos(k[2] * y + ph[2])
    v = mach * np.sin(a) + amp * np.sin(k[3] * x + ph[3])
    p = 1.0 / GAMMA * (1.0 + amp * np.cos(k[1] * x - k[0] * y))
    U = np.stack([rho, rho * u, rho * v, p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v)])
    wall = cloud["flags"] == 1
    mn = U[1, wall] * cloud["nx"][wall] + U[2, wall] * cloud["ny"][wall]
    U[1, wall] -= mn * cloud["nx"][wall]
    U[2, wall] -= mn * cloud["ny"][wall]
    return np.ascontiguousarray(U)


@pytest.fixture(scope="module")
def small():
    c = naca0012_cloud(130, 24, seed=11)          # 3250 points, 130 wall, 130 far field
    return c, oracle.split_stencils(c)


@pytest.mark.parametrize("order,limiter", [(1, 0.0), (2, 0.0), (2, 1.0)])
@pytest.mark.parametrize("reorder", [0, 1])
def test_residual_matches_oracle(small, order, limiter, reorder):
    c, m = small
    U = _state(c, 0.85, 1.0, seed=2)
    s = _solver(c, order=order, inner_iters=3, reorder=reorder, limiter_K=limiter, mach=0.85, aoa_deg=1.0)
    assert np.array_equal(s.stencil_masks(), m)       # the images are internal
    R = s.residual(_dev(U)).cpu().numpy()
    Ro, S = oracle.residual(c, m, U, order=order, inner=3, want_scale=True, limiter=limiter, boundary=1,
                            mach=0.85, aoa_deg=1.0)
    assert np.all(np.abs(R - Ro) <= 1e-12 * S), np.max(np.abs(R - Ro) / S)
    far = c["flags"] == 2
    assert np.all(np.abs(R[:, far]).max(axis=0) > 0.0)    # far-field points are evaluated
    Rp = oracle.residual(c, m, U, order=order, inner=3, limiter=limiter)
    wall = c["flags"] == 1
    assert np.all(np.abs(Rp[:, wall] - Ro[:, wall]).max(axis=0) > 1e-8)   # and the wall differs


@pytest.mark.parametrize("order,limiter", [(1, 0.0), (2, 0.0), (2, 1.0)])
def test_mixed_residual_matches_oracle(small, order, limiter):
    c, m = small
    U = _state(c, 0.85, 1.0, seed=3)
    s = _solver(c, order=order, inner_iters=3, reorder=1, limiter_K=limiter, precision=1, mach=0.85, aoa_deg=1.0)
    R = s.residual(_dev(U)).cpu().numpy()
    Ro, S = oracle.residual(c, m, U, order=order, inner=3, want_scale=True, limiter=limiter, boundary=1,
                            mach=0.85, aoa_deg=1.0)
    assert np.all(np.abs(R - Ro) <= 3e-5 * S), np.max(np.abs(R - Ro) / S)


@pytest.mark.parametrize("inner,limiter", [(0, 0.0), (3, 0.0), (0, 1.0), (1, 1.0), (3, 1.0)])
def test_q_derivatives_match_oracle(small, inner, limiter):
    c, m = small
    U = _state(c, 0.63, 2.0, seed=4)
    s = _solver(c, order=2, inner_iters=inner, limiter_K=limiter, mach=0.63, aoa_deg=2.0)
    qx, qy = (t.cpu().numpy() for t in s.q_derivatives(_dev(U)))
    _, ox, oy = oracle.residual(c, m, U, order=2, inner=inner, limiter=limiter, want_grad=True, boundary=1,
                                mach=0.63, aoa_deg=2.0)
    off, idx = c["nbr_offsets"], c["nbr_idx"]
    rows = np.repeat(np.arange(c["n"]), np.diff(off))
    d = np.hypot(c["x"][idx] - c["x"][rows], c["y"][idx] - c["y"][rows])
    q = oracle.q_variables(U)
    S = np.zeros_like(q)
    for k in range(4):
        term = (np.abs(q[k, idx] - q[k, rows]) + 0.5 * d * (np.hypot(ox[k, idx], oy[k, idx])
                                                            + np.hypot(ox[k, rows], oy[k, rows]))) / d
        S[k] = np.bincount(rows, weights=term, minlength=c["n"]) / np.diff(off)
    assert np.all(np.abs(qx - ox) <= 2e-12 * S)
    assert np.all(np.abs(qy - oy) <= 2e-12 * S)
    # the images change the first-order gradients at the boundary points only
    if inner == 0 and limiter == 0.0:
        _, px, py = oracle.residual(c, m, U, order=2, inner=0, want_grad=True)
        interior = c["flags"] == 0
        assert np.array_equal(ox[:, interior], px[:, interior])
        assert np.all(np.abs(ox[:, ~interior] - px[:, ~interior]).max(axis=0) > 0.0)


@pytest.mark.parametrize("scheme,order,limiter", [(1, 2, 0.0), (0, 2, 1.0), (1, 1, 0.0)])
def test_trajectory_matches_oracle(small, scheme, order, limiter):
    c, m = small
    mach, aoa = (0.85, 1.0) if limiter == 0.0 else (1.2, 0.0)
    U0 = oracle.freestream_state(c["n"], mach, aoa)
    iters = 20
    Uo, ho = oracle.solve(c, m, U0, iters, order=order, inner=3, scheme=scheme, cfl=0.2, mach=mach, aoa_deg=aoa,
                          limiter=limiter, boundary=1)
    s = _solver(c, order=order, inner_iters=3, time_scheme=scheme, cfl=0.2, mach=mach, aoa_deg=aoa,
                limiter_K=limiter, reorder=1)
    h = s.step(iters)
    U = s.get_state()
    assert np.max(np.abs(U - Uo) / (np.abs(Uo) + 1e-3)) < 1e-10
    assert np.allclose(h, ho, rtol=1e-9, atol=1e-14)
    far = c["flags"] == 2
    assert np.any(U[:, far] != oracle.freestream(mach, aoa)[:, None])   # far field not held
    cl, cd, _ = s.forces()
    clo, cdo, _ = oracle.forces(c, Uo, mach, aoa)
    assert abs(cl - clo) <= 1e-10 * max(abs(clo), abs(cdo)) and abs(cd - cdo) <= 1e-10 * max(abs(clo), abs(cdo))


@pytest.mark.parametrize("precision", [0, 1])
def test_free_stream_is_preserved_with_free_stream_images(precision):
    """On a cloud whose boundaries are all far field, U = U_inf gives R = 0
    exactly (the images carry the same free stream, bit for bit)."""
    import importlib
    import sys
    import os
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    half = importlib.import_module("test_oracle_kinetic")
    h = half.half_cloud("far", seed=5)
    c = half._csr(h, h["nb"])
    for aoa in (0.0, 23.0):
        s = _solver(c, order=2, inner_iters=3, precision=precision, mach=0.7, aoa_deg=aoa, limiter_K=1.0)
        R = s.residual().cpu().numpy()
        assert np.all(R == 0.0)


def test_batch_uses_each_cases_free_stream(small):
    """In a batch the far-field images carry the case's own free stream."""
    from paper_2403_13287_gb300.lskum import Solver
    c, m = small
    cases = [(c, 0.5, -2.0), (c, 0.85, 1.0), (c, 1.2, 4.0)]
    B = Solver.batch(cases, order=2, inner_iters=3, precision=0, reorder=1, boundary=1)
    Us = [_state(c, mach, aoa, seed=10 + k) for k, (_, mach, aoa) in enumerate(cases)]
    R = B.residual(_dev(np.concatenate(Us, axis=1))).cpu().numpy()
    for k, (_, mach, aoa) in enumerate(cases):
        first, count, _, _ = B.case_range(k)
        Ro, S = oracle.residual(c, m, Us[k], order=2, inner=3, want_scale=True, boundary=1, mach=mach,
                                aoa_deg=aoa)
        assert np.all(np.abs(R[:, first:first + count] - Ro) <= 1e-12 * S)


def test_derivative_calls_need_the_plain_mode(small):
    from paper_2403_13287_gb300.lskum import LskumError, LSKUM_ERR_ARG
    c, _ = small
    s = _solver(c, order=2)
    W = _dev(np.zeros((4, c["n"])))
    for call in (lambda: s.residual_vjp(W), lambda: s.step_vjp(W)):
        with pytest.raises(LskumError) as e:
            call()
        assert e.value.status == LSKUM_ERR_ARG
