"""Reverse-mode derivatives of the iteration and of the forces (needs a GPU).

lskum_step_vjp and lskum_forces_vjp against the complex-step oracle
(oracle/lskum_jvp.py) by the dot-product identity <w, J v> = <J^T w, v> and by
sampled entries; then d Cl / d (Hicks-Henne amplitudes) after unrolled RK4
iterations with checkpointing (paper_2403_13287_gb300/adjoint.py) against the
oracle's complex step through the same iterations and against central
differences (step 1e-6) of the GPU forward solve.

Tolerance: both sides compute exact derivatives up to rounding, so dot
products agree to 1e-10 of the sum of the magnitudes of their terms, and the
unrolled gradient to 1e-8 of its largest entry (rounding carried through the
iterations). Central differences carry O(h^2) truncation and O(eps/h)
rounding: 1e-5 relative. The nearest-neighbour distance in the time step has a
kink where two neighbours are equally near (the leading and trailing edge of
the mirror-symmetric contour): the derivative takes the first of them in row
order, as the oracle does, and the finite-difference checks use displacements
that keep the contour's mirror symmetry.
"""
import numpy as np
import pytest

import oracle
from oracle import lskum_jvp
from paper_2403_13287_gb300.cloudgen import hicks_henne_basis, naca0012_cloud, smooth_state

pytestmark = pytest.mark.gpu

MACH, AOA = 0.63, 2.0


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _solver(cloud, **kw):
    from paper_2403_13287_gb300.lskum import Solver
    kw.setdefault("mach", MACH)
    kw.setdefault("aoa_deg", AOA)
    return Solver(cloud, **kw)


@pytest.fixture(scope="module")
def small():
    c = naca0012_cloud(130, 24, seed=11)
    return c, oracle.split_stencils(c)


@pytest.mark.parametrize("scheme,order", [(0, 1), (0, 2), (1, 2)])
def test_step_vjp_dot_products(small, scheme, order):
    c, mask = small
    n = c["n"]
    U = smooth_state(c, MACH, AOA, amp=0.05, seed=5)
    rng = np.random.default_rng(7 + scheme + order)
    W = rng.standard_normal((4, n))
    s = _solver(c, order=order, inner_iters=3, time_scheme=scheme, reorder=1)
    Ub, xb, yb = (t.cpu().numpy() for t in s.step_vjp(_dev(W), _dev(U)))
    vU = rng.standard_normal((4, n)) * np.abs(U)
    vx = rng.standard_normal(n) * 1e-3
    vy = rng.standard_normal(n) * 1e-3
    kw = dict(scheme=scheme, order=order, inner=3, mach=MACH, aoa_deg=AOA)
    for dU, dx, dy, gpu in ((vU, None, None, np.sum(Ub * vU)), (None, vx, vy, np.sum(xb * vx) + np.sum(yb * vy))):
        Jv = lskum_jvp.iterate_jvp(c, mask, U, dU=dU, dx=dx, dy=dy, **kw)
        ref = np.sum(W * Jv)
        assert abs(gpu - ref) <= 1e-10 * np.sum(np.abs(W * Jv)), (gpu, ref)
    # a few entries of U_bar, each one complex-step iteration
    for k, p in ((0, 17), (1, 1234), (3, n - 5)):
        e = np.zeros((4, n))
        e[k, p] = 1.0
        ref = np.sum(W * lskum_jvp.iterate_jvp(c, mask, U, dU=e, **kw))
        assert abs(Ub[k, p] - ref) <= 1e-10 * (np.abs(Ub).max() + abs(ref))


def test_forces_vjp_dot_products(small):
    c, _ = small
    n = c["n"]
    U = smooth_state(c, MACH, AOA, amp=0.05, seed=6)
    s = _solver(c, order=2)
    s.set_state(U)
    rng = np.random.default_rng(3)
    vU = rng.standard_normal((4, n)) * np.abs(U)
    vx = rng.standard_normal(n) * 1e-3
    vy = rng.standard_normal(n) * 1e-3
    for clb, cdb in ((1.0, 0.0), (0.0, 1.0), (0.3, -2.0)):
        Ub, xb, yb = (t.cpu().numpy() for t in s.forces_vjp(clb, cdb))
        dcl, dcd = lskum_jvp.forces_jvp(c, U, dU=vU, mach=MACH, aoa_deg=AOA)
        ref = clb * dcl + cdb * dcd
        assert abs(np.sum(Ub * vU) - ref) <= 1e-12 * (abs(ref) + np.sum(np.abs(Ub * vU)))
        dcl, dcd = lskum_jvp.forces_jvp(c, U, dx=vx, dy=vy, mach=MACH, aoa_deg=AOA)
        ref = clb * dcl + cdb * dcd
        got = np.sum(xb * vx) + np.sum(yb * vy)
        assert abs(got - ref) <= 1e-12 * (abs(ref) + np.sum(np.abs(xb * vx)) + np.sum(np.abs(yb * vy)))


def test_step_vjp_is_the_same_in_a_mixed_context(small):
    c, _ = small
    n = c["n"]
    U = smooth_state(c, MACH, AOA, amp=0.05, seed=8)
    W = _dev(np.random.default_rng(1).standard_normal((4, n)))
    a = [t.cpu().numpy() for t in _solver(c, order=2, time_scheme=1, reorder=1).step_vjp(W, _dev(U))]
    b = [t.cpu().numpy() for t in _solver(c, order=2, time_scheme=1, reorder=1, precision=1).step_vjp(W, _dev(U))]
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_limited_step_vjp_dot_products(small):
    """One RK4 iteration with the limiter (K = 1, M 0.85) in reverse against
    the oracle's complex step through the same iteration; the directions
    leave the far-field states and the wall points fixed (tied choices of
    the limiter and of the nearest-neighbour distance sit there)."""
    c, mask = small
    n = c["n"]
    U = smooth_state(c, 0.85, 1.0, amp=0.05, seed=16)
    W = np.random.default_rng(2).standard_normal((4, n))
    s = _solver(c, order=2, time_scheme=1, reorder=1, limiter_K=1.0, mach=0.85, aoa_deg=1.0)
    Ub, xb, yb = (t.cpu().numpy() for t in s.step_vjp(_dev(W), _dev(U)))
    rng = np.random.default_rng(11)
    far, wall = c["flags"] == 2, c["flags"] == 1
    vU = rng.standard_normal((4, n)) * np.abs(U)
    vU[:, far] = 0.0
    vx = rng.standard_normal(n) * 1e-3
    vy = rng.standard_normal(n) * 1e-3
    vx[wall] = 0.0
    vy[wall] = 0.0
    kw = dict(scheme=1, order=2, inner=3, mach=0.85, aoa_deg=1.0, limiter=1.0)
    for dU, dx, dy, gpu in ((vU, None, None, np.sum(Ub * vU)), (None, vx, vy, np.sum(xb * vx) + np.sum(yb * vy))):
        Jv = lskum_jvp.iterate_jvp(c, mask, U, dU=dU, dx=dx, dy=dy, **kw)
        ref = np.sum(W * Jv)
        assert abs(gpu - ref) <= 1e-10 * np.sum(np.abs(W * Jv)), (gpu, ref)


# ---------------------------------------------------------------------------
# d Cl / d (Hicks-Henne amplitudes) through unrolled iterations
# ---------------------------------------------------------------------------
ITERS = 9


def _deformed(base, B, a):
    c = dict(base)
    c["y"] = base["y"] + a @ B
    return c


def _cl_after(cloud, U0):
    s = _solver(cloud, order=2, inner_iters=3, time_scheme=1, reorder=1)
    s.set_state(U0)
    s.step(ITERS, history=False)
    return s.forces(want_cp=False)[0]


def test_unrolled_cl_gradient_wrt_hicks_henne_amplitudes():
    from paper_2403_13287_gb300.adjoint import unrolled_force_gradient
    base = naca0012_cloud(64, 35, seed=4)           # grid order: the bump basis needs it
    B = hicks_henne_basis(base)
    a = np.random.default_rng(2024).uniform(-2e-3, 2e-3, B.shape[0])
    c = _deformed(base, B, a)
    U0 = oracle.freestream_state(c["n"], MACH, AOA)   # independent of the shape
    s = _solver(c, order=2, inner_iters=3, time_scheme=1, reorder=1)
    (cl, cd), (U0b, xb, yb), info = unrolled_force_gradient(s, _dev(U0), ITERS, cl_bar=1.0)
    g = B @ yb.cpu().numpy()
    assert info["checkpoint_every"] == 3 and info["recomputed_iterations"] == 6
    assert info["state_bytes_peak"] < info["state_bytes_unrolled"]
    # the oracle: complex step through the same 9 RK4 iterations, one amplitude at a time
    mask = oracle.split_stencils(c)
    ref = np.empty_like(g)
    for k in range(B.shape[0]):
        (clo, _), (dcl, _) = lskum_jvp.unrolled_forces(c, mask, U0, ITERS, dy=B[k], scheme=1, mach=MACH,
                                                       aoa_deg=AOA)
        ref[k] = dcl
    assert abs(cl - clo) <= 1e-10 * abs(clo)
    assert np.all(np.abs(g - ref) <= 1e-8 * np.abs(ref).max()), (g, ref)
    # central differences of the GPU solve along mirror-symmetric combinations
    h = 1e-6
    K = B.shape[0] // 2
    for k in range(K):
        d = np.zeros(B.shape[0])
        d[k] = d[K + k] = 1.0
        fd = (_cl_after(_deformed(base, B, a + h * d), U0) - _cl_after(_deformed(base, B, a - h * d), U0)) / (2 * h)
        assert abs(fd - (g[k] + g[K + k])) <= 1e-5 * np.abs(g).max(), (k, fd, g[k] + g[K + k])


def test_unrolled_cd_gradient_with_the_limiter():
    """dCd/d(amplitudes) through 9 RK4 iterations of the limited scheme
    (K = 1) at M 1.2, alpha 0: the checkpointed reverse sweep against the
    oracle's complex step through the same iterations. Both differentiate
    the branch the forward takes, with the same first-wins choices; a
    central difference would straddle the limiter's switches, so there is
    none here."""
    from paper_2403_13287_gb300.adjoint import unrolled_force_gradient
    base = naca0012_cloud(64, 35, seed=4)
    B = hicks_henne_basis(base)
    a = np.random.default_rng(2025).uniform(-2e-3, 2e-3, B.shape[0])
    c = _deformed(base, B, a)
    mach, aoa = 1.2, 0.0
    U0 = oracle.freestream_state(c["n"], mach, aoa)
    s = _solver(c, order=2, inner_iters=3, time_scheme=1, reorder=1, limiter_K=1.0, mach=mach, aoa_deg=aoa)
    (cl, cd), (U0b, xb, yb), info = unrolled_force_gradient(s, _dev(U0), ITERS, cl_bar=0.0, cd_bar=1.0)
    g = B @ yb.cpu().numpy()
    mask = oracle.split_stencils(c)
    ref = np.empty_like(g)
    for k in range(B.shape[0]):
        (_, cdo), (_, dcd) = lskum_jvp.unrolled_forces(c, mask, U0, ITERS, dy=B[k], scheme=1, mach=mach,
                                                       aoa_deg=aoa, limiter=1.0)
        ref[k] = dcd
    assert abs(cd - cdo) <= 1e-10 * abs(cdo)
    assert np.abs(ref).max() > 0
    assert np.all(np.abs(g - ref) <= 1e-8 * np.abs(ref).max()), (g, ref)
