"""Staged tiles of the mixed flux kernel (launch shapes 17-21; needs a GPU).

A staged CTA copies the q and grad q of its 64 points and of up to 160
neighbours outside the tile into shared memory, then runs the neighbour
loop on those rows; neighbours beyond the cap are read from global memory.
The arithmetic is the mixed form's, so the residual must meet the mixed
form's bar against the FP64 oracle (3e-5 of the summand scale S, see
test_gpu_mixed.py): in Morton order (every neighbour staged), in the
shuffled input order (most tiles overflow the cap, so both paths run), in
the kinetic boundary mode (images read from global memory) and in a batch
(bitwise equal to the single-case contexts with the same shape).
"""
import numpy as np
import pytest

import oracle
from paper_2403_13287_gb300.cloudgen import naca0012_cloud, smooth_state

pytestmark = pytest.mark.gpu

FIRST_STAGED = 17
LAST_STAGED = 21


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def cloud():
    return naca0012_cloud(130, 24, seed=11, shuffle=True)


@pytest.mark.parametrize("variant", range(FIRST_STAGED, LAST_STAGED + 1))
@pytest.mark.parametrize("reorder", [0, 1])
@pytest.mark.parametrize("order,limiter", [(1, 0.0), (2, 1.0)])
def test_staged_residual_matches_oracle(cloud, variant, reorder, order, limiter):
    from paper_2403_13287_gb300.lskum import Solver
    U = smooth_state(cloud, 0.85, 1.0, amp=0.05, seed=3)
    s = Solver(cloud, order=order, inner_iters=3, mach=0.85, aoa_deg=1.0, limiter_K=limiter, precision=1,
               reorder=reorder)
    s.set_tuning(variant, 0)
    R = s.residual(_dev(U)).cpu().numpy()
    s.close()
    m = oracle.split_stencils(cloud)
    Ro, S = oracle.residual(cloud, m, U, order=order, inner=3, limiter=limiter, want_scale=True)
    assert np.all(np.abs(R - Ro) <= 3e-5 * S + 1e-300)


def test_staged_kinetic_boundary_residual_matches_oracle(cloud):
    from paper_2403_13287_gb300.lskum import Solver
    U = smooth_state(cloud, 0.85, 1.0, amp=0.05, seed=4)
    s = Solver(cloud, order=2, inner_iters=3, mach=0.85, aoa_deg=1.0, precision=1, reorder=1, boundary=1)
    s.set_tuning(FIRST_STAGED, 0)
    R = s.residual(_dev(U)).cpu().numpy()
    s.close()
    m = oracle.split_stencils(cloud)
    Ro, S = oracle.residual(cloud, m, U, order=2, inner=3, want_scale=True, boundary=1, mach=0.85, aoa_deg=1.0)
    assert np.all(np.abs(R - Ro) <= 3e-5 * S + 1e-300)


def test_staged_trajectory_matches_the_streamed_kernel(cloud):
    """Five RK4 iterations with a staged shape and with the streamed shape of
    the same register budget (64 threads, 14 blocks, pipelined) agree to
    FP32 rounding."""
    from paper_2403_13287_gb300.lskum import Solver
    U0 = smooth_state(cloud, 1.2, 0.0, amp=0.05, seed=5)
    out = []
    for v in (7, FIRST_STAGED):
        s = Solver(cloud, order=2, inner_iters=3, time_scheme=1, mach=1.2, aoa_deg=0.0, limiter_K=1.0,
                   precision=1, reorder=1)
        s.set_tuning(v, 0)
        s.set_state(U0)
        h = s.step(5)
        out.append((h, s.get_state()))
        s.close()
    assert np.allclose(out[0][0], out[1][0], rtol=1e-5, atol=0)
    assert np.all(np.abs(out[0][1] - out[1][1]) <= 1e-5 * np.abs(out[0][1]).max(axis=1, keepdims=True))


def test_staged_batch_matches_single_contexts():
    from paper_2403_13287_gb300.lskum import Solver
    a, b = naca0012_cloud(130, 24, seed=11), naca0012_cloud(96, 20, seed=3)
    cases = [(a, 0.85, 1.0), (b, 0.63, 2.0)]
    kw = dict(order=2, inner_iters=3, time_scheme=1, limiter_K=1.0, precision=1, reorder=1)
    U0 = [smooth_state(c, m, al, amp=0.05, seed=30 + k) for k, (c, m, al) in enumerate(cases)]
    B = Solver.batch(cases, **kw)
    B.set_tuning(FIRST_STAGED, 0)
    B.set_state(np.concatenate(U0, axis=1))
    B.step(4)
    Ub = B.get_state()
    for k, (c, m, al) in enumerate(cases):
        s = Solver(c, mach=m, aoa_deg=al, **kw)
        s.set_tuning(FIRST_STAGED, 0)
        s.set_state(U0[k])
        s.step(4)
        first, count, _, _ = B.case_range(k)
        assert np.array_equal(Ub[:, first:first + count], s.get_state())
        s.close()
    B.close()
