"""Batched solves (lskum_create_batch) and the launch-shape autotuner (needs a GPU).

A batch runs every kernel once over the disjoint union of its cases, so each
point's arithmetic is the same as in a context of its own case: states must
agree bitwise with single-case contexts, and the per-case residues agree to
rounding of their summation grouping. The FP64 batch residual is also checked
against the oracle per case.
"""
import numpy as np
import pytest

import oracle
from paper_2403_13287_gb300.cloudgen import naca0012_cloud, smooth_state

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.fixture(scope="module")
def clouds():
    return naca0012_cloud(130, 24, seed=11), naca0012_cloud(96, 20, seed=3)


def _cases(clouds):
    a, b = clouds
    return [(a, 0.85, 1.0), (b, 0.63, 2.0), (a, 1.2, 0.0)]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("scheme", [0, 1])
def test_batch_matches_single_contexts(clouds, precision, scheme):
    from paper_2403_13287_gb300.lskum import Solver
    cases = _cases(clouds)
    kw = dict(order=2, inner_iters=3, time_scheme=scheme, limiter_K=1.0, precision=precision, reorder=1)
    B = Solver.batch(cases, **kw)
    assert B.ncases == 3
    U0 = [smooth_state(c, m, a, amp=0.05, seed=20 + k) for k, (c, m, a) in enumerate(cases)]
    B.set_state(np.concatenate(U0, axis=1))
    hb = B.step(7)
    Ub = B.get_state()
    for k, (c, m, a) in enumerate(cases):
        s = Solver(c, mach=m, aoa_deg=a, **kw)
        s.set_state(U0[k])
        h = s.step(7)
        first, count, _, _ = B.case_range(k)
        assert np.array_equal(Ub[:, first:first + count], s.get_state())
        # residue: sums grouped by warps of 32 points, which differ between the
        # two numberings; the mixed form sums R_rho^2 within a warp in FP32
        assert np.allclose(hb[:, k], h, rtol=1e-12 if precision == 0 else 1e-6, atol=0)
        cl, cd, cp = s.forces()
        clb, cdb, cpb = B.case_forces(k)
        assert np.array_equal(cp, cpb)
        assert abs(cl - clb) <= 1e-14 * max(abs(cl), abs(cd)) and abs(cd - cdb) <= 1e-14 * max(abs(cl), abs(cd))


def test_batch_starts_from_each_free_stream_and_residual_matches_oracle(clouds):
    from paper_2403_13287_gb300.lskum import Solver
    cases = _cases(clouds)
    B = Solver.batch(cases, order=2, inner_iters=3, precision=0, reorder=1)
    U = B.get_state()
    Us = []
    for k, (c, m, a) in enumerate(cases):
        first, count, _, _ = B.case_range(k)
        assert np.array_equal(U[:, first:first + count], np.repeat(oracle.freestream(m, a)[:, None], count, axis=1))
        Us.append(smooth_state(c, m, a, amp=0.05, seed=40 + k))
    R = B.residual(_dev(np.concatenate(Us, axis=1))).cpu().numpy()
    for k, (c, m, a) in enumerate(cases):
        first, count, _, _ = B.case_range(k)
        mask = oracle.split_stencils(c)
        Ro, S = oracle.residual(c, mask, Us[k], order=2, inner=3, want_scale=True)
        assert np.all(np.abs(R[:, first:first + count] - Ro) <= 1e-12 * S + 1e-300)


def test_autotune_keeps_the_state_and_picks_the_fastest(clouds):
    from paper_2403_13287_gb300.lskum import Solver
    cases = _cases(clouds)
    kw = dict(order=2, inner_iters=3, time_scheme=1, limiter_K=1.0, precision=1, reorder=1)
    U0 = np.concatenate([smooth_state(c, m, a, amp=0.05, seed=60 + k) for k, (c, m, a) in enumerate(cases)], axis=1)
    B = Solver.batch(cases, **kw)
    B.set_state(U0)
    t = B.autotune(reps=3)
    assert np.array_equal(B.get_state(), U0)           # tuning runs in residual mode and scratch buffers
    assert t["flux_ms"] > 0 and t["qgrad_ms"] > 0
    assert t["flux_ms"] <= t["flux_ms_default"] and t["qgrad_ms"] <= t["qgrad_ms_default"]
    assert t["flux_threads"] % 32 == 0 and t["qgrad_threads"] % 32 == 0


def test_every_launch_shape_gives_the_same_solution(clouds):
    """Shapes change only the compiler's register budget, and with it which
    FP32 multiply-adds are contracted: the states agree to FP32 rounding (the
    FP64 path has one shape and is bitwise reproducible)."""
    from paper_2403_13287_gb300.lskum import Solver
    c = clouds[0]
    U0 = smooth_state(c, 0.85, 1.0, amp=0.05, seed=70)
    ref = None
    for v in range(24):                                 # 24 flux shapes (17-21 staged), 6 q-derivative shapes
        s = Solver(c, order=2, inner_iters=3, time_scheme=1, mach=0.85, aoa_deg=1.0, limiter_K=1.0, precision=1)
        s.set_tuning(v, v % 6)
        s.set_state(U0)
        h = s.step(3)
        out = (h, s.get_state())
        if ref is None:
            ref = out
        assert np.allclose(out[0], ref[0], rtol=1e-5, atol=0)
        assert np.all(np.abs(out[1] - ref[1]) <= 1e-5 * np.abs(ref[1]).max(axis=1, keepdims=True))


def test_batch_arguments(clouds):
    from paper_2403_13287_gb300.lskum import LskumError, LSKUM_ERR_ARG, Solver
    a, _ = clouds
    tiny = naca0012_cloud(8, 2, seed=1)            # fewer than 32 points
    if tiny["n"] >= 32:
        pytest.skip("generator gave a larger cloud")
    with pytest.raises(LskumError) as e:
        Solver.batch([(a, 0.8, 0.0), (tiny, 0.8, 0.0)])
    assert e.value.status == LSKUM_ERR_ARG
    with pytest.raises(LskumError) as e:
        Solver.batch([(a, 0.0, 0.0)])
    assert e.value.status == LSKUM_ERR_ARG
    s1 = Solver(a, precision=1)
    with pytest.raises(LskumError) as e:
        s1.set_tuning(1000, 0)
    assert e.value.status == LSKUM_ERR_ARG
    f64 = Solver(a, precision=0)
    with pytest.raises(LskumError) as e:
        f64.autotune()
    assert e.value.status == LSKUM_ERR_ARG
    B = Solver.batch([(a, 0.8, 0.0), (a, 0.7, 1.0)])
    with pytest.raises(LskumError):
        B.forces()
    with pytest.raises(LskumError):
        B.case_forces(2)
