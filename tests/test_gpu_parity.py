"""CUDA path vs the FP64 CPU oracle, through the C ABI (needs a GPU).

Tolerances (FP64 path):
- sub-stencil masks and renumbering: bit-exact;
- residual: |R_gpu - R_oracle| <= 1e-12 * S per point and component, where S
  is the oracle's magnitude of the summed terms before cancellation
  (sum |LS weight| (|G(q~_i)| + |G(q~_0)|)); rounding of either side is a
  few ulp of S times the stencil's condition number;
- q-derivatives: 1e-12 of the summand scale of the least-squares sum;
- time step: 1e-14 relative;
- trajectories: 1e-10 relative in U after tens of iterations, the same for
  Cl and Cd.
"""
import numpy as np
import pytest

import oracle
from paper_2403_13287_gb300.cloudgen import naca0012_cloud

pytestmark = pytest.mark.gpu

GAMMA = 1.4


def _torch():
    import torch
    return torch


def _solver(cloud, **kw):
    from paper_2403_13287_gb300.lskum import Solver
    return Solver(cloud, **kw)


def _perturbed_state(cloud, mach, aoa, amp=0.05, seed=0):
    """Free stream times a smooth seeded perturbation (physical everywhere)."""
    rng = np.random.default_rng(seed)
    x, y = cloud["x"], cloud["y"]
    k = rng.uniform(1.0, 3.0, 4)
    ph = rng.uniform(0, 2 * np.pi, 4)
    a = np.radians(aoa)
    rho = 1.0 + amp * np.sin(k[0] * x + ph[0]) * np.cos(k[1] * y + ph[1])
    u = mach * np.cos(a) + amp * np.cos(k[2] * y + ph[2])
    v = mach * np.sin(a) + amp * np.sin(k[3] * x + ph[3])
    p = 1.0 / GAMMA * (1.0 + amp * np.cos(k[1] * x - k[0] * y))
    far = cloud["flags"] == 2
    U = np.stack([rho, rho * u, rho * v, p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v)])
    U[:, far] = oracle.freestream(mach, aoa)[:, None]
    wall = cloud["flags"] == 1
    mn = U[1, wall] * cloud["nx"][wall] + U[2, wall] * cloud["ny"][wall]
    U[1, wall] -= mn * cloud["nx"][wall]
    U[2, wall] -= mn * cloud["ny"][wall]
    return np.ascontiguousarray(U)


def _dev(a):
    torch = _torch()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def small():
    return naca0012_cloud(130, 24, seed=11)      # 3250 points: not a multiple of the block


@pytest.fixture(scope="module")
def ten_k():
    return naca0012_cloud(320, 30)                # the ~10k first-order workload


@pytest.mark.parametrize("reorder", [0, 1, 2])
def test_stencil_masks_bit_exact(small, reorder):
    s = _solver(small, reorder=reorder)
    assert np.array_equal(s.stencil_masks(), oracle.split_stencils(small))
    perm = s.permutation()
    assert np.array_equal(np.sort(perm), np.arange(small["n"]))
    if reorder == 0:
        assert np.array_equal(perm, np.arange(small["n"]))


def test_stencil_masks_bit_exact_10k_shuffled():
    c = naca0012_cloud(320, 30, seed=5, shuffle=True)
    s = _solver(c, reorder=1)
    assert np.array_equal(s.stencil_masks(), oracle.split_stencils(c))


def _grad_scale(cloud, q, gx, gy):
    off, idx = cloud["nbr_offsets"], cloud["nbr_idx"]
    n = cloud["n"]
    rows = np.repeat(np.arange(n), np.diff(off))
    dx = cloud["x"][idx] - cloud["x"][rows]
    dy = cloud["y"][idx] - cloud["y"][rows]
    d = np.hypot(dx, dy)
    S = np.zeros_like(q)
    for k in range(4):
        term = (np.abs(q[k, idx] - q[k, rows])
                + 0.5 * (np.abs(dx) * (np.abs(gx[k, idx]) + np.abs(gx[k, rows]))
                         + np.abs(dy) * (np.abs(gy[k, idx]) + np.abs(gy[k, rows])))) / d
        S[k] = np.bincount(rows, weights=term, minlength=n) / np.diff(off)
    return S


# inner 0 with the limiter: the first pass limits; 1: the one inner pass
# reads the first-order solve as its previous iterate too; 2 and 3: the
# iterates end in either buffer
@pytest.mark.parametrize("inner,limiter", [(0, 0.0), (1, 0.0), (2, 0.0), (3, 0.0),
                                           (0, 1.0), (1, 1.0), (2, 1.0), (3, 1.0)])
def test_q_derivatives_match_oracle(small, inner, limiter):
    U = _perturbed_state(small, 0.63, 2.0, seed=1)
    s = _solver(small, order=2, inner_iters=inner, limiter_K=limiter)
    qx, qy = s.q_derivatives(_dev(U))
    qx, qy = qx.cpu().numpy(), qy.cpu().numpy()
    q = oracle.q_variables(U)
    ox, oy = oracle.q_derivatives(small, q, inner=inner)
    S = _grad_scale(small, q, ox, oy)
    if limiter:
        ox, oy = oracle.limit_gradients(small, q, ox, oy, limiter)
        # the limiter really acts on this state
        assert np.mean(np.abs(ox) < np.abs(oracle.q_derivatives(small, q, inner=inner)[0])) > 0.05
    assert np.all(np.abs(qx - ox) <= 1e-12 * S)
    assert np.all(np.abs(qy - oy) <= 1e-12 * S)


@pytest.mark.parametrize("limiter", [1.0, 0.05])
def test_limited_q_derivatives_on_a_jump_and_a_constant_region(small, limiter):
    """A state with a jump (density x3, energy x5 upstream of x = 0.3) and
    the exact free stream elsewhere. Near the jump the gradients are large
    and the limiter acts; away from it every q_i - q_0 is exactly zero, so
    the largest shift d_m is 0 and the FP32 screen of d_m keeps every edge
    (its absolute margin). Both must match the oracle, the constant region
    exactly."""
    c = small
    U = oracle.freestream_state(c["n"], 0.85, 1.0).copy()
    jump = c["x"] < 0.3
    U[:3, jump] *= 3.0
    U[3, jump] *= 5.0
    U = np.ascontiguousarray(U)
    s = _solver(c, order=2, inner_iters=3, limiter_K=limiter)
    qx, qy = s.q_derivatives(_dev(U))
    qx, qy = qx.cpu().numpy(), qy.cpu().numpy()
    q = oracle.q_variables(U)
    ox, oy = oracle.q_derivatives(c, q, inner=3)
    S = _grad_scale(c, q, ox, oy)
    lx, ly = oracle.limit_gradients(c, q, ox, oy, limiter)
    assert np.mean(np.abs(lx) < np.abs(ox)) > 0.001            # the limiter acts at the jump
    assert np.any(np.all(S == 0.0, axis=0))                    # and some stencils see no variation
    assert np.all(np.abs(qx - lx) <= 1e-12 * S)
    assert np.all(np.abs(qy - ly) <= 1e-12 * S)


@pytest.mark.parametrize("order,limiter", [(1, 0.0), (2, 0.0), (2, 1.0)])
@pytest.mark.parametrize("reorder", [0, 1, 2])
def test_residual_matches_oracle(small, order, limiter, reorder):
    U = _perturbed_state(small, 0.85, 1.0, seed=2)
    s = _solver(small, order=order, inner_iters=3, reorder=reorder, limiter_K=limiter)
    R = s.residual(_dev(U)).cpu().numpy()
    m = oracle.split_stencils(small)
    Ro, S = oracle.residual(small, m, U, order=order, inner=3, want_scale=True, limiter=limiter)
    assert np.all(np.abs(R - Ro) <= 1e-12 * S)
    assert np.all(R[:, small["flags"] == 2] == 0.0)


def test_residual_of_freestream_is_exactly_zero(ten_k):
    s = _solver(ten_k, order=2, mach=1.2, aoa_deg=0.0)
    R = s.residual().cpu().numpy()
    assert np.all(R == 0.0)


def test_timestep_matches_oracle(small):
    U = _perturbed_state(small, 0.63, 2.0, seed=3)
    s = _solver(small, cfl=0.3)
    dt = s.timestep(_dev(U)).cpu().numpy()
    dto = oracle.timestep(small, U, 0.3)
    assert np.allclose(dt, dto, rtol=1e-14, atol=0)


def test_state_roundtrip_and_renumbering(small):
    U = _perturbed_state(small, 0.63, 2.0, seed=4)
    for reorder in (0, 1):
        s = _solver(small, reorder=reorder)
        s.set_state(U)
        assert np.array_equal(s.get_state(), U)
        t = _dev(U)
        s.set_state(t)
        out = _torch().empty_like(t)
        s.get_state(out)
        assert np.array_equal(out.cpu().numpy(), U)


@pytest.mark.parametrize("order,scheme,iters,mach,aoa,limiter,cloud_name", [
    (1, 0, 100, 0.63, 2.0, 0.0, "ten_k"),   # first-order forward Euler (the 10k workload)
    (2, 1, 30, 0.63, 2.0, 0.0, "ten_k"),    # the paper's scheme: second order, 3 inner its, no limiter
    (2, 1, 30, 0.85, 1.0, 1.0, "small"),    # second order, RK4, transonic, limited
    (2, 0, 40, 1.2, 0.0, 1.0, "small"),     # second order forward Euler, supersonic, limited
])
def test_trajectory_matches_oracle(request, order, scheme, iters, mach, aoa, limiter, cloud_name):
    cloud = request.getfixturevalue(cloud_name)
    m = oracle.split_stencils(cloud)
    U0 = oracle.freestream_state(cloud["n"], mach, aoa)
    Uo, ho = oracle.solve(cloud, m, U0, iters, order=order, inner=3, scheme=scheme, cfl=0.2,
                          mach=mach, aoa_deg=aoa, limiter=limiter)
    s = _solver(cloud, order=order, inner_iters=3, time_scheme=scheme, cfl=0.2, mach=mach,
                aoa_deg=aoa, limiter_K=limiter)
    h = s.step(iters)
    U = s.get_state()
    assert np.max(np.abs(U - Uo) / (np.abs(Uo) + 1e-3)) < 1e-10
    assert np.allclose(h, ho, rtol=1e-9, atol=1e-14)
    cl, cd, cp = s.forces()
    clo, cdo, cpo = oracle.forces(cloud, Uo, mach, aoa)
    assert abs(cl - clo) <= 1e-10 * max(abs(clo), abs(cdo))
    assert abs(cd - cdo) <= 1e-10 * max(abs(clo), abs(cdo))
    assert np.allclose(cp, cpo, rtol=0, atol=1e-10)


def test_reordering_does_not_change_the_solution(small):
    states = []
    for reorder in (0, 1, 2):
        s = _solver(small, order=2, time_scheme=1, mach=0.85, aoa_deg=1.0, reorder=reorder, limiter_K=1.0)
        s.step(10)
        states.append(s.get_state())
    assert np.array_equal(states[0], states[1]) and np.array_equal(states[0], states[2])


def _bandwidth(cloud, perm):
    """Largest |internal(p) - internal(i)| over the stencil edges."""
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    src = np.repeat(np.arange(cloud["n"]), np.diff(cloud["nbr_offsets"]))
    return int(np.max(np.abs(inv[src] - inv[cloud["nbr_idx"]])))


def test_rcm_numbering_is_a_permutation_that_narrows_the_stencil_band():
    c = naca0012_cloud(130, 24, seed=11, shuffle=True)
    s0 = _solver(c, reorder=0)
    s2 = _solver(c, reorder=2)
    p0, p2 = s0.permutation(), s2.permutation()
    assert np.array_equal(p0, np.arange(c["n"]))
    assert np.array_equal(np.sort(p2), np.arange(c["n"]))
    # shuffled input: the band of the stencil graph collapses under RCM
    assert _bandwidth(c, p2) * 10 < _bandwidth(c, p0)
    assert _bandwidth(c, p2) <= 2 * 130 + 10        # about one grid ring of the O-grid


def test_resume_continues_bitwise(small):
    """Checkpoint/resume: 6 iterations, state out, a new context, state in,
    4 more iterations equal 10 iterations in one run."""
    kw = dict(order=2, time_scheme=1, mach=0.85, aoa_deg=1.0, limiter_K=1.0, reorder=1)
    a = _solver(small, **kw)
    a.step(10)
    b = _solver(small, **kw)
    b.step(6)
    U6 = b.get_state()
    c = _solver(small, **kw)
    c.set_state(U6)
    c.step(4)
    assert np.array_equal(a.get_state(), c.get_state())


def test_runs_are_bitwise_deterministic(small):
    runs = []
    for _ in range(2):
        s = _solver(small, order=2, time_scheme=1, mach=0.85, aoa_deg=1.0, reorder=1, limiter_K=1.0)
        h = s.step(8)
        runs.append((s.get_state(), h))
    assert np.array_equal(runs[0][0], runs[1][0])
    assert np.array_equal(runs[0][1], runs[1][1])


def test_tiny_cartesian_stencil():
    """Nine points: one interior point with the 3x3 block around it, the ring
    held as far field (the hand-checked stencil of the oracle pins)."""
    h = 0.01
    offs = [(-1, -1), (-1, 0), (-1, 1), (0, -1), (0, 1), (1, -1), (1, 0), (1, 1)]
    pts = [(0.0, 0.0)] + [(h * a, h * b) for a, b in offs]
    rows = [list(range(1, 9))]
    for k in range(1, 9):
        a, b = offs[k - 1]
        rows.append(sorted([0] + [j + 1 for j, (c, d) in enumerate(offs)
                                  if (c, d) != (a, b) and abs(c - a) <= 1 and abs(d - b) <= 1]))
    off = np.zeros(10, np.int32)
    off[1:] = np.cumsum([len(r) for r in rows])
    cloud = {"n": 9, "x": np.array([p[0] for p in pts]), "y": np.array([p[1] for p in pts]),
             "nx": np.zeros(9), "ny": np.ones(9), "flags": np.array([0] + [2] * 8, np.int32),
             "nbr_offsets": off, "nbr_idx": np.array([i for r in rows for i in r], np.int32),
             "wall_order": np.zeros(0, np.int32)}
    U = _perturbed_state(cloud, 0.5, 10.0, amp=0.2, seed=9)
    U[:, 1:] = U[:, 1:] * (1 + 0.01 * np.arange(8))[None, :]
    for order in (1, 2):
        s = _solver(cloud, order=order, mach=0.5, aoa_deg=10.0)
        R = s.residual(_dev(U)).cpu().numpy()
        Ro, S = oracle.residual(cloud, oracle.split_stencils(cloud), U, order=order, inner=3,
                                want_scale=True)
        assert np.all(np.abs(R - Ro) <= 1e-12 * S)
        with pytest.raises(Exception):
            s.forces()


def _cloud_with(cloud, **changes):
    c = dict(cloud)
    c.update(changes)
    return c


def test_connectivity_and_argument_errors(small):
    from paper_2403_13287_gb300.lskum import LskumError, LSKUM_ERR_CONNECTIVITY, LSKUM_ERR_ARG
    idx = small["nbr_idx"].copy()
    idx[0] = 0                                              # self loop at point 0
    with pytest.raises(LskumError) as e:
        _solver(_cloud_with(small, nbr_idx=idx))
    assert e.value.status == LSKUM_ERR_CONNECTIVITY
    idx = small["nbr_idx"].copy()
    idx[1] = idx[0]                                         # duplicate
    with pytest.raises(LskumError) as e:
        _solver(_cloud_with(small, nbr_idx=idx))
    assert e.value.status == LSKUM_ERR_CONNECTIVITY
    idx = small["nbr_idx"].copy()
    idx[5] = small["n"]                                     # out of range
    with pytest.raises(LskumError) as e:
        _solver(_cloud_with(small, nbr_idx=idx))
    assert e.value.status == LSKUM_ERR_CONNECTIVITY
    nx = small["nx"].copy()
    nx[3] *= 2.0                                            # not a unit normal
    with pytest.raises(LskumError) as e:
        _solver(_cloud_with(small, nx=nx))
    assert e.value.status == LSKUM_ERR_ARG
    with pytest.raises(LskumError) as e:
        _solver(small, order=3)
    assert e.value.status == LSKUM_ERR_ARG


def test_degenerate_stencil_is_reported(small):
    from paper_2403_13287_gb300.lskum import LskumError, LSKUM_ERR_DEGENERATE_STENCIL
    # keep only the first two neighbours of interior point p: its x+/x-/y+/y-
    # sub-stencils cannot all have two points
    p = int(np.where(small["flags"] == 0)[0][40])
    off, idx = small["nbr_offsets"], small["nbr_idx"]
    rows = [list(idx[off[i]:off[i + 1]]) for i in range(small["n"])]
    rows[p] = rows[p][:2]
    new_off = np.zeros(small["n"] + 1, np.int32)
    new_off[1:] = np.cumsum([len(r) for r in rows])
    c = _cloud_with(small, nbr_offsets=new_off, nbr_idx=np.array([i for r in rows for i in r], np.int32))
    with pytest.raises(LskumError) as e:
        _solver(c)
    assert e.value.status == LSKUM_ERR_DEGENERATE_STENCIL
    assert ("point %d" % p) in str(e.value)


def test_nonphysical_state_is_rejected_and_step_rolls_back(small):
    from paper_2403_13287_gb300.lskum import LskumError, LSKUM_ERR_NONPHYSICAL
    s = _solver(small, order=2, time_scheme=0, cfl=50.0, mach=0.85, aoa_deg=1.0)
    U = _perturbed_state(small, 0.85, 1.0, amp=0.2, seed=5)
    s.set_state(U)
    with pytest.raises(LskumError) as e:
        s.step(200)
    assert e.value.status == LSKUM_ERR_NONPHYSICAL
    assert np.array_equal(s.get_state(), U)
    bad = U.copy()
    bad[3, 7] = -1.0                                        # negative energy -> p < 0
    with pytest.raises(LskumError) as e:
        s.set_state(bad)
    assert e.value.status == LSKUM_ERR_NONPHYSICAL


def test_launch_count_is_reported(small):
    s = _solver(small, order=2, inner_iters=3, time_scheme=1)
    before = s.launch_count()
    s.step(2)
    # per RK4 stage: 1 first-order + 3 inner gradient passes + 1 fused flux;
    # per iteration one residue reduction (two kernels)
    assert s.launch_count() - before == 2 * (4 * 5 + 2)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("scheme", [0, 1])
def test_graph_replay_matches_direct_launches(small, scheme, precision):
    """lskum_step replays a captured iteration as a CUDA graph; with kernel
    timing on it launches every kernel directly. Both give the same bits,
    also across calls with odd iteration counts (forward Euler captures two
    iterations, so odd counts end on the other q buffer)."""
    kw = dict(order=2, inner_iters=3, time_scheme=scheme, mach=0.85, aoa_deg=1.0, limiter_K=1.0,
              precision=precision)
    U0 = _perturbed_state(small, 0.85, 1.0, seed=3)
    runs = []
    for direct in (False, True):
        s = _solver(small, **kw)
        s.set_state(U0)
        if direct:
            s.profile(True)
        hist = [s.step(k) for k in (3, 1, 4, 2)]
        runs.append((np.concatenate(hist), s.get_state(), s.launch_count()))
    (h_g, U_g, n_g), (h_d, U_d, n_d) = runs
    assert np.array_equal(h_g, h_d)
    assert np.array_equal(U_g, U_d)
    assert n_g == n_d
    assert np.all(np.isfinite(h_g)) and np.all(h_g > 0)
