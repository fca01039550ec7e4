"""Pins of the complex-step derivative oracle (oracle/lskum_jvp.py), no GPU.

The derivative oracle restates the residual over complex numbers. It is tied
to the C oracle twice: its real arithmetic reproduces the C oracle's
residual, and its J v agrees with central differences of the C oracle (a
dropped term, a wrong sign or a transposed operand in either breaks one of
the two). The entry-wise VJP is checked against a brute-force transpose of
the full Jacobian on a tiny cloud.
"""
import numpy as np
import pytest

import oracle
from oracle import lskum_jvp
from paper_2403_13287_gb300.cloudgen import naca0012_cloud, smooth_state

GAMMA = 1.4


@pytest.fixture(scope="module")
def cloud():
    c = naca0012_cloud(48, 10, seed=4)
    return c, oracle.split_stencils(c)


def _state(c, amp=0.05, seed=3):
    return smooth_state(c, 0.63, 2.0, amp=amp, seed=seed)


@pytest.mark.parametrize("order", [1, 2])
def test_real_part_is_the_c_oracle_residual(cloud, order):
    c, mask = cloud
    U = _state(c)
    R_c, S = oracle.residual(c, mask, U, order=order, inner=3, want_scale=True)
    R_py = lskum_jvp.residual(c, mask, U, order=order, inner=3)
    # same steps and order; only erf comes from another library (cephes)
    assert np.all(np.abs(R_py - R_c) <= 1e-13 * S + 1e-300)


def _fd(c, mask, U, dU, dx, dy, order, eps):
    def R(s):
        cc = dict(c)
        cc["x"] = c["x"] + s * dx
        cc["y"] = c["y"] + s * dy
        return oracle.residual(cc, mask, U + s * dU, order=order, inner=3)
    return (R(eps) - R(-eps)) / (2 * eps)


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("what", ["U", "xy"])
def test_jvp_matches_central_differences_of_the_c_oracle(cloud, order, what):
    c, mask = cloud
    n = c["n"]
    U = _state(c)
    rng = np.random.default_rng(17)
    dU = np.zeros((4, n))
    dx = np.zeros(n)
    dy = np.zeros(n)
    if what == "U":
        dU = rng.standard_normal((4, n)) * np.abs(U)
    else:
        # displacements of the order of the local spacing
        dx = rng.standard_normal(n) * 0.01
        dy = rng.standard_normal(n) * 0.01
    J = lskum_jvp.jvp(c, mask, U, dU, dx, dy, order=order, inner=3)
    F = _fd(c, mask, U, dU, dx, dy, order, 1e-6)
    F2 = _fd(c, mask, U, dU, dx, dy, order, 2e-6)
    # Richardson: the difference error is O(eps^2); scale it from two steps
    err_fd = np.abs(F2 - F) + 1e-9 * np.max(np.abs(J))
    assert np.max(np.abs(J)) > 0
    assert np.all(np.abs(J - F) <= 10 * err_fd)
    assert np.max(np.abs(J - F)) <= 1e-6 * np.max(np.abs(J))


def test_jvp_is_linear_in_the_direction(cloud):
    c, mask = cloud
    n = c["n"]
    U = _state(c)
    rng = np.random.default_rng(5)
    a = rng.standard_normal((4, n)) * np.abs(U)
    b = rng.standard_normal((4, n)) * np.abs(U)
    Ja = lskum_jvp.jvp(c, mask, U, dU=a)
    Jb = lskum_jvp.jvp(c, mask, U, dU=b)
    Jab = lskum_jvp.jvp(c, mask, U, dU=2.0 * a - 3.0 * b)
    assert np.allclose(Jab, 2.0 * Ja - 3.0 * Jb, rtol=1e-12, atol=1e-12 * np.max(np.abs(Jab)))


def test_uniform_flow_has_no_derivative_along_the_free_stream(cloud):
    """R(U_inf + t U_inf) = 0 for every t (uniform states give dG = 0 on
    every edge), so J U_inf = 0 away from the wall, where the uniform state
    would carry normal momentum."""
    c, mask = cloud
    n = c["n"]
    Uinf = oracle.freestream(0.63, 2.0)
    U = np.repeat(Uinf[:, None], n, axis=1)
    J = lskum_jvp.jvp(c, mask, U, dU=U.copy())
    assert np.all(J == 0.0)


def test_vjp_entries_are_the_transposed_jacobian():
    """Brute force on a tiny cloud: build J column by column, compare J^T r."""
    c = naca0012_cloud(20, 5, seed=9)
    mask = oracle.split_stencils(c)
    n = c["n"]
    U = _state(c, amp=0.01, seed=8)
    rng = np.random.default_rng(2)
    r = rng.standard_normal((4, n))
    cols = []
    for k in range(4):
        for p in range(n):
            d = np.zeros((4, n))
            d[k, p] = 1.0
            cols.append(lskum_jvp.jvp(c, mask, U, dU=d).ravel())
    for name in ("dx", "dy"):
        for p in range(n):
            d = np.zeros(n)
            d[p] = 1.0
            cols.append(lskum_jvp.jvp(c, mask, U, **{name: d}).ravel())
    J = np.stack(cols, axis=1)                    # (4n) x (6n)
    full = J.T @ r.ravel()
    ent = ([("U", k, p) for k in range(4) for p in range(0, n, 7)]
           + [("x", p) for p in range(0, n, 5)] + [("y", p) for p in range(1, n, 5)])
    pos = {"x": 4 * n, "y": 5 * n}
    want = np.array([full[e[1] * n + e[2]] if e[0] == "U" else full[pos[e[0]] + e[1]] for e in ent])
    got = lskum_jvp.vjp_entries(c, mask, U, r, ent)
    assert np.allclose(got, want, rtol=1e-13, atol=1e-13 * np.max(np.abs(full)))


@pytest.mark.parametrize("scheme", [0, 1])
def test_iteration_real_part_is_the_c_oracle_step(cloud, scheme):
    c, mask = cloud
    U0 = _state(c, amp=0.02)
    Upy = lskum_jvp.iterate(c, mask, U0, scheme=scheme, mach=0.63, aoa_deg=2.0)
    Uc, _ = oracle.solve(c, mask, U0.copy(), 1, order=2, inner=3, scheme=scheme, cfl=0.2, mach=0.63,
                         aoa_deg=2.0)
    assert np.max(np.abs(Upy - Uc)) <= 1e-13 * np.max(np.abs(Uc))


def _symmetric_wall_displacement(c, rng, scale):
    """Random displacements whose wall part keeps the contour's mirror
    symmetry: the leading- and trailing-edge points keep their two equally
    near wall neighbours equally near, so the nearest-neighbour distance of
    the time step is differentiable along them (a central difference across
    its kink would average two slopes)."""
    n, W = c["n"], c["W"]
    dx = rng.standard_normal(n) * scale
    dy = rng.standard_normal(n) * scale
    half = W // 2
    lower = np.arange(half + 1, W)
    dx[lower] = dx[W - lower]
    dy[lower] = -dy[W - lower]
    dy[0] = dy[half] = 0.0
    return dx, dy


def test_unrolled_force_derivative_matches_central_differences_of_the_c_oracle():
    """d Cl / d (point displacement) after 3 RK4 iterations: complex step
    against central differences of orc_solve + orc_forces (an isotropic
    64 x 35 cloud, on which the unlimited second-order scheme is stable)."""
    c = naca0012_cloud(64, 35, seed=4)
    mask = oracle.split_stencils(c)
    n = c["n"]
    U0 = _state(c, amp=0.02)
    rng = np.random.default_rng(23)
    dx, dy = _symmetric_wall_displacement(c, rng, 0.01)
    (cl, cd), (dcl, dcd) = lskum_jvp.unrolled_forces(c, mask, U0, 3, dx=dx, dy=dy, scheme=1, mach=0.63,
                                                     aoa_deg=2.0)

    def forces(eps):
        cc = dict(c)
        cc["x"] = c["x"] + eps * dx
        cc["y"] = c["y"] + eps * dy
        U, _ = oracle.solve(cc, mask, U0.copy(), 3, order=2, inner=3, scheme=1, cfl=0.2, mach=0.63, aoa_deg=2.0)
        return oracle.forces(cc, U, 0.63, 2.0)[:2]

    cl_c, cd_c = forces(0.0)
    assert abs(cl - cl_c) <= 1e-13 * abs(cl_c) and abs(cd - cd_c) <= 1e-13 * abs(cd_c)
    fp, fm = forces(1e-6), forces(-1e-6)
    fd = [(a - b) / 2e-6 for a, b in zip(fp, fm)]
    assert abs(dcl - fd[0]) <= 1e-6 * abs(dcl) + 1e-9
    assert abs(dcd - fd[1]) <= 1e-6 * abs(dcd) + 1e-9
    # a rigid translation of every point changes nothing
    (_, _), (tcl, tcd) = lskum_jvp.unrolled_forces(c, mask, U0, 3, dx=np.ones(n), dy=np.ones(n), scheme=1,
                                                   mach=0.63, aoa_deg=2.0)
    assert tcl == 0.0 and tcd == 0.0


# ---------------------------------------------------------------------------
# the limiter (Venkatakrishnan, K > 0) in the derivative oracle
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def limited():
    c = naca0012_cloud(64, 16, seed=3)
    return c, oracle.split_stencils(c), smooth_state(c, 0.85, 1.0, amp=0.05, seed=2)


@pytest.mark.parametrize("K", [1.0, 0.3])
def test_limited_real_part_is_the_c_oracle_residual(limited, K):
    c, mask, U = limited
    R_c, S = oracle.residual(c, mask, U, order=2, inner=3, limiter=K, want_scale=True)
    R_py = lskum_jvp.residual(c, mask, U, order=2, inner=3, limiter=K)
    assert np.all(np.abs(R_py - R_c) <= 1e-13 * S + 1e-300)
    # the limiter acts on this state
    R_free = lskum_jvp.residual(c, mask, U, order=2, inner=3)
    assert np.max(np.abs(R_free - R_c)) > 1e-2 * np.max(S)


@pytest.mark.parametrize("what", ["U", "xy"])
def test_limited_jvp_matches_central_differences_of_the_c_oracle(limited, what):
    """The limiter is piecewise smooth: its choices (nearest neighbour,
    stencil extremes, the smallest shift factor) switch at ties, where a
    central difference straddles two branches. Far-field points all carry
    the free stream, so their q are tied stencil extremes; the nose and tail
    points of the mirror-symmetric contour have two nearest neighbours at
    equal distances. The directions here leave the far-field states and the
    wall points fixed, and the step (1e-5) stays inside one branch."""
    c, mask, U = limited
    n = c["n"]
    rng = np.random.default_rng(23)
    far = c["flags"] == 2
    dU = np.zeros((4, n))
    dx = np.zeros(n)
    dy = np.zeros(n)
    if what == "U":
        dU = rng.standard_normal((4, n)) * np.abs(U) * 1e-2
        dU[:, far] = 0.0
    else:
        dx = rng.standard_normal(n) * 1e-3
        dy = rng.standard_normal(n) * 1e-3
        wall = c["flags"] == 1
        dx[wall] = 0.0
        dy[wall] = 0.0
    J = lskum_jvp.jvp(c, mask, U, dU, dx, dy, order=2, inner=3, limiter=1.0)

    def R(s):
        cc = dict(c)
        cc["x"] = c["x"] + s * dx
        cc["y"] = c["y"] + s * dy
        return oracle.residual(cc, mask, U + s * dU, order=2, inner=3, limiter=1.0)
    F = (R(1e-5) - R(-1e-5)) / 2e-5
    assert np.max(np.abs(J)) > 0
    assert np.max(np.abs(J - F)) <= 1e-7 * np.max(np.abs(J))
