"""Pins of the CPU oracle to facts outside itself (no GPU).

Each check ties one oracle routine to something the paper or the mathematics
fixes independently of the oracle's own formula: closed forms, invariants,
brute-force quadrature, hand-worked examples and convergence orders.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2403_13287_gb300.cloudgen import naca0012_cloud

GAMMA = 1.4
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_prim(rng, m):
    rho = rng.uniform(0.3, 3.0, m)
    u1 = rng.uniform(-2.0, 2.0, m)
    u2 = rng.uniform(-2.0, 2.0, m)
    p = rng.uniform(0.2, 3.0, m)
    return rho, u1, u2, p


def _U(rho, u1, u2, p):
    E = p / (GAMMA - 1) + 0.5 * rho * (u1 * u1 + u2 * u2)
    return np.stack([rho, rho * u1, rho * u2, E])


def _cloud(x, y, nx, ny, flags, rows):
    """A hand-built cloud; rows[p] is the neighbour list of point p."""
    off = np.zeros(len(x) + 1, dtype=np.int32)
    off[1:] = np.cumsum([len(r) for r in rows])
    idx = np.array([i for r in rows for i in r], dtype=np.int32)
    return {"n": len(x), "x": np.asarray(x, float), "y": np.asarray(y, float),
            "nx": np.asarray(nx, float), "ny": np.asarray(ny, float),
            "flags": np.asarray(flags, np.int32), "nbr_offsets": off, "nbr_idx": idx,
            "wall_order": np.zeros(0, np.int32)}


# --------------------------------------------------------------------------
# q-variables (E13)
# --------------------------------------------------------------------------

def test_q_roundtrip():
    rng = np.random.default_rng(1)
    U = _U(*_rand_prim(rng, 2000))
    q = oracle.q_variables(U)
    U2 = oracle.U_from_q(q)
    assert np.max(np.abs(U2 - U) / np.abs(U).max(axis=0)) < 1e-14


def test_q_are_entropy_variables():
    """E13's q is the gradient of the entropy function eta = -rho s/(gamma-1),
    s = ln(p / rho^gamma), up to a constant shift of q1:
    q2..q4 = d eta/dU2..4 and q1 - d eta/dU1 = -(gamma + ln 2)/(gamma - 1)."""
    rng = np.random.default_rng(2)
    U = _U(*_rand_prim(rng, 50))
    q = oracle.q_variables(U)

    def eta(U):
        rho = U[0]
        p = (GAMMA - 1) * (U[3] - 0.5 * (U[1] ** 2 + U[2] ** 2) / rho)
        return -rho * (np.log(p) - GAMMA * np.log(rho)) / (GAMMA - 1)

    h = 1e-6
    grad = np.empty_like(U)
    for k in range(4):
        e = np.zeros((4, 1)); e[k] = h
        grad[k] = (eta(U + e) - eta(U - e)) / (2 * h)
    assert np.allclose(q[1:], grad[1:], rtol=1e-7, atol=1e-8)
    shift = q[0] - grad[0]
    assert np.allclose(shift, -(GAMMA + math.log(2.0)) / (GAMMA - 1), atol=1e-7)


def test_q_printed_code_value():
    """The printed q_variables code fixes q for gamma = 1.4 (ln(beta)*2.5).
    Worked by hand: rho = 1, u = (0, 0), p = 1/2 -> beta = 1, q = [0, 0, 0, -2];
    rho = e, u = (1, 0), p = e/2 -> beta = 1, q = [1 - 1, 2, 0, -2]."""
    U = _U(np.array([1.0, math.e]), np.array([0.0, 1.0]), np.array([0.0, 0.0]),
           np.array([0.5, math.e / 2]))
    q = oracle.q_variables(U)
    assert np.allclose(q[:, 0], [0, 0, 0, -2], atol=1e-15)
    assert np.allclose(q[:, 1], [0, 2, 0, -2], atol=1e-15)


# --------------------------------------------------------------------------
# Kinetic split fluxes
# --------------------------------------------------------------------------

def _euler_flux_textbook(rho, un, ut, p):
    E = p / (GAMMA - 1) + 0.5 * rho * (un * un + ut * ut)
    return np.array([rho * un, rho * un * un + p, rho * un * ut, un * (E + p)])


def test_split_fluxes_sum_to_euler_flux():
    rng = np.random.default_rng(3)
    for rho, un, ut, p in zip(*_rand_prim(rng, 500)):
        Gp = oracle.split_flux(rho, un, ut, p, +1)
        Gm = oracle.split_flux(rho, un, ut, p, -1)
        F = _euler_flux_textbook(rho, un, ut, p)
        scale = np.abs(Gp) + np.abs(Gm)
        assert np.all(np.abs(Gp + Gm - F) <= 4e-16 * scale + 1e-300)


def test_split_flux_mirror_and_supersonic_limits():
    rng = np.random.default_rng(4)
    flip = np.array([-1.0, 1.0, -1.0, -1.0])
    for rho, un, ut, p in zip(*_rand_prim(rng, 200)):
        Gm = oracle.split_flux(rho, un, ut, p, -1)
        Gp_mirror = oracle.split_flux(rho, -un, ut, p, +1)
        assert np.allclose(Gm, flip * Gp_mirror, rtol=1e-15, atol=1e-15)
    # S = un sqrt(beta) = 8: the backward half-range carries nothing
    rho, p = 1.0, 1.0 / GAMMA
    un = 8.0 / math.sqrt(rho / (2 * p))
    Gm = oracle.split_flux(rho, un, 0.3, p, -1)
    Gp = oracle.split_flux(rho, un, 0.3, p, +1)
    assert np.all(np.abs(Gm) < 1e-25 * np.abs(Gp).max())
    assert np.allclose(Gp, _euler_flux_textbook(rho, un, 0.3, p), rtol=1e-15)


def test_split_flux_matches_half_range_quadrature():
    """Brute force: integrate v1 * Psi * F over v1 > 0 for the 2D Maxwellian
    F = rho beta/pi exp(-beta |v - u|^2) with Psi = [1, v1, v2, |v|^2/2 + e_int],
    e_int = p/rho (1/(gamma-1) - 1) the non-translational energy per mass."""
    from scipy import integrate

    cases = [(1.0, 0.3, -0.2, 0.7), (0.6, -1.1, 0.5, 1.9), (2.2, 1.7, 0.0, 0.4)]
    for rho, u1, u2, p in cases:
        beta = rho / (2 * p)
        e_int = p / rho * (1.0 / (GAMMA - 1) - 1.0)
        sig = 1.0 / math.sqrt(beta)

        def F(v2, v1):
            return rho * beta / math.pi * math.exp(-beta * ((v1 - u1) ** 2 + (v2 - u2) ** 2))

        psis = [lambda v1, v2: 1.0, lambda v1, v2: v1, lambda v1, v2: v2,
                lambda v1, v2: 0.5 * (v1 * v1 + v2 * v2) + e_int]
        G = []
        for psi in psis:
            val, _ = integrate.dblquad(lambda v2, v1: v1 * psi(v1, v2) * F(v2, v1),
                                       0.0, u1 + 14 * sig, u2 - 14 * sig, u2 + 14 * sig,
                                       epsabs=1e-13, epsrel=1e-12)
            G.append(val)
        G = np.array(G)
        Gp = oracle.split_flux(rho, u1, u2, p, +1)
        assert np.allclose(Gp, G, rtol=1e-9, atol=1e-11), (Gp, G)


# --------------------------------------------------------------------------
# Stencil split (after E12)
# --------------------------------------------------------------------------

def test_split_stencils_hand_cloud():
    """Point 0 at the origin with normal n = (0.6, 0.8), tangent t = (0.8, -0.6).
    Neighbours at P = a t + b n have ds = a, dn = b; exact zeros join no set.
    (a, b) are chosen so that the products are exact in binary."""
    t = np.array([0.8, -0.6]); nn = np.array([0.6, 0.8])
    ab = [(-1.0, 0.0), (1.0, 0.0), (0.0, -1.0), (0.0, 1.0), (-2.0, 3.0), (0.5, -0.25)]
    xs = [0.0] + [a * t[0] + b * nn[0] for a, b in ab]
    ys = [0.0] + [a * t[1] + b * nn[1] for a, b in ab]
    c = _cloud(xs, ys, [0.6] + [1.0] * 6, [0.8] + [0.0] * 6, [0] * 7,
               [list(range(1, 7))] + [[0]] * 6)
    m = oracle.split_stencils(c)
    expect = []
    for a, b in ab:
        v = 0
        v |= oracle.XPOS if a < 0 else 0
        v |= oracle.XNEG if a > 0 else 0
        v |= oracle.YPOS if b < 0 else 0
        v |= oracle.YNEG if b > 0 else 0
        expect.append(v)
    assert list(m[:6]) == expect


# --------------------------------------------------------------------------
# Least-squares derivatives (E9, E14, E15)
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def small_cloud():
    return naca0012_cloud(64, 12, seed=7)


def test_ls_gradient_exact_for_linear_fields(small_cloud):
    c = small_cloud
    rng = np.random.default_rng(5)
    a = rng.normal(size=(4, 3))
    q = a[:, :1] + a[:, 1:2] * c["x"] + a[:, 2:3] * c["y"]
    for inner in (0, 3):
        qx, qy = oracle.q_derivatives(c, q, inner=inner)
        assert np.allclose(qx, a[:, 1:2], rtol=0, atol=1e-11)
        assert np.allclose(qy, a[:, 2:3], rtol=0, atol=1e-11)


def test_inner_iteration_fixed_point_for_quadratic_fields(small_cloud):
    """For quadratic q the exact gradient satisfies E15 exactly (the defect
    correction of E14 removes the whole second-order Taylor term), so one
    inner iteration started from it returns it."""
    c = small_cloud
    rng = np.random.default_rng(6)
    A = rng.normal(size=(4, 6))
    x, y = c["x"], c["y"]
    q = A[:, :1] + A[:, 1:2] * x + A[:, 2:3] * y + A[:, 3:4] * x * x + A[:, 4:5] * x * y + A[:, 5:6] * y * y
    gx = A[:, 1:2] + 2 * A[:, 3:4] * x + A[:, 4:5] * y
    gy = A[:, 2:3] + A[:, 4:5] * x + 2 * A[:, 5:6] * y
    qx, qy = oracle.q_derivatives_pass(c, q, gx, gy)
    scale = np.abs(A).max() * (1 + np.abs(x).max() + np.abs(y).max()) ** 2
    assert np.max(np.abs(qx - gx)) < 1e-9 * scale
    assert np.max(np.abs(qy - gy)) < 1e-9 * scale
    # and the first-order gradient is not exact (the correction matters)
    qx1, _ = oracle.q_derivatives(c, q, inner=0)
    assert np.max(np.abs(qx1 - gx)) > 1e-6 * scale


def test_inner_iterations_reduce_gradient_error_on_quadratics(small_cloud):
    c = small_cloud
    x, y = c["x"], c["y"]
    q = np.stack([x * x, x * y, y * y, 0.3 * x * x - y * y + x])
    gx = np.stack([2 * x, y, 0 * x, 0.6 * x + 1])
    interior = c["flags"] == 0
    errs = []
    for inner in (0, 1, 2, 3, 6):
        qx, _ = oracle.q_derivatives(c, q, inner=inner)
        errs.append(np.max(np.abs(qx - gx)[:, interior]))
    assert errs[1] < errs[0] and errs[3] < errs[1] and errs[4] < errs[3]


# --------------------------------------------------------------------------
# Flux residual (E10-E14)
# --------------------------------------------------------------------------

def _cartesian_stencil(h, theta, flag=0):
    """Point 0 at the origin, 8 neighbours on the 3x3 block of spacing h,
    rotated by theta; the point's normal is the rotated (0, 1), so its local
    frame is s = rotated x, n = rotated y."""
    offs = [(-1, -1), (-1, 0), (-1, 1), (0, -1), (0, 1), (1, -1), (1, 0), (1, 1)]
    c, s = math.cos(theta), math.sin(theta)
    pts = [(0.0, 0.0)] + [(h * a, h * b) for a, b in offs]
    xs = [c * a - s * b for a, b in pts]
    ys = [s * a + c * b for a, b in pts]
    nx, ny = -s, c
    rows = [list(range(1, 9))] + [[0]] * 8
    cl = _cloud(xs, ys, [nx] * 9, [ny] * 9, [flag] + [2] * 8, rows)
    return cl, offs


def test_first_order_residual_is_upwind_difference_on_cartesian_stencil():
    """On the symmetric 3x3 stencil the least-squares formula E11 reduces to
    one-sided differences against the mean of each side's three points:
    dGs+/ds = (G+(0) - mean_left G+)/h, dGs-/ds = (mean_right G- - G-(0))/h,
    and likewise in n. The frame is rotated by 0.3 rad, so the momentum
    residual is rotated back."""
    rng = np.random.default_rng(8)
    h, theta = 0.01, 0.3
    c, offs = _cartesian_stencil(h, theta)
    m = oracle.split_stencils(c)
    rho, u1, u2, p = _rand_prim(rng, 9)
    rho = 1 + 0.1 * (rho - 1); p = 0.7 + 0.05 * p
    U = _U(rho, u1 * 0.3, u2 * 0.3, p)
    q = oracle.q_variables(U)
    R = oracle.flux_residual(c, m, q, None, None, order=1)
    cth, sth = math.cos(theta), math.sin(theta)
    t = np.array([cth, sth]); nn = np.array([-sth, cth])

    def G(k, d, sign):
        us = u1[k] * 0.3 * t[0] + u2[k] * 0.3 * t[1]
        un = u1[k] * 0.3 * nn[0] + u2[k] * 0.3 * nn[1]
        if d == 0:
            g = oracle.split_flux(rho[k], us, un, p[k], sign)
            return g
        g = oracle.split_flux(rho[k], un, us, p[k], sign)
        return np.array([g[0], g[2], g[1], g[3]])

    left = [k + 1 for k, (a, b) in enumerate(offs) if a < 0]
    right = [k + 1 for k, (a, b) in enumerate(offs) if a > 0]
    below = [k + 1 for k, (a, b) in enumerate(offs) if b < 0]
    above = [k + 1 for k, (a, b) in enumerate(offs) if b > 0]
    Rl = ((G(0, 0, +1) - np.mean([G(k, 0, +1) for k in left], axis=0)) / h
          + (np.mean([G(k, 0, -1) for k in right], axis=0) - G(0, 0, -1)) / h
          + (G(0, 1, +1) - np.mean([G(k, 1, +1) for k in below], axis=0)) / h
          + (np.mean([G(k, 1, -1) for k in above], axis=0) - G(0, 1, -1)) / h)
    expect = np.array([Rl[0], Rl[1] * t[0] + Rl[2] * nn[0], Rl[1] * t[1] + Rl[2] * nn[1], Rl[3]])
    scale = np.abs(expect).max()
    assert np.allclose(R[:, 0], expect, rtol=0, atol=1e-11 * scale)
    # far-field points carry no residual
    assert np.all(R[:, 1:] == 0.0)


def test_wall_residual_drops_the_inward_normal_term():
    rng = np.random.default_rng(9)
    h = 0.02
    c, offs = _cartesian_stencil(h, 0.0, flag=0)
    cw, _ = _cartesian_stencil(h, 0.0, flag=1)
    m = oracle.split_stencils(c)
    rho, u1, u2, p = _rand_prim(rng, 9)
    U = _U(1 + 0.05 * rho, 0.2 * u1, 0.2 * u2, 0.7 + 0.05 * p)
    q = oracle.q_variables(U)
    Ri = oracle.flux_residual(c, m, q, None, None, order=1)
    Rw = oracle.flux_residual(cw, m, q, None, None, order=1)
    below = [k + 1 for k, (a, b) in enumerate(offs) if b < 0]
    pr = [(U[0, k], U[1, k] / U[0, k], U[2, k] / U[0, k],
           (GAMMA - 1) * (U[3, k] - 0.5 * (U[1, k] ** 2 + U[2, k] ** 2) / U[0, k])) for k in range(9)]

    def Gn(k):
        r, a, b, pp = pr[k]
        g = oracle.split_flux(r, b, a, pp, +1)
        return np.array([g[0], g[2], g[1], g[3]])
    dGn_plus = (Gn(0) - np.mean([Gn(k) for k in below], axis=0)) / h
    assert np.allclose(Ri[:, 0] - Rw[:, 0], dGn_plus, rtol=0, atol=1e-11 * np.abs(dGn_plus).max())


def test_freestream_is_preserved_exactly():
    c = naca0012_cloud(96, 16, seed=11)
    m = oracle.split_stencils(c)
    U = oracle.freestream_state(c["n"], 0.85, 1.0)
    for order in (1, 2):
        R = oracle.residual(c, m, U, order=order)
        assert np.all(R == 0.0)


def _box_cloud(k, jitter, seed):
    """Jittered k x k grid on [0,1]^2, normals (0, 1); the outer ring is
    far-field. Neighbours: the 5x5 block."""
    rng = np.random.default_rng(seed)
    h = 1.0 / (k - 1)
    I, J = np.meshgrid(np.arange(k), np.arange(k), indexing="xy")
    x = (I * h).ravel().astype(float)
    y = (J * h).ravel().astype(float)
    ring = (I == 0) | (J == 0) | (I == k - 1) | (J == k - 1)
    inner = ~ring.ravel()
    x[inner] += jitter * h * rng.uniform(-1, 1, inner.sum())
    y[inner] += jitter * h * rng.uniform(-1, 1, inner.sum())
    rows = []
    for j in range(k):
        for i in range(k):
            r = []
            for dj in range(-2, 3):
                for di in range(-2, 3):
                    if (di or dj) and 0 <= i + di < k and 0 <= j + dj < k:
                        r.append((j + dj) * k + i + di)
            rows.append(r)
    flags = np.where(ring.ravel(), 2, 0)
    n = k * k
    return _cloud(x, y, np.zeros(n), np.ones(n), flags, rows), h, I.ravel(), J.ravel()


def _smooth_state(x, y):
    rho = 1.0 + 0.2 * np.sin(2.0 * x + 1.0) * np.cos(1.5 * y)
    u1 = 0.5 + 0.2 * np.cos(1.7 * y - 0.4 * x)
    u2 = 0.1 + 0.15 * np.sin(1.3 * x + 0.8 * y)
    p = 0.7 + 0.1 * np.cos(x - 2.0 * y)
    return rho, u1, u2, p


def _exact_divergence(x, y):
    """dGx/dx + dGy/dy of the smooth state, by 4th-order central differences
    of the textbook Euler fluxes (independent of the split fluxes)."""
    def Gx(x, y):
        r, a, b, p = _smooth_state(x, y)
        return _euler_flux_textbook(r, a, b, p)

    def Gy(x, y):
        r, a, b, p = _smooth_state(x, y)
        g = _euler_flux_textbook(r, b, a, p)
        return np.array([g[0], g[2], g[1], g[3]])
    e = 1e-3
    dx = (-Gx(x + 2 * e, y) + 8 * Gx(x + e, y) - 8 * Gx(x - e, y) + Gx(x - 2 * e, y)) / (12 * e)
    dy = (-Gy(x, y + 2 * e) + 8 * Gy(x, y + e) - 8 * Gy(x, y - e) + Gy(x, y - 2 * e)) / (12 * e)
    return dx + dy


@pytest.mark.parametrize("order,jitter,inner,expect_rate",
                         [(1, 0.2, 0, 0.8), (2, 0.2, 30, 1.6), (2, 0.0, 3, 1.8)])
def test_residual_converges_to_euler_divergence(order, jitter, inner, expect_rate):
    """Consistency: on refined clouds, R(U) of a smooth state tends to div G(U)
    at the order of the scheme (1 for first order; 2 for the defect-corrected
    q-LSKUM). A dropped term, a wrong sign or a transposed operand in E11-E15
    breaks the rate. On jittered clouds the second-order rate needs the inner
    iterations of E15 converged (30 here): a few Jacobi sweeps leave an
    O(h rho^k) gradient error that shows up as first order at fine h."""
    errs = []
    for k in (21, 41, 81):
        c, h, I, J = _box_cloud(k, jitter, seed=k)
        m = oracle.split_stencils(c)
        U = _U(*_smooth_state(c["x"], c["y"]))
        R = oracle.residual(c, m, U, order=order, inner=inner)
        core = (I >= k // 4) & (I <= 3 * k // 4) & (J >= k // 4) & (J <= 3 * k // 4)
        D = _exact_divergence(c["x"][core], c["y"][core])
        errs.append(np.sqrt(np.mean((R[:, core] - D) ** 2)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > expect_rate, (errs, rates)


# --------------------------------------------------------------------------
# Time stepping, residue, forces
# --------------------------------------------------------------------------

def test_timestep_worked_example():
    with open(os.path.join(GOLDEN, "timestep_example.json")) as f:
        g = json.load(f)
    c = _cloud(g["x"], g["y"], [0, 0, 0], [1, 1, 1], [0, 0, 0], g["rows"])
    U = np.array(g["U"], dtype=float)
    dt = oracle.timestep(c, U, g["cfl"])
    assert np.allclose(dt, g["dt"], rtol=1e-14, atol=0)


def test_euler_and_rk4_on_linear_residual():
    """R(U) = lam (U - U*) has the exact one-step amplification
    1 - z (Euler) and 1 - z + z^2/2 - z^3/6 + z^4/24 (RK4), z = lam dt."""
    rng = np.random.default_rng(10)
    n = 7
    lam = rng.uniform(0.5, 2.0, (4, n))
    Ustar = rng.normal(size=(4, n))
    U0 = rng.normal(size=(4, n))
    dt = rng.uniform(0.05, 0.4, n)
    flags = np.zeros(n, np.int32)
    z = lam * dt[None, :]
    fn = lambda U: lam * (U - Ustar)  # noqa: E731
    U1, R0 = oracle.euler_step(flags, np.zeros(n), np.ones(n), np.zeros(4), dt, U0, fn)
    assert np.allclose(U1 - Ustar, (U0 - Ustar) * (1 - z), rtol=1e-14, atol=1e-14)
    assert np.allclose(R0, fn(U0), rtol=0, atol=0)
    U4, _ = oracle.rk4_step(flags, np.zeros(n), np.ones(n), np.zeros(4), dt, U0, fn)
    amp = 1 - z + z ** 2 / 2 - z ** 3 / 6 + z ** 4 / 24
    assert np.allclose(U4 - Ustar, (U0 - Ustar) * amp, rtol=1e-13, atol=1e-14)


def test_boundary_treatment_in_updates():
    """Wall points lose exactly their normal momentum; far-field points are
    reset to the free stream; interior points are untouched."""
    n = 3
    flags = np.array([0, 1, 2], np.int32)
    nx = np.array([0.0, 0.6, 1.0]); ny = np.array([1.0, 0.8, 0.0])
    Uinf = oracle.freestream(0.5, 3.0)
    U0 = np.array([[1.0, 1.1, 0.9], [0.3, 0.5, -0.2], [0.1, -0.4, 0.3], [2.0, 2.1, 1.9]])
    U1, _ = oracle.euler_step(flags, nx, ny, Uinf, np.ones(n), U0, lambda U: np.zeros_like(U))
    assert np.array_equal(U1[:, 0], U0[:, 0])
    assert abs(U1[1, 1] * 0.6 + U1[2, 1] * 0.8) < 1e-16
    t = np.array([0.8, -0.6])
    assert abs((U1[1, 1] * t[0] + U1[2, 1] * t[1]) - (0.5 * 0.8 + 0.4 * 0.6)) < 1e-15
    assert np.array_equal(U1[:, 2], Uinf)


def test_residue_worked_example():
    R = np.zeros((4, 4)); R[0] = [3.0, 0.0, 4.0, 0.0]; R[1:] = 7.0
    assert oracle.residue(R) == 5.0 / 4.0


def test_freestream_worked_example():
    U = oracle.freestream(0.5, 90.0)
    # rho = 1, u = (0, 0.5) up to cos(pi/2) rounding, p = 1/1.4
    assert U[0] == 1.0 and abs(U[1]) < 1e-16 and abs(U[2] - 0.5) < 1e-16
    assert abs(U[3] - (1 / 1.4 / 0.4 + 0.125)) < 1e-15


def _naca_area():
    # exact integral of 2 * 0.6 (0.2969 sqrt(x) - 0.1260 x - 0.3516 x^2 + 0.2843 x^3 - 0.1036 x^4) on [0,1]
    return 1.2 * (0.2969 * 2 / 3 - 0.1260 / 2 - 0.3516 / 3 + 0.2843 / 4 - 0.1036 / 5)


@pytest.mark.parametrize("a,b,cx,mach,aoa", [(0.3, -1.5, False, 0.5, 0.0), (0.1, 2.0, True, 0.8, 3.0)])
def test_forces_divergence_theorem(a, b, cx, mach, aoa):
    """A wall pressure with Cp = a + b*y (or a + b*x) integrates to the force
    -b * area * e_y (or e_x): the closed-contour integral of y n equals the
    enclosed area times e_y. The discrete sum is second order, so W = 2048
    points meet it to about 1e-4."""
    c = naca0012_cloud(2048, 3, seed=3)
    n = c["n"]
    qinf = 0.5 * mach * mach
    coord = c["x"] if cx else c["y"]
    p = 1 / GAMMA + qinf * (a + b * coord)
    U = _U(np.ones(n), np.zeros(n), np.zeros(n), p)
    cl, cd, cp = oracle.forces(c, U, mach, aoa)
    wall = c["wall_order"]
    assert np.allclose(cp, (a + b * coord)[wall], rtol=1e-12, atol=1e-12)
    A = _naca_area()
    fx, fy = (-b * A, 0.0) if cx else (0.0, -b * A)
    al = math.radians(aoa)
    assert abs(cl - (fy * math.cos(al) - fx * math.sin(al))) < 2e-4 * abs(b)
    assert abs(cd - (fx * math.cos(al) + fy * math.sin(al))) < 2e-4 * abs(b)


def test_mirror_symmetric_cloud_gives_zero_lift_at_zero_incidence():
    c = naca0012_cloud(128, 24, seed=5, mirror=True)
    m = oracle.split_stencils(c)
    U0 = oracle.freestream_state(c["n"], 0.63, 0.0)
    U, hist = oracle.solve(c, m, U0, 30, order=2, inner=3, scheme=1, cfl=0.2, mach=0.63, aoa_deg=0.0,
                           limiter=1.0)
    cl, cd, cp = oracle.forces(c, U, 0.63, 0.0)
    assert abs(cl) < 1e-11 and cd != 0.0
    # the state itself is mirror-symmetric: point (i, j) <-> (W - i, j)
    W = c["W"]
    i = np.arange(c["n"]) % W
    j = np.arange(c["n"]) // W
    mi = j * W + (W - i) % W
    assert np.allclose(U[0], U[0][mi], rtol=0, atol=1e-12)
    assert np.allclose(U[1], U[1][mi], rtol=0, atol=1e-12)
    assert np.allclose(U[2], -U[2][mi], rtol=0, atol=1e-12)


# --------------------------------------------------------------------------
# Venkatakrishnan limiter (optional; not in the paper)
# --------------------------------------------------------------------------

def _line_cloud(q_values, h=0.1):
    """Point 0 at the origin with neighbours at (+-h, 0), (0, +-h)."""
    xs = [0.0, h, -h, 0.0, 0.0]
    ys = [0.0, 0.0, 0.0, h, -h]
    c = _cloud(xs, ys, [0.0] * 5, [1.0] * 5, [0] + [2] * 4, [[1, 2, 3, 4], [0, 3, 4], [0, 3, 4],
                                                             [0, 1, 2], [0, 1, 2]])
    q = np.zeros((4, 5))
    q[0] = q_values
    return c, q


def test_limiter_keeps_linear_fields_on_symmetric_stencils():
    """For q linear, each half shift is half a neighbour difference, inside
    [q_min - q_0, q_max - q_0] by a factor 2, where f >= 1: no limiting."""
    c, q = _line_cloud([0.0, 0.3, -0.3, 0.2, -0.2])
    gx = np.zeros((4, 5)); gy = np.zeros((4, 5))
    gx[0, 0], gy[0, 0] = 3.0, 2.0
    lx, ly = oracle.limit_gradients(c, q, gx, gy, 1e-6)
    # the largest shift is exactly D/2, where f = 1 up to rounding
    assert abs(lx[0, 0] - 3.0) < 1e-14 and abs(ly[0, 0] - 2.0) < 1e-14


def test_limiter_worked_value():
    """Hand value of the published function: with D/d = 1 and e = 0,
    f = (1 + 2)/(1 + 2 + 1) = 3/4. Neighbour values 0.1 and -0.5 around q_0 = 0
    and grad (2, 0): shifts +-0.1 on the x edges; D+ = 0.1 -> f = 3/4,
    D- = -0.5 -> f(-0.5, -0.1) = (0.25 + 0.1)/(0.25 + 0.02 + 0.05) = 1.09375 (> 1)."""
    c, q = _line_cloud([0.0, 0.1, -0.5, 0.0, 0.0])
    gx = np.zeros((4, 5)); gy = np.zeros((4, 5))
    gx[0, 0] = 2.0
    lx, _ = oracle.limit_gradients(c, q, gx, gy, 1e-9)
    assert abs(lx[0, 0] - 2.0 * 0.75) < 1e-9


def test_limiter_flattens_extrema_and_bounds_reconstruction():
    """At a local maximum (q_0 above every neighbour) the limited gradient is
    ~0 for e -> 0; in general the limited shifts +-(P_i - P_0).grad/2 stay
    within the neighbour range (f d <= D for e = 0)."""
    c, q = _line_cloud([1.0, 0.3, 0.2, 0.5, 0.4])
    gx = np.full((4, 5), 0.0); gy = np.zeros((4, 5))
    gx[0, 0] = 4.0
    lx, _ = oracle.limit_gradients(c, q, gx, gy, 1e-9)
    assert abs(lx[0, 0]) < 1e-12
    rng = np.random.default_rng(12)
    cl = naca0012_cloud(64, 12, seed=2)
    qq = rng.normal(size=(4, cl["n"]))
    ox, oy = oracle.q_derivatives(cl, qq, inner=0)
    lx, ly = oracle.limit_gradients(cl, qq, ox, oy, 1e-9)
    off, idx = cl["nbr_offsets"], cl["nbr_idx"]
    for p in range(cl["n"]):
        nb = idx[off[p]:off[p + 1]]
        dx = cl["x"][nb] - cl["x"][p]
        dy = cl["y"][nb] - cl["y"][p]
        for k in range(4):
            qs = np.concatenate([[qq[k, p]], qq[k, nb]])
            shift = 0.5 * (dx * lx[k, p] + dy * ly[k, p])
            lo, hi = qs.min() - qq[k, p], qs.max() - qq[k, p]
            assert np.all(shift <= hi + 1e-9) and np.all(-shift <= hi + 1e-9)
            assert np.all(shift >= lo - 1e-9) and np.all(-shift >= lo - 1e-9)
