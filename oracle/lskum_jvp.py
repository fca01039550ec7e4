"""Exact directional derivatives of the q-LSKUM residual, for checking its
vector-Jacobian product (VJP).

TEST INFRASTRUCTURE ONLY: the tests use this module; the CUDA product path
never imports it.

The residual R(U; x, y) of the scheme (E13 q-variables; E15 q-derivatives
with the E14 modified variables and `inner` Jacobi iterations; the kinetic
split fluxes of each x+/x-/y+/y- sub-stencil closed by the least-squares
formula E11; the sum E10) is written out again here in plain numpy, in the
same steps and the same order as the C oracle, but over complex numbers.
The complex-step method (W. Squire and G. Trapp, SIAM Review 40 (1998)
110-112; J. Martins, P. Sturdza and J. Alonso, ACM TOMS 29 (2003) 245-262)
then gives the Jacobian-vector product J v without a difference quotient:
for an analytic f, Im f(z + i h v) / h = f'(z) v + O(h^2), and with
h = 1e-30 the O(h^2) term is far below rounding. Discrete choices (the
sub-stencil masks, the positivity checks) use real parts only, and erf of a
complex argument is its first-order expansion erf(a) + i b erf'(a),
which is exact to O(b^2).

The VJP of a seeded R_bar is then checked entry by entry:
(J^T R_bar)_k = <R_bar, J e_k>, one complex-step residual per entry.

Derivatives with respect to x and y hold the frame normals, the
connectivity and the sub-stencil membership fixed (they are inputs of the
scheme, not functions of the coordinates).

The module is pinned against the C oracle: its real part is the C oracle's
residual, and its J v agrees with central differences of the C oracle.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf as _erf_real

XPOS, XNEG, YPOS, YNEG = 1, 2, 4, 8
INTERIOR, WALL, FARFIELD = 0, 1, 2

_TWO_OVER_SQRT_PI = 2.0 / math.sqrt(math.pi)


def _erf(z):
    """erf on the complex-step lattice: erf(a) + i b (2/sqrt(pi)) exp(-a^2)."""
    if not np.iscomplexobj(z):
        return _erf_real(z)
    a = z.real
    return _erf_real(a) + 1j * z.imag * (_TWO_OVER_SQRT_PI * np.exp(-a * a))


class _Edges:
    """CSR edge lists: src (owner point), dst (neighbour)."""

    def __init__(self, cloud):
        off = np.asarray(cloud["nbr_offsets"], dtype=np.int64)
        self.n = int(cloud["n"])
        self.off = off
        self.src = np.repeat(np.arange(self.n), np.diff(off))
        self.dst = np.asarray(cloud["nbr_idx"], dtype=np.int64)

    def rowsum(self, vals):
        """Per-point sum over the point's CSR row, in CSR order (as the C loop)."""
        out = np.zeros(self.n, dtype=vals.dtype)
        np.add.at(out, self.src, vals)
        return out


def q_from_U(U, gamma=1.4):
    """E13: q = [ln rho + ln(beta)/(gamma-1) - beta |u|^2, 2 beta u1, 2 beta u2, -2 beta]."""
    rho = U[0]
    u1 = U[1] / rho
    u2 = U[2] / rho
    p = (gamma - 1.0) * (U[3] - 0.5 * rho * (u1 * u1 + u2 * u2))
    beta = 0.5 * rho / p
    return np.stack([np.log(rho) + np.log(beta) / (gamma - 1.0) - beta * (u1 * u1 + u2 * u2),
                     2.0 * beta * u1, 2.0 * beta * u2, -2.0 * beta])


def _prim_from_q(qt, gamma):
    """Inverse of E13 for q[4, m]: (rho, u1, u2, p)."""
    beta = -0.5 * qt[3]
    if np.any(beta.real <= 0.0):
        raise ValueError("reconstructed state with beta <= 0")
    u1 = qt[1] / (2.0 * beta)
    u2 = qt[2] / (2.0 * beta)
    rho = np.exp(qt[0] - np.log(beta) / (gamma - 1.0) + beta * (u1 * u1 + u2 * u2))
    p = rho / (2.0 * beta)
    return rho, u1, u2, p


def _split_flux(gamma, rho, un, ut, p, sign):
    """Half-range-moment split flux along a direction (un normal, ut transverse);
    components [mass, normal momentum, transverse momentum, energy]."""
    beta = 0.5 * rho / p
    S = un * np.sqrt(beta)
    A = 0.5 * (1.0 + sign * _erf(S))
    B = np.exp(-S * S) / (2.0 * np.sqrt(math.pi * beta))
    rhoE = p / (gamma - 1.0) + 0.5 * rho * (un * un + ut * ut)
    return np.stack([rho * (un * A + sign * B),
                     (p + rho * un * un) * A + sign * rho * un * B,
                     rho * ut * (un * A + sign * B),
                     (rhoE + p) * un * A + sign * (rhoE + 0.5 * p) * B])


def _frame_flux(gamma, prim, tx, ty, nx, ny, direction, sign):
    """Split flux along s (direction 0) or n (1) in frame order [mass, s-mom, n-mom, energy]."""
    rho, u1, u2, p = prim
    us = u1 * tx + u2 * ty
    un = u1 * nx + u2 * ny
    if direction == 0:
        return _split_flux(gamma, rho, us, un, p, sign)
    g = _split_flux(gamma, rho, un, us, p, sign)
    return np.stack([g[0], g[2], g[1], g[3]])


def _gradient_pass(E, dx, dy, q, gx_old=None, gy_old=None):
    """One least-squares solve of E15 (first order when gx_old is None)."""
    sxx = E.rowsum(dx * dx)
    sxy = E.rowsum(dx * dy)
    syy = E.rowsum(dy * dy)
    det = sxx * syy - sxy * sxy
    gx = np.empty_like(q)
    gy = np.empty_like(q)
    for k in range(4):
        dq = q[k][E.dst] - q[k][E.src]
        if gx_old is not None:
            dq = dq - 0.5 * (dx * (gx_old[k][E.dst] - gx_old[k][E.src])
                             + dy * (gy_old[k][E.dst] - gy_old[k][E.src]))
        sxq = E.rowsum(dx * dq)
        syq = E.rowsum(dy * dq)
        gx[k] = (syy * sxq - sxy * syq) / det
        gy[k] = (sxx * syq - sxy * sxq) / det
    return gx, gy


def _first_per_point(src, key, order, n):
    """For every point, the position (into the edge arrays) of its entry with
    the smallest real key, the earliest in `order` among equal keys; -1 for a
    point without entries."""
    pick = np.full(n, -1, dtype=np.int64)
    if len(src) == 0:
        return pick
    o = np.lexsort((order, key, src))
    first = np.ones(len(o), dtype=bool)
    first[1:] = src[o][1:] != src[o][:-1]
    pick[src[o][first]] = o[first]
    return pick


def _limit(E, dx, dy, q, gx, gy, K):
    """Venkatakrishnan's limiter exactly as the C oracle's limit_gradients
    takes it, over complex numbers: every choice (the nearest neighbour, the
    stencil maximum and minimum, the smallest f over all reconstruction
    shifts) is made on real parts, with the C loops' first-wins tie order,
    and the chosen complex values are carried through."""
    n = E.n
    ne = len(E.dst)
    eidx = np.arange(ne)
    dist = np.sqrt(dx * dx + dy * dy)
    near = _first_per_point(E.src, dist.real, eidx, n)
    h = dist[near]
    eps2 = (K * h) * (K * h) * (K * h)
    gx = gx.copy()
    gy = gy.copy()
    for k in range(4):
        q0 = q[k]
        qi = q[k][E.dst]
        # stencil extremes over P_0 and its neighbours (P_0 wins ties, then CSR order)
        amax = _first_per_point(E.src, -qi.real, eidx, n)
        amin = _first_per_point(E.src, qi.real, eidx, n)
        qmax = np.where(qi[amax].real > q0.real, qi[amax], q0)
        qmin = np.where(qi[amin].real < q0.real, qi[amin], q0)
        half = 0.5 * (dx * gx[k][E.src] + dy * gy[k][E.src])
        # the shifts -half then +half of every member, in the C loop's order
        d = np.concatenate([-half, half])
        s2 = np.concatenate([E.src, E.src])
        ordr = np.concatenate([2 * eidx, 2 * eidx + 1])
        D = np.where(d.real > 0.0, (qmax - q0)[s2], (qmin - q0)[s2])
        e2 = eps2[s2]
        f = (D * D + e2 + 2.0 * D * d) / (D * D + 2.0 * d * d + D * d + e2)
        f = np.where(d.real != 0.0, f, 1.0 + 0.0 * f)
        best = _first_per_point(s2, f.real, ordr, n)
        phi = np.where(f[best].real < 1.0, f[best], 1.0 + 0.0 * f[best])
        gx[k] = gx[k] * phi
        gy[k] = gy[k] * phi
    return gx, gy


def _residual(cloud, mask, U, x, y, order, inner, gamma, limiter=0.0):
    E = _Edges(cloud)
    n = E.n
    nx = np.asarray(cloud["nx"], dtype=np.float64)
    ny = np.asarray(cloud["ny"], dtype=np.float64)
    flags = np.asarray(cloud["flags"])
    mask = np.asarray(mask, dtype=np.uint8)
    dx = x[E.dst] - x[E.src]
    dy = y[E.dst] - y[E.src]
    q = q_from_U(U, gamma)
    if order == 2:
        gx, gy = _gradient_pass(E, dx, dy, q)
        for _ in range(inner):
            gx, gy = _gradient_pass(E, dx, dy, q, gx, gy)
        if limiter > 0.0:
            gx, gy = _limit(E, dx, dy, q, gx, gy, limiter)
        qt_i = np.stack([q[k][E.dst] - 0.5 * (dx * gx[k][E.dst] + dy * gy[k][E.dst]) for k in range(4)])
        qt_0 = np.stack([q[k][E.src] - 0.5 * (dx * gx[k][E.src] + dy * gy[k][E.src]) for k in range(4)])
    else:
        qt_i = q[:, E.dst]
        qt_0 = q[:, E.src]
    prim_i = _prim_from_q(qt_i, gamma)
    prim_0 = _prim_from_q(qt_0, gamma)
    tx, ty = ny[E.src], -nx[E.src]
    enx, eny = nx[E.src], ny[E.src]
    ds = dx * tx + dy * ty
    dn = dx * enx + dy * eny
    Rl = np.zeros((4, n), dtype=np.result_type(U, x, y, np.float64))
    subs = ((XPOS, 0, +1.0), (XNEG, 0, -1.0), (YPOS, 1, +1.0), (YNEG, 1, -1.0))
    for sub, (bit, direction, sign) in enumerate(subs):
        inside = (mask & bit) != 0
        # the sub-stencil's own sums: terms of other edges are left out
        Gi = _frame_flux(gamma, prim_i, tx, ty, enx, eny, direction, sign)
        G0 = _frame_flux(gamma, prim_0, tx, ty, enx, eny, direction, sign)
        sel = inside.astype(np.float64)
        sss = E.rowsum(sel * ds * ds)
        ssn = E.rowsum(sel * ds * dn)
        snn = E.rowsum(sel * dn * dn)
        det = sss * snn - ssn * ssn
        used = flags != FARFIELD
        if sub == 2:
            used &= flags != WALL                       # no dGn+/dn at the wall
        safe = np.where(used, det, 1.0)
        for k in range(4):
            dG = sel * (Gi[k] - G0[k])
            ssG = E.rowsum(ds * dG)
            snG = E.rowsum(dn * dG)
            if direction == 0:
                d = (snn * ssG - ssn * snG) / safe
            else:
                d = (sss * snG - ssn * ssG) / safe
            Rl[k] += np.where(used, d, 0.0)
    tx, ty = ny, -nx
    return np.stack([Rl[0], Rl[1] * tx + Rl[2] * nx, Rl[1] * ty + Rl[2] * ny, Rl[3]])


def residual(cloud, mask, U, order=2, inner=3, gamma=1.4, limiter=0.0):
    """R(U) of the scheme in real arithmetic (equals the C oracle's); limiter
    K > 0 applies Venkatakrishnan's limiter to the last iterate."""
    x = np.asarray(cloud["x"], dtype=np.float64)
    y = np.asarray(cloud["y"], dtype=np.float64)
    return _residual(cloud, mask, np.asarray(U, dtype=np.float64), x, y, order, inner, gamma, limiter)


def jvp(cloud, mask, U, dU=None, dx=None, dy=None, order=2, inner=3, gamma=1.4, h=1e-30, limiter=0.0):
    """J v = dR/dU dU + dR/dx dx + dR/dy dy at (U, x, y), by complex step.
    With the limiter the derivative is that of the branch the real parts
    select (the limiter is piecewise smooth)."""
    U = np.asarray(U, dtype=np.float64).astype(np.complex128)
    x = np.asarray(cloud["x"], dtype=np.float64).astype(np.complex128)
    y = np.asarray(cloud["y"], dtype=np.float64).astype(np.complex128)
    if dU is not None:
        U = U + 1j * h * np.asarray(dU, dtype=np.float64)
    if dx is not None:
        x = x + 1j * h * np.asarray(dx, dtype=np.float64)
    if dy is not None:
        y = y + 1j * h * np.asarray(dy, dtype=np.float64)
    return _residual(cloud, mask, U, x, y, order, inner, gamma, limiter).imag / h


def vjp_entries(cloud, mask, U, R_bar, entries, order=2, inner=3, gamma=1.4, limiter=0.0):
    """Selected entries of the VJP J^T R_bar: entries is a list of
    ("U", component, point), ("x", point) or ("y", point); each is
    <R_bar, J e> for the unit direction e of that entry."""
    n = int(cloud["n"])
    out = np.empty(len(entries))
    for j, ent in enumerate(entries):
        if ent[0] == "U":
            d = np.zeros((4, n))
            d[ent[1], ent[2]] = 1.0
            Jv = jvp(cloud, mask, U, dU=d, order=order, inner=inner, gamma=gamma, limiter=limiter)
        else:
            d = np.zeros(n)
            d[ent[1]] = 1.0
            Jv = jvp(cloud, mask, U, **{"d" + ent[0]: d}, order=order, inner=inner, gamma=gamma,
                     limiter=limiter)
        out[j] = float(np.sum(R_bar * Jv))
    return out


# ---------------------------------------------------------------------------
# The pseudo-time iteration and the forces over complex numbers, the same
# steps as the C oracle's orc_timestep, orc_euler_step / orc_rk4_step and
# orc_forces, for derivatives of Cl and Cd after unrolled iterations.
# ---------------------------------------------------------------------------
def _timestep(E, U, x, y, cfl, gamma):
    """dt = CFL dmin / (|u| + 3 sqrt(p/rho)), dmin the nearest neighbour's
    distance. dmin is a minimum: at a tie (the leading and trailing edge of a
    mirror-symmetric contour have two nearest neighbours at equal distance) it
    has a kink, and its derivative here is that of the first nearest
    neighbour in row order, ranked by the real squared distance."""
    rho = U[0]
    u1 = U[1] / rho
    u2 = U[2] / rho
    p = (gamma - 1.0) * (U[3] - 0.5 * rho * (u1 * u1 + u2 * u2))
    speed = np.sqrt(u1 * u1 + u2 * u2) + 3.0 * np.sqrt(p / rho)
    dx = x[E.dst] - x[E.src]
    dy = y[E.dst] - y[E.src]
    d2 = dx * dx + dy * dy
    d = np.sqrt(d2)
    order = np.lexsort((np.arange(len(d)), d2.real, E.src))
    first = np.ones(len(order), dtype=bool)
    first[1:] = E.src[order][1:] != E.src[order][:-1]
    dmin = np.zeros(E.n, dtype=d.dtype)
    dmin[E.src[order][first]] = d[order][first]
    return cfl * dmin / speed


def _boundary(U, flags, nx, ny, Uinf):
    """Wall points lose the normal momentum, far-field points take U_inf."""
    U = U.copy()
    wall = flags == WALL
    mn = U[1, wall] * nx[wall] + U[2, wall] * ny[wall]
    U[1, wall] = U[1, wall] - mn * nx[wall]
    U[2, wall] = U[2, wall] - mn * ny[wall]
    far = flags == FARFIELD
    U[:, far] = np.asarray(Uinf)[:, None]
    return U


def _freestream(mach, aoa_deg, gamma):
    a = math.radians(aoa_deg)
    rho, u1, u2, p = 1.0, mach * math.cos(a), mach * math.sin(a), 1.0 / gamma
    return np.array([rho, rho * u1, rho * u2, p / (gamma - 1.0) + 0.5 * rho * (u1 * u1 + u2 * u2)])


def _iterate(cloud, mask, U, x, y, scheme, cfl, mach, aoa_deg, order, inner, gamma, limiter=0.0):
    """One pseudo-time iteration: forward Euler (E16) or RK4 with dt frozen."""
    E = _Edges(cloud)
    flags = np.asarray(cloud["flags"])
    nx = np.asarray(cloud["nx"], dtype=np.float64)
    ny = np.asarray(cloud["ny"], dtype=np.float64)
    Uinf = _freestream(mach, aoa_deg, gamma)
    dt = _timestep(E, U, x, y, cfl, gamma)

    def R(V):
        return _residual(cloud, mask, V, x, y, order, inner, gamma, limiter)

    if scheme == 0:
        return _boundary(U - dt * R(U), flags, nx, ny, Uinf)
    R0 = R(U)
    U1 = _boundary(U - 0.5 * dt * R0, flags, nx, ny, Uinf)
    R1 = R(U1)
    U2 = _boundary(U - 0.5 * dt * R1, flags, nx, ny, Uinf)
    R2 = R(U2)
    U3 = _boundary(U - dt * R2, flags, nx, ny, Uinf)
    R3 = R(U3)
    return _boundary(U - dt / 6.0 * (R0 + 2.0 * R1 + 2.0 * R2 + R3), flags, nx, ny, Uinf)


def _forces(cloud, U, x, y, mach, aoa_deg, gamma):
    """Cl, Cd: Cp = (p - p_inf)/q_inf on the closed wall contour, arc-length
    weights ds = (|P_{w+1} - P_w| + |P_w - P_{w-1}|)/2, (cx, cy) = -sum Cp n ds."""
    w = np.asarray(cloud["wall_order"], dtype=np.int64)
    wn, wp = np.roll(w, -1), np.roll(w, 1)
    nx = np.asarray(cloud["nx"], dtype=np.float64)[w]
    ny = np.asarray(cloud["ny"], dtype=np.float64)[w]
    rho = U[0, w]
    u1 = U[1, w] / rho
    u2 = U[2, w] / rho
    p = (gamma - 1.0) * (U[3, w] - 0.5 * rho * (u1 * u1 + u2 * u2))
    c = (p - 1.0 / gamma) / (0.5 * mach * mach)
    dsn = np.sqrt((x[wn] - x[w]) ** 2 + (y[wn] - y[w]) ** 2)
    dsp = np.sqrt((x[w] - x[wp]) ** 2 + (y[w] - y[wp]) ** 2)
    ds = 0.5 * (dsn + dsp)
    cx = -np.sum(c * nx * ds)
    cy = -np.sum(c * ny * ds)
    a = math.radians(aoa_deg)
    return cy * math.cos(a) - cx * math.sin(a), cx * math.cos(a) + cy * math.sin(a)


def _unrolled(cloud, mask, U0, x, y, iters, scheme, cfl, mach, aoa_deg, order, inner, gamma, limiter=0.0):
    U = U0
    for _ in range(iters):
        U = _iterate(cloud, mask, U, x, y, scheme, cfl, mach, aoa_deg, order, inner, gamma, limiter)
    return U


def iterate(cloud, mask, U, scheme=1, cfl=0.2, mach=0.63, aoa_deg=2.0, order=2, inner=3, gamma=1.4,
            limiter=0.0):
    """One iteration in real arithmetic (equals the C oracle's)."""
    x = np.asarray(cloud["x"], dtype=np.float64)
    y = np.asarray(cloud["y"], dtype=np.float64)
    return _iterate(cloud, mask, np.asarray(U, dtype=np.float64), x, y, scheme, cfl, mach, aoa_deg, order,
                    inner, gamma, limiter)


def iterate_jvp(cloud, mask, U, dU=None, dx=None, dy=None, scheme=1, cfl=0.2, mach=0.63, aoa_deg=2.0,
                order=2, inner=3, gamma=1.4, h=1e-30, limiter=0.0):
    """J v of one iteration U^n -> U^{n+1}, by complex step."""
    U, x, y = _lift(cloud, U, dU, dx, dy, h)
    return _iterate(cloud, mask, U, x, y, scheme, cfl, mach, aoa_deg, order, inner, gamma, limiter).imag / h


def forces_jvp(cloud, U, dU=None, dx=None, dy=None, mach=0.63, aoa_deg=2.0, gamma=1.4, h=1e-30):
    """(dCl, dCd) along (dU, dx, dy), by complex step."""
    U, x, y = _lift(cloud, U, dU, dx, dy, h)
    cl, cd = _forces(cloud, U, x, y, mach, aoa_deg, gamma)
    return cl.imag / h, cd.imag / h


def unrolled_forces(cloud, mask, U0, iters, dx=None, dy=None, scheme=1, cfl=0.2, mach=0.63, aoa_deg=2.0,
                    order=2, inner=3, gamma=1.4, h=1e-30, limiter=0.0):
    """(Cl, Cd) after `iters` iterations from U0, and their derivatives along
    a displacement (dx, dy) of the points (frame normals and connectivity fixed)."""
    U, x, y = _lift(cloud, U0, None, dx, dy, h)
    U = _unrolled(cloud, mask, U, x, y, iters, scheme, cfl, mach, aoa_deg, order, inner, gamma, limiter)
    cl, cd = _forces(cloud, U, x, y, mach, aoa_deg, gamma)
    return (float(np.real(cl)), float(np.real(cd))), (float(np.imag(cl)) / h, float(np.imag(cd)) / h)


def _lift(cloud, U, dU, dx, dy, h):
    U = np.asarray(U, dtype=np.float64).astype(np.complex128)
    x = np.asarray(cloud["x"], dtype=np.float64).astype(np.complex128)
    y = np.asarray(cloud["y"], dtype=np.float64).astype(np.complex128)
    if dU is not None:
        U = U + 1j * h * np.asarray(dU, dtype=np.float64)
    if dx is not None:
        x = x + 1j * h * np.asarray(dx, dtype=np.float64)
    if dy is not None:
        y = y + 1j * h * np.asarray(dy, dtype=np.float64)
    return U, x, y
