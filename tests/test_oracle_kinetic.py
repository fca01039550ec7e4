"""Pins of the oracle's kinetic boundary mode (no GPU).

The mode gives a wall or far-field point the mirror image of each neighbour
across its tangent line; the image of a wall point's neighbour carries the
specularly reflected gas, that of a far-field point the free stream with zero
gradient, and the point is then treated by the interior formulas. The pins
build that augmented stencil out of real points instead: a cloud on one side
of a straight line, and the same cloud with its mirror images added as points
of their own, whose line points are plain interior points. The interior
formulas of the second cloud (pinned by the plain-mode tests) must give the
kinetic residual of the first at every original point.

Wall: the mirror points carry the reflected state (v -> -v for the line
y = 0). With the wall states tangential (v = 0) and the free stream along the
line (alpha = 0), the second cloud is mirror-symmetric, every operation at a
mirror point is the negation of one at its original, and the two residuals
agree bitwise up to the gradient at the line points (read by the inner
iterations), whose symmetric part cancels only to rounding. Rotating both
clouds breaks the symmetry by rounding too.

Far field: the mirror points carry the free stream. Their gradients are zero
(all their neighbours carry the free stream) when the line points do too, or
at first order, and the residuals agree bitwise.
"""
import numpy as np
import pytest

import oracle

C, R_ROWS, K = 16, 8, 10


def _knn(x, y, k):
    d2 = (x[:, None] - x[None, :]) ** 2 + (y[:, None] - y[None, :]) ** 2
    np.fill_diagonal(d2, np.inf)
    return [list(np.argsort(d2[p], kind="stable")[:k]) for p in range(len(x))]


def half_cloud(line_kind, seed=0, tie_free=False):
    """Rows j = 0..R-1 of a jittered grid above the line y = 0; row 0 lies on
    the line (columns 1..C-2) and is a wall (normal (0, 1), into the fluid) or
    far field (normal (0, -1), outward). Side columns and the top row are far
    field with outward normals; interior points get random frames.
    tie_free: jitter the edges too and keep line points out of each other's
    stencils, so that no offset has an exactly zero component in any frame
    (a rotated copy then splits its stencils the same way)."""
    rng = np.random.default_rng(seed)
    pts, fl, nrm, row = [], [], [], []
    for j in range(R_ROWS):
        for i in range(C):
            if j == 0 and i in (0, C - 1):
                continue
            jit = tie_free or (0 < i < C - 1)
            x = i + (rng.uniform(-0.2, 0.2) if jit else 0.0)
            yj = 0.0 if j == 0 else j + (rng.uniform(-0.2, 0.2) if (tie_free or j < R_ROWS - 1) else 0.0)
            if j == 0:
                f, n = (1, (0.0, 1.0)) if line_kind == "wall" else (2, (0.0, -1.0))
            elif j == R_ROWS - 1 and i in (0, C - 1):
                f, n = 2, ((-1.0 if i == 0 else 1.0) / np.sqrt(2.0), 1.0 / np.sqrt(2.0))
            elif j == R_ROWS - 1:
                f, n = 2, (0.0, 1.0)
            elif i in (0, C - 1):
                f, n = 2, (-1.0 if i == 0 else 1.0, 0.0)
            else:
                th = rng.uniform(0, 2 * np.pi)
                f, n = 0, (np.cos(th), np.sin(th))
            pts.append((x, yj)); fl.append(f); nrm.append(n); row.append(j)
    x = np.array([p[0] for p in pts]); y = np.array([p[1] for p in pts])
    row = np.array(row)
    if tie_free:
        d2 = (x[:, None] - x[None, :]) ** 2 + (y[:, None] - y[None, :]) ** 2
        np.fill_diagonal(d2, np.inf)
        line = row == 0
        d2[np.ix_(line, line)] = np.inf
        nb = [list(np.argsort(d2[p], kind="stable")[:K]) for p in range(len(x))]
    else:
        nb = _knn(x, y, K)
    return {"x": x, "y": y, "nx": np.array([n[0] for n in nrm]), "ny": np.array([n[1] for n in nrm]),
            "flags": np.array(fl, np.int32), "row": row, "nb": nb}


def _csr(h, nb):
    off = np.zeros(len(nb) + 1, np.int32)
    off[1:] = np.cumsum([len(r) for r in nb])
    return {"n": len(nb), "x": h["x"], "y": h["y"], "nx": h["nx"], "ny": h["ny"], "flags": h["flags"],
            "nbr_offsets": off, "nbr_idx": np.array([i for r in nb for i in r], np.int32),
            "wall_order": np.zeros(0, np.int32)}


def mirrored_cloud(h):
    """The half cloud plus the mirror image (x, -y) of every point off the
    line, with mirrored normals and the original's flag; line points become
    interior points whose stencil is their neighbours followed by the mirror
    images of those off the line. Returns (cloud, mirror map)."""
    n = len(h["x"])
    off_line = np.nonzero(h["row"] > 0)[0]
    mir = np.arange(n)
    mir[off_line] = n + np.arange(len(off_line))
    x = np.concatenate([h["x"], h["x"][off_line]])
    y = np.concatenate([h["y"], -h["y"][off_line]])
    nx = np.concatenate([h["nx"], h["nx"][off_line]])
    ny = np.concatenate([h["ny"], -h["ny"][off_line]])
    flags = np.concatenate([h["flags"], h["flags"][off_line]]).astype(np.int32)
    flags[np.nonzero(h["row"] == 0)[0]] = 0
    nb = [list(r) for r in h["nb"]]
    for p in np.nonzero(h["row"] == 0)[0]:
        nb[p] = nb[p] + [int(mir[k]) for k in h["nb"][p] if h["row"][k] > 0]
    nb += [[int(mir[k]) for k in h["nb"][j]] for j in off_line]
    e = {"x": x, "y": y, "nx": nx, "ny": ny, "flags": flags}
    return _csr(e, nb), mir, off_line


def _state(x, y, seed, mach, aoa):
    rng = np.random.default_rng(seed)
    k = rng.uniform(0.2, 0.5, 4)
    a = np.radians(aoa)
    rho = 1.0 + 0.1 * np.sin(k[0] * x + 0.3) * np.cos(k[1] * y)
    u = mach * np.cos(a) + 0.1 * np.cos(k[2] * y - 0.2 * x)
    v = mach * np.sin(a) + 0.1 * np.sin(k[3] * x + 0.1 * y)
    p = (1.0 + 0.1 * np.cos(k[1] * x - k[0] * y)) / 1.4
    return rho, u, v, p


def _U(rho, u, v, p):
    return np.stack([rho, rho * u, rho * v, p / 0.4 + 0.5 * rho * (u * u + v * v)])


def _rotate(c, th):
    cs, sn = np.cos(th), np.sin(th)
    out = dict(c)
    out["x"], out["y"] = cs * c["x"] - sn * c["y"], sn * c["x"] + cs * c["y"]
    out["nx"], out["ny"] = cs * c["nx"] - sn * c["ny"], sn * c["nx"] + cs * c["ny"]
    return out


def _rotate_U(U, th):
    cs, sn = np.cos(th), np.sin(th)
    V = U.copy()
    V[1], V[2] = cs * U[1] - sn * U[2], sn * U[1] + cs * U[2]
    return V


def _transpose(c):
    """x <-> y (exact): the line y = 0 becomes the line x = 0"""
    out = dict(c)
    out["x"], out["y"], out["nx"], out["ny"] = c["y"], c["x"], c["ny"], c["nx"]
    return out


def _transpose_U(U):
    return U[[0, 2, 1, 3]]


CASES = [(1, 3, 0.0), (2, 0, 0.0), (2, 3, 0.0), (2, 3, 1.0)]


@pytest.mark.parametrize("line", ["y=0", "x=0"])
@pytest.mark.parametrize("order,inner,lim", CASES)
def test_kinetic_wall_is_the_interior_scheme_on_the_mirrored_cloud(order, inner, lim, line):
    h = half_cloud("wall")
    H = _csr(h, h["nb"])
    E, mir, off_line = mirrored_cloud(h)
    rho, u, v, p = _state(h["x"], h["y"], 5, 0.6, 0.0)
    v[h["row"] == 0] = 0.0                                # tangential gas on the wall
    UH = _U(rho, u, v, p)
    UE = np.concatenate([UH, UH[:, off_line] * np.array([[1], [1], [-1], [1]])], axis=1)
    if line == "x=0":                                     # the wall x = 0, normal (1, 0)
        H, E, UH, UE = _transpose(H), _transpose(E), _transpose_U(UH), _transpose_U(UE)
    aoa = 90.0 if line == "x=0" else 0.0                  # free stream along the wall
    RH, S = oracle.residual(H, oracle.split_stencils(H), UH, order=order, inner=inner, limiter=lim,
                            boundary=1, mach=0.6, aoa_deg=aoa, want_scale=True)
    RE = oracle.residual(E, oracle.split_stencils(E), UE, order=order, inner=inner, limiter=lim,
                         boundary=1, mach=0.6, aoa_deg=aoa)
    n = H["n"]
    if line == "y=0" and (order == 1 or inner == 0):
        assert np.array_equal(RH, RE[:, :n])
    else:
        # inner iterations read the gradient at the wall points, whose normal
        # derivative of the even components is zero only up to the rounding
        # of the sums over the neighbours and then over their mirror images;
        # along x = 0 the free stream (cos 90 deg != 0 in floating point) is
        # tangential only to rounding
        assert np.all(np.abs(RH - RE[:, :n]) <= 1e-13 * S), np.max(np.abs(RH - RE[:, :n]) / S)
    # and the images matter: the plain wall reading differs at the wall
    RP = oracle.residual(H, oracle.split_stencils(H), UH, order=order, inner=inner, limiter=lim)
    wall = h["row"] == 0
    assert np.all(np.abs(RP[:, wall] - RH[:, wall]).max(axis=0) > 1e-8)


@pytest.mark.parametrize("order,inner,lim", [c for c in CASES if c[2] == 0.0])
def test_kinetic_wall_on_a_tilted_line(order, inner, lim):
    """The same pin with both clouds rotated by 0.4 rad (and the gas with
    them): the mirror symmetry now holds to rounding, 1e-12 of the scale.
    Without the limiter: it scales each component of grad q in the global
    frame, and a reflection across a tilted line mixes the components q1 and
    q2, so a mirror point limits differently from the reflection of its
    original's limited gradient (the images carry the latter)."""
    th = 0.4
    h = half_cloud("wall", seed=3, tie_free=True)
    H = _csr(h, h["nb"])
    E, mir, off_line = mirrored_cloud(h)
    rho, u, v, p = _state(h["x"], h["y"], 6, 0.6, 0.0)
    v[h["row"] == 0] = 0.0
    UH = _U(rho, u, v, p)
    UE = np.concatenate([UH, UH[:, off_line] * np.array([[1], [1], [-1], [1]])], axis=1)
    Hr, Er = _rotate(H, th), _rotate(E, th)
    UHr, UEr = _rotate_U(UH, th), _rotate_U(UE, th)
    kw = dict(order=order, inner=inner, limiter=lim, boundary=1, mach=0.6, aoa_deg=np.degrees(th))
    mH, mE = oracle.split_stencils(Hr), oracle.split_stencils(Er)
    # no exact ties: the rotation keeps every sub-stencil membership
    assert np.array_equal(mH, oracle.split_stencils(H)) and np.array_equal(mE, oracle.split_stencils(E))
    RH, S = oracle.residual(Hr, mH, UHr, want_scale=True, **kw)
    RE = oracle.residual(Er, mE, UEr, **kw)
    n = H["n"]
    assert np.all(np.abs(RH - RE[:, :n]) <= 1e-12 * S + 1e-300)


@pytest.mark.parametrize("order,inner,lim,line_at_inf", [(1, 3, 0.0, False), (2, 0, 0.0, True),
                                                         (2, 0, 1.0, True), (1, 3, 1.0, False)])
def test_kinetic_far_field_is_the_interior_scheme_with_free_stream_outside(order, inner, lim, line_at_inf):
    mach, aoa = 0.7, 3.0
    h = half_cloud("far", seed=1)
    H = _csr(h, h["nb"])
    E, mir, off_line = mirrored_cloud(h)
    UH = _U(*_state(h["x"], h["y"], 7, mach, aoa))
    Uinf = oracle.freestream(mach, aoa)
    if line_at_inf:
        UH[:, h["row"] == 0] = Uinf[:, None]
    UE = np.concatenate([UH, np.repeat(Uinf[:, None], len(off_line), axis=1)], axis=1)
    kw = dict(order=order, inner=inner, limiter=lim, boundary=1, mach=mach, aoa_deg=aoa)
    RH = oracle.residual(H, oracle.split_stencils(H), UH, **kw)
    RE, qxE, qyE = oracle.residual(E, oracle.split_stencils(E), UE, want_grad=True, **kw)
    n = H["n"]
    if order == 2:
        # the mirror points' gradients are zero, as the images' are
        assert np.all(qxE[:, n:] == 0.0) and np.all(qyE[:, n:] == 0.0)
    assert np.array_equal(RH, RE[:, :n])
    line = h["row"] == 0
    assert np.all(np.abs(RH[:, line]).max(axis=0) > 1e-8)


@pytest.mark.parametrize("order", [1, 2])
def test_kinetic_mode_preserves_the_free_stream(order):
    """U = U_inf everywhere. With far-field boundaries only, R = 0 exactly at
    every point for any flow angle (the images carry U_inf too). With a wall,
    R = 0 exactly everywhere if the free stream is tangential to it (alpha = 0
    on the line y = 0: the reflected gas equals the gas); otherwise the wall
    points see the reflected stream and R != 0 there (at first order R stays
    0 elsewhere; at second order the wall gradients reach their neighbours)."""
    f = half_cloud("far", seed=2)
    F = _csr(f, f["nb"])
    for aoa in (0.0, 7.0, -30.0):
        U = oracle.freestream_state(F["n"], 0.8, aoa)
        R = oracle.residual(F, oracle.split_stencils(F), U, order=order, inner=3, limiter=1.0, boundary=1,
                            mach=0.8, aoa_deg=aoa)
        assert np.all(R == 0.0)
    h = half_cloud("wall", seed=2)
    H = _csr(h, h["nb"])
    m = oracle.split_stencils(H)
    wall = h["row"] == 0
    for aoa in (0.0, 7.0):
        U = oracle.freestream_state(H["n"], 0.8, aoa)
        R = oracle.residual(H, m, U, order=order, inner=3, boundary=1, mach=0.8, aoa_deg=aoa)
        if aoa == 0.0:
            assert np.all(R == 0.0)
        else:
            assert np.all(np.abs(R[:, wall]).max(axis=0) > 1e-6)
            if order == 1:
                assert np.all(R[:, ~wall] == 0.0)


def test_kinetic_far_field_points_are_updated():
    """Plain reading: far-field points stay at U_inf. Kinetic mode: they move
    with the flow, and the wall keeps zero normal momentum."""
    h = half_cloud("wall", seed=4)
    H = _csr(h, h["nb"])
    m = oracle.split_stencils(H)
    rho, u, v, p = _state(h["x"], h["y"], 8, 0.5, 0.0)
    U0 = _U(rho, u, v, p)
    far = H["flags"] == 2
    Uinf = oracle.freestream(0.5, 0.0)
    U0[:, far] = Uinf[:, None]
    U0[2, h["row"] == 0] = 0.0
    Up, _ = oracle.solve(H, m, U0, 3, mach=0.5, aoa_deg=0.0, boundary=0)
    Uk, hk = oracle.solve(H, m, U0, 3, mach=0.5, aoa_deg=0.0, boundary=1)
    assert np.all(Up[:, far] == Uinf[:, None])
    assert np.any(Uk[:, far] != Uinf[:, None])
    wall = H["flags"] == 1
    assert np.all(Uk[2, wall] == 0.0)                     # normal (0, 1): rho v = 0
    assert np.all(np.isfinite(hk))
