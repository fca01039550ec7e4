"""Seeded synthetic NACA 0012 point clouds for q-LSKUM.

This module builds inputs only: point coordinates, normals, point flags and
connectivity. It holds none of the method's arithmetic (no stencil split, no
least squares, no fluxes), so both the CPU oracle and the CUDA path can take
their inputs from it.

The paper's own clouds (an O-type distribution of 614,400 points with 1280
points on the airfoil, and levels of 1M to 64M points; Sec. 4 and Sec. 5) are
not published. These clouds take their shape instead:

* W wall points on the analytic NACA 0012 contour (closed trailing edge,
  half-thickness 0.6 (0.2969 sqrt(x) - 0.1260 x - 0.3516 x^2 + 0.2843 x^3
  - 0.1036 x^4)), cosine chord spacing, counter-clockwise from the trailing
  edge;
* L layers offset with geometric growth along rays that start at each wall
  point in the direction of its outward normal, smoothed around the contour
  so that the trailing-edge corner does not fan out in a single column, the last layer on a far-field circle of radius 15 chords centred at
  mid-chord (each normal ray is cut at that circle);
* seeded uniform jitter of +-`jitter` of the local tangential/normal spacing on
  interior points (wall points stay on the contour, far-field points on the
  circle);
* flags 0 interior, 1 wall, 2 far-field; wall points carry the contour's
  outward normal, interior points the direction of their generating ray
  (wall-aligned frames), far-field points the radial normal;
* connectivity: the points within 1.8 x the local spacing, measured per
  direction in the point's frame ((dt/h_t)^2 + (dn/h_n)^2 <= 1.8^2, with h_t,
  h_n the local tangential and normal grid spacings), searched among the
  7x7 block of grid neighbours, always including the 3x3 block; then each
  half-plane of the point's frame (the body side of wall points excepted)
  is topped up to two clearly-inside neighbours, nearest first; at most 25,
  ordered by that distance (ties by index).

Point index of grid node (i, j) is j*W + i (layer-major) unless `shuffle`.
"""
from __future__ import annotations

import os

import numpy as np

FLAG_INTERIOR = 0
FLAG_WALL = 1
FLAG_FARFIELD = 2

_CENTRE = (0.5, 0.0)
_MAX_DEGREE = 25


def _naca0012_half_thickness(x):
    return 0.6 * (0.2969 * np.sqrt(x) - 0.1260 * x - 0.3516 * x**2
                  + 0.2843 * x**3 - 0.1036 * x**4)


def naca0012_wall(W: int):
    """Wall points and outward unit normals, counter-clockwise from the TE.

    The contour parameter is phi_k = 2 pi k / W, x = (1 + cos phi)/2 (cosine
    spacing); the upper surface is phi in (0, pi), the lower one is its mirror
    image, built by reflection so that the contour is exactly symmetric.
    Returns (xw, yw, nxw, nyw) as float64 arrays of length W.
    """
    if W < 8 or W % 2:
        raise ValueError("W must be even and >= 8")
    half = W // 2
    phi = 2.0 * np.pi * np.arange(half + 1) / W          # 0 .. pi (TE .. LE)
    x = 0.5 * (1.0 + np.cos(phi))
    x[0], x[half] = 1.0, 0.0
    y = _naca0012_half_thickness(x)
    y[0], y[half] = 0.0, 0.0
    # Tangent d(x, y)/dphi on the upper surface. sqrt(x) = cos(phi/2) there,
    # so d sqrt(x)/dphi = -sin(phi/2)/2 has no 0/0 at the leading edge.
    dx = -0.5 * np.sin(phi)
    dsqrt = -0.5 * np.sin(0.5 * phi)
    dpoly = (-0.1260 - 2 * 0.3516 * x + 3 * 0.2843 * x**2 - 4 * 0.1036 * x**3) * dx
    dy = 0.6 * (0.2969 * dsqrt + dpoly)
    # Counter-clockwise traversal: outward normal = (dy, -dx)/|.|
    nrm = np.hypot(dx, dy)
    nrm[0] = 1.0                     # TE corner: replaced below
    nx = dy / nrm
    ny = -dx / nrm
    nx[0], ny[0] = 1.0, 0.0          # trailing-edge corner: bisector
    nx[half], ny[half] = -1.0, 0.0   # leading edge
    xw = np.empty(W); yw = np.empty(W); nxw = np.empty(W); nyw = np.empty(W)
    xw[:half + 1], yw[:half + 1], nxw[:half + 1], nyw[:half + 1] = x, y, nx, ny
    lower = np.arange(half + 1, W)
    mirror = W - lower
    xw[lower], yw[lower] = x[mirror], -y[mirror]
    nxw[lower], nyw[lower] = nx[mirror], -ny[mirror]
    return xw, yw, nxw, nyw


def _ray_lengths(xw, yw, nxw, nyw, radius):
    """Distance t along each outward normal ray to the far-field circle."""
    cx, cy = _CENTRE
    ox, oy = xw - cx, yw - cy
    b = nxw * ox + nyw * oy
    c = ox * ox + oy * oy - radius * radius
    return -b + np.sqrt(b * b - c)


def _ray_directions(nxw, nyw, sweeps):
    """Outward ray directions: the wall normals' angle, smoothed around the
    closed contour by `sweeps` Jacobi sweeps of a (1/4, 1/2, 1/4) filter, so
    that the 160-degree jump of the normal at the trailing-edge corner is
    spread over a few dozen columns instead of one. The filter is symmetric,
    so a mirror-symmetric contour keeps mirror-symmetric rays."""
    th = np.unwrap(np.arctan2(nyw, nxw))
    W = th.shape[0]
    ext = th.copy()
    for _ in range(sweeps):
        left = np.roll(ext, 1)
        right = np.roll(ext, -1)
        left[0] -= 2.0 * np.pi      # periodic unwrap across the seam
        right[W - 1] += 2.0 * np.pi
        ext = 0.25 * left + 0.5 * ext + 0.25 * right
    return np.cos(ext), np.sin(ext)


def _growth_fractions(L, first_fraction):
    """g_j, j = 0..L, geometric with g_0 = 0, g_L = 1 and g_1 ~ first_fraction."""
    if first_fraction * L >= 1.0:
        return np.arange(L + 1) / L
    lo, hi = 1.0 + 1e-12, min(4.0, float(np.exp(600.0 / L)))
    for _ in range(200):
        r = 0.5 * (lo + hi)
        g1 = (r - 1.0) / (r**L - 1.0)
        if g1 > first_fraction:
            lo = r
        else:
            hi = r
    r = 0.5 * (lo + hi)
    return (r ** np.arange(L + 1) - 1.0) / (r**L - 1.0)


def _connectivity(x, y, W, L, flags, fnx, fny, ht, hn, radius_factor, max_degree, reach=3,
                  chunk=1 << 16):
    """CSR rows from grid candidates (i + di, j + dj), |di|, |dj| <= reach.

    Distances are measured in the point's frame (tangent (ny, -nx), normal
    (nx, ny)) in units of its local tangential and normal spacings:
    d^2 = (dt/h_t)^2 + (dn/h_n)^2. A candidate is kept if d <= radius_factor
    or it is in the 3x3 block of grid neighbours. Quadrant balance: each
    half-plane dt < 0, dt > 0, dn < 0, dn > 0 (dn < 0 not for wall points,
    which have the body there) then receives the nearest further candidates
    lying clearly inside it (|component| >= 0.05 |offset|) until it holds
    two. Rows are ordered by d, ties by index, at most max_degree entries.
    """
    n = W * (L + 1)
    offs = [(di, dj) for dj in range(-reach, reach + 1) for di in range(-reach, reach + 1)
            if di or dj]
    D = len(offs)
    deg = np.zeros(n, dtype=np.int64)
    rows = np.full((n, max_degree), -1, dtype=np.int32)
    r2 = radius_factor * radius_factor
    big = np.iinfo(np.int64).max

    def rows_of(s):
        # the rows of points [s, e): written to disjoint slices, so chunks run concurrently
        e = min(n, s + chunk)
        m = e - s
        p = np.arange(s, e)
        i = p % W
        j = p // W
        cand = np.empty((m, D), dtype=np.int64)
        blk = np.empty(D, dtype=bool)
        for k, (di, dj) in enumerate(offs):
            jj = j + dj
            cand[:, k] = np.where((jj >= 0) & (jj <= L), jj * W + (i + di) % W, -1)
            blk[k] = abs(di) <= 1 and abs(dj) <= 1
        valid = cand >= 0
        cs = np.where(valid, cand, 0)
        dx = x[cs] - x[p, None]
        dy = y[cs] - y[p, None]
        dt = dx * fny[p, None] - dy * fnx[p, None]
        dn = dx * fnx[p, None] + dy * fny[p, None]
        d2 = (dt / ht[p, None]) ** 2 + (dn / hn[p, None]) ** 2
        keep = valid & (blk[None, :] | (d2 <= r2))
        dist = np.sqrt(dx * dx + dy * dy)
        halves = [dt < -0.05 * dist, dt > 0.05 * dist, dn < -0.05 * dist, dn > 0.05 * dist]
        for h, inside in enumerate(halves):
            inside = inside & valid
            if h == 2:
                inside = inside & (flags[p, None] != 1)
            have = (keep & inside).sum(axis=1, keepdims=True)
            need = np.maximum(0, 2 - have)
            pool = inside & ~keep
            dp = np.where(pool, d2, np.inf)
            # admit the `need` nearest, and any candidate tied with the last
            # one admitted (mirror images of a point on the symmetry axis)
            ds = np.sort(dp, axis=1)
            cut = np.take_along_axis(ds, np.maximum(need - 1, 0), 1)
            keep |= pool & (need > 0) & (dp <= cut)
        # cap: block members first, then by distance; a tie group that the
        # cap would split (mirror images) is dropped whole
        dk = np.where(keep, d2, np.inf)
        nb = ~blk[None, :].repeat(m, 0)
        o = np.lexsort((np.where(keep, cand, big), dk, nb), axis=1)
        if D > max_degree:
            dso = np.take_along_axis(dk, o, 1)
            nbo = np.take_along_axis(nb, o, 1)
            last_d, last_b = dso[:, max_degree - 1:max_degree], nbo[:, max_degree - 1:max_degree]
            next_d, next_b = dso[:, max_degree:max_degree + 1], nbo[:, max_degree:max_degree + 1]
            split = np.isfinite(next_d) & (next_d == last_d) & (next_b == last_b)
            in_cap = np.zeros_like(keep)
            np.put_along_axis(in_cap, o[:, :max_degree], True, 1)
            keep &= in_cap & ~(split & (dk == last_d) & (nb == last_b))
        dk = np.where(keep, d2, np.inf)
        o = np.lexsort((np.where(keep, cand, big), dk), axis=1)[:, :max_degree]
        ck = np.take_along_axis(np.where(keep, cand, -1), o, 1)
        deg[s:e] = keep.sum(axis=1)
        rows[s:e] = ck.astype(np.int32)

    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1))) as ex:
        list(ex.map(rows_of, range(0, n, chunk)))
    offsets = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=offsets[1:])
    mask = np.arange(max_degree)[None, :] < deg[:, None]
    return offsets.astype(np.int32), rows[mask].astype(np.int32)


def naca0012_cloud(W: int = 320, L: int = 30, seed: int = 2403_13287,
                   jitter: float = 0.10, radius: float = 15.0,
                   mirror: bool = False, shuffle: bool = False,
                   radius_factor: float = 1.8, max_degree: int = _MAX_DEGREE,
                   ray_smoothing: int | None = None):
    """Build a synthetic NACA 0012 cloud of W*(L+1) points.

    Returns a dict with float64 arrays x, y, nx, ny; int32 flags; int32 CSR
    connectivity nbr_offsets (n+1) and nbr_idx (nnz); int32 wall_order (the
    wall points counter-clockwise from the trailing edge); and the grid sizes.
    `mirror` draws the jitter on the upper half and reflects it, so the cloud
    is mirror-symmetric about y = 0 (points on the axis move along it only).
    `shuffle` applies a seeded random permutation of the point order.
    """
    if L < 2:
        raise ValueError("need L >= 2 layers")
    if ray_smoothing is None:
        ray_smoothing = max(8, W // 4)
    rng = np.random.Generator(np.random.PCG64(seed))
    xw, yw, nxw, nyw = naca0012_wall(W)
    rxw, ryw = _ray_directions(nxw, nyw, ray_smoothing)
    half = W // 2
    lower = np.arange(half + 1, W)
    rxw[lower], ryw[lower] = rxw[W - lower], -ryw[W - lower]   # exact symmetry
    rxw[0], ryw[0], rxw[half], ryw[half] = 1.0, 0.0, -1.0, 0.0
    t = _ray_lengths(xw, yw, rxw, ryw, radius)
    seg = np.hypot(np.roll(xw, -1) - xw, np.roll(yw, -1) - yw)
    mean_wall_spacing = seg.mean()
    g = _growth_fractions(L, mean_wall_spacing / t.mean())
    # nominal grid, layer-major (j, i)
    X = xw[None, :] + (t[None, :] * g[:, None]) * rxw[None, :]
    Y = yw[None, :] + (t[None, :] * g[:, None]) * ryw[None, :]
    # the far-field layer sits exactly on the circle
    fx, fy = xw + t * rxw - _CENTRE[0], yw + t * ryw - _CENTRE[1]
    X[L] = _CENTRE[0] + radius * fx / np.hypot(fx, fy)
    Y[L] = _CENTRE[1] + radius * fy / np.hypot(fx, fy)
    if mirror:
        half = W // 2
        lower = np.arange(half + 1, W)
        X[:, lower] = X[:, W - lower]
        Y[:, lower] = -Y[:, W - lower]
        Y[:, 0] = 0.0
        Y[:, half] = 0.0
    ht = 0.5 * (np.hypot(np.roll(X, -1, 1) - X, np.roll(Y, -1, 1) - Y)
                + np.hypot(X - np.roll(X, 1, 1), Y - np.roll(Y, 1, 1)))
    dn = np.hypot(np.diff(X, axis=0), np.diff(Y, axis=0))
    hn = np.empty_like(X)
    hn[0] = dn[0]
    hn[L] = dn[L - 1]
    hn[1:L] = 0.5 * (dn[:-1] + dn[1:])
    # jitter (interior layers only)
    txw, tyw = ryw, -rxw
    a = rng.uniform(-1.0, 1.0, size=(L + 1, W))
    b = rng.uniform(-1.0, 1.0, size=(L + 1, W))
    if mirror:
        half = W // 2
        lower = np.arange(half + 1, W)
        # reflection maps the tangent to minus the mirrored tangent and the
        # normal to the mirrored normal
        a[:, lower] = -a[:, W - lower]
        b[:, lower] = b[:, W - lower]
        a[:, 0] = 0.0      # TE axis: tangent is vertical, keep on axis
        a[:, half] = 0.0   # LE axis
    dX = jitter * (a * ht * txw[None, :] + b * hn * rxw[None, :])
    dY = jitter * (a * ht * tyw[None, :] + b * hn * ryw[None, :])
    dX[0] = dX[L] = 0.0
    dY[0] = dY[L] = 0.0
    X = X + dX
    Y = Y + dY
    if mirror:
        half = W // 2
        Y[:, 0] = 0.0
        Y[:, half] = 0.0
    n = W * (L + 1)
    x = X.reshape(n).copy()
    y = Y.reshape(n).copy()
    nx = np.tile(rxw, L + 1)
    ny = np.tile(ryw, L + 1)
    nx[:W], ny[:W] = nxw, nyw
    ffx = X[L] - _CENTRE[0]
    ffy = Y[L] - _CENTRE[1]
    ffr = np.hypot(ffx, ffy)
    nx[L * W:] = ffx / ffr
    ny[L * W:] = ffy / ffr
    flags = np.zeros(n, dtype=np.int32)
    flags[:W] = FLAG_WALL
    flags[L * W:] = FLAG_FARFIELD
    offsets, idx = _connectivity(x, y, W, L, flags, nx, ny, ht.reshape(n), hn.reshape(n),
                                 radius_factor, max_degree)
    wall_order = np.arange(W, dtype=np.int32)
    if shuffle:
        perm = np.random.Generator(np.random.PCG64(seed + 1)).permutation(n)  # new -> old
        inv = np.empty(n, dtype=np.int64)
        inv[perm] = np.arange(n)                                              # old -> new
        x, y, nx, ny, flags = x[perm], y[perm], nx[perm], ny[perm], flags[perm]
        deg = np.diff(offsets.astype(np.int64))[perm]
        new_off = np.zeros(n + 1, dtype=np.int64)
        np.cumsum(deg, out=new_off[1:])
        starts = offsets[:-1].astype(np.int64)[perm]
        pos = np.repeat(starts - new_off[:-1], deg) + np.arange(new_off[-1])
        idx = inv[idx[pos]].astype(np.int32)
        offsets = new_off.astype(np.int32)
        wall_order = inv[wall_order].astype(np.int32)
    return {
        "n": n, "W": W, "L": L,
        "x": np.ascontiguousarray(x), "y": np.ascontiguousarray(y),
        "nx": np.ascontiguousarray(nx), "ny": np.ascontiguousarray(ny),
        "flags": flags, "nbr_offsets": offsets, "nbr_idx": idx,
        "wall_order": wall_order,
    }


# Named workloads: (W, L). Point counts are W*(L+1). Second-order workloads use
# near-isotropic layering (L ~ W ln(30)/(2 pi), log-polar): on strongly
# stretched outer cells the Jacobi inner iterations of E15 go unstable.
CLOUDS = {
    "naca0012_10k": (320, 30),        # 9,920 points (first-order workload)
    "naca0012_160k": (512, 311),      # 159,744 points
    "naca0012_640k": (1024, 624),     # 640,000 points
    "naca0012_2p5m": (2560, 975),     # 2,498,560 points
    "naca0012_10m": (5120, 1952),     # 9,999,360 points
}


def smooth_state(cloud, mach, aoa_deg, amp=0.05, seed=0, gamma=1.4):
    """A seeded smooth perturbation of the free stream (rho = 1, p = 1/gamma,
    |u| = mach) as conserved variables U[4, n]: density, velocity and pressure
    each vary by about `amp` on a scale of a chord. Far-field points carry the
    free stream, wall points have no normal momentum. An input for tests and
    timing: every stencil sees a non-uniform state."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x, y = cloud["x"], cloud["y"]
    k = rng.uniform(1.0, 3.0, 4)
    ph = rng.uniform(0.0, 2.0 * np.pi, 4)
    a = np.radians(aoa_deg)
    rho = 1.0 + amp * np.sin(k[0] * x + ph[0]) * np.cos(k[1] * y + ph[1])
    u = mach * np.cos(a) + amp * np.cos(k[2] * y + ph[2])
    v = mach * np.sin(a) + amp * np.sin(k[3] * x + ph[3])
    p = (1.0 + amp * np.cos(k[1] * x - k[0] * y)) / gamma
    far = cloud["flags"] == FLAG_FARFIELD
    rho[far], u[far], v[far], p[far] = 1.0, mach * np.cos(a), mach * np.sin(a), 1.0 / gamma
    U = np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])
    wall = cloud["flags"] == FLAG_WALL
    mn = U[1, wall] * cloud["nx"][wall] + U[2, wall] * cloud["ny"][wall]
    U[1, wall] -= mn * cloud["nx"][wall]
    U[2, wall] -= mn * cloud["ny"][wall]
    return np.ascontiguousarray(U)


def hicks_henne_basis(cloud, peaks=(0.2, 0.4, 0.6, 0.8), width=3.0):
    """Point displacements of 2*len(peaks) Hicks-Henne bumps (R. Hicks and
    P. Henne, J. Aircraft 15 (1978) 407-412) on a cloud built in grid order
    (not shuffled): B[k] is the y-displacement of every point per unit
    amplitude of bump k, so y(a) = y + a @ B. Bump k (peak position x_k,
    b(x) = sin(pi x^(ln 0.5 / ln x_k))^width on the chord x in [0, 1]) moves
    the upper surface outward for k < len(peaks), the lower surface outward
    after; interior points of the same grid column follow with the smooth
    decay (1 + cos(pi j / L)) / 2 of their layer j, so the far-field layer
    stays put. The frame normals are not changed."""
    W, L = cloud["W"], cloud["L"]
    n = cloud["n"]
    if n != W * (L + 1):
        raise ValueError("hicks_henne_basis needs a cloud in grid order (shuffle=False)")
    xw, yw = cloud["x"][:W], cloud["y"][:W]
    half = W // 2
    col = np.arange(n) % W
    layer = np.arange(n) // W
    decay = 0.5 * (1.0 + np.cos(np.pi * layer / L))
    xc = np.clip(xw, 0.0, 1.0)
    upper = np.zeros(W, dtype=bool)
    upper[1:half] = True
    lower = np.zeros(W, dtype=bool)
    lower[half + 1:] = True
    B = np.zeros((2 * len(peaks), n))
    for k, xp in enumerate(peaks):
        m = np.log(0.5) / np.log(xp)
        b = np.sin(np.pi * xc ** m) ** width
        bu = np.where(upper, b, 0.0)
        bl = np.where(lower, -b, 0.0)
        B[k] = bu[col] * decay
        B[len(peaks) + k] = bl[col] * decay
    return B
