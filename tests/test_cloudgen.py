"""Checks of the seeded NACA 0012 cloud generator (inputs only, no GPU)."""
import numpy as np
import pytest

from paper_2403_13287_gb300.cloudgen import naca0012_cloud, naca0012_wall, CLOUDS


@pytest.fixture(scope="module")
def cloud():
    return naca0012_cloud(128, 16, seed=21)


def test_same_seed_same_bytes():
    a = naca0012_cloud(64, 10, seed=3)
    b = naca0012_cloud(64, 10, seed=3)
    c = naca0012_cloud(64, 10, seed=4)
    for k in ("x", "y", "nx", "ny", "flags", "nbr_offsets", "nbr_idx"):
        assert a[k].tobytes() == b[k].tobytes()
    assert a["x"].tobytes() != c["x"].tobytes()


def test_csr_well_formed(cloud):
    n = cloud["n"]
    off, idx = cloud["nbr_offsets"], cloud["nbr_idx"]
    assert off.dtype == np.int32 and idx.dtype == np.int32
    assert off[0] == 0 and off[-1] == len(idx) and np.all(np.diff(off) >= 3)
    assert np.all(np.diff(off) <= 25)
    assert idx.min() >= 0 and idx.max() < n
    rows = np.repeat(np.arange(n), np.diff(off))
    assert np.all(idx != rows)
    pairs = rows.astype(np.int64) * n + idx
    assert len(np.unique(pairs)) == len(pairs)
    # quadrant balance: interior points have at least two neighbours clearly
    # inside each half-plane of their frame
    dx = cloud["x"][idx] - cloud["x"][rows]
    dy = cloud["y"][idx] - cloud["y"][rows]
    nx, ny = cloud["nx"][rows], cloud["ny"][rows]
    dt, dn = dx * ny - dy * nx, dx * nx + dy * ny
    dist = np.hypot(dx, dy)
    interior = cloud["flags"][rows] == 0
    for half in (dt < -0.05 * dist, dt > 0.05 * dist, dn < -0.05 * dist, dn > 0.05 * dist):
        cnt = np.bincount(rows[half & interior], minlength=n)
        assert np.all(cnt[cloud["flags"] == 0] >= 2)


def test_geometry(cloud):
    W, L = cloud["W"], cloud["L"]
    x, y, f = cloud["x"], cloud["y"], cloud["flags"]
    wall = f == 1
    far = f == 2
    assert wall.sum() == W and far.sum() == W
    # wall points on the closed-trailing-edge NACA 0012 contour
    xt = x[wall]
    yt = 0.6 * (0.2969 * np.sqrt(xt) - 0.1260 * xt - 0.3516 * xt**2 + 0.2843 * xt**3 - 0.1036 * xt**4)
    assert np.allclose(np.abs(y[wall]), yt, atol=1e-15)
    assert np.allclose(np.hypot(x[far] - 0.5, y[far]), 15.0, rtol=1e-14)
    # unit normals; wall normals point out of the body (away from mid-chord axis)
    assert np.allclose(np.hypot(cloud["nx"], cloud["ny"]), 1.0, rtol=1e-14)
    # interior points lie outside the body and inside the far-field circle
    inner = f == 0
    r = np.hypot(x[inner] - 0.5, y[inner])
    assert r.max() < 15.0
    xi, yi = x[inner], y[inner]
    over = (xi >= 0) & (xi <= 1)
    xo = xi[over]
    yto = 0.6 * (0.2969 * np.sqrt(xo) - 0.1260 * xo - 0.3516 * xo**2 + 0.2843 * xo**3 - 0.1036 * xo**4)
    assert np.all(np.abs(yi[over]) > yto)


def test_wall_normals_are_outward_and_contour_closed():
    xw, yw, nxw, nyw = naca0012_wall(200)
    # signed area of the counter-clockwise contour is positive and close to the
    # exact area of NACA 0012 (0.0821...)
    area = 0.5 * np.sum(xw * np.roll(yw, -1) - np.roll(xw, -1) * yw)
    assert 0.080 < area < 0.083
    # the outward normal points away from the polygon: a small step along it
    # increases the distance to the chord line on the upper/lower surfaces
    up = yw > 1e-9
    assert np.all(nyw[up] > 0) and np.all(nyw[yw < -1e-9] < 0)


def test_mirror_cloud_is_symmetric():
    c = naca0012_cloud(64, 10, seed=9, mirror=True)
    W = c["W"]
    n = c["n"]
    i = np.arange(n) % W
    j = np.arange(n) // W
    mi = j * W + (W - i) % W
    assert np.array_equal(c["x"], c["x"][mi])
    assert np.array_equal(c["y"], -c["y"][mi])
    assert np.array_equal(c["nx"], c["nx"][mi])
    assert np.array_equal(c["ny"], -c["ny"][mi])
    off, idx = c["nbr_offsets"], c["nbr_idx"]
    for p in range(n):
        a = set(idx[off[p]:off[p + 1]].tolist())
        b = set(mi[idx[off[mi[p]]:off[mi[p] + 1]]].tolist())
        assert a == b


def test_shuffle_is_a_relabelling():
    a = naca0012_cloud(48, 8, seed=5)
    b = naca0012_cloud(48, 8, seed=5, shuffle=True)
    # same multiset of points; edges map through the permutation
    key_a = np.lexsort((a["y"], a["x"]))
    key_b = np.lexsort((b["y"], b["x"]))
    assert np.array_equal(a["x"][key_a], b["x"][key_b])
    old_of_new = np.empty(a["n"], np.int64)
    old_of_new[key_b] = key_a
    ea = set()
    for p in range(a["n"]):
        for e in range(a["nbr_offsets"][p], a["nbr_offsets"][p + 1]):
            ea.add((p, int(a["nbr_idx"][e])))
    eb = set()
    for p in range(b["n"]):
        for e in range(b["nbr_offsets"][p], b["nbr_offsets"][p + 1]):
            eb.add((int(old_of_new[p]), int(old_of_new[b["nbr_idx"][e]])))
    assert ea == eb
    assert np.array_equal(old_of_new[b["wall_order"]], a["wall_order"])


def test_named_workload_sizes():
    assert {k: W * (L + 1) for k, (W, L) in CLOUDS.items()} == {
        "naca0012_10k": 9920, "naca0012_160k": 159744, "naca0012_640k": 640000,
        "naca0012_2p5m": 2498560, "naca0012_10m": 9999360}
