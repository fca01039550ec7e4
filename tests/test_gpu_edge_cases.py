"""Edge cases of the CUDA path against the oracle (needs a GPU): the largest
stencils the library takes (25 neighbours), rows of uneven length in the
same 32-point slice, frames rotated at random, a degree beyond the limit,
an empty cloud, and the smallest stencil in the mixed form.

Tolerances as in test_gpu_parity (FP64: 1e-12 S) and test_gpu_mixed
(mixed: 3e-5 S), S the magnitude of the summed terms before cancellation.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _solver(cloud, **kw):
    from paper_2403_13287_gb300.lskum import Solver
    return Solver(cloud, **kw)


def knn_cloud(m=23, k_max=25, seed=1):
    """A jittered m x m grid on the unit square (529 points: 16 full warps
    and a ragged tail of 17), each point joined to its
    k nearest neighbours with k cycling through 12..k_max (rows of uneven
    length), random unit frame normals; the outer ring is far field."""
    rng = np.random.default_rng(seed)
    g = np.linspace(0.0, 1.0, m)
    X, Y = np.meshgrid(g, g)
    h = g[1] - g[0]
    x = (X + rng.uniform(-0.2, 0.2, X.shape) * h).ravel()
    y = (Y + rng.uniform(-0.2, 0.2, Y.shape) * h).ravel()
    n = x.size
    ring = ((X == 0) | (X == 1) | (Y == 0) | (Y == 1)).ravel()
    d2 = (x[:, None] - x[None, :]) ** 2 + (y[:, None] - y[None, :]) ** 2
    np.fill_diagonal(d2, np.inf)
    order = np.argsort(d2, axis=1, kind="stable")
    ks = 12 + (np.arange(n) % (k_max - 11))
    ks[ring] = k_max
    rows = [order[p, :ks[p]] for p in range(n)]
    off = np.zeros(n + 1, np.int32)
    off[1:] = np.cumsum([len(r) for r in rows])
    th = rng.uniform(0, 2 * np.pi, n)
    return {"n": n, "x": x, "y": y, "nx": np.cos(th), "ny": np.sin(th),
            "flags": np.where(ring, 2, 0).astype(np.int32), "nbr_offsets": off,
            "nbr_idx": np.concatenate(rows).astype(np.int32), "wall_order": np.zeros(0, np.int32)}


def _state(cloud, seed=3, amp=0.05):
    rng = np.random.default_rng(seed)
    x, y = cloud["x"], cloud["y"]
    k = rng.uniform(1.0, 3.0, 4)
    rho = 1.0 + amp * np.sin(k[0] * x) * np.cos(k[1] * y)
    u = 0.6 + amp * np.cos(k[2] * y)
    v = 0.1 + amp * np.sin(k[3] * x)
    p = (1.0 + amp * np.cos(k[1] * x - k[0] * y)) / 1.4
    return np.stack([rho, rho * u, rho * v, p / 0.4 + 0.5 * rho * (u * u + v * v)])


@pytest.fixture(scope="module")
def knn():
    c = knn_cloud()
    return c, oracle.split_stencils(c)


def test_knn_cloud_has_the_largest_and_uneven_rows(knn):
    c, _ = knn
    deg = np.diff(c["nbr_offsets"])
    assert deg.max() == 25 and deg.min() == 12
    # a 32-point slice mixes short and long rows
    assert len(set(deg[:32])) > 5


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("reorder", [0, 1, 2])
def test_residual_on_the_largest_stencils(knn, precision, order, reorder):
    c, mask = knn
    U = _state(c)
    s = _solver(c, order=order, inner_iters=3, precision=precision, reorder=reorder, mach=0.6, aoa_deg=9.0)
    assert np.array_equal(s.stencil_masks(), mask)
    R = s.residual(_dev(U)).cpu().numpy()
    Ro, S = oracle.residual(c, mask, U, order=order, inner=3, want_scale=True)
    tol = 1e-12 if precision == 0 else 3e-5
    assert np.all(np.abs(R - Ro) <= tol * S), np.max(np.abs(R - Ro) / S)


def test_trajectory_on_the_largest_stencils(knn):
    c, mask = knn
    U0 = _state(c)
    far = c["flags"] == 2
    U0[:, far] = oracle.freestream(0.6, 9.0)[:, None]
    s = _solver(c, order=2, inner_iters=3, time_scheme=1, mach=0.6, aoa_deg=9.0, reorder=1)
    s.set_state(U0)
    s.step(5)
    Uo, _ = oracle.solve(c, mask, U0.copy(), 5, order=2, inner=3, scheme=1, cfl=0.2, mach=0.6, aoa_deg=9.0)
    assert np.max(np.abs(s.get_state() - Uo) / np.abs(Uo).max(axis=1, keepdims=True)) <= 1e-10


def test_degree_limit_and_empty_cloud(knn):
    from paper_2403_13287_gb300.lskum import LskumError, LSKUM_ERR_ARG, LSKUM_ERR_CONNECTIVITY
    c, _ = knn
    # one row with 26 neighbours
    n = c["n"]
    rows = [list(c["nbr_idx"][c["nbr_offsets"][p]:c["nbr_offsets"][p + 1]]) for p in range(n)]
    extra = [j for j in range(n) if j != 0 and j not in rows[0]][:26 - len(rows[0])]
    rows[0] = rows[0] + extra
    off = np.zeros(n + 1, np.int32)
    off[1:] = np.cumsum([len(r) for r in rows])
    bad = dict(c, nbr_offsets=off, nbr_idx=np.concatenate(rows).astype(np.int32))
    with pytest.raises(LskumError) as e:
        _solver(bad)
    assert e.value.status == LSKUM_ERR_CONNECTIVITY
    empty = {"n": 0, "x": np.zeros(0), "y": np.zeros(0), "nx": np.zeros(0), "ny": np.zeros(0),
             "flags": np.zeros(0, np.int32), "nbr_offsets": np.zeros(1, np.int32),
             "nbr_idx": np.zeros(0, np.int32), "wall_order": np.zeros(0, np.int32)}
    with pytest.raises(LskumError) as e:
        _solver(empty)
    assert e.value.status == LSKUM_ERR_ARG


def cartesian9():
    """The nine-point Cartesian stencil: one interior point, eight far-field
    points joined to their grid neighbours."""
    h = 0.01
    offs = [(-1, -1), (-1, 0), (-1, 1), (0, -1), (0, 1), (1, -1), (1, 0), (1, 1)]
    pts = [(0.0, 0.0)] + [(h * a, h * b) for a, b in offs]
    rows = [list(range(1, 9))]
    for a, b in offs:
        rows.append(sorted([0] + [j + 1 for j, (cc, d) in enumerate(offs)
                                  if (cc, d) != (a, b) and abs(cc - a) <= 1 and abs(d - b) <= 1]))
    off = np.zeros(10, np.int32)
    off[1:] = np.cumsum([len(r) for r in rows])
    return {"n": 9, "x": np.array([p[0] for p in pts]), "y": np.array([p[1] for p in pts]),
            "nx": np.zeros(9), "ny": np.ones(9), "flags": np.array([0] + [2] * 8, np.int32),
            "nbr_offsets": off, "nbr_idx": np.array([i for r in rows for i in r], np.int32),
            "wall_order": np.zeros(0, np.int32)}


def test_smallest_stencil_in_the_mixed_form():
    cloud = cartesian9()
    U = _state(cloud, amp=0.2)
    for order in (1, 2):
        s = _solver(cloud, order=order, precision=1, mach=0.5, aoa_deg=10.0)
        R = s.residual(_dev(U)).cpu().numpy()
        Ro, S = oracle.residual(cloud, oracle.split_stencils(cloud), U, order=order, inner=3, want_scale=True)
        assert np.all(np.abs(R - Ro) <= 3e-5 * S + 1e-300)


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_of_ragged_cases(knn, precision):
    """A batch whose cases end inside warps and blocks: 36, 529 and 49
    points (a case needs at least 32, so a warp spans at most two cases).
    The residual of each case against the oracle, and five iterations
    against single-case contexts (bitwise)."""
    from paper_2403_13287_gb300.lskum import Solver, LskumError, LSKUM_ERR_ARG
    c, _ = knn
    a, b = knn_cloud(m=6, seed=2), knn_cloud(m=7, seed=3)
    cases = [(a, 0.5, 10.0), (c, 0.6, 9.0), (b, 1.3, -4.0)]
    kw = dict(order=2, inner_iters=3, time_scheme=1, precision=precision, reorder=1)
    B = Solver.batch(cases, **kw)
    Us = [_state(cl, seed=50 + k, amp=0.1) for k, (cl, m, al) in enumerate(cases)]
    R = B.residual(_dev(np.concatenate(Us, axis=1))).cpu().numpy()
    tol = 1e-12 if precision == 0 else 3e-5
    for k, (cl, m, al) in enumerate(cases):
        first, count, _, _ = B.case_range(k)
        assert count == cl["n"]
        Ro, S = oracle.residual(cl, oracle.split_stencils(cl), Us[k], order=2, inner=3, want_scale=True)
        assert np.all(np.abs(R[:, first:first + count] - Ro) <= tol * S + 1e-300)
    U0 = []
    for cl, m, al in cases:
        u = _state(cl, seed=7, amp=0.05)
        u[:, cl["flags"] == 2] = oracle.freestream(m, al)[:, None]
        U0.append(u)
    B.set_state(np.concatenate(U0, axis=1))
    B.step(5)
    Ub = B.get_state()
    for k, (cl, m, al) in enumerate(cases):
        s = Solver(cl, mach=m, aoa_deg=al, **kw)
        s.set_state(U0[k])
        s.step(5)
        first, count, _, _ = B.case_range(k)
        assert np.array_equal(Ub[:, first:first + count], s.get_state())
    with pytest.raises(LskumError) as e:
        Solver.batch([(cartesian9(), 0.5, 0.0), (c, 0.6, 9.0)], **kw)
    assert e.value.status == LSKUM_ERR_ARG
