"""lskum_residual_vjp against the complex-step derivative oracle (needs a GPU).

Entry-wise: sampled entries of U_bar, x_bar and y_bar are <R_bar, J e_k>
from the oracle, one complex-step residual each. At larger sizes: the
dot-product identity <R_bar, J v> = <J^T R_bar, v> with the oracle's J v.

Tolerance: both sides compute the exact derivative up to rounding; the
entries are sums over a point's two-ring of products whose magnitudes the
check bounds by the entry's own absolute-value sum, so the comparison is
relative to max|entry| over the sample at 1e-10 (rounding of the E11/E15
closures is a few ulp times the stencil condition number, ~1e3 here).
"""
import numpy as np
import pytest

import oracle
from oracle import lskum_jvp
from paper_2403_13287_gb300.cloudgen import naca0012_cloud, smooth_state

pytestmark = pytest.mark.gpu

MACH, AOA = 0.63, 2.0


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _solver(cloud, **kw):
    from paper_2403_13287_gb300.lskum import Solver
    kw.setdefault("mach", MACH)
    kw.setdefault("aoa_deg", AOA)
    return Solver(cloud, **kw)


@pytest.fixture(scope="module")
def small():
    c = naca0012_cloud(130, 24, seed=11)        # 3250 points, several blocks and a ragged tail
    return c, oracle.split_stencils(c)


def _sample(n, rng, m_u=48, m_xy=24):
    pts = rng.choice(n, size=m_u, replace=False)
    ent = [("U", int(rng.integers(4)), int(p)) for p in pts]
    ent += [("x", int(p)) for p in rng.choice(n, size=m_xy, replace=False)]
    ent += [("y", int(p)) for p in rng.choice(n, size=m_xy, replace=False)]
    return ent


def _pick(ent, Ub, xb, yb):
    out = []
    for e in ent:
        if e[0] == "U":
            out.append(Ub[e[1], e[2]])
        elif e[0] == "x":
            out.append(xb[e[1]])
        else:
            out.append(yb[e[1]])
    return np.array(out)


@pytest.mark.parametrize("order,reorder", [(1, 0), (2, 0), (2, 1)])
def test_vjp_entries_match_the_oracle(small, order, reorder):
    c, mask = small
    n = c["n"]
    U = smooth_state(c, MACH, AOA, amp=0.05, seed=3)
    rng = np.random.default_rng(100 + order)
    Rb = rng.standard_normal((4, n))
    s = _solver(c, order=order, inner_iters=3, reorder=reorder)
    Ub, xb, yb = (t.cpu().numpy() for t in s.residual_vjp(_dev(Rb), _dev(U)))
    ent = _sample(n, rng)
    want = lskum_jvp.vjp_entries(c, mask, U, Rb, ent, order=order, inner=3)
    got = _pick(ent, Ub, xb, yb)
    scale = np.max(np.abs(want))
    assert scale > 0
    assert np.all(np.abs(got - want) <= 1e-10 * scale), np.max(np.abs(got - want)) / scale


def test_vjp_of_the_context_state_and_far_field(small):
    """U = NULL uses the context's state; far-field rows of R_bar have no effect (R = 0 there)."""
    c, _ = small
    n = c["n"]
    U = smooth_state(c, MACH, AOA, amp=0.05, seed=4)
    s = _solver(c, order=2)
    s.set_state(U)
    rng = np.random.default_rng(9)
    Rb = rng.standard_normal((4, n))
    a = [t.cpu().numpy() for t in s.residual_vjp(_dev(Rb))]
    b = [t.cpu().numpy() for t in s.residual_vjp(_dev(Rb), _dev(U))]
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    Rb2 = Rb.copy()
    Rb2[:, c["flags"] == 2] = 123.0
    d = [t.cpu().numpy() for t in s.residual_vjp(_dev(Rb2), _dev(U))]
    for x, y in zip(b, d):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("order", [1, 2])
def test_dot_product_identity_at_160k(order):
    """<R_bar, J v> (oracle, complex step) = <J^T R_bar, v> (GPU) on the 160k-point cloud.

    The coordinate product runs through the inverse least-squares normal
    matrices of the sub-stencils, whose condition number reaches 1.3e10 at
    the four leading- and trailing-edge wall points of this cloud (x+-
    sub-stencils); rounding amplified there is about 1e-10 of the
    first-order coordinate product, so that one takes 1e-9 (a wrong term
    would be off by 1e-3 or more)."""
    c = naca0012_cloud(512, 311)
    mask = oracle.split_stencils(c)
    n = c["n"]
    U = smooth_state(c, MACH, AOA, amp=0.05, seed=5)
    rng = np.random.default_rng(31)
    Rb = rng.standard_normal((4, n))
    s = _solver(c, order=order, inner_iters=3, reorder=1)
    Ub, xb, yb = (t.cpu().numpy() for t in s.residual_vjp(_dev(Rb), _dev(U)))
    vU = rng.standard_normal((4, n)) * np.abs(U)
    h = 1e-3 * np.median(np.abs(np.diff(c["x"])))
    vx = rng.standard_normal(n) * h
    vy = rng.standard_normal(n) * h
    for dU, dx, dy, lhs_gpu, tol in ((vU, None, None, np.sum(Ub * vU), 1e-10),
                                     (None, vx, vy, np.sum(xb * vx) + np.sum(yb * vy), 1e-9 if order == 1 else 1e-10)):
        Jv = lskum_jvp.jvp(c, mask, U, dU=dU, dx=dx, dy=dy, order=order, inner=3)
        lhs = np.sum(Rb * Jv)
        mag = np.sum(np.abs(Rb * Jv))
        assert abs(lhs_gpu - lhs) <= tol * mag, (lhs_gpu, lhs, mag)


def test_vjp_is_deterministic_and_precision_independent(small):
    c, _ = small
    n = c["n"]
    U = smooth_state(c, MACH, AOA, amp=0.05, seed=6)
    Rb = np.random.default_rng(4).standard_normal((4, n))
    f64 = _solver(c, order=2, reorder=1)
    a = [t.cpu().numpy() for t in f64.residual_vjp(_dev(Rb), _dev(U))]
    b = [t.cpu().numpy() for t in f64.residual_vjp(_dev(Rb), _dev(U))]
    mixed = _solver(c, order=2, reorder=1, precision=1)
    m = [t.cpu().numpy() for t in mixed.residual_vjp(_dev(Rb), _dev(U))]
    for x, y, z in zip(a, b, m):
        assert np.array_equal(x, y)
        assert np.array_equal(x, z)        # the VJP runs in FP64 on the same geometry


def test_vjp_arguments(small):
    from paper_2403_13287_gb300.lskum import LskumError, LSKUM_ERR_ARG
    c, _ = small
    Rb = _dev(np.zeros((4, c["n"])))
    # the limiter is differentiated by the FP64 product only
    sm = _solver(c, order=2, limiter_K=1.0, precision=1)
    with pytest.raises(LskumError) as e:
        sm.residual_vjp(Rb, fp32=True)
    assert e.value.status == LSKUM_ERR_ARG
    sk = _solver(c, order=2, boundary=1)
    with pytest.raises(LskumError) as e:
        sk.residual_vjp(Rb)
    assert e.value.status == LSKUM_ERR_ARG
    s1 = _solver(c, order=2)
    Ub, xb, yb = s1.residual_vjp(Rb, want_xy=False)
    assert xb is None and yb is None and float(Ub.abs().max()) == 0.0


def test_autograd_function(small):
    import torch
    from paper_2403_13287_gb300.lskum import residual_fn
    c, _ = small
    n = c["n"]
    s = _solver(c, order=2)
    U0 = smooth_state(c, MACH, AOA, amp=0.05, seed=7)
    U = _dev(U0).requires_grad_(True)
    xy = _dev(np.stack([c["x"], c["y"]])).requires_grad_(True)
    W = _dev(np.random.default_rng(8).standard_normal((4, n)))
    R = residual_fn(s, U, xy)
    assert torch.equal(R.detach(), s.residual(_dev(U0)))
    (R * W).sum().backward()
    Ub, xb, yb = s.residual_vjp(W, _dev(U0))
    assert torch.equal(U.grad, Ub)
    assert torch.equal(xy.grad, torch.stack([xb, yb]))


@pytest.mark.parametrize("order", [1, 2])
def test_fp32_vjp_agrees_with_fp64(small, order):
    """The FP32 product (mixed context) against the FP64 product, entry by
    entry relative to each output's largest entry, and by the dot-product
    identity against the oracle. U_bar agrees to FP32 rounding amplified by
    the stencil closures (2e-4); the coordinate cotangents carry the weight
    cotangents R_bar . (G(q~_i) - G(q~_0)), where the FP32 flux difference
    cancels, so they agree only to 2e-2 (use the FP64 product for them)."""
    from paper_2403_13287_gb300.lskum import LskumError, LSKUM_ERR_ARG
    c, mask = small
    n = c["n"]
    U = smooth_state(c, MACH, AOA, amp=0.05, seed=12)
    Rb = np.random.default_rng(40 + order).standard_normal((4, n))
    s64 = _solver(c, order=order, inner_iters=3, reorder=1)
    s32 = _solver(c, order=order, inner_iters=3, reorder=1, precision=1)
    a = [t.cpu().numpy() for t in s64.residual_vjp(_dev(Rb), _dev(U))]
    b = [t.cpu().numpy() for t in s32.residual_vjp(_dev(Rb), _dev(U), fp32=True)]
    for x, y, tol in zip(a, b, (2e-4, 2e-2, 2e-2)):
        scale = np.abs(x).max(axis=-1, keepdims=True)
        assert np.all(np.abs(x - y) <= tol * scale), np.max(np.abs(x - y) / scale)
    vU = np.random.default_rng(3).standard_normal((4, n)) * np.abs(U)
    Jv = lskum_jvp.jvp(c, mask, U, dU=vU, order=order, inner=3)
    ref = np.sum(Rb * Jv)
    assert abs(np.sum(b[0] * vU) - ref) <= 2e-4 * np.sum(np.abs(Rb * Jv))
    with pytest.raises(LskumError) as e:
        s64.residual_vjp(_dev(Rb), _dev(U), fp32=True)
    assert e.value.status == LSKUM_ERR_ARG


# ---------------------------------------------------------------------------
# the limiter (Venkatakrishnan, limiter_K > 0)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("K,reorder", [(1.0, 0), (1.0, 1), (0.3, 1)])
def test_limited_vjp_entries_match_the_oracle(small, K, reorder):
    """The limiter is piecewise smooth; both sides differentiate the branch
    the forward takes, with the same first-wins choices (stencil extremes,
    the largest reconstruction shift, the nearest neighbour), so ties such
    as the far-field points' equal states give the same one-sided
    derivative on both sides."""
    c, mask = small
    n = c["n"]
    U = smooth_state(c, 0.85, 1.0, amp=0.05, seed=13)
    rng = np.random.default_rng(200 + reorder)
    Rb = rng.standard_normal((4, n))
    s = _solver(c, order=2, inner_iters=3, reorder=reorder, limiter_K=K, mach=0.85, aoa_deg=1.0)
    Ub, xb, yb = (t.cpu().numpy() for t in s.residual_vjp(_dev(Rb), _dev(U)))
    ent = _sample(n, rng)
    want = lskum_jvp.vjp_entries(c, mask, U, Rb, ent, order=2, inner=3, limiter=K)
    got = _pick(ent, Ub, xb, yb)
    scale = np.max(np.abs(want))
    assert scale > 0
    assert np.all(np.abs(got - want) <= 1e-10 * scale), np.max(np.abs(got - want)) / scale
    # the limiter's terms matter here: the unlimited product differs
    s0 = _solver(c, order=2, inner_iters=3, reorder=reorder, mach=0.85, aoa_deg=1.0)
    U0b = s0.residual_vjp(_dev(Rb), _dev(U))[0].cpu().numpy()
    assert np.max(np.abs(U0b - Ub)) > 1e-3 * np.max(np.abs(Ub))


def test_limited_dot_product_identity_at_160k():
    """<R_bar, J v> (oracle, complex step, limiter K = 1) = <J^T R_bar, v>
    (GPU) on the 160k-point cloud at M 1.2 with the limiter active; the
    directions leave the far-field states and the wall points fixed (tied
    choices there are kinks, where a directional derivative has two sides)."""
    c = naca0012_cloud(512, 311)
    mask = oracle.split_stencils(c)
    n = c["n"]
    U = smooth_state(c, 1.2, 0.0, amp=0.05, seed=15)
    rng = np.random.default_rng(41)
    Rb = rng.standard_normal((4, n))
    s = _solver(c, order=2, inner_iters=3, reorder=1, limiter_K=1.0, mach=1.2, aoa_deg=0.0)
    Ub, xb, yb = (t.cpu().numpy() for t in s.residual_vjp(_dev(Rb), _dev(U)))
    far, wall = c["flags"] == 2, c["flags"] == 1
    vU = rng.standard_normal((4, n)) * np.abs(U)
    vU[:, far] = 0.0
    h = 1e-3 * np.median(np.abs(np.diff(c["x"])))
    vx = rng.standard_normal(n) * h
    vy = rng.standard_normal(n) * h
    vx[wall] = 0.0
    vy[wall] = 0.0
    for dU, dx, dy, lhs_gpu in ((vU, None, None, np.sum(Ub * vU)),
                                (None, vx, vy, np.sum(xb * vx) + np.sum(yb * vy))):
        Jv = lskum_jvp.jvp(c, mask, U, dU=dU, dx=dx, dy=dy, order=2, inner=3, limiter=1.0)
        lhs = np.sum(Rb * Jv)
        mag = np.sum(np.abs(Rb * Jv))
        assert abs(lhs_gpu - lhs) <= 1e-10 * mag, (lhs_gpu, lhs, mag)
