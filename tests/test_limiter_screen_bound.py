"""The FP32 screen of the limiter's largest shift (no GPU).

The FP64 limiter pass finds d_m = max_e |h_e . (sx, sy)| per component. It
first bounds every edge's FP64 value with FP32 arithmetic and evaluates in
FP64 only the edges whose upper bound reaches the largest lower bound, which
keeps d_m bit for bit the plain loop's provided that, for every edge,

    fl32(v - c) <= |r|  and  fl32(v + c) >= |r|,

with r the FP64 value fma(h_x, sx, h_y * sy), v = |fl32(a + b)|,
a = fl32(hf_x sf), b = fl32(hf_y tf) (hf, sf, tf: h, sx, sy rounded to FP32)
and c = fl32(2^-20 (|a| + |b|) + 2^-120). This test restates that FP32
arithmetic in numpy (round to nearest, subnormals kept, as the kernel's
translation unit compiles) and checks both inequalities on random edges,
including strong cancellation, tiny and huge gradients, and underflow.
"""
import numpy as np

MARGIN = np.float32(2.0 ** -20)
TINY = np.float32(2.0 ** -120)


def _screen(h, s, t):
    """FP32 bounds (lo, hi) and the FP64 value |r| of each edge, as the
    kernel forms them (h: (m, 2) float64, s, t: (m,) float64)."""
    hf = h.astype(np.float32)
    sf = s.astype(np.float32)
    tf = t.astype(np.float32)
    a = hf[:, 0] * sf
    b = hf[:, 1] * tf
    v = np.abs(a + b)
    # fmaf(MARGIN, |a| + |b|, TINY): one rounding of the exact value; the
    # float64 product of two floats is exact, the sum with TINY is rounded
    # once more in float64, far below the slack of the bound
    S = np.abs(a) + np.abs(b)
    c = (np.float64(MARGIN) * S.astype(np.float64) + np.float64(TINY)).astype(np.float32)
    lo = v - c
    hi = v + c
    # FP64: fma(h_x, sx, h_y * sy), one rounding after an exact product plus
    # the rounded product h_y * sy (longdouble keeps the fused step exact
    # enough for a check at 2^-20 relative)
    p = h[:, 1] * t
    r = np.abs((h[:, 0].astype(np.longdouble) * s.astype(np.longdouble) + p.astype(np.longdouble)).astype(np.float64))
    return lo, hi, r


def _check(h, s, t):
    with np.errstate(over="ignore", invalid="ignore", under="ignore"):
        lo, hi, r = _screen(h, s, t)
    ok = np.isfinite(lo) & np.isfinite(hi)
    # non-finite bounds mark the edge as a candidate in the kernel: nothing to check
    assert np.all(lo[ok].astype(np.float64) <= r[ok])
    assert np.all(hi[ok].astype(np.float64) >= r[ok])
    return ok.mean()


def test_random_edges():
    rng = np.random.default_rng(0)
    m = 400_000
    h = rng.uniform(-2.0, 2.0, (m, 2)) * 10.0 ** rng.uniform(-4, 1, (m, 1))
    s = rng.standard_normal(m) * 10.0 ** rng.uniform(-6, 4, m)
    t = rng.standard_normal(m) * 10.0 ** rng.uniform(-6, 4, m)
    assert _check(h, s, t) == 1.0


def test_cancelling_edges():
    """h_x sx and h_y sy nearly opposite: the FP32 sum loses every digit,
    the margin (relative to |a| + |b|) must still cover it."""
    rng = np.random.default_rng(1)
    m = 400_000
    h = rng.uniform(0.1, 1.0, (m, 2))
    s = rng.standard_normal(m)
    t = -(h[:, 0] * s) / h[:, 1] * (1.0 + rng.uniform(-1e-6, 1e-6, m))
    assert _check(h, s, t) == 1.0


def test_tiny_and_huge_gradients():
    rng = np.random.default_rng(2)
    m = 200_000
    h = rng.uniform(-1.0, 1.0, (m, 2))
    # subnormal and underflowing FP32 values, and values near the FP32 maximum
    s = rng.standard_normal(m) * 10.0 ** rng.choice([-44.0, -40.0, -38.0, -30.0, 30.0, 37.0], m)
    t = rng.standard_normal(m) * 10.0 ** rng.choice([-44.0, -40.0, -38.0, -30.0, 30.0, 37.0], m)
    frac = _check(h, s, t)
    assert frac > 0.5            # most edges stay finite and are checked


def test_the_maximum_edge_is_always_kept():
    """On stencils of up to 25 edges with near-ties, the candidate set taken
    as the kernel takes it holds the edge of the FP64 maximum."""
    rng = np.random.default_rng(3)
    for _ in range(2000):
        deg = int(rng.integers(2, 26))
        h = rng.uniform(-1.0, 1.0, (deg, 2)) * 0.01
        g = rng.standard_normal(2) * 10.0 ** rng.uniform(-3, 3)
        # near-ties: copies of one edge perturbed in the last bits
        k = int(rng.integers(0, deg))
        h[rng.integers(0, deg, 3)] = h[k] * (1.0 + rng.uniform(-1e-15, 1e-15, (3, 1)))
        s = np.full(deg, g[0])
        t = np.full(deg, g[1])
        lo, hi, r = _screen(h, s, t)
        L = max(0.0, float(np.max(lo)))
        cand = ~(hi < np.float32(L))
        assert r[cand].max() == r.max()
