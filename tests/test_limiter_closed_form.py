"""The q-derivative kernels apply Venkatakrishnan's limiter in a closed form:
phi = min over every reconstruction shift +-d_e (both signs, all edges) of
f(D, d), with D the stencil maximum minus q_0 for a positive shift and the
minimum minus q_0 for a negative one, equals f(x_m, d_m) when
x_m = min(D+, -D-) < 2 d_m (d_m the largest |d_e|), and 1 otherwise.
Checked here, without a GPU, against the brute-force minimum over the shifts
on random stencils, including the degenerate cases (a side with no spread,
all shifts zero)."""
import numpy as np


def f(D, d, eps2):
    # Venkatakrishnan's function of the limiter (the form the oracle evaluates)
    return (D * D + eps2 + 2.0 * D * d) / (D * D + 2.0 * d * d + D * d + eps2)


def brute(Dp, Dm, shifts, eps2):
    phi = 1.0
    for h in shifts:
        for d in (h, -h):
            if d > 0.0:
                phi = min(phi, f(Dp, d, eps2))
            elif d < 0.0:
                phi = min(phi, f(Dm, d, eps2))
    return phi


def closed(Dp, Dm, shifts, eps2):
    dm = max(abs(h) for h in shifts)
    xm = min(Dp, -Dm)
    return f(xm, dm, eps2) if xm < 2.0 * dm else 1.0


def test_closed_form_equals_the_minimum_over_all_shifts():
    rng = np.random.default_rng(2024)
    worst = 0.0
    for trial in range(20000):
        k = int(rng.integers(1, 12))
        scale = 10.0 ** rng.uniform(-6, 1)
        shifts = rng.normal(0.0, scale, k)
        Dp = abs(rng.normal(0.0, scale * rng.uniform(0.1, 4.0)))
        Dm = -abs(rng.normal(0.0, scale * rng.uniform(0.1, 4.0)))
        if trial % 7 == 0:
            Dp = 0.0                         # q_0 is the stencil maximum
        if trial % 11 == 0:
            Dm = 0.0                         # q_0 is the stencil minimum
        if trial % 13 == 0:
            shifts[:] = 0.0                  # no shift at all: phi = 1
        eps2 = (rng.uniform(0.0, 2.0) * scale) ** 3
        b = brute(Dp, Dm, shifts, eps2)
        c = closed(Dp, Dm, shifts, eps2)
        assert 0.0 <= c <= 1.0
        worst = max(worst, abs(b - c))
    # equal up to rounding of f (a few units in the last place of 1)
    assert worst <= 4e-16, worst


def test_closed_form_threshold_is_exact():
    """f(x, d) < 1 exactly when x < 2d: N - M = d (x - 2d), eps cancels."""
    for d in (1e-3, 0.5, 7.0):
        for eps2 in (0.0, 1e-9, 0.3):
            assert abs(f(2.0 * d, d, eps2) - 1.0) <= 2e-16
            assert f(1.999 * d, d, eps2) < 1.0
            assert f(2.001 * d, d, eps2) > 1.0
