"""The oracle's OpenMP build (used to time it on all host cores and to run the
long converged solves) gives the serial build's results bit for bit: points
are independent within every pass and each point's sums stay serial."""
import numpy as np
import pytest

import oracle
from paper_2403_13287_gb300.cloudgen import naca0012_cloud, smooth_state


@pytest.fixture
def threads_back():
    yield
    oracle.set_threads(1)


def _runs(cloud, m, U):
    out = [oracle.residual(cloud, m, U, order=2, inner=3, limiter=1.0, want_scale=True, want_grad=True)]
    out.append(oracle.residual(cloud, m, U, order=2, inner=3, boundary=1, mach=0.85, aoa_deg=1.0))
    out.append(oracle.solve(cloud, m, U, 3, order=2, inner=3, scheme=1, cfl=0.3, mach=0.85, aoa_deg=1.0,
                            limiter=1.0))
    out.append(oracle.solve(cloud, m, U, 3, order=1, scheme=0, cfl=0.3, mach=0.85, aoa_deg=1.0))
    out.append(oracle.timestep(cloud, U, 0.3))
    return out


def _flat(x):
    if isinstance(x, (tuple, list)):
        return [a for y in x for a in _flat(y)]
    return [np.asarray(x)]


def test_openmp_build_is_bitwise_serial(threads_back):
    cloud = naca0012_cloud(64, 20, seed=3)
    m = oracle.split_stencils(cloud)
    U = smooth_state(cloud, 0.85, 1.0, amp=0.05, seed=2)
    assert oracle.set_threads(1) == 1
    serial = _flat(_runs(cloud, m, U))
    got = oracle.set_threads(4)
    if got == 1:
        pytest.skip("the compiler has no OpenMP")
    assert got == 4
    threaded = _flat(_runs(cloud, m, U))
    assert len(serial) == len(threaded)
    for a, b in zip(serial, threaded):
        assert np.array_equal(a, b)


def test_openmp_build_reports_errors(threads_back):
    """A non-physical state is refused by both builds."""
    cloud = naca0012_cloud(64, 20, seed=3)
    m = oracle.split_stencils(cloud)
    U = smooth_state(cloud, 0.85, 1.0, amp=0.05, seed=2)
    U[3, 100] = -1.0
    for t in (1, 4):
        oracle.set_threads(t)
        with pytest.raises(oracle.OracleError) as e:
            oracle.residual(cloud, m, U, order=2, inner=3)
        assert e.value.rc == oracle.ERR_NONPHYSICAL
