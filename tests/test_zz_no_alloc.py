"""The allocation-free q-derivative entry point against the context-based one.

lskum_q_derivatives_noalloc serves callers that cannot allocate device memory
where they call from (a caching allocator that owns the GPU's memory, a loop
that must not pay cudaMalloc's device synchronisation, a fixed budget); its
scratch is one static device array shared by every call. Two calls in a row
with different states must each agree with lskum_q_derivatives of a context
on the same state, and the FP64 CPU oracle's q-derivatives, within the
q-derivative tolerance of the parity tests (1e-12 of the summand scale of the
least-squares sum), so nothing left in the shared scratch by one call leaks
into the next. Arrays of the wrong size and malformed CSR rows are refused
before or by the kernels, without any read outside the caller's arrays.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2403_13287_gb300.cloudgen import naca0012_cloud

pytestmark = pytest.mark.gpu

GAMMA = 1.4


def _state(cloud, seed, amp=0.05, mach=0.7, aoa=3.0):
    rng = np.random.default_rng(seed)
    x, y = cloud["x"], cloud["y"]
    k = rng.uniform(1.0, 3.0, 4)
    a = np.radians(aoa)
    rho = 1.0 + amp * np.sin(k[0] * x) * np.cos(k[1] * y)
    u = mach * np.cos(a) + amp * np.cos(k[2] * y)
    v = mach * np.sin(a) + amp * np.sin(k[3] * x)
    p = 1.0 / GAMMA * (1.0 + amp * np.cos(k[1] * x - k[0] * y))
    return np.ascontiguousarray(np.stack([rho, rho * u, rho * v, p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v)]))


def _summand_scale(cloud, U, gx, gy):
    """Mean over the stencil of (|dq| + |d|(|grad q_i| + |grad q_0|)/2)/|d| per point and component."""
    rho = U[0]
    u, v = U[1] / rho, U[2] / rho
    p = (GAMMA - 1) * (U[3] - 0.5 * rho * (u * u + v * v))
    beta = rho / (2 * p)
    q = np.stack([np.log(rho) + np.log(beta) / (GAMMA - 1) - beta * (u * u + v * v),
                  2 * beta * u, 2 * beta * v, -2 * beta])
    off, idx = cloud["nbr_offsets"], cloud["nbr_idx"]
    rows = np.repeat(np.arange(cloud["n"]), np.diff(off))
    dx = cloud["x"][idx] - cloud["x"][rows]
    dy = cloud["y"][idx] - cloud["y"][rows]
    d = np.hypot(dx, dy)
    S = np.zeros_like(q)
    for k in range(4):
        term = (np.abs(q[k, idx] - q[k, rows])
                + 0.5 * (np.abs(dx) * (np.abs(gx[k, idx]) + np.abs(gx[k, rows]))
                         + np.abs(dy) * (np.abs(gy[k, idx]) + np.abs(gy[k, rows])))) / d
        S[k] = np.bincount(rows, weights=term, minlength=cloud["n"]) / np.diff(off)
    return S


def _q_rounding_scale(cloud, q):
    """Mean over the stencil of (|q_i| + |q_0|)/|d| per point and component:
    the CUDA path forms q with the device log, the oracle with glibc's, so
    their q differ in the last bit; this term admits that difference."""
    off, idx = cloud["nbr_offsets"], cloud["nbr_idx"]
    rows = np.repeat(np.arange(cloud["n"]), np.diff(off))
    d = np.hypot(cloud["x"][idx] - cloud["x"][rows], cloud["y"][idx] - cloud["y"][rows])
    Q = np.zeros_like(q)
    for k in range(4):
        Q[k] = np.bincount(rows, weights=(np.abs(q[k, idx]) + np.abs(q[k, rows])) / d,
                           minlength=cloud["n"]) / np.diff(off)
    return Q


def test_noalloc_q_derivatives_match_the_context_entry_point_twice():
    import torch
    from paper_2403_13287_gb300 import lskum

    cloud = naca0012_cloud(130, 24, seed=3)
    n = cloud["n"]
    inner = 3
    solver = lskum.Solver(cloud, order=2, inner_iters=inner, limiter_K=0.0)
    dev = lambda a, t=torch.float64: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", t)  # noqa: E731
    x, y = dev(cloud["x"]), dev(cloud["y"])
    off, idx = dev(cloud["nbr_offsets"], torch.int32), dev(cloud["nbr_idx"], torch.int32)
    for call, seed in enumerate((1, 2)):
        U = _state(cloud, seed)
        Ud = dev(U)
        qx = torch.full((4, n), float("nan"), dtype=torch.float64, device="cuda")
        qy = torch.full_like(qx, float("nan"))
        lskum.q_derivatives_noalloc(x, y, off, idx, Ud, qx, qy, gamma=GAMMA, inner_iters=inner)
        rx, ry = solver.q_derivatives(Ud)
        qx, qy, rx, ry = (t.cpu().numpy() for t in (qx, qy, rx, ry))
        q = oracle.q_variables(U, GAMMA)
        ox, oy = oracle.q_derivatives(cloud, q, inner=inner)
        S = _summand_scale(cloud, U, ox, oy)
        assert np.all(np.isfinite(qx)) and np.all(np.isfinite(qy)), "call %d" % call
        assert np.all(np.abs(qx - rx) <= 1e-12 * S), "call %d" % call
        assert np.all(np.abs(qy - ry) <= 1e-12 * S), "call %d" % call
        # against the oracle, whose q is rounded by another log: a few ulp of
        # q over the stencil's spacing on top of the summand scale
        So = S + 1e-3 * _q_rounding_scale(cloud, q)
        assert np.all(np.abs(qx - ox) <= 1e-12 * So), "call %d vs the oracle" % call
        assert np.all(np.abs(qy - oy) <= 1e-12 * So), "call %d vs the oracle" % call
    solver.close()


def test_noalloc_refuses_short_arrays_and_malformed_rows():
    import torch
    from paper_2403_13287_gb300 import lskum

    cloud = naca0012_cloud(64, 12, seed=3)
    n = cloud["n"]
    dev = lambda a, t=torch.float64: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", t)  # noqa: E731
    x, y = dev(cloud["x"]), dev(cloud["y"])
    off, idx = dev(cloud["nbr_offsets"], torch.int32), dev(cloud["nbr_idx"], torch.int32)
    U = dev(_state(cloud, 1))
    qx = torch.empty((4, n), dtype=torch.float64, device="cuda")
    qy = torch.empty_like(qx)
    short = torch.empty(4 * n - 1, dtype=torch.float64, device="cuda")
    with pytest.raises(lskum.LskumError) as e:
        lskum.q_derivatives_noalloc(x, y, off, idx, U, short, qy)
    assert e.value.status == lskum.LSKUM_ERR_ARG
    with pytest.raises(lskum.LskumError) as e:
        lskum.q_derivatives_noalloc(x, y, off, idx[:-1], U, qx, qy)
    assert e.value.status == lskum.LSKUM_ERR_ARG
    # rows that run backwards and past nbr_offsets[n]: refused by the wrapper
    bad = off.clone()
    nnz = int(cloud["nbr_offsets"][-1])
    bad[5], bad[6] = off[6], off[5]
    bad[9] = nnz + 10
    with pytest.raises(lskum.LskumError) as e:
        lskum.q_derivatives_noalloc(x, y, bad, idx, U, qx, qy)
    assert e.value.status == lskum.LSKUM_ERR_CONNECTIVITY
    # and by the kernels' own row checks, through the C entry point itself;
    # nbr_idx is padded past nbr_offsets[n] + 10, so every read stays inside
    # this test's allocation
    idx_pad = torch.cat([idx, torch.zeros(64, dtype=torch.int32, device="cuda")])
    L = lskum._noalloc_lib()
    P = ctypes.c_void_p
    st = L.lskum_q_derivatives_noalloc(n, P(x.data_ptr()), P(y.data_ptr()), P(bad.data_ptr()),
                                       P(idx_pad.data_ptr()), P(U.data_ptr()), GAMMA, 3, P(qx.data_ptr()),
                                       P(qy.data_ptr()), P(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert st == lskum.LSKUM_ERR_CONNECTIVITY
    assert "nbr_offsets" in L.lskum_last_error(None).decode()
    # a good call after the refused ones gives the oracle's derivatives
    lskum.q_derivatives_noalloc(x, y, off, idx, U, qx, qy)
    Uh = U.cpu().numpy()
    q = oracle.q_variables(Uh, GAMMA)
    ox, oy = oracle.q_derivatives(cloud, q, inner=3)
    So = _summand_scale(cloud, Uh, ox, oy) + 1e-3 * _q_rounding_scale(cloud, q)
    assert np.all(np.abs(qx.cpu().numpy() - ox) <= 1e-12 * So)
    assert np.all(np.abs(qy.cpu().numpy() - oy) <= 1e-12 * So)


def test_noalloc_rejects_sizes_beyond_its_static_scratch():
    import torch
    from paper_2403_13287_gb300 import lskum

    n = lskum.LSKUM_NOALLOC_MAX_POINTS + 1
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    off = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    U = torch.zeros((4, n), dtype=torch.float64, device="cuda")
    with pytest.raises(lskum.LskumError) as e:
        lskum.q_derivatives_noalloc(x, x, off, off, U, U, U)
    assert e.value.status == lskum.LSKUM_ERR_ARG
    assert "static scratch" in str(e.value)
