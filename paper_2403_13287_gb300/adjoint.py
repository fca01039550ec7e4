"""Reverse sweeps through unrolled q-LSKUM iterations.

Cl and Cd after K pseudo-time iterations from U^0 are differentiated with
respect to U^0 and the point coordinates by running the iterations backwards
with lskum_step_vjp (one iteration in reverse) and lskum_forces_vjp (the force
integrals). The forward states the reverse sweep needs are kept every s
iterations (checkpoints) and recomputed segment by segment, s = ceil(sqrt(K))
by default: memory for about 2 sqrt(K) states instead of K, for one extra
forward pass. This module only orders calls of the C ABI; every product runs
in the library's kernels.
"""
from __future__ import annotations

import math


def unrolled_force_gradient(solver, U0, iters, cl_bar=1.0, cd_bar=0.0, case=0, every=None):
    """Forces after `iters` iterations of `solver` from U0 ([4, n] float64
    CUDA tensor) and the cotangents of cl_bar Cl + cd_bar Cd.

    Returns ((Cl, Cd), (U0_bar, x_bar, y_bar), info), the cotangents as CUDA
    tensors in the solver's input order; info reports the checkpoint interval,
    the recomputed iterations and the bytes of stored states. The solver's
    state is left at the forward result."""
    import torch

    K = int(iters)
    s = int(every) if every else max(1, math.ceil(math.sqrt(K)))
    n = solver.n

    def snapshot():
        out = torch.empty((4, n), dtype=torch.float64, device="cuda")
        solver.get_state(out=out)
        return out

    solver.set_state(U0)
    ckpt = {}
    for k in range(K):
        if k % s == 0:
            ckpt[k] = snapshot()
        solver.step(1, history=False)
    UK = snapshot()
    if solver.ncases > 1:
        cl, cd, _ = solver.case_forces(case, want_cp=False)
    else:
        cl, cd, _ = solver.forces(want_cp=False)
    xb = torch.zeros(n, dtype=torch.float64, device="cuda")
    yb = torch.zeros(n, dtype=torch.float64, device="cuda")
    Ub, _, _ = solver.forces_vjp(cl_bar, cd_bar, case=case, xy_bar=(xb, yb))
    recomputed = 0
    peak_states = len(ckpt)
    for a in reversed(range(0, K, s)):
        b = min(a + s, K)
        states = [ckpt[a]]
        solver.set_state(ckpt[a])
        for _ in range(a + 1, b):
            solver.step(1, history=False)
            recomputed += 1
            states.append(snapshot())
        peak_states = max(peak_states, len(ckpt) + len(states) - 1)
        for k in reversed(range(a, b)):
            Ub, _, _ = solver.step_vjp(Ub, U=states[k - a], xy_bar=(xb, yb))
    solver.set_state(UK)
    info = {"iterations": K, "checkpoint_every": s, "checkpoints": len(ckpt), "recomputed_iterations": recomputed,
            "state_bytes_peak": peak_states * 4 * n * 8, "state_bytes_unrolled": K * 4 * n * 8}
    return (cl, cd), (Ub, xb, yb), info
