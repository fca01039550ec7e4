"""Python access to the plain FP64 CPU oracle of the q-LSKUM hot path.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the bench's CPU
baseline use this package; the CUDA product path never imports it. The
arithmetic lives in `lskum_oracle.c` (serial, FP64, compiled with
-ffp-contract=off); this module only builds it with gcc and marshals numpy
arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lskum_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
# the same source built with -fopenmp: the points of each pass shared out
# among host threads (bitwise the same results), for timing on all cores
_LIB_OMP = os.path.join(_BUILD, "liboracle_omp.so")

OK = 0
ERR_DEGENERATE = 3
ERR_NONPHYSICAL = 6

XPOS, XNEG, YPOS, YNEG = 1, 2, 4, 8

_lib = None
_libs = {}
_threads = 1

_d = ctypes.c_double
_i64 = ctypes.c_int64
_int = ctypes.c_int
_p = ctypes.c_void_p

RESIDUAL_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double), ctypes.c_void_p)


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (plain gcc, -O2, no
    FMA contraction); openmp=True builds liboracle_omp.so from the same source
    with -fopenmp (returns None if the compiler has no OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    out = _LIB_OMP if openmp else _LIB
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
        return out
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-Wall", "-fopenmp" if openmp else "-Wno-unknown-pragmas",
           "-o", tmp, _SRC, "-lm"]
    if openmp:
        r = subprocess.run(cmd, capture_output=True)
        if r.returncode != 0:
            return None
    else:
        subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def set_threads(threads: int) -> int:
    """Host threads for the oracle calls that follow: 1 (the default) uses the
    serial build; more uses the OpenMP build (same bits). Returns the number
    of threads in effect (1 if OpenMP is not available)."""
    global _lib, _threads
    threads = max(1, int(threads))
    if threads > 1 and build(openmp=True) is None:
        threads = 1
    _threads = threads
    _lib = None
    L = lib()
    return int(L.orc_set_threads(threads)) if threads > 1 else 1


def threads() -> int:
    return _threads


def lib():
    global _lib
    if _lib is None:
        key = "omp" if _threads > 1 else "serial"
        if key not in _libs:
            _libs[key] = _declare(ctypes.CDLL(build(openmp=True) if key == "omp" else build()))
        _lib = _libs[key]
    return _lib


def _declare(L):
    L.orc_set_threads.argtypes = [_int]
    L.orc_set_threads.restype = _int
    L.orc_split_stencils.argtypes = [_i64] + [_p] * 7
    L.orc_q_variables.argtypes = [_i64, _d, _p, _p]
    L.orc_U_from_q.argtypes = [_i64, _d, _p, _p]
    L.orc_split_flux.argtypes = [_d, _d, _d, _d, _d, _int, _p]
    L.orc_split_flux.restype = None
    L.orc_euler_flux.argtypes = [_d, _d, _d, _d, _d, _p]
    L.orc_euler_flux.restype = None
    L.orc_q_derivatives.argtypes = [_i64, _p, _p, _p, _p, _p, _int, _p, _p]
    L.orc_q_derivatives_pass.argtypes = [_i64] + [_p] * 9
    L.orc_flux_residual.argtypes = [_i64, _d] + [_p] * 11 + [_int, _p, _p]
    L.orc_timestep.argtypes = [_i64, _d, _d] + [_p] * 5 + [_p]
    L.orc_freestream.argtypes = [_d, _d, _d, _p]
    L.orc_freestream.restype = None
    L.orc_residue.argtypes = [_i64, _p]
    L.orc_residue.restype = _d
    L.orc_euler_step.argtypes = [_i64, _p, _p, _p, _p, _p, _p, RESIDUAL_FN, _p, _p]
    L.orc_rk4_step.argtypes = [_i64, _p, _p, _p, _p, _p, _p, RESIDUAL_FN, _p, _p]
    L.orc_residual.argtypes = [_i64, _d] + [_p] * 8 + [_int, _int, _d] + [_p] * 5
    L.orc_limit_gradients.argtypes = [_i64, _p, _p, _p, _p, _p, _d, _p, _p]
    L.orc_forces.argtypes = [_i64, _d, _d, _d, _p, _p, _p, _p, _p, _i64, _p, _p, _p, _p]
    L.orc_solve.argtypes = ([_i64, _d] + [_p] * 8 + [_int, _int, _d, _int, _d, _d, _d, _int, _p, _p])
    L.orc_residual_bc.argtypes = [_i64, _d] + [_p] * 8 + [_int, _int, _d, _int, _d, _d] + [_p] * 5
    L.orc_solve_bc.argtypes = ([_i64, _d] + [_p] * 8 + [_int, _int, _d, _int, _int, _d, _d, _d, _int, _p, _p])
    return L


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


class OracleError(RuntimeError):
    def __init__(self, rc, what):
        super().__init__("oracle %s failed with status %d" % (what, rc))
        self.rc = rc


def _check(rc, what):
    if rc != OK:
        raise OracleError(rc, what)


def split_stencils(cloud):
    n = cloud["n"]
    idx = _i32(cloud["nbr_idx"])
    mask = np.zeros(idx.shape[0], dtype=np.uint8)
    _check(lib().orc_split_stencils(n, _ptr(_f64(cloud["x"])), _ptr(_f64(cloud["y"])),
                                    _ptr(_f64(cloud["nx"])), _ptr(_f64(cloud["ny"])),
                                    _ptr(_i32(cloud["nbr_offsets"])), _ptr(idx), _ptr(mask)),
           "split_stencils")
    return mask


def q_variables(U, gamma=1.4):
    U = _f64(U)
    n = U.shape[1]
    q = np.empty_like(U)
    _check(lib().orc_q_variables(n, gamma, _ptr(U), _ptr(q)), "q_variables")
    return q


def U_from_q(q, gamma=1.4):
    q = _f64(q)
    U = np.empty_like(q)
    _check(lib().orc_U_from_q(q.shape[1], gamma, _ptr(q), _ptr(U)), "U_from_q")
    return U


def split_flux(rho, un, ut, p, sign, gamma=1.4):
    G = np.empty(4)
    lib().orc_split_flux(gamma, rho, un, ut, p, sign, _ptr(G))
    return G


def euler_flux(rho, un, ut, p, gamma=1.4):
    G = np.empty(4)
    lib().orc_euler_flux(gamma, rho, un, ut, p, _ptr(G))
    return G


def q_derivatives(cloud, q, inner=3):
    q = _f64(q)
    n = cloud["n"]
    qx = np.empty_like(q)
    qy = np.empty_like(q)
    _check(lib().orc_q_derivatives(n, _ptr(_f64(cloud["x"])), _ptr(_f64(cloud["y"])),
                                   _ptr(_i32(cloud["nbr_offsets"])), _ptr(_i32(cloud["nbr_idx"])),
                                   _ptr(q), inner, _ptr(qx), _ptr(qy)), "q_derivatives")
    return qx, qy


def q_derivatives_pass(cloud, q, qx_old=None, qy_old=None):
    """One least-squares solve of E15: first order if qx_old is None, else one inner iteration."""
    q = _f64(q)
    qx = np.empty_like(q)
    qy = np.empty_like(q)
    ox = _f64(qx_old) if qx_old is not None else None
    oy = _f64(qy_old) if qy_old is not None else None
    _check(lib().orc_q_derivatives_pass(cloud["n"], _ptr(_f64(cloud["x"])), _ptr(_f64(cloud["y"])),
                                        _ptr(_i32(cloud["nbr_offsets"])), _ptr(_i32(cloud["nbr_idx"])),
                                        _ptr(q), _ptr(ox), _ptr(oy), _ptr(qx), _ptr(qy)),
           "q_derivatives_pass")
    return qx, qy


def limit_gradients(cloud, q, qx, qy, K):
    """Venkatakrishnan-limited copies of the gradients (qx, qy) for q."""
    q = _f64(q)
    gx = _f64(qx).copy()
    gy = _f64(qy).copy()
    _check(lib().orc_limit_gradients(cloud["n"], _ptr(_f64(cloud["x"])), _ptr(_f64(cloud["y"])),
                                     _ptr(_i32(cloud["nbr_offsets"])), _ptr(_i32(cloud["nbr_idx"])),
                                     _ptr(q), float(K), _ptr(gx), _ptr(gy)), "limit_gradients")
    return gx, gy


def flux_residual(cloud, mask, q, qx, qy, order=2, gamma=1.4, want_scale=False):
    n = cloud["n"]
    q = _f64(q)
    qx = _f64(qx) if qx is not None else np.zeros_like(q)
    qy = _f64(qy) if qy is not None else np.zeros_like(q)
    R = np.empty_like(q)
    sc = np.empty_like(q) if want_scale else None
    _check(lib().orc_flux_residual(n, gamma, _ptr(_f64(cloud["x"])), _ptr(_f64(cloud["y"])),
                                   _ptr(_f64(cloud["nx"])), _ptr(_f64(cloud["ny"])),
                                   _ptr(_i32(cloud["flags"])), _ptr(_i32(cloud["nbr_offsets"])),
                                   _ptr(_i32(cloud["nbr_idx"])),
                                   _ptr(np.ascontiguousarray(mask, dtype=np.uint8)),
                                   _ptr(q), _ptr(qx), _ptr(qy), order, _ptr(R), _ptr(sc)),
           "flux_residual")
    return (R, sc) if want_scale else R


def residual(cloud, mask, U, order=2, inner=3, gamma=1.4, want_scale=False, want_grad=False,
             limiter=0.0, boundary=0, mach=0.0, aoa_deg=0.0):
    """R(U) of the whole scheme; optional error scale and q-derivatives.
    boundary=1: kinetic boundary mode, mach/aoa_deg give the free stream."""
    n = cloud["n"]
    U = _f64(U)
    R = np.empty_like(U)
    sc = np.empty_like(U) if want_scale else None
    qx = np.empty_like(U) if want_grad else None
    qy = np.empty_like(U) if want_grad else None
    _check(lib().orc_residual_bc(n, gamma, _ptr(_f64(cloud["x"])), _ptr(_f64(cloud["y"])),
                                 _ptr(_f64(cloud["nx"])), _ptr(_f64(cloud["ny"])),
                                 _ptr(_i32(cloud["flags"])), _ptr(_i32(cloud["nbr_offsets"])),
                                 _ptr(_i32(cloud["nbr_idx"])),
                                 _ptr(np.ascontiguousarray(mask, dtype=np.uint8)),
                                 order, inner, float(limiter), int(boundary), float(mach), float(aoa_deg),
                                 _ptr(U), _ptr(R), _ptr(sc), _ptr(qx), _ptr(qy)),
           "residual")
    out = [R]
    if want_scale:
        out.append(sc)
    if want_grad:
        out += [qx, qy]
    return out[0] if len(out) == 1 else tuple(out)


def timestep(cloud, U, cfl, gamma=1.4):
    U = _f64(U)
    dt = np.empty(cloud["n"])
    _check(lib().orc_timestep(cloud["n"], gamma, cfl, _ptr(_f64(cloud["x"])), _ptr(_f64(cloud["y"])),
                              _ptr(_i32(cloud["nbr_offsets"])), _ptr(_i32(cloud["nbr_idx"])),
                              _ptr(U), _ptr(dt)), "timestep")
    return dt


def freestream(mach, aoa_deg, gamma=1.4):
    U = np.empty(4)
    lib().orc_freestream(gamma, mach, aoa_deg, _ptr(U))
    return U


def freestream_state(n, mach, aoa_deg, gamma=1.4):
    return np.ascontiguousarray(np.repeat(freestream(mach, aoa_deg, gamma)[:, None], n, axis=1))


def residue(R):
    R = _f64(R)
    return lib().orc_residue(R.shape[1], _ptr(R))


def _step(fn, n, flags, nx, ny, Uinf, dt, U, residual_cb):
    """Run one oracle time step with a Python residual callback R = f(U)."""
    def cb(Up, Rp, _user):
        try:
            Ua = np.ctypeslib.as_array(Up, shape=(4 * n,)).reshape(4, n)
            Ra = np.ctypeslib.as_array(Rp, shape=(4 * n,)).reshape(4, n)
            Ra[...] = residual_cb(Ua.copy())
            return 0
        except Exception:  # noqa: BLE001 - surfaced as a non-zero status
            return -2
    cfn = RESIDUAL_FN(cb)
    U = _f64(U).copy()
    R0 = np.empty_like(U)
    _check(fn(n, _ptr(_i32(flags)), _ptr(_f64(nx)), _ptr(_f64(ny)), _ptr(_f64(Uinf)),
              _ptr(_f64(dt)), _ptr(U), cfn, None, _ptr(R0)), "time step")
    return U, R0


def euler_step(flags, nx, ny, Uinf, dt, U, residual_cb):
    return _step(lib().orc_euler_step, len(flags), flags, nx, ny, Uinf, dt, U, residual_cb)


def rk4_step(flags, nx, ny, Uinf, dt, U, residual_cb):
    return _step(lib().orc_rk4_step, len(flags), flags, nx, ny, Uinf, dt, U, residual_cb)


def forces(cloud, U, mach, aoa_deg, gamma=1.4):
    """(Cl, Cd, Cp[wall order])."""
    U = _f64(U)
    wo = _i32(cloud["wall_order"])
    cp = np.empty(wo.shape[0])
    cl = ctypes.c_double()
    cd = ctypes.c_double()
    _check(lib().orc_forces(cloud["n"], gamma, mach, aoa_deg, _ptr(U),
                            _ptr(_f64(cloud["x"])), _ptr(_f64(cloud["y"])),
                            _ptr(_f64(cloud["nx"])), _ptr(_f64(cloud["ny"])),
                            wo.shape[0], _ptr(wo), ctypes.byref(cl), ctypes.byref(cd), _ptr(cp)),
           "forces")
    return cl.value, cd.value, cp


def solve(cloud, mask, U0, n_iters, order=2, inner=3, scheme=1, cfl=0.2, mach=0.63,
          aoa_deg=2.0, gamma=1.4, limiter=0.0, boundary=0):
    """Algorithm 1 for n_iters iterations; returns (U, residue history).
    boundary=1: kinetic boundary mode."""
    U = _f64(U0).copy()
    hist = np.zeros(n_iters)
    _check(lib().orc_solve_bc(cloud["n"], gamma, _ptr(_f64(cloud["x"])), _ptr(_f64(cloud["y"])),
                              _ptr(_f64(cloud["nx"])), _ptr(_f64(cloud["ny"])),
                              _ptr(_i32(cloud["flags"])), _ptr(_i32(cloud["nbr_offsets"])),
                              _ptr(_i32(cloud["nbr_idx"])),
                              _ptr(np.ascontiguousarray(mask, dtype=np.uint8)),
                              order, inner, float(limiter), int(boundary), scheme, cfl, mach, aoa_deg,
                              n_iters, _ptr(U), _ptr(hist)),
           "solve")
    return U, hist
