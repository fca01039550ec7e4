"""Thin Python binding of the C ABI in include/lskum.h (liblskum.so).

Argument marshalling only: every step of the hot path runs in the CUDA
kernels of the shared library. Device arrays are torch CUDA tensors (float64,
contiguous, component-major [4, n]); host arrays are numpy arrays. There is
no CPU fallback: if the library cannot be loaded, importing its functions
raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LSKUM_OK = 0
LSKUM_ERR_ARG = 1
LSKUM_ERR_CONNECTIVITY = 2
LSKUM_ERR_DEGENERATE_STENCIL = 3
LSKUM_ERR_CUDA = 4
LSKUM_ERR_OOM = 5
LSKUM_ERR_NONPHYSICAL = 6
LSKUM_ERR_TIMEOUT = 7

LSKUM_BOUNDARY_PLAIN = 0
LSKUM_BOUNDARY_KINETIC = 1

LSKUM_KERNEL_FLUX = 0
LSKUM_KERNEL_QGRAD = 1

_STATUS_NAMES = {0: "LSKUM_OK", 1: "LSKUM_ERR_ARG", 2: "LSKUM_ERR_CONNECTIVITY",
                 3: "LSKUM_ERR_DEGENERATE_STENCIL", 4: "LSKUM_ERR_CUDA", 5: "LSKUM_ERR_OOM",
                 6: "LSKUM_ERR_NONPHYSICAL", 7: "LSKUM_ERR_TIMEOUT"}


class lskum_config(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int), ("inner_iters", ctypes.c_int),
                ("time_scheme", ctypes.c_int), ("cfl", ctypes.c_double),
                ("mach", ctypes.c_double), ("aoa_deg", ctypes.c_double),
                ("gamma", ctypes.c_double), ("precision", ctypes.c_int),
                ("reorder", ctypes.c_int), ("limiter_K", ctypes.c_double), ("boundary", ctypes.c_int)]


class LskumError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (_STATUS_NAMES.get(status, str(status)), message))
        self.status = status


_lib = None
_p = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int


def library_path() -> str:
    return _build.LIB


class lskum_case(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("nx", ctypes.c_void_p), ("ny", ctypes.c_void_p), ("flags", ctypes.c_void_p),
                ("nbr_offsets", ctypes.c_void_p), ("nbr_idx", ctypes.c_void_p), ("n_wall", ctypes.c_int64),
                ("wall_order", ctypes.c_void_p), ("mach", ctypes.c_double), ("aoa_deg", ctypes.c_double)]


class lskum_tuning(ctypes.Structure):
    _fields_ = [("flux_variant", ctypes.c_int), ("flux_threads", ctypes.c_int), ("flux_min_blocks", ctypes.c_int),
                ("qgrad_variant", ctypes.c_int), ("qgrad_threads", ctypes.c_int),
                ("qgrad_min_blocks", ctypes.c_int), ("flux_ms", ctypes.c_double), ("qgrad_ms", ctypes.c_double),
                ("flux_ms_default", ctypes.c_double), ("qgrad_ms_default", ctypes.c_double)]


def load(build_if_missing: bool = True):
    """Load liblskum.so (building it first if asked and needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise ImportError("liblskum.so not found at %s: run __graft_entry__.build()" % path)
    L = ctypes.CDLL(path)
    L.lskum_create.argtypes = [_i64, _p, _p, _p, _p, _p, _p, _p, _i64, _p,
                               ctypes.POINTER(lskum_config), _p, ctypes.POINTER(_p)]
    L.lskum_create.restype = _int
    L.lskum_destroy.argtypes = [_p]
    L.lskum_destroy.restype = None
    L.lskum_last_error.argtypes = [_p]
    L.lskum_last_error.restype = ctypes.c_char_p
    L.lskum_step.argtypes = [_p, _int, _p]
    L.lskum_residual.argtypes = [_p, _p, _p]
    L.lskum_create_batch.argtypes = [_int, ctypes.POINTER(lskum_case), ctypes.POINTER(lskum_config), _p,
                                     ctypes.POINTER(_p)]
    L.lskum_create_batch.restype = _int
    L.lskum_case_count.argtypes = [_p]
    L.lskum_case_count.restype = _int
    L.lskum_case_range.argtypes = [_p, _int, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                   ctypes.POINTER(_i64)]
    L.lskum_case_forces.argtypes = [_p, _int, _p, _p, _p]
    L.lskum_autotune.argtypes = [_p, _int, ctypes.POINTER(lskum_tuning)]
    L.lskum_set_tuning.argtypes = [_p, _int, _int]
    L.lskum_mixed_fp64_points.argtypes = [_p, ctypes.POINTER(ctypes.c_int64)]
    L.lskum_residual_vjp.argtypes = [_p, _p, _p, _p, _p, _p, _int]
    L.lskum_step_vjp.argtypes = [_p, _p, _p, _p, _p, _p, _int]
    L.lskum_forces_vjp.argtypes = [_p, _int, ctypes.c_double, ctypes.c_double, _p, _p, _p, _int]
    L.lskum_q_derivatives.argtypes = [_p, _p, _p, _p]
    L.lskum_timestep.argtypes = [_p, _p, _p]
    L.lskum_forces.argtypes = [_p, _p, _p, _p]
    L.lskum_get_state.argtypes = [_p, _p, _int]
    L.lskum_set_state.argtypes = [_p, _p, _int]
    L.lskum_get_stencil_masks.argtypes = [_p, _p]
    L.lskum_get_permutation.argtypes = [_p, _p]
    L.lskum_launch_count.argtypes = [_p]
    L.lskum_launch_count.restype = _i64
    L.lskum_profile.argtypes = [_p, _int]
    L.lskum_kernel_time.argtypes = [_p, _int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i64)]
    for name in ("lskum_case_range", "lskum_case_forces", "lskum_autotune", "lskum_set_tuning",
                 "lskum_step_vjp", "lskum_forces_vjp", "lskum_mixed_fp64_points"):
        getattr(L, name).restype = _int
    for name in ("lskum_step", "lskum_residual", "lskum_residual_vjp", "lskum_q_derivatives", "lskum_timestep",
                 "lskum_forces", "lskum_get_state", "lskum_set_state", "lskum_get_stencil_masks",
                 "lskum_get_permutation", "lskum_profile", "lskum_kernel_time"):
        getattr(L, name).restype = _int
    _lib = L
    return L


def _stream_ptr(stream):
    if stream is not None:
        return int(stream)
    try:
        import torch
        return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
    except Exception:  # noqa: BLE001
        return 0


def _np_ptr(a):
    return a.ctypes.data_as(_p)


def _dev_ptr(t):
    if t is None:
        return None
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return _p(t.data_ptr())


class Solver:
    """A q-LSKUM context (lskum_ctx) on the current CUDA device."""

    def __init__(self, cloud, order=2, inner_iters=3, time_scheme=1, cfl=0.2, mach=0.63,
                 aoa_deg=2.0, gamma=1.4, precision=0, reorder=0, limiter_K=0.0, stream=None, boundary=0):
        L = load()
        self._L = L
        self.n = int(cloud["n"])
        self.cfg = lskum_config(order, inner_iters, time_scheme, cfl, mach, aoa_deg, gamma,
                                precision, reorder, limiter_K, boundary)
        self._keep = {k: np.ascontiguousarray(cloud[k], dtype=np.float64) for k in ("x", "y", "nx", "ny")}
        for k in ("flags", "nbr_offsets", "nbr_idx"):
            self._keep[k] = np.ascontiguousarray(cloud[k], dtype=np.int32)
        wo = cloud.get("wall_order")
        self._keep["wall_order"] = np.ascontiguousarray(wo if wo is not None else np.zeros(0), dtype=np.int32)
        self.nnz = int(self._keep["nbr_offsets"][-1])
        self.n_wall = int(self._keep["wall_order"].shape[0])
        stream_ptr = _stream_ptr(stream)
        ctx = _p()
        k = self._keep
        st = L.lskum_create(self.n, _np_ptr(k["x"]), _np_ptr(k["y"]), _np_ptr(k["nx"]), _np_ptr(k["ny"]),
                            _np_ptr(k["flags"]), _np_ptr(k["nbr_offsets"]), _np_ptr(k["nbr_idx"]),
                            self.n_wall, _np_ptr(k["wall_order"]), ctypes.byref(self.cfg),
                            _p(stream_ptr) if stream_ptr else None, ctypes.byref(ctx))
        if st != LSKUM_OK:
            raise LskumError(st, L.lskum_last_error(None).decode())
        self._ctx = ctx
        self.ncases = 1

    @classmethod
    def batch(cls, cases, order=2, inner_iters=3, time_scheme=1, cfl=0.2, gamma=1.4, precision=1, reorder=1,
              limiter_K=0.0, stream=None, boundary=0):
        """One context over several independent solves (lskum_create_batch).
        cases: a list of (cloud, mach, aoa_deg); clouds may repeat."""
        self = cls.__new__(cls)
        L = load()
        self._L = L
        self.cfg = lskum_config(order, inner_iters, time_scheme, cfl, cases[0][1], cases[0][2], gamma,
                                precision, reorder, limiter_K, boundary)
        keep, arr = {}, (lskum_case * len(cases))()
        for k, (cloud, mach, aoa) in enumerate(cases):
            key = id(cloud)
            if key not in keep:
                d = {f: np.ascontiguousarray(cloud[f], dtype=np.float64) for f in ("x", "y", "nx", "ny")}
                for f in ("flags", "nbr_offsets", "nbr_idx"):
                    d[f] = np.ascontiguousarray(cloud[f], dtype=np.int32)
                wo = cloud.get("wall_order")
                d["wall_order"] = np.ascontiguousarray(wo if wo is not None else np.zeros(0), dtype=np.int32)
                keep[key] = d
            d = keep[key]
            a = arr[k]
            a.n = int(cloud["n"])
            for f in ("x", "y", "nx", "ny", "flags", "nbr_offsets", "nbr_idx", "wall_order"):
                setattr(a, f, d[f].ctypes.data)
            a.n_wall = int(d["wall_order"].shape[0])
            a.mach = float(mach)
            a.aoa_deg = float(aoa)
        self._keep = keep
        ctx = _p()
        stream_ptr = _stream_ptr(stream)
        st = L.lskum_create_batch(len(cases), arr, ctypes.byref(self.cfg), _p(stream_ptr) if stream_ptr else None,
                                  ctypes.byref(ctx))
        if st != LSKUM_OK:
            raise LskumError(st, L.lskum_last_error(None).decode())
        self._ctx = ctx
        self.ncases = int(L.lskum_case_count(ctx))
        self.n = sum(int(c[0]["n"]) for c in cases)
        self.nnz = sum(int(np.asarray(c[0]["nbr_offsets"])[-1]) for c in cases)
        self.n_wall = sum(int(keep[id(c[0])]["wall_order"].shape[0]) for c in cases)
        return self

    def case_range(self, k):
        """(first, count, wall_first, wall_count) of case k in caller-visible arrays."""
        v = [_i64() for _ in range(4)]
        self._check(self._L.lskum_case_range(self._ctx, int(k), *[ctypes.byref(x) for x in v]))
        return tuple(int(x.value) for x in v)

    def case_forces(self, k, want_cp=True):
        nw = self.case_range(k)[3]
        cl = ctypes.c_double()
        cd = ctypes.c_double()
        cp = np.zeros(nw) if want_cp else None
        self._check(self._L.lskum_case_forces(self._ctx, int(k), ctypes.byref(cl), ctypes.byref(cd),
                                              _np_ptr(cp) if want_cp else None))
        return cl.value, cd.value, cp

    def autotune(self, reps=5):
        """Time every launch shape of the mixed kernels on this context and keep the fastest."""
        t = lskum_tuning()
        self._check(self._L.lskum_autotune(self._ctx, int(reps), ctypes.byref(t)))
        return {f: getattr(t, f) for f, _ in lskum_tuning._fields_}

    def set_tuning(self, flux_variant, qgrad_variant):
        self._check(self._L.lskum_set_tuning(self._ctx, int(flux_variant), int(qgrad_variant)))

    def mixed_fp64_points(self):
        """Points whose least-squares closures run in FP64 (mixed contexts; 0 for FP64)."""
        v = ctypes.c_int64(0)
        self._check(self._L.lskum_mixed_fp64_points(self._ctx, ctypes.byref(v)))
        return int(v.value)

    def _check(self, st):
        if st != LSKUM_OK:
            raise LskumError(st, self._L.lskum_last_error(self._ctx).decode())

    def close(self):
        if getattr(self, "_ctx", None):
            self._L.lskum_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    # --- hot path ---
    def step(self, n_iters, history=True):
        """n_iters iterations; the residue history ([n_iters], or [n_iters, ncases] for a batch)."""
        hist = np.zeros((n_iters, self.ncases) if self.ncases > 1 else n_iters) if history else None
        self._check(self._L.lskum_step(self._ctx, int(n_iters), _np_ptr(hist) if history else None))
        return hist

    def residual(self, U=None, out=None):
        import torch
        if out is None:
            out = torch.empty((4, self.n), dtype=torch.float64, device="cuda")
        self._check(self._L.lskum_residual(self._ctx, _dev_ptr(U), _dev_ptr(out)))
        return out

    def residual_vjp(self, R_bar, U=None, want_U=True, want_xy=True, fp32=False):
        """(U_bar, x_bar, y_bar) = (dR/dU, dR/dx, dR/dy)^T R_bar at U (the
        context's state if None); the unrequested ones are None. fp32: the
        product in FP32 (mixed contexts)."""
        import torch
        Ub = torch.empty((4, self.n), dtype=torch.float64, device="cuda") if want_U else None
        xb = torch.empty(self.n, dtype=torch.float64, device="cuda") if want_xy else None
        yb = torch.empty_like(xb) if want_xy else None
        self._check(self._L.lskum_residual_vjp(self._ctx, _dev_ptr(U), _dev_ptr(R_bar), _dev_ptr(Ub),
                                               _dev_ptr(xb), _dev_ptr(yb), LSKUM_VJP_FP32 if fp32 else 0))
        return Ub, xb, yb

    def step_vjp(self, U_bar_next, U=None, want_U=True, want_xy=True, U_bar=None, xy_bar=None):
        """(U_bar, x_bar, y_bar): one iteration U^n -> U^{n+1} differentiated
        in reverse at U^n = U (the context's state if None). Pass xy_bar
        (x_bar, y_bar tensors) to add the coordinate cotangents into them."""
        import torch
        Ub = U_bar if U_bar is not None else (
            torch.empty((4, self.n), dtype=torch.float64, device="cuda") if want_U else None)
        xb, yb, flags = self._xy_out(want_xy, xy_bar)
        self._check(self._L.lskum_step_vjp(self._ctx, _dev_ptr(U), _dev_ptr(U_bar_next), _dev_ptr(Ub),
                                           _dev_ptr(xb), _dev_ptr(yb), flags))
        return Ub, xb, yb

    def forces_vjp(self, cl_bar=1.0, cd_bar=0.0, case=0, want_U=True, want_xy=True, xy_bar=None):
        """(U_bar, x_bar, y_bar) of cl_bar Cl + cd_bar Cd at the context's state
        (coordinate cotangents added into xy_bar if given)."""
        import torch
        Ub = torch.empty((4, self.n), dtype=torch.float64, device="cuda") if want_U else None
        xb, yb, flags = self._xy_out(want_xy, xy_bar)
        self._check(self._L.lskum_forces_vjp(self._ctx, int(case), float(cl_bar), float(cd_bar), _dev_ptr(Ub),
                                             _dev_ptr(xb), _dev_ptr(yb), flags))
        return Ub, xb, yb

    def _xy_out(self, want_xy, xy_bar):
        import torch
        if xy_bar is not None:
            return xy_bar[0], xy_bar[1], LSKUM_VJP_ACCUMULATE_XY
        if not want_xy:
            return None, None, 0
        xb = torch.empty(self.n, dtype=torch.float64, device="cuda")
        return xb, torch.empty_like(xb), 0

    def q_derivatives(self, U=None):
        import torch
        qx = torch.empty((4, self.n), dtype=torch.float64, device="cuda")
        qy = torch.empty_like(qx)
        self._check(self._L.lskum_q_derivatives(self._ctx, _dev_ptr(U), _dev_ptr(qx), _dev_ptr(qy)))
        return qx, qy

    def timestep(self, U=None):
        import torch
        dt = torch.empty(self.n, dtype=torch.float64, device="cuda")
        self._check(self._L.lskum_timestep(self._ctx, _dev_ptr(U), _dev_ptr(dt)))
        return dt

    def forces(self, want_cp=True):
        cl = ctypes.c_double()
        cd = ctypes.c_double()
        cp = np.zeros(self.n_wall) if want_cp else None
        self._check(self._L.lskum_forces(self._ctx, ctypes.byref(cl), ctypes.byref(cd),
                                         _np_ptr(cp) if want_cp else None))
        return cl.value, cd.value, cp

    # --- state ---
    def get_state(self, out=None):
        """State U as a [4, n] array: into `out` (a CUDA tensor or a contiguous
        float64 numpy array) or a new host numpy array."""
        if isinstance(out, np.ndarray):
            if not (out.dtype == np.float64 and out.flags.c_contiguous and out.size == 4 * self.n):
                raise TypeError("expected a contiguous float64 array of 4*n values")
            self._check(self._L.lskum_get_state(self._ctx, _np_ptr(out), 1))
            return out
        if out is not None:
            self._check(self._L.lskum_get_state(self._ctx, _dev_ptr(out), 0))
            return out
        U = np.empty((4, self.n))
        self._check(self._L.lskum_get_state(self._ctx, _np_ptr(U), 1))
        return U

    def set_state(self, U):
        if isinstance(U, np.ndarray):
            Uh = np.ascontiguousarray(U, dtype=np.float64)
            self._check(self._L.lskum_set_state(self._ctx, _np_ptr(Uh), 1))
        else:
            self._check(self._L.lskum_set_state(self._ctx, _dev_ptr(U), 0))

    def stencil_masks(self):
        m = np.empty(self.nnz, dtype=np.uint8)
        self._check(self._L.lskum_get_stencil_masks(self._ctx, _np_ptr(m)))
        return m

    def permutation(self):
        p = np.empty(self.n, dtype=np.int32)
        self._check(self._L.lskum_get_permutation(self._ctx, _np_ptr(p)))
        return p

    def launch_count(self):
        return int(self._L.lskum_launch_count(self._ctx))

    # --- kernel timing ---
    def profile(self, enable=True):
        self._check(self._L.lskum_profile(self._ctx, 1 if enable else 0))

    def kernel_time(self, kernel_class):
        """(summed milliseconds, launches) of one kernel class since profile(True)."""
        ms = ctypes.c_double()
        cnt = _i64()
        self._check(self._L.lskum_kernel_time(self._ctx, int(kernel_class), ctypes.byref(ms), ctypes.byref(cnt)))
        return ms.value, cnt.value


LSKUM_NOALLOC_MAX_POINTS = 131072
LSKUM_VJP_ACCUMULATE_XY = 1
LSKUM_VJP_FP32 = 2


PROBE_FP64_FMA = 0
PROBE_FP32_FMA = 1
PROBE_FP32X2_FMA = 2


def probe_peak(kind, reps=5, stream=None):
    """Measured FMA peak of the current device in GFLOP/s (lskum_probe_peak):
    kind 0 FP64, 1 FP32, 2 packed FP32x2."""
    L = load()
    if not hasattr(L, "_probe_ready"):
        L.lskum_probe_peak.argtypes = [_int, _int, _p, ctypes.POINTER(ctypes.c_double)]
        L.lskum_probe_peak.restype = _int
        L._probe_ready = True
    g = ctypes.c_double()
    stream_ptr = _stream_ptr(stream)
    st = L.lskum_probe_peak(int(kind), int(reps), _p(stream_ptr) if stream_ptr else None, ctypes.byref(g))
    if st != LSKUM_OK:
        raise LskumError(st, "lskum_probe_peak failed")
    return g.value


def _noalloc_lib():
    L = load()
    if not hasattr(L, "_noalloc_ready"):
        L.lskum_q_derivatives_noalloc.argtypes = [_i64, _p, _p, _p, _p, _p, ctypes.c_double, _int,
                                                  _p, _p, _p]
        L.lskum_q_derivatives_noalloc.restype = _int
        L._noalloc_ready = True
    return L


def q_derivatives_noalloc(x, y, nbr_offsets, nbr_idx, U, qx, qy, gamma=1.4, inner_iters=3,
                          stream=None):
    """lskum_q_derivatives_noalloc on caller-owned CUDA tensors (no context,
    no device allocation): x, y float64[n]; nbr_offsets int32[n+1]; nbr_idx
    int32[nnz]; U float64[4, n]; qx, qy float64[4, n] written."""
    import torch
    L = _noalloc_lib()
    for t, dt in ((nbr_offsets, torch.int32), (nbr_idx, torch.int32)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dt and t.is_contiguous()):
            raise TypeError("expected a contiguous int32 CUDA tensor")
    n = int(x.shape[0])
    # sizes and devices: the C entry sees plain pointers and cannot check them
    for t in (x, y, U, qx, qy):
        _dev_ptr(t)                       # contiguous float64 CUDA tensors, else TypeError
    need = ((x, n), (y, n), (nbr_offsets, n + 1), (U, 4 * n), (qx, 4 * n), (qy, 4 * n))
    for t, size in need:
        if t.numel() != size:
            raise LskumError(LSKUM_ERR_ARG, "an array has %d entries where %d are needed" % (t.numel(), size))
    dev = torch.cuda.current_device()
    for t in (x, y, nbr_offsets, nbr_idx, U, qx, qy):
        if t.device.index != dev:
            raise LskumError(LSKUM_ERR_ARG, "an array is on cuda:%d, the current device is cuda:%d"
                             % (t.device.index, dev))
    # the CSR rows: non-decreasing from 0, and nbr_idx long enough for them
    # (one scalar read back)
    bad = (nbr_offsets[0] != 0) | (nbr_offsets[1:] < nbr_offsets[:-1]).any()
    nnz = int(torch.where(bad, torch.full_like(nbr_offsets[-1], -1), nbr_offsets[-1]).item())
    if nnz < 0:
        raise LskumError(LSKUM_ERR_CONNECTIVITY, "nbr_offsets does not start at 0 or decreases")
    if nbr_idx.numel() < nnz:
        raise LskumError(LSKUM_ERR_ARG, "nbr_idx has %d entries, nbr_offsets[n] = %d" % (nbr_idx.numel(), nnz))
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    st = L.lskum_q_derivatives_noalloc(n, _dev_ptr(x), _dev_ptr(y), _p(nbr_offsets.data_ptr()),
                                       _p(nbr_idx.data_ptr()), _dev_ptr(U), float(gamma),
                                       int(inner_iters), _dev_ptr(qx), _dev_ptr(qy),
                                       _p(int(stream)) if stream else None)
    if st != LSKUM_OK:
        raise LskumError(st, L.lskum_last_error(None).decode())


def _residual_fn_class():
    import torch

    class ResidualFn(torch.autograd.Function):
        """R = residual(U) with backward by lskum_residual_vjp. `xy` ([2, n],
        the solver's own coordinates, which the forward does not read) is the
        handle through which coordinate gradients flow."""

        @staticmethod
        def forward(ctx, solver, U, xy):
            U = U.contiguous()
            ctx.solver = solver
            ctx.save_for_backward(U)
            return solver.residual(U)

        @staticmethod
        def backward(ctx, R_bar):
            (U,) = ctx.saved_tensors
            want_U, want_xy = ctx.needs_input_grad[1], ctx.needs_input_grad[2]
            Ub, xb, yb = ctx.solver.residual_vjp(R_bar.contiguous(), U, want_U=want_U, want_xy=want_xy)
            return None, Ub, (torch.stack([xb, yb]) if want_xy else None)

    return ResidualFn


_ResidualFn = None


def residual_fn(solver, U, xy=None):
    """Differentiable residual: R(U) of `solver`'s scheme as a torch op.
    U is a [4, n] float64 CUDA tensor; xy, if given, is a [2, n] float64 CUDA
    tensor holding the solver's coordinates, to receive dR/dxy gradients."""
    global _ResidualFn
    if _ResidualFn is None:
        _ResidualFn = _residual_fn_class()
    if xy is not None and tuple(xy.shape) != (2, solver.n):
        raise ValueError("xy must have shape [2, n]")
    return _ResidualFn.apply(solver, U, xy)
