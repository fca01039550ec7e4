"""The C ABI library builds, loads and exports every entry point that
include/lskum.h declares (no GPU needed; no compute call is made)."""
import ctypes
import os
import re

from paper_2403_13287_gb300 import build as lbuild
from paper_2403_13287_gb300 import lskum

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "lskum.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lskum_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lskum_create", "lskum_step", "lskum_residual", "lskum_forces",
                     "lskum_q_derivatives", "lskum_timestep", "lskum_get_state",
                     "lskum_set_state", "lskum_destroy", "lskum_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    path = lbuild.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_config_struct_matches_header_layout():
    # order, inner_iters, time_scheme (3 ints, padded to 16), 4 doubles, 2 ints, 1 double
    assert ctypes.sizeof(lskum.lskum_config) == 64
    assert lskum.lskum_config.cfl.offset == 16
    assert lskum.lskum_config.precision.offset == 48
    assert lskum.lskum_config.limiter_K.offset == 56


def test_create_rejects_bad_arguments_without_touching_the_gpu():
    L = lskum.load()
    ctx = ctypes.c_void_p()
    cfg = lskum.lskum_config(2, 3, 1, 0.2, 0.5, 0.0, 1.4, 0, 0, 0.0)
    st = L.lskum_create(0, None, None, None, None, None, None, None, 0, None, ctypes.byref(cfg), None,
                        ctypes.byref(ctx))
    assert st == lskum.LSKUM_ERR_ARG and not ctx.value
    assert b"out of range" in L.lskum_last_error(None)
