"""The C ABI library builds, loads and exports every entry point that
include/lskum.h declares (no GPU needed; no compute call is made)."""
import ctypes
import os
import re
import subprocess

from paper_2403_13287_gb300 import build as lbuild
from paper_2403_13287_gb300 import lskum

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lskum.h")


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


def test_config_struct_matches_header_layout(tmp_path):
    """ctypes' lskum_config against the C compiler's layout of the header's"""
    fields = [f[0] for f in lskum.lskum_config._fields_]
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "lskum.h"\nint main(void) {\n'
                   '  printf("%zu\\n", sizeof(lskum_config));\n'
                   + "".join('  printf("%%zu\\n", offsetof(lskum_config, %s));\n' % f for f in fields)
                   + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got[0] == ctypes.sizeof(lskum.lskum_config)
    assert got[1:] == [getattr(lskum.lskum_config, f).offset for f in fields]


def test_create_rejects_bad_arguments_without_touching_the_gpu():
    L = lskum.load()
    ctx = ctypes.c_void_p()
    cfg = lskum.lskum_config(2, 3, 1, 0.2, 0.5, 0.0, 1.4, 0, 0, 0.0, 0)
    st = L.lskum_create(0, None, None, None, None, None, None, None, 0, None, ctypes.byref(cfg), None,
                        ctypes.byref(ctx))
    assert st == lskum.LSKUM_ERR_ARG and not ctx.value
    assert b"out of range" in L.lskum_last_error(None)


def test_create_rejects_an_unknown_boundary_mode_without_touching_the_gpu():
    import numpy as np
    L = lskum.load()
    ctx = ctypes.c_void_p()
    cfg = lskum.lskum_config(2, 3, 1, 0.2, 0.5, 0.0, 1.4, 0, 0, 0.0, 2)
    x = np.zeros(3); nx = np.ones(3)
    fl = np.zeros(3, np.int32); off = np.array([0, 2, 4, 6], np.int32); idx = np.array([1, 2, 0, 2, 0, 1], np.int32)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    st = L.lskum_create(3, p(x), p(x), p(nx), p(x), p(fl), p(off), p(idx), 0, None, ctypes.byref(cfg), None,
                        ctypes.byref(ctx))
    assert st == lskum.LSKUM_ERR_ARG and not ctx.value
    assert b"boundary" in L.lskum_last_error(None)


def test_create_rejects_clouds_beyond_the_layout_limits_without_touching_the_gpu():
    """The mixed form packs a neighbour index into 28 bits: 2^28 points are
    refused (before any input array is read), as is n = 2^31 in either form."""
    import numpy as np
    L = lskum.load()
    ctx = ctypes.c_void_p()
    x = np.zeros(4)
    off = np.zeros(5, np.int32)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    for n, precision, what in ((1 << 28, 1, b"2^28"), (1 << 31, 0, b"out of range")):
        cfg = lskum.lskum_config(2, 3, 1, 0.2, 0.5, 0.0, 1.4, precision, 0, 0.0, 0)
        st = L.lskum_create(n, p(x), p(x), p(x), p(x), p(off), p(off), p(off), 0, None, ctypes.byref(cfg), None,
                            ctypes.byref(ctx))
        assert st == lskum.LSKUM_ERR_ARG and not ctx.value
        assert what in L.lskum_last_error(None)
