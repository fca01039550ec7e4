"""The FP64 split fluxes take erf(S) and exp(-S^2) from one Taylor table
(csrc/fp64_tables.h, written by csrc/gen_fp64_tables.py). Checked here without a
GPU: the committed table is what the generator writes, and the table's two
Horner chains reproduce erf and exp(-S^2) to about one unit in the last place
of 1 on a dense grid (the device code runs the same chains with fused
multiply-adds)."""
import math
import os
import re
import subprocess
import sys

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2403_13287_gb300", "csrc")


def _table():
    txt = open(os.path.join(CSRC, "fp64_tables.h")).read()
    body = txt.split("kErfExpTable", 1)[1].split("= {", 1)[1].split("};", 1)[0]
    rows = re.findall(r"\{([^{}]*)\}", body)
    return np.array([[float.fromhex(v.strip()) for v in r.split(",")] for r in rows])


def test_table_is_the_generator_output(tmp_path):
    pytest.importorskip("mpmath")
    src = os.path.join(CSRC, "gen_fp64_tables.py")
    work = tmp_path / "csrc"
    work.mkdir()
    (work / "gen_fp64_tables.py").write_text(open(src).read())
    subprocess.run([sys.executable, str(work / "gen_fp64_tables.py")], check=True)
    assert (work / "fp64_tables.h").read_text() == open(os.path.join(CSRC, "fp64_tables.h")).read()


def test_table_reproduces_erf_and_exp():
    T = _table()
    step, deg = 1024, 4
    assert T.shape == (6 * step + 1, 2 * deg + 4)
    assert np.all(T[:, 0] == np.arange(6 * step + 1) / step)
    S = np.linspace(-6.0, 6.0, 400001)
    a = np.abs(S)
    k = np.minimum(np.rint(a * step).astype(int), 6 * step)
    d = a - T[k, 0]
    c = T[k, 1:deg + 2]
    e = T[k, deg + 2:2 * deg + 3]
    erf = c[:, deg]
    ex = e[:, deg]
    for n in range(deg - 1, -1, -1):
        erf = erf * d + c[:, n]
        ex = ex * d + e[:, n]
    erf = np.copysign(erf, S)
    ref_erf = np.array([math.erf(x) for x in S])
    assert np.max(np.abs(erf - ref_erf)) <= 2.3e-16
    assert np.max(np.abs(ex - np.exp(-S * S))) <= 2.3e-16
    # near 0, where erf is small: within the truncation bound
    # d^5/5! 2/sqrt(pi) max|H_4| = 3e-18 at |d| = 1/2048 plus two units in the
    # last place of erf itself, far below one unit of 1 (the split fluxes take
    # erf only through 1 +- erf)
    small = np.abs(S) < 0.5
    assert np.all((np.abs(erf - ref_erf) <= 5e-18 + 2 * np.spacing(np.abs(ref_erf)))[small])
    # half a grid step off the nodes as well (the largest |d| of the device)
    off = (np.arange(6 * step) + 0.5) / step
    assert np.max(np.abs(np.array([math.erf(x) for x in off]) -
                         np.array([np.polyval(T[j, deg + 1:0:-1], 0.5 / step) for j in range(6 * step)]))) <= 2.3e-16


def _exp_consts():
    txt = open(os.path.join(CSRC, "fp64_tables.h")).read()
    def const(name):
        return float.fromhex(re.search(r"#define %s (\S+)" % name, txt).group(1))
    body = txt.split("kExp2Table", 1)[1].split("= {", 1)[1].split("};", 1)[0]
    T = np.array([float.fromhex(v.strip()) for v in body.split(",") if v.strip()])
    return const("LSKUM_EXP_INV_L"), const("LSKUM_EXP_L_HI"), const("LSKUM_EXP_L_LO"), T


def test_exp_table_reproduces_exp():
    """The table-driven exp of the device, step by step in double precision
    (numpy rounds each operation; the device fuses multiply-adds)."""
    inv_l, l_hi, l_lo, T = _exp_consts()
    N = 4096
    assert T.shape == (N,) and T[0] == 1.0 and np.all(np.diff(T) > 0)
    assert np.all(np.abs(T - np.array([2.0 ** (j / N) for j in range(N)])) <= np.spacing(T))
    # the head of ln2/4096 has 31 significant bits, so n * head is exact for
    # |n| < 2^22 (|x| < 706 gives |n| < 4.18e6)
    m, e = math.frexp(l_hi)
    assert m * 2.0 ** 31 == int(m * 2.0 ** 31)
    assert abs((l_hi + l_lo) - math.log(2) / N) <= 1e-20
    x = np.concatenate([np.linspace(-705.9, 705.9, 200001), np.linspace(-5.0, 5.0, 200001)])
    kd = np.rint(x * inv_l)
    n = kd.astype(np.int64)
    assert np.max(np.abs(n)) < 2 ** 22
    r = (x - kd * l_hi) - kd * l_lo
    assert np.max(np.abs(r)) <= math.log(2) / (2 * N) * (1 + 1e-9)
    p = ((r / 6 + 0.5) * r + 1) * r + 1
    # the exponent-field scaling by 2^(m + k), k = -1 as for rho/2, stays normal
    for k in (0, -1):
        sc = (n >> 12) + k
        tp = T[n & (N - 1)] * p
        assert np.all((np.frexp(tp)[1] - 1 + sc) >= -1022)
        got = tp * np.ldexp(1.0, sc.astype(np.int32))
        rel = np.abs(got - np.ldexp(np.exp(x), k)) / np.ldexp(np.exp(x), k)
        assert np.max(rel) <= 4.5e-16
