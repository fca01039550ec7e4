"""The FP64 split fluxes take erf(S) and exp(-S^2) from one Taylor table
(csrc/erf_table.h, written by csrc/gen_erf_table.py). Checked here without a
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
    txt = open(os.path.join(CSRC, "erf_table.h")).read()
    body = txt.split("= {", 1)[1]
    rows = re.findall(r"\{([^{}]*)\}", body)
    return np.array([[float.fromhex(v.strip()) for v in r.split(",")] for r in rows])


def test_table_is_the_generator_output(tmp_path):
    pytest.importorskip("mpmath")
    src = os.path.join(CSRC, "gen_erf_table.py")
    work = tmp_path / "csrc"
    work.mkdir()
    (work / "gen_erf_table.py").write_text(open(src).read())
    subprocess.run([sys.executable, str(work / "gen_erf_table.py")], check=True)
    assert (work / "erf_table.h").read_text() == open(os.path.join(CSRC, "erf_table.h")).read()


def test_table_reproduces_erf_and_exp():
    T = _table()
    assert T.shape == (193, 20)
    assert np.all(T[:, 0] == np.arange(193) / 32.0)
    S = np.linspace(-6.0, 6.0, 400001)
    a = np.abs(S)
    k = np.minimum(np.rint(a * 32).astype(int), 192)
    d = a - T[k, 0]
    c = T[k, 1:10]
    e = T[k, 10:19]
    erf = c[:, 8]
    ex = e[:, 8]
    for n in range(7, -1, -1):
        erf = erf * d + c[:, n]
        ex = ex * d + e[:, n]
    erf = np.copysign(erf, S)
    ref_erf = np.array([math.erf(x) for x in S])
    assert np.max(np.abs(erf - ref_erf)) <= 2.3e-16
    assert np.max(np.abs(ex - np.exp(-S * S))) <= 2.3e-16
    # half a grid step off the nodes as well (the largest |d| of the device)
    off = (np.arange(192) + 0.5) / 32.0
    assert np.max(np.abs(np.array([math.erf(x) for x in off]) -
                         np.array([np.polyval(T[j, 9:0:-1], 1 / 64) for j in range(192)]))) <= 2.3e-16
