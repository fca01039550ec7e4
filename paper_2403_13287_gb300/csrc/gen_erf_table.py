"""Write erf_table.h: Taylor coefficients of erf(s) and exp(-s^2) on a grid.

The FP64 split fluxes need erf(S) and exp(-S^2) of the same S. On the grid
s_k = k/32, k = 0..192 (0 <= s <= 6), each row holds s_k and the degree-8
Taylor coefficients in d = s - s_k of

    erf(s_k + d)      : c_n = erf^(n)(s_k) / n!
    exp(-(s_k + d)^2) : e_n = (-1)^n H_n(s_k) exp(-s_k^2) / n!

(H_n the physicists' Hermite polynomials, d^n/dx^n exp(-x^2) =
(-1)^n H_n(x) exp(-x^2), and erf' = 2/sqrt(pi) exp(-x^2), so
c_n = 2/sqrt(pi) e_{n-1} / n for n >= 1). With |d| <= 1/64 the first
omitted terms are below 1e-18, so each function comes out of one table row
and two Horner chains to about one unit in the last place of 1. The values
are computed with mpmath at 50 significant digits and written as exactly
rounded hexadecimal doubles.

Run from the repository root:  python paper_2403_13287_gb300/csrc/gen_erf_table.py
"""
import os

import mpmath as mp

mp.mp.dps = 50
STEP = 32          # grid points per unit of s
KMAX = 192         # s_k up to 6
DEG = 8


def hermite(n, x):
    h0, h1 = mp.mpf(1), 2 * x
    if n == 0:
        return h0
    for k in range(1, n):
        h0, h1 = h1, 2 * x * h1 - 2 * k * h0
    return h1


def row(k):
    s = mp.mpf(k) / STEP
    g = mp.e ** (-s * s)
    e = [(-1) ** n * hermite(n, s) * g / mp.factorial(n) for n in range(DEG + 1)]
    c = [mp.erf(s)] + [2 / mp.sqrt(mp.pi) * e[n - 1] / n for n in range(1, DEG + 1)]
    return [s] + c + e


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    rows = [row(k) for k in range(KMAX + 1)]
    width = 1 + 2 * (DEG + 1)
    lines = [
        "// Generated by gen_erf_table.py (mpmath, 50 digits): do not edit.",
        "// Row k: s_k = k/%d, then the degree-%d Taylor coefficients in d = s - s_k" % (STEP, DEG),
        "// of erf(s) (c_0..c_%d) and of exp(-s^2) (e_0..e_%d); one padding entry." % (DEG, DEG),
        "#pragma once",
        "",
        "#define LSKUM_ERF_STEP %d" % STEP,
        "#define LSKUM_ERF_KMAX %d" % KMAX,
        "#define LSKUM_ERF_DEG %d" % DEG,
        "#define LSKUM_ERF_ROW %d" % (width + 1),
        "",
        "__device__ __align__(16) const double kErfExpTable[%d][%d] = {" % (KMAX + 1, width + 1),
    ]
    for r in rows:
        vals = [float(v).hex() for v in r] + ["0x0.0p+0"]
        lines.append("    {" + ", ".join(vals) + "},")
    lines.append("};")
    with open(os.path.join(here, "erf_table.h"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
