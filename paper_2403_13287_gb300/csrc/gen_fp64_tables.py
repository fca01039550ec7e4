"""Write fp64_tables.h: the tables of the FP64 flux kernel's elementary functions.

1. erf(S) and exp(-S^2), Taylor coefficients on a grid.

The FP64 split fluxes need erf(S) and exp(-S^2) of the same S. On the grid
s_k = k/1024, k = 0..6144 (0 <= s <= 6), each row holds s_k and the degree-4
Taylor coefficients in d = s - s_k of

    erf(s_k + d)      : c_n = erf^(n)(s_k) / n!
    exp(-(s_k + d)^2) : e_n = (-1)^n H_n(s_k) exp(-s_k^2) / n!

(H_n the physicists' Hermite polynomials, d^n/dx^n exp(-x^2) =
(-1)^n H_n(x) exp(-x^2), and erf' = 2/sqrt(pi) exp(-x^2), so
c_n = 2/sqrt(pi) e_{n-1} / n for n >= 1). With |d| <= 1/2048 the first
omitted terms, d^5/5! times |H_5(s) exp(-s^2)| <= 32 (or 2/sqrt(pi) |H_4|
<= 14 for erf), are below 1e-17, so each function comes out of one table
row and a Horner chain of 4 steps to about one unit in the last place of 1.
The split fluxes take erf only through 1 +- erf(S), so this absolute error
is the measure. A finer grid with a lower degree means fewer FP64
operations per evaluation for a larger table (576 KB): the FP64 pipe, not
the cache, bounds the kernels that use it. The values are computed with
mpmath at 50 significant digits and written as exactly rounded
hexadecimal doubles.

2. exp(x), table-driven (P. T. P. Tang, ACM Trans. Math. Software 15 (1989)
144-157): x = n ln2/4096 + r with |r| <= ln2/8192 and n = 4096 m + j, so
exp(x) = 2^m 2^(j/4096) p(r), p the degree-3 Taylor polynomial of exp
(truncation r^4/24 below 3e-18). The table holds 2^(j/4096), j = 0..4095,
exactly rounded (32 KB); ln2/4096 is split into a head with 31 significant
bits (so that n * head is exact for |n| < 2^22, which covers |x| < 708) and
the rounded remainder.

Run from the repository root:  python paper_2403_13287_gb300/csrc/gen_fp64_tables.py
"""
import os

import mpmath as mp

mp.mp.dps = 50
STEP = 1024        # grid points per unit of s
KMAX = 6144        # s_k up to 6
DEG = 4
EXP_N = 4096       # entries of the 2^(j/N) table
EXP_HEAD_BITS = 31 # significant bits of the head of ln2/N


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
        "// Generated by gen_fp64_tables.py (mpmath, 50 digits): do not edit.",
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
    # exp: 2^(j/512) and the split of ln2/512
    L = mp.log(2) / EXP_N
    m_, e_ = mp.frexp(L)                       # L = m_ 2^e_, 1/2 <= m_ < 1
    head = mp.ldexp(mp.floor(mp.ldexp(m_, EXP_HEAD_BITS)), e_ - EXP_HEAD_BITS)
    tail = L - head
    lines += [
        "",
        "// exp(x) = 2^m 2^(j/%d) p(r), x = (%d m + j) ln2/%d + r (Tang's table-driven method)" % (EXP_N, EXP_N, EXP_N),
        "#define LSKUM_EXP_N %d" % EXP_N,
        "#define LSKUM_EXP_LOG2N %d" % (EXP_N.bit_length() - 1),
        "#define LSKUM_EXP_INV_L %s   // %d/ln2" % (float(EXP_N / mp.log(2)).hex(), EXP_N),
        "#define LSKUM_EXP_L_HI %s    // ln2/%d, %d significant bits" % (float(head).hex(), EXP_N, EXP_HEAD_BITS),
        "#define LSKUM_EXP_L_LO %s    // ln2/%d - LSKUM_EXP_L_HI" % (float(tail).hex(), EXP_N),
        "__device__ __align__(16) const double kExp2Table[%d] = {" % EXP_N,
    ]
    vals = [float(mp.mpf(2) ** (mp.mpf(j) / EXP_N)).hex() for j in range(EXP_N)]
    for j in range(0, EXP_N, 4):
        lines.append("    " + ", ".join(vals[j:j + 4]) + ",")
    lines.append("};")
    with open(os.path.join(here, "fp64_tables.h"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
