"""Writes special_tables.inc, the tables of special.cuh: the coefficients of the
scaled complementary error function erfcx(x) = exp(x^2) erfc(x), and 2^(j/64)
for j = 0..63 (the table of the exponential), each rounded to the nearest double.

    python paper_2509_06347_b300/csrc/gen_special_tables.py

On [0, 8): 128 intervals of width 1/16; on each, the degree-7 polynomial in
s = x - centre that interpolates erfcx at the 8 Chebyshev points of the
interval (evaluated with mpmath at 40 digits), converted to monomial
coefficients.  On [8, inf): g(z) = x sqrt(pi) erfcx(x) with z = 64 / x^2 in
(0, 1], interpolated at 11 Chebyshev points of [0, 1] by a degree-10
polynomial in z (g is smooth there: its asymptotic series in z has terms
(2k-1)!! (z/128)^k).  The script prints the largest relative error of both
parts against mpmath, evaluated with double-precision Horner steps.
"""
import os

import mpmath as mp
import numpy as np

mp.mp.dps = 40
WIDTH, N_INT, DEG = 1.0 / 16.0, 128, 7
DEG_TAIL = 10


def erfcx(x):
    return mp.exp(x * x) * mp.erfc(x)


def cheb_points(n, a, b):
    k = np.arange(n)
    t = np.cos((2 * k + 1) * np.pi / (2 * n))
    return [mp.mpf(a) + (mp.mpf(b) - mp.mpf(a)) * (mp.mpf(float(v)) + 1) / 2 for v in t]


def monomial_fit(points, values, deg, origin):
    V = mp.matrix([[(p - origin) ** j for j in range(deg + 1)] for p in points])
    c = mp.lu_solve(V, mp.matrix(values))
    return [float(c[j]) for j in range(deg + 1)]


def horner(c, s):
    h = c[-1]
    for a in reversed(c[:-1]):
        h = h * s + a
    return h


def main():
    rows, worst = [], 0.0
    for i in range(N_INT):
        a, b = i * WIDTH, (i + 1) * WIDTH
        c = (a + b) / 2
        pts = cheb_points(DEG + 1, a, b)
        co = monomial_fit(pts, [erfcx(p) for p in pts], DEG, mp.mpf(c))
        rows.append([c] + co)
        for x in np.linspace(a, b, 33):
            ref = erfcx(mp.mpf(float(x)))
            worst = max(worst, float(abs((horner(co, float(x) - c) - ref) / ref)))
    pts = cheb_points(DEG_TAIL + 1, 0.0, 1.0)

    def g(z):
        x = 8 / mp.sqrt(z)
        return x * mp.sqrt(mp.pi) * erfcx(x)

    tail = monomial_fit(pts, [g(p) for p in pts], DEG_TAIL, mp.mpf(0))
    worst_tail = 0.0
    for z in np.linspace(1e-9, 1.0, 257):
        ref = g(mp.mpf(float(z)))
        worst_tail = max(worst_tail, float(abs((horner(tail, float(z)) - ref) / ref)))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "special_tables.inc")
    with open(out, "w") as f:
        f.write("// Generated by gen_special_tables.py.  erfcx on [0, 8) in 128 intervals of width 1/16,\n")
        f.write("// rows {centre, a0..a7, 0} of the degree-7 polynomial in x - centre; then the\n")
        f.write(f"// degree-{DEG_TAIL} polynomial in z = 64 / x^2 of x sqrt(pi) erfcx(x) for x >= 8.\n")
        f.write(f"// Largest relative error (double Horner vs mpmath): {worst:.2e} on [0, 8), "
                f"{worst_tail:.2e} beyond.\n")
        f.write(f"__device__ __align__(16) const double kErfcxTable[{N_INT}][10] = {{\n")
        for r in rows:
            f.write("    {" + ", ".join(repr(float(v)) for v in r) + ", 0.0},\n")
        f.write("};\n")
        f.write(f"__device__ const double kErfcxTail[{DEG_TAIL + 1}] = {{"
                + ", ".join(repr(v) for v in tail) + "};\n")
        f.write("// 2^(j/64), j = 0..63\n")
        f.write("__device__ const double kExp2Table[64] = {"
                + ", ".join(repr(float(mp.mpf(2) ** (mp.mpf(j) / 64))) for j in range(64)) + "};\n")
    print(out, f"worst relative error {worst:.3e} (table), {worst_tail:.3e} (tail)")


if __name__ == "__main__":
    main()
