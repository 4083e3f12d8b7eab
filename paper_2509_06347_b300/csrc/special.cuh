// The exponential and the complementary error function of the half-space
// Maxwellian moments and of the time integrals (Sec 2.3, and the KFVS flux of
// the coarse levels), built for kernels bound by the FP64 pipe, where every
// FP64 instruction counts and table loads, integer and FP32 work are nearly
// free.
//
// exp(x), x <= 0, follows Tang's table-driven method (ACM TOMS 15, 1989):
// x = (64 k + j) ln2/64 + r with |r| <= ln2/128, exp(x) = 2^k 2^(j/64) e^r,
// e^r from its degree-5 Taylor polynomial (truncation below 3.5e-17), 2^(j/64)
// from a table, 2^k added to the exponent bits: about 12 FP64 instructions
// against about 19 for the library exp.  Results below 2^-1009 (x <= -700)
// are returned as 0, and so is erfc(x) for x^2 >= 700 (below 2^-1000).
//
// The moments already hold E = exp(-lambda U^2), so
//   erfc(x) = E * erfcx(x)          (x >= 0)
//   erfc(x) = 2 - E * erfcx(-x)     (x < 0),   x^2 = lambda U^2,
// with the scaled function erfcx(x) = exp(x^2) erfc(x) taken from piecewise
// polynomials: 128 intervals of width 1/16 on [0, 8) with a degree-7
// interpolant at Chebyshev points on each, and beyond 8 a degree-10
// polynomial in z = 64 / x^2 of x sqrt(pi) erfcx(x) (coefficients written by
// gen_special_tables.py from mpmath; largest relative error 3.6e-16).  That costs
// about 10 FP64 instructions against about 75 for a library erfc; the table
// lookups and the interval index run on the load and FP32 pipes.
#pragma once

#include <cuda_runtime.h>

#include "dword.cuh"

namespace cgks {

#include "special_tables.inc"

// exp(x) for x <= 0 (x > 0 is outside its use and not handled; NaN -> NaN)
__device__ __forceinline__ double exp_neg(double x) {
  if (!(x > -700.0)) return x != x ? x : 0.0;
  // n = round(x 64 / ln2) in the low bits of t (round-to-nearest by the 1.5 * 2^52 shift)
  const double t = fma(x, 92.33248261689366, 6755399441055744.0);
  const int n = __double2loint(t);
  const double nd = t - 6755399441055744.0;
  // r = x - n ln2/64, with ln2/64 = L1 + L2 (L1 has 21 significant bits)
  double r = fma(nd, -0.010830417275428772, x);
  r = fma(nd, -7.420820373486988e-09, r);
  double q = fma(r, 1.0 / 120.0, 1.0 / 24.0);
  q = fma(q, r, 1.0 / 6.0);
  q = fma(q, r, 0.5);
  q = fma(q, r, 1.0);
  const double T = __ldg(&kExp2Table[n & 63]);
  const double m = fma(T, r * q, T);  // 2^(j/64) e^r, in [0.99, 2)
  // times 2^k, k = floor(n / 64) >= -1010: add k to the exponent field
  return __hiloint2double(__double2hiint(m) + ((n >> 6) << 20), __double2loint(m));
}

// erfcx(x) for x >= 0 (also +inf -> 0; NaN -> NaN)
__device__ __forceinline__ double erfcx_pos(double x) {
  if (x < 8.0) {
    // interval index from the FP32 value: off by one only within an FP32
    // rounding of a boundary, where the neighbouring polynomial is as accurate
    const int i = min(max(static_cast<int>(__double2float_rz(x) * 16.0f), 0), 127);
    const double2* row = reinterpret_cast<const double2*>(kErfcxTable[i]);
    const double2 r0 = __ldg(row), r1 = __ldg(row + 1), r2 = __ldg(row + 2), r3 = __ldg(row + 3),
                  r4 = __ldg(row + 4);
    const double s = x - r0.x;
    double h = r4.x;
    h = fma(h, s, r3.y);
    h = fma(h, s, r3.x);
    h = fma(h, s, r2.y);
    h = fma(h, s, r2.x);
    h = fma(h, s, r1.y);
    h = fma(h, s, r1.x);
    h = fma(h, s, r0.y);
    return h;
  }
  const double r = 1.0 / x;
  const double z = 64.0 * r * r;
  double g = kErfcxTail[10];
#pragma unroll
  for (int k = 9; k >= 0; --k) g = fma(g, z, kErfcxTail[k]);
  return g * r * 0.56418958354775628;  // 1 / sqrt(pi)
}

__device__ __forceinline__ dword exp_neg(dword x) { return dword(exp_neg(static_cast<double>(x))); }

__device__ __forceinline__ double erfc_with_exp(double x, double E) {
  const double h = erfcx_pos(fabs(x));
  return x >= 0.0 ? E * h : fma(-E, h, 2.0);
}

__device__ __forceinline__ dword erfc_with_exp(dword x, dword E) {
  const dword h(erfcx_pos(fabs(static_cast<double>(x))));
  return x < dword(0.0) ? dword(2.0) - E * h : E * h;
}

}  // namespace cgks
