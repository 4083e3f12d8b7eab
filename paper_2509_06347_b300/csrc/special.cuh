// The complementary error function of the half-space Maxwellian moments
// (Sec 2.3, and the KFVS flux of the coarse levels), built for a kernel bound
// by the FP64 pipe.  The moments already hold E = exp(-lambda U^2), so
//   erfc(x) = E * erfcx(x)          (x >= 0)
//   erfc(x) = 2 - E * erfcx(-x)     (x < 0),   x^2 = lambda U^2,
// with the scaled function erfcx(x) = exp(x^2) erfc(x) taken from piecewise
// polynomials: 128 intervals of width 1/16 on [0, 8) with a degree-7
// interpolant at Chebyshev points on each, and beyond 8 a degree-10
// polynomial in z = 64 / x^2 of x sqrt(pi) erfcx(x) (coefficients written by
// gen_erfcx_table.py from mpmath; largest relative error 3.6e-16).  That costs
// about 10 FP64 instructions against about 75 for a library erfc; the table
// lookups and the interval index run on the load and FP32 pipes.
#pragma once

#include <cuda_runtime.h>

#include "dword.cuh"

namespace cgks {

#include "erfcx_table.inc"

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

__device__ __forceinline__ double erfc_with_exp(double x, double E) {
  const double h = erfcx_pos(fabs(x));
  return x >= 0.0 ? E * h : fma(-E, h, 2.0);
}

__device__ __forceinline__ dword erfc_with_exp(dword x, dword E) {
  const dword h(erfcx_pos(fabs(static_cast<double>(x))));
  return x < dword(0.0) ? dword(2.0) - E * h : E * h;
}

}  // namespace cgks
