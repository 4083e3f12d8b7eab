// Double-word ("double-float") arithmetic on the FP32 pipes: a value is the
// unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2, carrying about
// 48 significant bits (unit roundoff u^2 with u = 2^-24, about 3.6e-15).  On
// B300 an FP32 FMA issues at ~58x the FP64 rate, so a double-word add (11 FP32
// operations) or multiply (7) costs a fraction of one FP64 operation.
//
// Building blocks (error-free transformations):
//   TwoSum      Knuth, The Art of Computer Programming vol. 2, Sec 4.2.2;
//   Fast2Sum    Dekker, "A floating-point technique for extending the
//               available precision", Numer. Math. 18 (1971);
//   TwoProd     with a fused multiply-add;
// and the double-word algorithms of Joldes, Muller and Popescu, "Tight and
// rigorous error bounds for basic building blocks of double-word arithmetic",
// ACM TOMS 44(2), 2017: the "sloppy" double-word sum (absolute error of order
// u^2 (|x| + |y|)), the double-word product with FMAs, and a double-word
// quotient refined by Newton corrections.  The square root takes one Newton
// step from the FP32 root.  exp and erfc go through the FP64 functions.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace cgks {

// the FP64 overloads stay visible next to the double-word ones below
using ::erfc;
using ::exp;
using ::fabs;
using ::sqrt;
using ::pow;

struct dword {
  float hi, lo;
  dword() = default;
  __host__ __device__ constexpr dword(float h, float l) : hi(h), lo(l) {}
  // exact for |x| in float range up to the 48-bit rounding of the split; a
  // compile-time constant folds to two float literals
  __host__ __device__ constexpr explicit dword(double x)
      : hi(static_cast<float>(x)), lo(static_cast<float>(x - static_cast<double>(static_cast<float>(x)))) {}
  __host__ __device__ constexpr explicit dword(int x) : hi(static_cast<float>(x)), lo(0.0f) {}
  __host__ __device__ explicit operator double() const { return static_cast<double>(hi) + static_cast<double>(lo); }
};

namespace dw {
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ dword add(dword x, dword y) {
  float s, e;
  two_sum(x.hi, y.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(x.lo, y.lo));
  float h, l;
  fast_two_sum(s, e, h, l);
  return dword(h, l);
}
__device__ __forceinline__ dword add(dword x, float y) {
  float s, e;
  two_sum(x.hi, y, s, e);
  e = __fadd_rn(e, x.lo);
  float h, l;
  fast_two_sum(s, e, h, l);
  return dword(h, l);
}
__device__ __forceinline__ dword mul(dword x, dword y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  float h, l;
  fast_two_sum(p, e, h, l);
  return dword(h, l);
}
__device__ __forceinline__ dword mul(dword x, float y) {
  const float p = __fmul_rn(x.hi, y);
  float e = __fmaf_rn(x.hi, y, -p);
  e = __fmaf_rn(x.lo, y, e);
  float h, l;
  fast_two_sum(p, e, h, l);
  return dword(h, l);
}
// x / y: q1 = x.hi / y.hi from the FP32 reciprocal, then two corrections
// q_{k+1} = (x - q y).hi / y.hi with the remainder formed in double-word.
__device__ __forceinline__ dword div(dword x, dword y) {
  const float r = __frcp_rn(y.hi);
  const float q1 = __fmul_rn(x.hi, r);
  dword t = mul(y, q1);
  dword rem = add(x, dword(-t.hi, -t.lo));
  const float q2 = __fmul_rn(rem.hi, r);
  t = mul(y, q2);
  rem = add(rem, dword(-t.hi, -t.lo));
  const float q3 = __fmul_rn(rem.hi, r);
  float h, l;
  fast_two_sum(q1, q2, h, l);
  return add(dword(h, l), q3);
}
// sqrt(x), x >= 0: s0 = sqrtf(x.hi), s = s0 + (x - s0^2) / (2 s0)
__device__ __forceinline__ dword sqrt(dword x) {
  if (!(x.hi > 0.0f)) return dword(0.0f, 0.0f);
  const float s0 = __fsqrt_rn(x.hi);
  const float p = __fmul_rn(s0, s0);
  const float pe = __fmaf_rn(s0, s0, -p);
  // x - s0^2 (its leading part cancels, so the float sum below is exact enough)
  const float d = __fadd_rn(__fadd_rn(__fsub_rn(x.hi, p), -pe), x.lo);
  const float c = __fdiv_rn(d, __fmul_rn(2.0f, s0));
  float h, l;
  fast_two_sum(s0, c, h, l);
  return dword(h, l);
}
}  // namespace dw

__device__ __forceinline__ dword operator-(dword x) { return dword(-x.hi, -x.lo); }
__device__ __forceinline__ dword operator+(dword x, dword y) { return dw::add(x, y); }
__device__ __forceinline__ dword operator-(dword x, dword y) { return dw::add(x, -y); }
__device__ __forceinline__ dword operator*(dword x, dword y) { return dw::mul(x, y); }
__device__ __forceinline__ dword operator/(dword x, dword y) { return dw::div(x, y); }
// int operands are small exact integers (loop indices, signs)
__device__ __forceinline__ dword operator*(int a, dword x) { return dw::mul(x, static_cast<float>(a)); }
__device__ __forceinline__ dword operator*(dword x, int a) { return dw::mul(x, static_cast<float>(a)); }
__device__ __forceinline__ dword& operator+=(dword& x, dword y) { return x = x + y; }
__device__ __forceinline__ dword& operator-=(dword& x, dword y) { return x = x - y; }
__device__ __forceinline__ dword& operator*=(dword& x, dword y) { return x = x * y; }
__device__ __forceinline__ bool operator>(dword x, dword y) { return x.hi > y.hi || (x.hi == y.hi && x.lo > y.lo); }
__device__ __forceinline__ bool operator<(dword x, dword y) { return y > x; }
__device__ __forceinline__ dword fabs(dword x) { return (x.hi < 0.0f || (x.hi == 0.0f && x.lo < 0.0f)) ? -x : x; }
__device__ __forceinline__ dword sqrt(dword x) { return dw::sqrt(x); }
__device__ __forceinline__ dword to_dword(double x) { return dword(x); }
__device__ __forceinline__ dword exp(dword x) { return dword(::exp(static_cast<double>(x))); }
__device__ __forceinline__ dword pow(dword x, dword y) {
  return dword(::pow(static_cast<double>(x), static_cast<double>(y)));
}
__device__ __forceinline__ dword erfc(dword x) { return dword(::erfc(static_cast<double>(x))); }

// scalar-generic helpers used by the templated flux code
template <typename S>
__device__ __forceinline__ S scal(double c) { return S(c); }
template <typename S>
__device__ __forceinline__ double to_double(S x) { return static_cast<double>(x); }

}  // namespace cgks
