// Double-word ("double-float") numbers on the FP32 pipe: a value is the unevaluated sum hi + lo of
// two floats with |lo| <= ulp(hi) / 2, about 48 significant bits.  GB300 issues FP32 arithmetic
// about 60 times faster than FP64, so vectors held and updated in this form keep the streaming
// passes bound by memory bandwidth (8 bytes per element, as FP64) instead of by the FP64 units,
// at a unit roundoff of about 2^-47 instead of FP32's 2^-24.
//
// Building blocks are error-free transformations: TwoSum (Knuth, TAOCP vol. 2, 4.2.2), Fast2Sum
// (Dekker 1971, valid when |a| >= |b| or a = 0) and TwoProd with one FMA.  Addition is the
// accurate double-word sum and multiplication the double-word product of Joldes, Muller &
// Popescu, "Tight and rigorous error bounds for basic building blocks of double-word arithmetic",
// ACM Trans. Math. Softw. 44 (2017): relative errors below 3u^2 / (1 - 4u) and 5u^2 (u = 2^-24).
// The *_rn intrinsics keep the compiler from contracting or reassociating the error terms.
#pragma once
#include <cuda_runtime.h>

namespace bmr {

struct __align__(8) dw {
  float hi, lo;
  dw() = default;
  __host__ __device__ constexpr dw(int i) : hi((float)i), lo(0.0f) {}
  __device__ explicit dw(float f) : hi(f), lo(0.0f) {}
  // round-to-nearest split of a double: hi = fl32(d), lo = fl32(d - hi) (FP64 arithmetic)
  __device__ explicit dw(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __device__ static dw make(float h, float l) {
    dw z;
    z.hi = h;
    z.lo = l;
    return z;
  }
};

__device__ __forceinline__ double to_double(dw x) { return (double)x.hi + (double)x.lo; }

// s + t == a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}
// s + t == a + b exactly when |a| >= |b|
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  t = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ dw dw_add(dw x, dw y) {
  float sh, sl, th, tl, vh, vl, zh, zl;
  two_sum(x.hi, y.hi, sh, sl);
  two_sum(x.lo, y.lo, th, tl);
  const float c = __fadd_rn(sl, th);
  fast_two_sum(sh, c, vh, vl);
  const float w = __fadd_rn(tl, vl);
  fast_two_sum(vh, w, zh, zl);
  return dw::make(zh, zl);
}

__device__ __forceinline__ dw dw_mul(dw x, dw y) {
  const float ch = __fmul_rn(x.hi, y.hi);
  const float cl1 = __fmaf_rn(x.hi, y.hi, -ch);  // ch + cl1 == x.hi * y.hi exactly
  const float tl0 = __fmul_rn(x.lo, y.lo);
  const float tl1 = __fmaf_rn(x.hi, y.lo, tl0);
  const float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
  const float cl3 = __fadd_rn(cl1, cl2);
  float zh, zl;
  fast_two_sum(ch, cl3, zh, zl);
  return dw::make(zh, zl);
}

// a * b + c for the streaming passes: the product of the high parts exactly (TwoProd), the cross
// terms by FMA, then one error-free sum with c.hi and a Fast2Sum renormalisation (15 FP32
// operations instead of 28 for dw_add(dw_mul)).  The error is a few u^2 (|a b| + |c|): under
// cancellation it is absolute rather than relative, i.e. of the order of the rounding already
// present in the double-word operands, which is what an update w - h u or a dot product needs.
__device__ __forceinline__ dw dw_fma(dw a, dw b, dw c) {
  const float ph = __fmul_rn(a.hi, b.hi);
  float pl = __fmaf_rn(a.hi, b.hi, -ph);
  pl = __fmaf_rn(a.hi, b.lo, pl);
  pl = __fmaf_rn(a.lo, b.hi, pl);
  float sh, sl, zh, zl;
  two_sum(ph, c.hi, sh, sl);
  sl = __fadd_rn(sl, __fadd_rn(pl, c.lo));
  fast_two_sum(sh, sl, zh, zl);
  return dw::make(zh, zl);
}

__device__ __forceinline__ dw operator-(dw x) { return dw::make(-x.hi, -x.lo); }
__device__ __forceinline__ dw operator+(dw x, dw y) { return dw_add(x, y); }
__device__ __forceinline__ dw operator-(dw x, dw y) { return dw_add(x, -y); }
__device__ __forceinline__ dw operator*(dw x, dw y) { return dw_mul(x, y); }
__device__ __forceinline__ dw& operator+=(dw& x, dw y) { return x = dw_add(x, y); }
__device__ __forceinline__ dw& operator-=(dw& x, dw y) { return x = dw_add(x, -y); }
__device__ __forceinline__ dw& operator*=(dw& x, dw y) { return x = dw_mul(x, y); }

}  // namespace bmr
