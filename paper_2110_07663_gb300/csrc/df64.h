// Double-float ("df64") arithmetic on the FP32 pipe.
//
// A df64 value is the unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2, about
// 48 significant bits.  GB300 executes FP32 FMAs at 64 times its FP64 rate, so the two kernels of
// this path that are bound by arithmetic (the sum-factorised operator and the FDM solves) can
// compute to about FP64 accuracy several times faster in df64 than in FP64 while their vectors
// stay FP64 in memory.
//
// The operations are the classical error-free transformations: Knuth's TwoSum, Dekker's
// FastTwoSum, and TwoProd by FMA (Dekker 1971; Knuth, TAOCP vol. 2; Hida, Li and Bailey's
// double-double library describes the same combinations).  Addition is the "sloppy" variant:
// its error is bounded relative to |a| + |b| (not |a + b|), the same kind of bound an FP64 sum
// of products has.  Every step uses the _rn intrinsics, which the compiler never contracts or
// reassociates.  Range: FP32's exponent range; a value below about 1e-30 in magnitude loses
// low-order bits (its lo part leaves the normal range), so callers keep operands well inside
// [1e-30, 1e30] (the operator inputs of this path are O(1) solution and residual vectors and
// geometric factors of order 1e-6 to 1e2).
#pragma once

#include <cuda_runtime.h>

namespace se {

using ::fma;  // the df64 overload below must not hide the FP64 and FP32 ones inside namespace se

struct __align__(8) df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  // nearest df64 of an FP64 value: hi = fl32(d), lo = fl32(d - hi) (d - hi is exact in FP64)
  __host__ __device__ explicit df64(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ df64 df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df64(s, e);
}

__device__ __forceinline__ df64 df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df64(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  const df64 s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }

__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}

__device__ __forceinline__ df64& operator+=(df64& a, df64 b) {
  a = a + b;
  return a;
}

// a * b + c with one renormalisation
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const df64 s = df_two_sum(c.hi, p);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, c.lo)));
}

// Conversion between a kernel's storage type IO and its arithmetic type T.
template <class IO, class T>
__device__ __forceinline__ IO io_cast(T v) {
  return static_cast<IO>(v);
}

template <class T>
struct is_df64 {
  static constexpr bool value = false;
};
template <>
struct is_df64<df64> {
  static constexpr bool value = true;
};

}  // namespace se
