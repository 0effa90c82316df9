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

// ---- conversions without the FP64 pipe
// GB300's FP64 pipe (2 lanes per clock per SM) also executes the FP32 <-> FP64 conversions, so
// converting every operand of a df64 kernel that way (4 FP64-pipe instructions per value in,
// 3 out) kept that pipe 40% busy and stalled the FP32 work.  These conversions use integer and
// FP32 instructions on the bit patterns instead.

// FP64 -> df64: hi = the FP64 value truncated to 24 significant bits (exponent rebiased), lo =
// the next 23 bits of its significand, scaled (|lo| < ulp(hi); about 47 bits in all).  Values
// outside 2^-103 <= |d| < 2^128 (zero, tiny, huge, inf, NaN) take the FP64 route above.
__device__ __forceinline__ df64 df_from_double(double d) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(d);
  const unsigned hw = (unsigned)(bits >> 32), lw = (unsigned)bits;
  const int ex = (int)((hw >> 20) & 0x7FFu);
  if (ex < 920 || ex > 1150) return df64(d);
  const unsigned sign = hw & 0x80000000u;
  const unsigned mh = ((hw & 0xFFFFFu) << 3) | (lw >> 29);                    // top 23 bits
  const float hi = __uint_as_float(sign | ((unsigned)(ex - 896) << 23) | mh);
  const float frac = __fsub_rn(__uint_as_float(0x3F800000u | ((lw >> 6) & 0x7FFFFFu)), 1.0f);
  const float scale = __uint_as_float(sign | ((unsigned)(ex - 919) << 23));   // 2^(ex - 1046)
  return df64(hi, __fmul_rn(frac, scale));
}

// FP32 -> FP64 bit pattern (exact for normal numbers; FP32 subnormals become signed zero).
__device__ __forceinline__ double f32_to_f64_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xFFu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned long long mant = (unsigned long long)(u & 0x7FFFFFu) << 29;
  const unsigned long long e64 = ex == 255u ? 2047ull : (unsigned long long)(ex + 896u);
  const unsigned long long b = ex == 0u ? sign : (sign | (e64 << 52) | mant);
  return __longlong_as_double((long long)b);
}

// df64 -> FP64: one FP64 addition of the two exactly converted parts.
__device__ __forceinline__ double df_to_double(df64 v) {
  return f32_to_f64_bits(v.hi) + f32_to_f64_bits(v.lo);
}

template <class T>
struct is_df64 {
  static constexpr bool value = false;
};
template <>
struct is_df64<df64> {
  static constexpr bool value = true;
};

// ---- dot products
// Accumulator of a df64 dot product: s is the running FP32 sum of the leading product terms,
// kept error-free by TwoSum; c collects every lower-order part (the TwoProd error, the cross
// terms, the TwoSum errors) in plain FP32.  The pair is renormalised once, at the end: 12 FP32
// instructions per term instead of the 15 of a df64 FMA, with an error bound relative to the sum
// of the terms' magnitudes (as for an FP64 dot product).
struct df_acc {
  float s = 0.0f, c = 0.0f;
};

__device__ __forceinline__ void df_acc_fma(df_acc& A, df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const df64 t = df_two_sum(A.s, p);
  A.s = t.hi;
  A.c = __fadd_rn(A.c, __fadd_rn(t.lo, e));
}

// A + B of two accumulators, renormalised
__device__ __forceinline__ df64 df_acc_merge(const df_acc& A, const df_acc& B) {
  const df64 t = df_two_sum(A.s, B.s);
  return df_fast_two_sum(t.hi, __fadd_rn(t.lo, __fadd_rn(A.c, B.c)));
}

__device__ __forceinline__ df64 df_acc_value(const df_acc& A) { return df_fast_two_sum(A.s, A.c); }

// Conversion between a kernel's storage type IO and its arithmetic type T.
template <class IO, class T>
__device__ __forceinline__ IO io_cast(T v) {
  if constexpr (is_df64<T>::value && !is_df64<IO>::value) return df_to_double(v);
  else return static_cast<IO>(v);
}
template <class T, class IO>
__device__ __forceinline__ T from_io(IO v) {
  if constexpr (is_df64<T>::value && !is_df64<IO>::value) return df_from_double((double)v);
  else return T(v);
}

}  // namespace se
