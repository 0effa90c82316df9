// Device helpers shared by the reduction kernels: unique-node weights applied by exponent
// arithmetic and a deterministic block reduction (fixed shuffle tree).
#pragma once

#include "se_internal.h"

namespace se {

// log2 of the multiplicity stored in the low bits of a point flag (1, 2, 4, 8 -> 0..3)
__device__ __forceinline__ int mult_log2(uint8_t f) { return __ffs(f & 0x0F) - 1; }

// a * 2^-k for k in 0..3 by exponent arithmetic (integer ops only).  Values whose exponent
// would underflow (|a| < 2^-1019, including zero and subnormals) give 0; NaN/Inf pass through.
__device__ __forceinline__ double scale_pow2(double a, int k) {
  const long long b = __double_as_longlong(a);
  const long long e = (b >> 52) & 0x7FF;
  const long long r = b - ((long long)k << 52);
  return __longlong_as_double(e == 0x7FF ? b : (e > k ? r : 0LL));
}

// The FP32 form: |a| < 2^-123 (zero and subnormals included) gives 0; NaN/Inf pass through.
__device__ __forceinline__ float scale_pow2(float a, int k) {
  const int b = __float_as_int(a);
  const int e = (b >> 23) & 0xFF;
  return __int_as_float(e == 0xFF ? b : (e > k ? b - (k << 23) : 0));
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block-reduce K values (deterministic shuffle tree); result valid in thread 0.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double (*sh)[RED_THREADS / 32]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = warp_sum(v[k]);
    if (lane == 0) sh[k][warp] = s;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = lane < RED_THREADS / 32 ? sh[k][lane] : 0.0;
      v[k] = warp_sum(s);
    }
  }
  __syncthreads();
}

}  // namespace se
