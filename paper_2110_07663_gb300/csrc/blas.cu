// Vector kernels of the Krylov solvers and smoothers: fused updates and deterministic
// unique-node inner products.
//
// GB300 executes FP64 at ~1/62 of its FP32 rate, so a streaming FP64 kernel has a budget of
// about one FP64 FMA per 11 bytes moved.  Inner products therefore apply the 1/multiplicity
// weight (1, 1/2, 1/4 or 1/8, exact powers of two) to one operand by lowering its binary
// exponent with integer instructions, leaving one FP64 FMA per point and product.
#include <algorithm>

#include "se_internal.h"
#include "reduce.h"

namespace se {

// Generic fused elementwise + reduction kernel.  Op provides:
//   static constexpr int K (number of reduced values, >= 1),
//   struct V (the values one point loads),
//   __device__ void setup()   (loop-invariant scalars, read once per thread into the op's copy),
//   __device__ V load(int64_t i) const,
//   __device__ void apply(int64_t i, const V& v, double (&acc)[K]) const   (stores, sums),
//   __device__ void finalize(const double* sums)   (K sums, called once by the last block).
// A thread walks its points (grid stride) U at a time: all loads of the U points are issued
// before the first store, since a store could alias a later point's load and would otherwise
// hold it back.  U = 4 for ops that load two vectors, 2 for more.  The grid is the blocks that
// are resident at once (fused_blocks), so no block waits for a second wave.  The points and the
// order of each thread's sums are those of the plain grid-stride loop over that grid.
constexpr int FUSED_U = 4;

template <class Op>
__global__ void __launch_bounds__(RED_THREADS) fused_kernel(Op op_in, int64_t n,
                                                            double* __restrict__ partial,
                                                            unsigned* __restrict__ counter) {
  constexpr int K = Op::K;
  constexpr int U = sizeof(typename Op::V) <= 24 ? FUSED_U : 2;
  Op op = op_in;
  op.setup();
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  const int64_t stride = (int64_t)gridDim.x * RED_THREADS;
  int64_t i = (int64_t)blockIdx.x * RED_THREADS + threadIdx.x;
  for (; i + (U - 1) * stride < n; i += U * stride) {
    typename Op::V v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = op.load(i + u * stride);
#pragma unroll
    for (int u = 0; u < U; ++u) op.apply(i + u * stride, v[u], acc);
  }
  for (; i < n; i += stride) op.apply(i, op.load(i), acc);
  {
    __shared__ double sh[K][RED_THREADS / 32];
    __shared__ bool last;
    double (&v)[K] = acc;
    block_sum<K>(v, sh);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < K; ++k) partial[(int64_t)blockIdx.x * K + k] = v[k];
      __threadfence();
      const unsigned t = atomicAdd(counter, 1u);
      last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double w[K];
#pragma unroll
    for (int k = 0; k < K; ++k) w[k] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += RED_THREADS)
#pragma unroll
      for (int k = 0; k < K; ++k) w[k] += __ldcg(partial + (int64_t)b * K + k);
    block_sum<K>(w, sh);
    if (threadIdx.x == 0) {
      op.finalize(w);
      *counter = 0u;
    }
  }
}

// Blocks of fused_kernel<Op> resident on the device at once (at most RED_MAX_BLOCKS), once per
// op type; the device's SM count, not a fixed one.
template <class Op>
static int64_t fused_blocks() {
  static const int64_t cap = [] {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fused_kernel<Op>, RED_THREADS, 0) != cudaSuccess ||
        sms < 1 || per_sm < 1)
      return (int64_t)RED_MAX_BLOCKS;
    return std::min<int64_t>(RED_MAX_BLOCKS, (int64_t)sms * per_sm);
  }();
  return cap;
}

template <class Op>
static int run_fused(const Op& op, int64_t n, Scratch& sc, cudaStream_t s, int kind, double bytes,
                     double flops) {
  ProfScope prof(kind, s, (double)n, bytes, flops);
  const unsigned blocks = grid_for(n, RED_THREADS, fused_blocks<Op>());
  fused_kernel<Op><<<blocks, RED_THREADS, 0, s>>>(op, n, sc.partial, sc.counter);
  SE_LAUNCH_CHECK();
  return SE_OK;
}

// ------------------------------------------------------------------ ops
struct DotOp {  // dst = (a, b)
  static constexpr int K = 1;
  const double* a;
  const double* b;
  const uint8_t* pf;
  double* dst;
  struct V { double a, b; uint8_t f; };
  __device__ void setup() {}
  __device__ V load(int64_t i) const { return {a[i], b[i], pf[i]}; }
  __device__ void apply(int64_t, const V& v, double (&acc)[1]) const {
    acc[0] = fma(scale_pow2(v.a, mult_log2(v.f)), v.b, acc[0]);
  }
  __device__ void finalize(const double* s) const { *dst = s[0]; }
};

int dot_weighted(const Level& lv, const double* a, const double* b, double* dst_dev, Scratch& sc,
                 cudaStream_t s) {
  return run_fused(DotOp{a, b, lv.pflag, dst_dev}, lv.L, sc, s, SE_K_KRYLOV, lv.L * 17.0, lv.L * 2.0);
}

// ------------------------------------------------------------------ simple elementwise kernels
template <class Tin, class Tout>
__global__ void convert_kernel(const Tin* __restrict__ in, Tout* __restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (Tout)in[i];
}
template <class Tin, class Tout>
int convert(const Tin* in, Tout* out, int64_t n, cudaStream_t s) {
  convert_kernel<Tin, Tout><<<grid_for(n, 256), 256, 0, s>>>(in, out, n);
  SE_LAUNCH_CHECK();
  return SE_OK;
}
template int convert<double, float>(const double*, float*, int64_t, cudaStream_t);
template int convert<float, double>(const float*, double*, int64_t, cudaStream_t);
template int convert<double, double>(const double*, double*, int64_t, cudaStream_t);
template int convert<float, float>(const float*, float*, int64_t, cudaStream_t);

template <class T>
int fill_zero(T* x, int64_t n, cudaStream_t s) {
  SE_CUDA(cudaMemsetAsync(x, 0, n * sizeof(T), s));
  return SE_OK;
}
template int fill_zero<double>(double*, int64_t, cudaStream_t);
template int fill_zero<float>(float*, int64_t, cudaStream_t);

// out may alias x or y (element-wise read before write)
template <class T>
__global__ void axpby_kernel(T a, const T* x, T b, const T* y, T* out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a * x[i] + b * y[i];
}
template <class T>
int axpby(T a, const T* x, T b, const T* y, T* out, int64_t n, cudaStream_t s) {
  ProfScope prof(SE_K_KRYLOV, s, (double)n, 3.0 * n * sizeof(T), 3.0 * n);
  axpby_kernel<T><<<grid_for(n, 256), 256, 0, s>>>(a, x, b, y, out, n);
  SE_LAUNCH_CHECK();
  return SE_OK;
}
template int axpby<double>(double, const double*, double, const double*, double*, int64_t, cudaStream_t);
template int axpby<float>(float, const float*, float, const float*, float*, int64_t, cudaStream_t);

template <class T>
__global__ void scale_mul_kernel(const T* __restrict__ a, const T* __restrict__ b,
                                 T* __restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i] * b[i];
}
template <class T>
int scale_mul(const T* a, const T* b, T* out, int64_t n, cudaStream_t s) {
  ProfScope prof(SE_K_JACOBI, s, (double)n, 3.0 * n * sizeof(T), (double)n);
  scale_mul_kernel<T><<<grid_for(n, 256), 256, 0, s>>>(a, b, out, n);
  SE_LAUNCH_CHECK();
  return SE_OK;
}
template int scale_mul<double>(const double*, const double*, double*, int64_t, cudaStream_t);
template int scale_mul<float>(const float*, const float*, float*, int64_t, cudaStream_t);

// Chebyshev recurrence step of Algorithm 2 (one pass):
//   s = dinv .* sv (Jacobi surrogate) or s = sv (Schwarz output, already S A d)
//   x = x + d (x = d when `first`), r = r - s, d = c1 d + c2 r
// from_r (the first step): d is not stored; d = scale r and s = scale (S A r) (the operator and
// smoother were applied to r itself: by linearity S A (scale r) = scale S A r).
// last: the final x += d of Algorithm 2 is done here, and r and d (no longer needed) are not
// written: x = x + d + (c1 d + c2 r).
// GB300 issues FP64 at 2 instructions/clk/SM, below the rate at which HBM delivers this
// kernel's 4-6 words per point, so the recurrence is evaluated with its constants folded into
// FMAs (3-5 FP64 instructions per point instead of 6-8): mathematically the same update, with
// the rounding of an FMA chain.  The constants are formed on the host in FP64:
//   k_d = 1 + c1, k_r = scale (1 + c1) + c2, c1s = c1 scale, k_s = -scale,
//   k_sl = -c2 scale (from_r) or -c2, the weight of the surrogate output in the last update.
// RS (FROM_R only): the smoothed residual of the first step is dinv .* rin, formed here.
// In FP64 the last step with RS is bound by the FP64 pipe (about 4 instructions per point against
// 4-5 words): it factors dinv out of its two terms.
constexpr int CHEB_U = 2;

template <class T, bool FIRST, bool FROM_R, bool LAST, bool RS = false>
__global__ void cheb_update_kernel(T* __restrict__ x, T* __restrict__ d, T* __restrict__ r,
                                   const T* __restrict__ sv, const T* __restrict__ dinv, int64_t n,
                                   T c1, T c2, T scale, T k_d, T k_r, T c1s, T k_s, T k_sl,
                                   const T* __restrict__ rin) {
  // CHEB_U points per thread, blockDim apart (coalesced): every load of the CHEB_U points is
  // issued before the first store
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x * CHEB_U + threadIdx.x;
  T s0[CHEB_U], di[CHEB_U], r0[CHEB_U], d0[CHEB_U], x0[CHEB_U];
#pragma unroll
  for (int u = 0; u < CHEB_U; ++u) {
    const int64_t i = i0 + (int64_t)u * blockDim.x;
    if (i < n) {
      s0[u] = sv[i];
      di[u] = dinv ? dinv[i] : T(1);
      r0[u] = RS ? rin[i] : r[i];
      d0[u] = FROM_R ? T(0) : d[i];
      x0[u] = FIRST ? T(0) : x[i];
    }
  }
#pragma unroll
  for (int u = 0; u < CHEB_U; ++u) {
    const int64_t i = i0 + (int64_t)u * blockDim.x;
    if (i >= n) break;
    if constexpr (RS && LAST) {
      // x + dinv (k_r rin + k_sl s): three FP64 instructions per point (the form below takes
      // four with the scaled residual formed first; this kernel is bound by the FP64 pipe)
      const T u2 = fma(k_r, r0[u], k_sl * s0[u]);
      x[i] = FIRST ? di[u] * u2 : fma(di[u], u2, x0[u]);
      continue;
    }
    if (RS) r0[u] = di[u] * r0[u];
    if constexpr (LAST) {
      // x + d + c1 d + c2 (r - s)
      const T w = dinv ? k_sl * di[u] : k_sl;
      const T t = FIRST ? w * s0[u] : fma(w, s0[u], x0[u]);
      x[i] = FROM_R ? fma(k_r, r0[u], t) : fma(k_d, d0[u], fma(c2, r0[u], t));
    } else if constexpr (FROM_R) {
      // d = scale r: x + d, r - scale s, c1 d + c2 r'
      const T w = dinv ? k_s * di[u] : k_s;
      const T rv = fma(w, s0[u], r0[u]);
      x[i] = FIRST ? scale * r0[u] : fma(scale, r0[u], x0[u]);
      r[i] = rv;
      d[i] = fma(c1s, r0[u], c2 * rv);
    } else {
      const T sval = dinv ? di[u] * s0[u] : s0[u];
      const T rv = r0[u] - sval;
      x[i] = FIRST ? d0[u] : x0[u] + d0[u];
      r[i] = rv;
      d[i] = fma(c1, d0[u], c2 * rv);
    }
  }
}
template <class T>
int cheb_update(T* x, T* d, T* r, const T* sv, const T* dinv, int64_t n, T c1, T c2, bool first,
                cudaStream_t s, T scale, bool from_r, bool last, const T* rin, int prof_p) {
  SE_CHECK(!rin || (from_r && dinv), SE_EINVAL, "cheb_update: a scaled residual needs the first step and dinv");
  const double words = 2.0 + (dinv ? 1.0 : 0.0) + (from_r ? 0.0 : 1.0) + (first ? 0.0 : 1.0) +
                       (last ? 1.0 : 3.0);
  ProfScope prof(SE_K_CHEBY_UPD, s, (double)n, words * n * sizeof(T), 6.0 * n, prof_variant<T>(prof_p));
  const unsigned g = grid_for((n + CHEB_U - 1) / CHEB_U, 256);
  const int key = (rin ? 8 : 0) + (first ? 4 : 0) + (from_r ? 2 : 0) + (last ? 1 : 0);
  const double C1 = (double)c1, C2 = (double)c2, SC = (double)scale;
  const T k_d = T(1.0 + C1), k_r = T(SC * (1.0 + C1) + C2), c1s = T(C1 * SC), k_s = T(-SC);
  const T k_sl = T(from_r ? -C2 * SC : -C2);
  switch (key) {
#define SE_CHEB_CASE(K, F, R, L, RS)                                                             \
  case K:                                                                                        \
    cheb_update_kernel<T, F, R, L, RS><<<g, 256, 0, s>>>(x, d, r, sv, dinv, n, c1, c2, scale, k_d, \
                                                         k_r, c1s, k_s, k_sl, rin);              \
    break;
    SE_CHEB_CASE(0, false, false, false, false) SE_CHEB_CASE(1, false, false, true, false)
    SE_CHEB_CASE(2, false, true, false, false) SE_CHEB_CASE(3, false, true, true, false)
    SE_CHEB_CASE(4, true, false, false, false) SE_CHEB_CASE(5, true, false, true, false)
    SE_CHEB_CASE(6, true, true, false, false) SE_CHEB_CASE(7, true, true, true, false)
    SE_CHEB_CASE(10, false, true, false, true) SE_CHEB_CASE(11, false, true, true, true)
    SE_CHEB_CASE(14, true, true, false, true) SE_CHEB_CASE(15, true, true, true, true)
#undef SE_CHEB_CASE
  }
  SE_LAUNCH_CHECK();
  return SE_OK;
}
template int cheb_update<double>(double*, double*, double*, const double*, const double*, int64_t,
                                 double, double, bool, cudaStream_t, double, bool, bool, const double*,
                                 int);
template int cheb_update<float>(float*, float*, float*, const float*, const float*, int64_t, float,
                                float, bool, cudaStream_t, float, bool, bool, const float*, int);

// ------------------------------------------------------------------ FPCG kernels (FP64)
struct AlphaOp {  // pw = (p, w); alpha = rz / pw
  static constexpr int K = 1;
  const double* p;
  const double* w;
  const uint8_t* pf;
  double* scal;
  struct V { double p, w; uint8_t f; };
  __device__ void setup() {}
  __device__ V load(int64_t i) const { return {p[i], w[i], pf[i]}; }
  __device__ void apply(int64_t, const V& v, double (&acc)[1]) const {
    acc[0] = fma(scale_pow2(v.p, mult_log2(v.f)), v.w, acc[0]);
  }
  __device__ void finalize(const double* s) const {
    scal[SC_PW] = s[0];
    scal[SC_ALPHA] = scal[SC_RZ] / s[0];
  }
};

struct UpdateXROp {  // x += alpha p; r2 = r - alpha w; rr = (r2, r2)
  static constexpr int K = 1;
  double* x;
  const double* p;
  const double* r;
  const double* w;
  double* r2;
  const uint8_t* pf;
  double* scal;
  double alpha;
  struct V { double x, p, r, w; uint8_t f; };
  __device__ void setup() { alpha = scal[SC_ALPHA]; }
  __device__ V load(int64_t i) const { return {x[i], p[i], r[i], w[i], pf[i]}; }
  __device__ void apply(int64_t i, const V& v, double (&acc)[1]) const {
    x[i] = fma(alpha, v.p, v.x);
    const double rv = fma(-alpha, v.w, v.r);
    r2[i] = rv;
    acc[0] = fma(scale_pow2(rv, mult_log2(v.f)), rv, acc[0]);
  }
  __device__ void finalize(const double* s) const { scal[SC_RR] = s[0]; }
};

struct BetaOp {  // zr = (z, r2); zro = (z, r); beta = (zr - zro)/rz; rz = zr
  static constexpr int K = 2;
  const double* z;
  const double* r2;
  const double* r;
  const uint8_t* pf;
  double* scal;
  struct V { double z, r2, r; uint8_t f; };
  __device__ void setup() {}
  __device__ V load(int64_t i) const { return {z[i], r2[i], r[i], pf[i]}; }
  __device__ void apply(int64_t, const V& v, double (&acc)[2]) const {
    const double zw = scale_pow2(v.z, mult_log2(v.f));
    acc[0] = fma(zw, v.r2, acc[0]);
    acc[1] = fma(zw, v.r, acc[1]);
  }
  __device__ void finalize(const double* s) const {
    scal[SC_BETA] = (s[0] - s[1]) / scal[SC_RZ];
    scal[SC_RZ] = s[0];
  }
};

struct RZInitOp {  // rz = (r, z); rr = (r, r); r0 = rr
  static constexpr int K = 2;
  const double* r;
  const double* z;
  const uint8_t* pf;
  double* scal;
  struct V { double r, z; uint8_t f; };
  __device__ void setup() {}
  __device__ V load(int64_t i) const { return {r[i], z[i], pf[i]}; }
  __device__ void apply(int64_t, const V& v, double (&acc)[2]) const {
    const double rw = scale_pow2(v.r, mult_log2(v.f));
    acc[0] = fma(rw, v.z, acc[0]);
    acc[1] = fma(rw, v.r, acc[1]);
  }
  __device__ void finalize(const double* s) const {
    scal[SC_RZ] = s[0];
    scal[SC_RR] = s[1];
    scal[SC_R0] = s[1];
  }
};

__global__ void pupdate_kernel(double* __restrict__ p, const double* __restrict__ z,
                               const double* __restrict__ scal, int64_t n) {
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x * FUSED_U + threadIdx.x;
  const double beta = scal[SC_BETA];
  double pv[FUSED_U], zv[FUSED_U];
#pragma unroll
  for (int u = 0; u < FUSED_U; ++u) {
    const int64_t i = i0 + (int64_t)u * blockDim.x;
    if (i < n) {
      pv[u] = p[i];
      zv[u] = z[i];
    }
  }
#pragma unroll
  for (int u = 0; u < FUSED_U; ++u) {
    const int64_t i = i0 + (int64_t)u * blockDim.x;
    if (i < n) p[i] = fma(beta, pv[u], zv[u]);
  }
}

int fpcg_init(const Level& lv, const double* r, const double* z, Scratch& sc, cudaStream_t s) {
  return run_fused(RZInitOp{r, z, lv.pflag, sc.scal}, lv.L, sc, s, SE_K_KRYLOV, lv.L * 17.0,
                   lv.L * 4.0);
}
int fpcg_alpha(const Level& lv, const double* p, const double* w, Scratch& sc, cudaStream_t s) {
  return run_fused(AlphaOp{p, w, lv.pflag, sc.scal}, lv.L, sc, s, SE_K_KRYLOV, lv.L * 17.0,
                   lv.L * 2.0);
}
int fpcg_update(const Level& lv, double* x, const double* p, const double* r, const double* w,
                double* r2, Scratch& sc, cudaStream_t s) {
  return run_fused(UpdateXROp{x, p, r, w, r2, lv.pflag, sc.scal}, lv.L, sc, s, SE_K_KRYLOV,
                   lv.L * 49.0, lv.L * 6.0);
}
int fpcg_beta(const Level& lv, const double* z, const double* r2, const double* r, Scratch& sc,
              cudaStream_t s) {
  return run_fused(BetaOp{z, r2, r, lv.pflag, sc.scal}, lv.L, sc, s, SE_K_KRYLOV, lv.L * 25.0,
                   lv.L * 4.0);
}
int fpcg_pupdate(const Level& lv, double* p, const double* z, Scratch& sc, cudaStream_t s) {
  ProfScope prof(SE_K_KRYLOV, s, (double)lv.L, lv.L * 24.0, lv.L * 2.0);
  pupdate_kernel<<<grid_for((lv.L + FUSED_U - 1) / FUSED_U, 256), 256, 0, s>>>(p, z, sc.scal, lv.L);
  SE_LAUNCH_CHECK();
  return SE_OK;
}

// ------------------------------------------------------------------ Gram-Schmidt kernels (FP64)
struct DotToSlotOp {  // scal[slot] = (a, b)
  static constexpr int K = 1;
  const double* a;
  const double* b;
  const uint8_t* pf;
  double* scal;
  int slot;
  struct V { double a, b; uint8_t f; };
  __device__ void setup() {}
  __device__ V load(int64_t i) const { return {a[i], b[i], pf[i]}; }
  __device__ void apply(int64_t, const V& v, double (&acc)[1]) const {
    acc[0] = fma(scale_pow2(v.a, mult_log2(v.f)), v.b, acc[0]);
  }
  __device__ void finalize(const double* s) const { scal[slot] = s[0]; }
};

struct AxpyDotOp {  // w -= scal[hslot] v; scal[nslot] = (w, vnext) (vnext may be w itself)
  static constexpr int K = 1;
  double* w;
  const double* v;
  const double* vnext;
  const uint8_t* pf;
  double* scal;
  int hslot, nslot;
  double h;
  struct V { double v, w, vn; uint8_t f; };
  __device__ void setup() { h = scal[hslot]; }
  __device__ V load(int64_t i) const { return {v[i], w[i], vnext ? vnext[i] : 0.0, pf[i]}; }
  __device__ void apply(int64_t i, const V& q, double (&acc)[1]) const {
    const double wv = fma(-h, q.v, q.w);
    w[i] = wv;
    acc[0] = fma(scale_pow2(wv, mult_log2(q.f)), vnext && vnext != w ? q.vn : wv, acc[0]);
  }
  __device__ void finalize(const double* s) const { scal[nslot] = s[0]; }
};

__global__ void scale_by_inv_sqrt_kernel(double* __restrict__ out, const double* __restrict__ in,
                                         const double* __restrict__ scal, int slot, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[i] * (1.0 / sqrt(scal[slot]));
}

// out = in / sqrt(scal[slot])  (one division per thread)
int scale_inv_sqrt(double* out, const double* in, double* scal, int slot, int64_t n, cudaStream_t s) {
  ProfScope prof(SE_K_KRYLOV, s, (double)n, 16.0 * n, (double)n);
  scale_by_inv_sqrt_kernel<<<grid_for(n, 256), 256, 0, s>>>(out, in, scal, slot, n);
  SE_LAUNCH_CHECK();
  return SE_OK;
}
int dot_to_slot(const Level& lv, const double* a, const double* b, Scratch& sc, int slot,
                cudaStream_t s) {
  return run_fused(DotToSlotOp{a, b, lv.pflag, sc.scal, slot}, lv.L, sc, s, SE_K_KRYLOV,
                   lv.L * 17.0, lv.L * 2.0);
}
int axpy_dot(const Level& lv, double* w, const double* v, const double* vnext, Scratch& sc,
             int hslot, int nslot, cudaStream_t s) {
  return run_fused(AxpyDotOp{w, v, vnext, lv.pflag, sc.scal, hslot, nslot}, lv.L, sc, s,
                   SE_K_KRYLOV, lv.L * (vnext ? 33.0 : 25.0), lv.L * 4.0);
}

// x += sum_j y_j z_j for host coefficients y (up to 8 vectors per pass)
__global__ void lincomb_kernel(double* __restrict__ x, const double* const* __restrict__ zs,
                               const double* __restrict__ y, int m, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = x[i];
  for (int j = 0; j < m; ++j) acc = fma(y[j], zs[j][i], acc);
  x[i] = acc;
}
int lincomb(double* x, const double* const* zs_dev, const double* y_dev, int m, int64_t n,
            cudaStream_t s) {
  ProfScope prof(SE_K_KRYLOV, s, (double)n, (m + 2.0) * 8.0 * n, 2.0 * m * n);
  lincomb_kernel<<<grid_for(n, 256), 256, 0, s>>>(x, zs_dev, y_dev, m, n);
  SE_LAUNCH_CHECK();
  return SE_OK;
}

}  // namespace se

using namespace se;

extern "C" int se_dot(se_mesh_t m, const double* a, const double* b, double* out_host, void* stream) {
  SE_CHECK(m && a && b && out_host, SE_EINVAL, "se_dot: null argument");
  cudaStream_t s = as_stream(stream, m->stream);
  SE_TRY(dot_weighted(m->fine, a, b, m->scratch.scal + SC_TMP, m->scratch, s));
  SE_CUDA(cudaMemcpyAsync(out_host, m->scratch.scal + SC_TMP, sizeof(double), cudaMemcpyDeviceToHost, s));
  SE_CUDA(cudaStreamSynchronize(s));
  return SE_OK;
}

namespace se {
// x += alpha p; r_old = r; r = r - alpha w; rr = (r, r): the in-place variant used by the
// device-driven (graph) solver, whose captured pointers cannot be swapped between iterations.
struct UpdateXR2Op {
  static constexpr int K = 1;
  double* x;
  const double* p;
  double* r;
  const double* w;
  double* r_old;
  const uint8_t* pf;
  double* scal;
  double alpha;
  struct V { double x, p, r, w; uint8_t f; };
  __device__ void setup() { alpha = scal[SC_ALPHA]; }
  __device__ V load(int64_t i) const { return {x[i], p[i], r[i], w[i], pf[i]}; }
  __device__ void apply(int64_t i, const V& v, double (&acc)[1]) const {
    x[i] = fma(alpha, v.p, v.x);
    r_old[i] = v.r;
    const double rv = fma(-alpha, v.w, v.r);
    r[i] = rv;
    acc[0] = fma(scale_pow2(rv, mult_log2(v.f)), rv, acc[0]);
  }
  __device__ void finalize(const double* s) const { scal[SC_RR] = s[0]; }
};

int fpcg_update_inplace(const Level& lv, double* x, const double* p, double* r, const double* w,
                        double* r_old, Scratch& sc, cudaStream_t s) {
  return run_fused(UpdateXR2Op{x, p, r, w, r_old, lv.pflag, sc.scal}, lv.L, sc, s, SE_K_KRYLOV,
                   lv.L * 57.0, lv.L * 6.0);
}
}  // namespace se
