// ALU roofs of this GPU for the roofline of the arithmetic-bound kernels (FP64 operator and FDM,
// FP32 FDM): the fused multiply-add throughput in FP64, FP32, and FP32 in packed pairs
// (fma.rn.f32x2, two lanes per instruction), measured with independent FMA chains per thread;
// and the warp-level TF32 tensor-core rate (mma.sync) that a tensor-core FDM would run on.
// This is measurement infrastructure; the paper has no counterpart.
#include <algorithm>

#include "se_internal.h"

namespace se {

constexpr int PROBE_CHAINS = 8;
__device__ float g_probe_sink32;   // written only if a chain reaches an impossible value: keeps
__device__ double g_probe_sink64;  // the chains live without a store per thread

template <int KIND>
__global__ void __launch_bounds__(256) fma_probe_kernel(int iters, float a32, float b32, double a64,
                                                        double b64) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (KIND == 0) {
    double x[PROBE_CHAINS];
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = 1e-3 * (t + c);
#pragma unroll 1
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = fma(x[c], a64, b64);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) s += x[c];
    if (s == 12345.678) g_probe_sink64 = s;  // never true (each chain tends to b / (1 - a))
  } else if constexpr (KIND == 1) {
    float x[PROBE_CHAINS];
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = 1e-3f * (t + c);
#pragma unroll 1
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = fmaf(x[c], a32, b32);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) s += x[c];
    if (s == 12345.678f) g_probe_sink32 = s;
  } else {
    float2 x[PROBE_CHAINS];
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = make_float2(1e-3f * (t + c), 2e-3f * (t + c));
    const float2 a2 = make_float2(a32, a32), b2 = make_float2(b32, b32);
#pragma unroll 1
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) s += x[c].x + x[c].y;
    if (s == 12345.678f) g_probe_sink32 = s;
  }
}

// Warp-level tensor-core rate for the FP32 contractions' tensor-core question: independent
// chains of mma.sync m16n8k8 with TF32 operands and FP32 accumulators (16 x 8 x 8 multiply-adds
// per instruction and warp); operands stay in registers, so only the tensor pipe is exercised.
constexpr int MMA_CHAINS = 4;
__global__ void __launch_bounds__(256) tf32_mma_probe_kernel(int iters, float seed) {
  unsigned a[4], b[2];
  const float av = seed * (1 + (threadIdx.x & 7)), bv = seed * (2 + (threadIdx.x & 3));
#pragma unroll
  for (int q = 0; q < 4; ++q) asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(a[q]) : "f"(av + q));
#pragma unroll
  for (int q = 0; q < 2; ++q) asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(b[q]) : "f"(bv + q));
  float c[MMA_CHAINS][4];
#pragma unroll
  for (int k = 0; k < MMA_CHAINS; ++k)
#pragma unroll
    for (int q = 0; q < 4; ++q) c[k][q] = 0.f;
#pragma unroll 1
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < MMA_CHAINS; ++k)
      asm volatile(
          "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};"
          : "+f"(c[k][0]), "+f"(c[k][1]), "+f"(c[k][2]), "+f"(c[k][3])
          : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  float sum = 0.f;
#pragma unroll
  for (int k = 0; k < MMA_CHAINS; ++k) sum += c[k][0] + c[k][1] + c[k][2] + c[k][3];
  if (sum == 12345.678f) g_probe_sink32 = sum;  // never true for these operands
}

static int run_mma_probe(int sms, cudaStream_t s, double* tflops) {
  const int iters = 4096, threads = 256;
  int per_sm = 0;
  SE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tf32_mma_probe_kernel, threads, 0));
  SE_CHECK(per_sm >= 1, SE_ECUDA, "mma probe: no resident block");
  const int blocks = sms * per_sm;
  cudaEvent_t e0, e1;
  SE_CUDA(cudaEventCreate(&e0));
  SE_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int st = SE_OK;
  for (int rep = 0; rep < 4 && st == SE_OK; ++rep) {
    cudaEventRecord(e0, s);
    tf32_mma_probe_kernel<<<blocks, threads, 0, s>>>(iters, 1e-3f);
    cudaEventRecord(e1, s);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      set_error("mma probe: launch failed");
      st = SE_ECUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != SE_OK) return st;
  const double warps = (double)blocks * threads / 32.0;
  const double macs = warps * iters * MMA_CHAINS * 16.0 * 8.0 * 8.0;
  *tflops = 2.0 * macs / (best * 1e-3) / 1e12;
  return SE_OK;
}

template <int KIND>
static int run_probe(int sms, cudaStream_t s, double* tflops) {
  // FP64 issues at 1/64 of the FP32 rate: fewer iterations keep its launch near the others'
  const int iters = KIND == 0 ? 1024 : 16384;
  const int threads = 256;
  int per_sm = 0;
  SE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_probe_kernel<KIND>, threads, 0));
  SE_CHECK(per_sm >= 1, SE_ECUDA, "fma probe: no resident block");
  const int blocks = sms * per_sm;
  cudaEvent_t e0, e1;
  SE_CUDA(cudaEventCreate(&e0));
  SE_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int st = SE_OK;
  for (int rep = 0; rep < 4 && st == SE_OK; ++rep) {  // first launch warms up
    cudaEventRecord(e0, s);
    fma_probe_kernel<KIND><<<blocks, threads, 0, s>>>(iters, 0.999999f, 1e-7f, 0.999999999, 1e-9);
    cudaEventRecord(e1, s);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      set_error("fma probe: launch failed");
      st = SE_ECUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != SE_OK) return st;
  const double fmas = (double)blocks * threads * iters * PROBE_CHAINS * (KIND == 2 ? 2 : 1);
  *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
  return SE_OK;
}

}  // namespace se

using namespace se;

extern "C" int se_prof_fma_peak(int kind, double* tflops, int* sms, void* stream) {
  SE_CHECK(tflops && kind >= 0 && kind <= 3, SE_EINVAL, "se_prof_fma_peak: bad argument");
  int dev = 0, n = 0;
  SE_CUDA(cudaGetDevice(&dev));
  SE_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
  if (sms) *sms = n;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (kind) {
    case 0: return run_probe<0>(n, s, tflops);
    case 1: return run_probe<1>(n, s, tflops);
    case 2: return run_probe<2>(n, s, tflops);
    default: return run_mma_probe(n, s, tflops);
  }
}
