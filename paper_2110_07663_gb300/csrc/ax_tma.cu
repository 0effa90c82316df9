// FP32 local Ax with TMA bulk-copy pipelining (sm_100+ async proxy).
//
// Persistent blocks walk over groups of NE consecutive elements.  One thread streams each
// group's u block and its six geometric-factor blocks (contiguous in the [6][L] layout) into a
// shared-memory stage with cp.async.bulk, completion counted by an mbarrier transaction count;
// two stages alternate, so the loads of the next group run while the current one is contracted.
// The contractions are those of ax_local_kernel (sum factorisation, 12N+15 flops per point).
// Every mbarrier wait is bounded (wall clock, ~1 s): on expiry the kernel records SE_ETIMEOUT in
// the level's status word, waits (bounded) for the copies it issued, and returns.
// Only for even N: then every element block (N^3 floats) is a multiple of 16 bytes, as the bulk
// copy requires for sizes and addresses.
#include <cstdint>

#include "se_internal.h"

namespace se {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ long long gtimer() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait for phase `parity` of `bar`; false on expiry (status recorded).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, long long limit_ns,
                                                  int* pstatus) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = gtimer();
  while (!mbar_try_wait(bar, parity)) {
    if (gtimer() - t0 > limit_ns) {
      atomicExch(pstatus, SE_ETIMEOUT);
      return false;
    }
  }
  return true;
}

constexpr long long PIPE_LIMIT_NS = 1000000000LL;

// Residual form (RES): an eighth block per group, b, comes through the same pipeline, and the
// output is b / multiplicity - A_L u; the multiplicity follows from the element's place in the
// lattice (copies = product over directions of 2 on an interior element interface, else 1), or,
// for a level that is a union of several lattices (nx = 0), from the point flags.
template <int N, bool RES>
__global__ void __launch_bounds__(512) ax_tma_kernel(int64_t E, int NE, int64_t ngroups,
                                                     const float* __restrict__ u,
                                                     const float* __restrict__ G, int64_t L,
                                                     const float* __restrict__ Dg,
                                                     float* __restrict__ y,
                                                     const float* __restrict__ sub, int nx,
                                                     int ny, int nz,
                                                     const uint8_t* __restrict__ pflag,
                                                     int* __restrict__ pstatus) {
  constexpr int N2 = N * N, N3 = N * N * N, A = RES ? 8 : 7;  // blocks per stage
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int S = NE * N3;                       // floats per element-group block
  float* stage0 = reinterpret_cast<float*>(smem_raw);   // stage s: u at s*A*S, G at +S, b at +7S
  float* swr = stage0 + 2 * A * S;
  float* sws = swr + S;
  float* sD = sws + S;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sD + ((N2 + 3) / 4) * 4 + 4);
  const int tid = threadIdx.x;
  const int le = tid / N2, ij = tid - le * N2;
  const int i = ij % N, j = ij / N;
  for (int t = tid; t < N2; t += blockDim.x) sD[t] = Dg[t];
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int st, int64_t g) {
    const int64_t e0 = g * NE;
    const int ne = (int)((E - e0) < NE ? (E - e0) : NE);
    const unsigned bytes = (unsigned)(ne * N3 * sizeof(float));
    float* dst = stage0 + st * A * S;
    mbar_arrive_expect_tx(&bars[st], (unsigned)A * bytes);
    bulk_load(dst, u + e0 * N3, bytes, &bars[st]);
#pragma unroll
    for (int c = 0; c < 6; ++c) bulk_load(dst + (c + 1) * S, G + c * L + e0 * N3, bytes, &bars[st]);
    if (RES) bulk_load(dst + 7 * S, sub + e0 * N3, bytes, &bars[st]);
  };
  int64_t g = blockIdx.x;
  if (tid == 0) {
    if (g < ngroups) issue(0, g);
    if (g + gridDim.x < ngroups) issue(1, g + gridDim.x);
  }
  float Dri[N], Drj[N], Dci[N], Dcj[N];
#pragma unroll
  for (int l = 0; l < N; ++l) {
    Dri[l] = sD[i * N + l];
    Drj[l] = sD[j * N + l];
    Dci[l] = sD[l * N + i];
    Dcj[l] = sD[l * N + j];
  }
  unsigned phases = 0u;  // bit s: parity of the next completion of stage s
  int st = 0;
  bool ok = true;
  for (; g < ngroups; g += gridDim.x) {
    const bool expired = !mbar_wait_bounded(&bars[st], (phases >> st) & 1u, PIPE_LIMIT_NS, pstatus);
    if (__syncthreads_or(expired)) {  // the whole block leaves together
      ok = false;
      break;
    }
    phases ^= 1u << st;
    const int64_t e0 = g * NE;
    const bool valid = (e0 + le) < E;
    const float* cu = stage0 + st * A * S + le * N3;
    const float* cg = cu + S;
    // residual form: b / multiplicity of this thread's outputs, read from the stage before the
    // stage is handed to the next copy
    float bw[N];
    if (RES && valid) {
      const int64_t e = e0 + le;
      if (nx > 0) {
        const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
        auto shared2 = [](int a, int ea, int na) { return (a == 0 && ea > 0) || (a == N - 1 && ea < na - 1); };
        const float wxy = (shared2(i, ex, nx) ? 0.5f : 1.f) * (shared2(j, ey, ny) ? 0.5f : 1.f);
#pragma unroll
        for (int k = 0; k < N; ++k) bw[k] = cu[7 * S + ij + N2 * k] * (wxy * (shared2(k, ez, nz) ? 0.5f : 1.f));
      } else {
#pragma unroll
        for (int k = 0; k < N; ++k) {
          const int mlog = __ffs(pflag[e * N3 + ij + N2 * k] & 0x0F) - 1;
          bw[k] = cu[7 * S + ij + N2 * k] * __int_as_float((127 - mlog) << 23);
        }
      }
    }
    float ru[N], ry[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      ru[k] = valid ? cu[ij + N2 * k] : 0.f;
      ry[k] = 0.f;
    }
    if (valid) {
#pragma unroll
      for (int k = 0; k < N; ++k) {
        float ur = 0.f, us = 0.f, ut = 0.f;
#pragma unroll
        for (int l = 0; l < N; ++l) {
          ur += Dri[l] * cu[l + N * j + N2 * k];
          us += Drj[l] * cu[i + N * l + N2 * k];
          ut += sD[k * N + l] * ru[l];
        }
        const int pt = ij + N2 * k;
        const float grr = cg[pt], grs = cg[S + pt], grt = cg[2 * S + pt];
        const float gss = cg[3 * S + pt], gst = cg[4 * S + pt], gtt = cg[5 * S + pt];
        swr[le * N3 + pt] = grr * ur + grs * us + grt * ut;
        sws[le * N3 + pt] = grs * ur + gss * us + gst * ut;
        const float wt = grt * ur + gst * us + gtt * ut;
#pragma unroll
        for (int l = 0; l < N; ++l) ry[l] += sD[k * N + l] * wt;
      }
    }
    __syncthreads();  // stage st fully read; swr/sws complete
    if (tid == 0 && g + 2 * (int64_t)gridDim.x < ngroups) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(st, g + 2 * (int64_t)gridDim.x);
    }
    if (valid) {
      const float* cwr = swr + le * N3;
      const float* cws = sws + le * N3;
      float* yo = y + (e0 + le) * N3;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        float acc = ry[k];
#pragma unroll
        for (int l = 0; l < N; ++l) {
          acc += Dci[l] * cwr[l + N * j + N2 * k];
          acc += Dcj[l] * cws[i + N * l + N2 * k];
        }
        yo[ij + N2 * k] = RES ? bw[k] - acc : acc;
      }
    }
    __syncthreads();  // swr/sws free for the next group
    st ^= 1;
  }
  if (!ok && tid == 0) {
    // wait (bounded) for copies still in flight before the block's shared memory goes away
    for (int s2 = 0; s2 < 2; ++s2) mbar_wait_bounded(&bars[s2], (phases >> s2) & 1u, PIPE_LIMIT_NS, pstatus);
  }
}

template <int N, bool RES>
static int launch_ax_tma_t(const Level& lv, const float* u, float* y, int NE, const float* sub,
                           cudaStream_t s) {
  constexpr int N3 = N * N * N, A = RES ? 8 : 7;
  SE_CHECK(lv.pstatus, SE_EINVAL, "ax_tma: level without a status word");
  const int threads = NE * N * N;
  const size_t smem = (size_t)((2 * A + 2) * NE * N3 + ((N * N + 3) / 4) * 4 + 4) * sizeof(float) +
                      2 * sizeof(uint64_t);
  static const cudaError_t attr = cudaFuncSetAttribute(
      ax_tma_kernel<N, RES>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  SE_CUDA(attr);
  int per_sm = 0;
  SE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ax_tma_kernel<N, RES>, threads, smem));
  SE_CHECK(per_sm >= 1, SE_ECUDA, "ax_tma: no resident block fits (NE=%d)", NE);
  int dev = 0, sms = 0;
  SE_CUDA(cudaGetDevice(&dev));
  SE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t groups = (lv.E + NE - 1) / NE;
  int64_t grid = (int64_t)sms * per_sm;
  if (grid > groups) grid = groups;
  ax_tma_kernel<N, RES><<<(unsigned)grid, threads, smem, s>>>(lv.E, NE, groups, u, lv.G32, lv.L,
                                                               lv.D32, y, sub, lv.nel[0],
                                                               lv.nel[1], lv.nel[2], lv.pflag,
                                                               lv.pstatus);
  SE_LAUNCH_CHECK();
  return SE_OK;
}

template <int N>
static int launch_ax_tma(const Level& lv, const float* u, float* y, int NE, const float* sub,
                         cudaStream_t s) {
  return sub ? launch_ax_tma_t<N, true>(lv, u, y, NE, sub, s)
             : launch_ax_tma_t<N, false>(lv, u, y, NE, sub, s);
}

// Elements per group of the pipelined kernel (tuned value, else 2 groups of N^2 threads).
int ax_tma_group(int p) {
  const int N = p + 1;
  const int t = tile_get(p, true).ax_ne;
  // shared memory for the residual form (18 blocks of the group): the plain form (16) then fits too
  if (t >= 1 && t * N * N <= 512 && 18 * t * N * N * N * 4 <= 200 * 1024) return t;
  int ne = 256 / (N * N);
  if (ne < 1) ne = 1;
  while (ne > 1 && 18 * ne * N * N * N * 4 > 200 * 1024) --ne;
  return ne;
}

bool ax_tma_supported(int p) { return (p + 1) % 2 == 0 && p + 1 >= 2 && p + 1 <= 10; }

int ax_local_tma(const Level& lv, const float* u, float* y, cudaStream_t s, const float* sub) {
  const int NE = ax_tma_group(lv.p);
  switch (lv.N) {
    case 2: return launch_ax_tma<2>(lv, u, y, NE, sub, s);
    case 4: return launch_ax_tma<4>(lv, u, y, NE, sub, s);
    case 6: return launch_ax_tma<6>(lv, u, y, NE, sub, s);
    case 8: return launch_ax_tma<8>(lv, u, y, NE, sub, s);
    case 10: return launch_ax_tma<10>(lv, u, y, NE, sub, s);
    default: set_error("ax_tma: unsupported N=%d", lv.N); return SE_EINVAL;
  }
}

int level_pipeline_take(const Level& lv, cudaStream_t s) {
  if (!lv.pstatus) return SE_OK;
  int h = 0;
  SE_CUDA(cudaStreamSynchronize(s));
  SE_CUDA(cudaMemcpy(&h, lv.pstatus, sizeof(int), cudaMemcpyDeviceToHost));
  if (h == 0) return SE_OK;
  SE_TRY(dzero(lv.pstatus, sizeof(int), s));
  set_error("p = %d level: a pipelined kernel's bounded wait expired (results invalid)", lv.p);
  return SE_ETIMEOUT;
}

}  // namespace se
