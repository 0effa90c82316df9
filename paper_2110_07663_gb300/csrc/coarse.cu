// Coarsest level (p = 1): assembled 27-point operator and a persistent Jacobi-PCG solve.
//
// The paper solves the coarse system with one BoomerAMG V-cycle (Sec. 2.3.2), a third-party
// library; here the coarse problem is solved by Jacobi-preconditioned CG to a relative tolerance.
// The p = 1 element matrices are assembled into rows over global lattice nodes (27 entries each,
// summed over the up to 8 elements sharing the row node in a fixed order: deterministic), and the
// whole CG iteration runs in ONE cooperative launch: blocks meet at a grid barrier between the
// matrix-vector product and each inner product.  Every wait is bounded by a wall-clock limit after
// which the kernel records SE_ETIMEOUT and returns.
#include <cooperative_groups.h>

#include <mutex>

#include "pmg_internal.h"

namespace se {

constexpr long long BARRIER_TIMEOUT_NS = 2000000000LL;  // 2 s

__device__ __forceinline__ long long global_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier over `nblocks` blocks: bar[0] arrival count, bar[1] generation.  Returns false if
// this or another block gave up waiting (status[0] != 0).
__device__ bool grid_barrier(unsigned* bar, int* status, unsigned nblocks, long long timeout_ns) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u) + 1u;
    if (arrived == nblocks) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = global_ns();
      while (*vgen == gen) {
        __nanosleep(64);
        if (*(volatile int*)status != 0) break;
        if (global_ns() - t0 > timeout_ns) {
          atomicExch(status, SE_ETIMEOUT);
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int*)status == 0;
}

// ------------------------------------------------------------------ assembly
// Row g, slot (dI+1) + 3(dJ+1) + 9(dK+1): sum over elements containing both nodes of the
// element-matrix entry A^e_ab = sum_q (grad_ref phi_a)^T G(q) (grad_ref phi_b) (p = 1, 8 points).
__global__ void coarse_assemble_kernel(int nx, int ny, int nz, int64_t n, int64_t L,
                                       const double* __restrict__ G,
                                       const uint8_t* __restrict__ pflag,
                                       double* __restrict__ A, double* __restrict__ dinv,
                                       int* __restrict__ g2l) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 27 * n) return;
  const int slot = (int)(t / n);
  const int64_t g = t - (int64_t)slot * n;
  const int NX = nx + 1, NY = ny + 1;
  const int I = (int)(g % NX), J = (int)((g / NX) % NY), K = (int)(g / ((int64_t)NX * NY));
  const int dI = slot % 3 - 1, dJ = (slot / 3) % 3 - 1, dK = slot / 9 - 1;
  const int I2 = I + dI, J2 = J + dJ, K2 = K + dK;
  double v = 0.0;
  bool row_free = true, col_free = true;
  int first_local = -1;
  // D for p = 1: h_0' = -1/2, h_1' = +1/2 at both points
  for (int ez = K - 1; ez <= K; ++ez) {
    if (ez < 0 || ez >= nz) continue;
    for (int ey = J - 1; ey <= J; ++ey) {
      if (ey < 0 || ey >= ny) continue;
      for (int ex = I - 1; ex <= I; ++ex) {
        if (ex < 0 || ex >= nx) continue;
        const int ia = I - ex, ja = J - ey, ka = K - ez;
        const int64_t e = ex + (int64_t)nx * (ey + (int64_t)ny * ez);
        const int64_t la = e * 8 + ia + 2 * (ja + 2 * ka);
        if (first_local < 0) first_local = (int)la;
        row_free = (pflag[la] & PF_FREE) != 0;
        const int ib = I2 - ex, jb = J2 - ey, kb = K2 - ez;
        if (ib < 0 || ib > 1 || jb < 0 || jb > 1 || kb < 0 || kb > 1) continue;
        col_free = (pflag[e * 8 + ib + 2 * (jb + 2 * kb)] & PF_FREE) != 0;
        for (int q = 0; q < 8; ++q) {
          const int l = q & 1, m = (q >> 1) & 1, nn = q >> 2;
          const double ga[3] = {(ia ? 0.5 : -0.5) * (m == ja) * (nn == ka),
                                (ja ? 0.5 : -0.5) * (l == ia) * (nn == ka),
                                (ka ? 0.5 : -0.5) * (l == ia) * (m == ja)};
          const double gb[3] = {(ib ? 0.5 : -0.5) * (m == jb) * (nn == kb),
                                (jb ? 0.5 : -0.5) * (l == ib) * (nn == kb),
                                (kb ? 0.5 : -0.5) * (l == ib) * (m == jb)};
          const int64_t pq = e * 8 + q;
          const double grr = G[pq], grs = G[L + pq], grt = G[2 * L + pq];
          const double gss = G[3 * L + pq], gst = G[4 * L + pq], gtt = G[5 * L + pq];
          v += ga[0] * (grr * gb[0] + grs * gb[1] + grt * gb[2]) +
               ga[1] * (grs * gb[0] + gss * gb[1] + gst * gb[2]) +
               ga[2] * (grt * gb[0] + gst * gb[1] + gtt * gb[2]);
        }
      }
    }
  }
  const bool keep = row_free && col_free && I2 >= 0 && I2 < NX && J2 >= 0 && J2 < NY && K2 >= 0 &&
                    K2 < nz + 1;
  A[(int64_t)slot * n + g] = keep ? v : 0.0;
  if (slot == 13) {
    dinv[g] = row_free ? 1.0 / v : 0.0;
    g2l[g] = first_local;
  }
}

int coarse_setup(Level& lv, Allocs& allocs, cudaStream_t s) {
  SE_CHECK(lv.p == 1, SE_EINVAL, "coarse level must have p = 1 (got %d)", lv.p);
  const int64_t n = lv.n_global;
  SE_TRY(dmalloc(allocs, &lv.Ac, 27 * n));
  SE_TRY(dmalloc(allocs, &lv.cdinv, n));
  SE_TRY(dmalloc(allocs, &lv.g2l, n));
  SE_TRY(dmalloc(allocs, &lv.l2g, lv.L));
  coarse_assemble_kernel<<<grid_for(27 * n, 256), 256, 0, s>>>(lv.nel[0], lv.nel[1], lv.nel[2], n,
                                                              lv.L, lv.G64, lv.pflag, lv.Ac,
                                                              lv.cdinv, lv.g2l);
  SE_LAUNCH_CHECK();
  return local_to_global(lv, lv.l2g, s);
}

// ------------------------------------------------------------------ persistent Jacobi-PCG
template <class T>
struct CoarseArgs {
  int64_t n, L;
  int NX, NY, NZ;
  const double* A;
  const double* dinv;
  const int* g2l;
  const int* l2g;
  const T* rin;
  T* xout;
  double *x, *r, *z, *p, *q, *partA, *partB;
  unsigned* bar;
  int* status;
  double tol;
  int maxit;
  long long timeout_ns;
};

constexpr int CG_THREADS = 256;

__device__ __forceinline__ void block_reduce2(double& a, double& b, double* sh) {
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    sh[2 * w] = a;
    sh[2 * w + 1] = b;
  }
  __syncthreads();
  if (w == 0) {
    a = lane < CG_THREADS / 32 ? sh[2 * lane] : 0.0;
    b = lane < CG_THREADS / 32 ? sh[2 * lane + 1] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
  }
  __syncthreads();
}

// Every block sums the per-block partials in block order with one warp (same result everywhere).
__device__ __forceinline__ void sum_partials(const double* part, int nb, double& a, double& b,
                                             double* sh) {
  if (threadIdx.x < 32) {
    double sa = 0.0, sb = 0.0;
    for (int k = threadIdx.x; k < nb; k += 32) {
      sa += __ldcg(part + 2 * k);
      sb += __ldcg(part + 2 * k + 1);
    }
    for (int o = 16; o > 0; o >>= 1) {
      sa += __shfl_down_sync(0xffffffffu, sa, o);
      sb += __shfl_down_sync(0xffffffffu, sb, o);
    }
    if (threadIdx.x == 0) {
      sh[0] = sa;
      sh[1] = sb;
    }
  }
  __syncthreads();
  a = sh[0];
  b = sh[1];
  __syncthreads();
}

template <class T>
__global__ void __launch_bounds__(CG_THREADS) coarse_pcg_kernel(CoarseArgs<T> c) {
  __shared__ double sh[2 * CG_THREADS / 32 + 2];
  const unsigned nb = gridDim.x;
  const int64_t stride = (int64_t)gridDim.x * CG_THREADS;
  const int64_t t0 = (int64_t)blockIdx.x * CG_THREADS + threadIdx.x;
  double a0 = 0.0, a1 = 0.0;
  for (int64_t g = t0; g < c.n; g += stride) {
    const double rv = (double)c.rin[c.g2l[g]];
    const double zv = c.dinv[g] * rv;
    c.r[g] = rv;
    c.x[g] = 0.0;
    c.z[g] = zv;
    c.p[g] = zv;
    a0 = fma(rv, zv, a0);
    a1 = fma(rv, rv, a1);
  }
  block_reduce2(a0, a1, sh);
  if (threadIdx.x == 0) {
    c.partB[2 * blockIdx.x] = a0;
    c.partB[2 * blockIdx.x + 1] = a1;
  }
  int it = 0;
  if (grid_barrier(c.bar, c.status, nb, c.timeout_ns)) {
    double rz, rr0;
    sum_partials(c.partB, nb, rz, rr0, sh);
    const double tol2 = c.tol * c.tol * rr0;
    bool ok = true;
    while (rr0 > 0.0 && it < c.maxit) {
      // q = A p, (p, q)
      a0 = 0.0;
      for (int64_t g = t0; g < c.n; g += stride) {
        const int I = (int)(g % c.NX), J = (int)((g / c.NX) % c.NY), K = (int)(g / ((int64_t)c.NX * c.NY));
        double acc = 0.0;
#pragma unroll
        for (int sl = 0; sl < 27; ++sl) {
          const int dI = sl % 3 - 1, dJ = (sl / 3) % 3 - 1, dK = sl / 9 - 1;
          const int I2 = I + dI, J2 = J + dJ, K2 = K + dK;
          if (I2 < 0 || I2 >= c.NX || J2 < 0 || J2 >= c.NY || K2 < 0 || K2 >= c.NZ) continue;
          acc = fma(c.A[sl * c.n + g], c.p[g + dI + (int64_t)c.NX * (dJ + (int64_t)c.NY * dK)], acc);
        }
        c.q[g] = acc;
        a0 = fma(c.p[g], acc, a0);
      }
      a1 = 0.0;
      block_reduce2(a0, a1, sh);
      if (threadIdx.x == 0) {
        c.partA[2 * blockIdx.x] = a0;
        c.partA[2 * blockIdx.x + 1] = 0.0;
      }
      if (!(ok = grid_barrier(c.bar, c.status, nb, c.timeout_ns))) break;
      double pq, unused;
      sum_partials(c.partA, nb, pq, unused, sh);
      const double alpha = rz / pq;
      a0 = 0.0;
      a1 = 0.0;
      for (int64_t g = t0; g < c.n; g += stride) {
        c.x[g] = fma(alpha, c.p[g], c.x[g]);
        const double rv = fma(-alpha, c.q[g], c.r[g]);
        c.r[g] = rv;
        const double zv = c.dinv[g] * rv;
        c.z[g] = zv;
        a0 = fma(rv, zv, a0);
        a1 = fma(rv, rv, a1);
      }
      block_reduce2(a0, a1, sh);
      if (threadIdx.x == 0) {
        c.partB[2 * blockIdx.x] = a0;
        c.partB[2 * blockIdx.x + 1] = a1;
      }
      if (!(ok = grid_barrier(c.bar, c.status, nb, c.timeout_ns))) break;
      double rz_new, rr;
      sum_partials(c.partB, nb, rz_new, rr, sh);
      ++it;
      if (rr <= tol2) break;
      const double beta = rz_new / rz;
      rz = rz_new;
      for (int64_t g = t0; g < c.n; g += stride) c.p[g] = fma(beta, c.p[g], c.z[g]);
      if (!(ok = grid_barrier(c.bar, c.status, nb, c.timeout_ns))) break;
    }
    if (ok) {
      for (int64_t l = t0; l < c.L; l += stride) c.xout[l] = (T)c.x[c.l2g[l]];
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) c.status[1] = it;
}

int coarse_alloc(const Level& lv, Allocs& allocs, CoarseWork* w) {
  const int64_t n = lv.n_global;
  int dev = 0, sms = 0, per_sm = 0;
  SE_CUDA(cudaGetDevice(&dev));
  SE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  SE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coarse_pcg_kernel<double>, CG_THREADS, 0));
  int per_sm32 = 0;
  SE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm32, coarse_pcg_kernel<float>, CG_THREADS, 0));
  if (per_sm32 < per_sm) per_sm = per_sm32;
  SE_CHECK(per_sm >= 1, SE_ECUDA, "coarse solver kernel cannot be resident");
  int64_t want = (n + CG_THREADS - 1) / CG_THREADS;
  const int64_t cap = (int64_t)sms * (per_sm < 2 ? per_sm : 2);
  if (want > cap) want = cap;
  if (want < 1) want = 1;
  w->nblocks = (int)want;
  SE_TRY(dmalloc(allocs, &w->x, n));
  SE_TRY(dmalloc(allocs, &w->r, n));
  SE_TRY(dmalloc(allocs, &w->z, n));
  SE_TRY(dmalloc(allocs, &w->p, n));
  SE_TRY(dmalloc(allocs, &w->q, n));
  SE_TRY(dmalloc(allocs, &w->partial, 4 * (size_t)w->nblocks));
  SE_TRY(dmalloc(allocs, &w->bar, 2));
  SE_TRY(dmalloc(allocs, &w->status, 2));
  SE_CUDA(cudaMemset(w->bar, 0, 2 * sizeof(unsigned)));
  SE_CUDA(cudaMemset(w->status, 0, 2 * sizeof(int)));
  return SE_OK;
}

template <class T>
int coarse_solve(const Level& lv, CoarseWork& w, const T* r_l, T* x_l, double tol, int maxit,
                 cudaStream_t s) {
  CoarseArgs<T> a;
  a.n = lv.n_global;
  a.L = lv.L;
  a.NX = lv.NX;
  a.NY = lv.NY;
  a.NZ = lv.NZ;
  a.A = lv.Ac;
  a.dinv = lv.cdinv;
  a.g2l = lv.g2l;
  a.l2g = lv.l2g;
  a.rin = r_l;
  a.xout = x_l;
  a.x = w.x;
  a.r = w.r;
  a.z = w.z;
  a.p = w.p;
  a.q = w.q;
  a.partA = w.partial;
  a.partB = w.partial + 2 * w.nblocks;
  a.bar = w.bar;
  a.status = w.status;
  a.tol = tol;
  a.maxit = maxit;
  a.timeout_ns = BARRIER_TIMEOUT_NS;
  ProfScope prof(SE_K_COARSE, s, (double)lv.n_global, 0.0, 0.0);
  SE_CUDA(cudaMemsetAsync(w.bar, 0, 2 * sizeof(unsigned), s));
  SE_CUDA(cudaMemsetAsync(w.status, 0, 2 * sizeof(int), s));
  void* args[] = {&a};
  SE_CUDA(cudaLaunchCooperativeKernel((const void*)coarse_pcg_kernel<T>, dim3(w.nblocks),
                                      dim3(CG_THREADS), args, 0, s));
  return SE_OK;
}

template int coarse_solve<double>(const Level&, CoarseWork&, const double*, double*, double, int, cudaStream_t);
template int coarse_solve<float>(const Level&, CoarseWork&, const float*, float*, double, int, cudaStream_t);

// ------------------------------------------------------------------ self-test of the wait limit
__global__ void barrier_timeout_kernel(unsigned* bar, int* status, long long timeout_ns) {
  // one more arrival is expected than blocks exist: nobody can pass, every block times out
  grid_barrier(bar, status, gridDim.x + 1, timeout_ns);
}

}  // namespace se

using namespace se;

extern "C" int se_selftest_wait_timeout(double timeout_ms) {
  SE_CHECK(timeout_ms > 0 && timeout_ms <= 5000, SE_EINVAL, "timeout_ms must be in (0, 5000]");
  unsigned* bar = nullptr;
  int* status = nullptr;
  SE_CUDA(cudaMalloc(&bar, 2 * sizeof(unsigned)));
  SE_CUDA(cudaMalloc(&status, 2 * sizeof(int)));
  SE_CUDA(cudaMemset(bar, 0, 2 * sizeof(unsigned)));
  SE_CUDA(cudaMemset(status, 0, 2 * sizeof(int)));
  barrier_timeout_kernel<<<4, 32>>>(bar, status, (long long)(timeout_ms * 1e6));
  cudaError_t e = cudaDeviceSynchronize();
  int h[2] = {0, 0};
  cudaMemcpy(h, status, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(bar);
  cudaFree(status);
  SE_CHECK(e == cudaSuccess, SE_ECUDA, "selftest kernel failed: %s", cudaGetErrorString(e));
  if (h[0] == SE_ETIMEOUT) {
    set_error("device wait gave up after %.1f ms (expected in this self-test)", timeout_ms);
    return SE_ETIMEOUT;
  }
  set_error("device wait did not report a timeout");
  return SE_ECUDA;
}

// ------------------------------------------------------------------ coarse solve, no allocation
// Scratch of se_pmg_coarse_solve_noalloc: the five CG vectors (x, r, z, p, q) of at most
// NOALLOC_MAX_N coarse nodes, the per-block partial sums, and four 32-bit words at the end
// (barrier count and generation, status, iteration count).  It lives in the library's static
// device memory: every GPU that loads the library holds it until the process exits.
namespace se {
constexpr int64_t NOALLOC_MAX_N = 1 << 17;        // 131072 coarse (p = 1) global nodes
constexpr int NOALLOC_MAX_BLOCKS = 1024;
constexpr int64_t NOALLOC_WORDS = 5 * NOALLOC_MAX_N + 4 * NOALLOC_MAX_BLOCKS + 2;
static __device__ __align__(256) double g_coarse_scratch[NOALLOC_WORDS];

static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[64] = {};  // device address of g_coarse_scratch, per device

// Host code must not use g_coarse_scratch itself (that name is a host-side stand-in): the
// device address is looked up once per device, with that device current.
static int noalloc_scratch(double** out) {
  int dev = 0;
  SE_CUDA(cudaGetDevice(&dev));
  SE_CHECK(dev >= 0 && dev < 64, SE_EINVAL, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    SE_CUDA(cudaGetSymbolAddress(&p, g_coarse_scratch));
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return SE_OK;
}
}  // namespace se

extern "C" int se_pmg_coarse_solve_noalloc(se_pmg_t P, const double* r, double* x, int* iters,
                                           void* stream) {
  SE_CHECK(P && r && x, SE_EINVAL, "se_pmg_coarse_solve_noalloc: null argument");
  const Level& c = *P->lv[P->nlev - 1];
  SE_CHECK(c.n_global <= NOALLOC_MAX_N, SE_EINVAL,
           "se_pmg_coarse_solve_noalloc: coarse level has %lld nodes, above the static limit of %lld",
           (long long)c.n_global, (long long)NOALLOC_MAX_N);
  SE_CHECK(P->cw.nblocks <= NOALLOC_MAX_BLOCKS, SE_EINVAL,
           "se_pmg_coarse_solve_noalloc: %d blocks above the static limit %d", P->cw.nblocks,
           NOALLOC_MAX_BLOCKS);
  double* base = nullptr;
  SE_TRY(noalloc_scratch(&base));
  cudaStream_t s = as_stream(stream, P->stream);
  CoarseWork w;
  w.nblocks = P->cw.nblocks;  // same grid as se_pmg_coarse_solve: same summation order
  w.x = base;
  w.r = base + NOALLOC_MAX_N;
  w.z = base + 2 * NOALLOC_MAX_N;
  w.p = base + 3 * NOALLOC_MAX_N;
  w.q = base + 4 * NOALLOC_MAX_N;
  w.partial = base + 5 * NOALLOC_MAX_N;
  w.bar = reinterpret_cast<unsigned*>(base + 5 * NOALLOC_MAX_N + 4 * NOALLOC_MAX_BLOCKS);
  w.status = reinterpret_cast<int*>(w.bar + 2);
  // coarse_solve zeroes the barrier and status words before its launch; the vectors are fully
  // written before they are read
  SE_TRY(coarse_solve<double>(c, w, r, x, P->desc.coarse_tol, P->desc.coarse_maxit, s));
  int h[2] = {0, 0};
  SE_CUDA(cudaMemcpyAsync(h, w.status, sizeof(h), cudaMemcpyDeviceToHost, s));
  SE_CUDA(cudaStreamSynchronize(s));
  if (iters) *iters = h[1];
  SE_CHECK(h[0] == 0, SE_ETIMEOUT, "coarse solve: a grid barrier wait ran out");
  return SE_OK;
}
