// Coarsest level (p = 1): assembled 27-point operator and a persistent Jacobi-PCG solve.
//
// The paper solves the coarse system with one BoomerAMG V-cycle (Sec. 2.2.2), a third-party
// library; here the coarse problem is solved by Jacobi-preconditioned CG to a relative tolerance.
// The p = 1 element matrices are assembled into rows over global lattice nodes (27 entries each,
// summed over the up to 8 elements sharing the row node in a fixed order: deterministic), and the
// whole CG iteration runs in ONE cooperative launch.  On this part a grid-wide synchronisation
// costs microseconds and a chain of dependent FP64 operations about 0.1 us per link, so the
// iteration is the pipelined form of preconditioned CG (one synchronisation per iteration, which
// carries all three inner products and orders the neighbour reads of the operator product).
// Every wait is bounded by a wall-clock limit after which the kernel records SE_ETIMEOUT and
// returns.
#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "pmg_internal.h"

namespace se {

constexpr long long BARRIER_TIMEOUT_NS = 2000000000LL;  // 2 s

__device__ __forceinline__ long long global_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr int CG_THREADS = 256;

// Sums of three values over the block, left in thread 0.  Every thread posts its values to shared
// memory; with three warps or more, warp k adds value k (lane l: entries l, l + 32, ... in order,
// then a shuffle tree), otherwise warp 0 adds all three: a fixed order (deterministic), few
// warp-wide FP64 additions (each occupies the SM's 2-lane FP64 pipe for 16 cycles) and a short
// chain of dependent ones.
__device__ __forceinline__ void block_sum3(double (&v)[3], double* red) {
  __shared__ double s3[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) red[k * blockDim.x + threadIdx.x] = v[k];
  __syncthreads();
  const unsigned w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (blockDim.x >= 96) {
    if (w < 3) {
      double acc = red[w * blockDim.x + lane];
      for (unsigned i = lane + 32; i < blockDim.x; i += 32) acc += red[w * blockDim.x + i];
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
      if (lane == 0) s3[w] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      v[0] = s3[0];
      v[1] = s3[1];
      v[2] = s3[2];
    }
  } else if (threadIdx.x < 32) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double acc = red[k * blockDim.x + threadIdx.x];
      for (unsigned i = threadIdx.x + 32; i < blockDim.x; i += 32) acc += red[k * blockDim.x + i];
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
      v[k] = acc;
    }
  }
}

// Pairwise sum of K register values in a fixed order: depth ceil(log2 K) instead of K - 1 (a
// dependent FP64 addition costs far more here than an independent one).
template <int K>
__device__ __forceinline__ double pairwise_sum(const double (&a)[K]) {
  if constexpr (K == 1) {
    return a[0];
  } else {
    constexpr int H = K / 2;
    double lo[H], hi[K - H];
#pragma unroll
    for (int i = 0; i < H; ++i) lo[i] = a[i];
#pragma unroll
    for (int i = 0; i < K - H; ++i) hi[i] = a[H + i];
    return pairwise_sum<H>(lo) + pairwise_sum<K - H>(hi);
  }
}

__device__ __forceinline__ unsigned atomic_add_release(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ unsigned load_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier that sums three values over the grid.  count is a monotonic arrival counter
// (zeroed before the launch): the k-th call of every block is complete once count reaches
// (k + 1) * nblocks.  Each block (index blk among the nblocks that share count) posts its sums
// to part[parity][blk] (4 doubles, the 4th
// unused) and arrives with a release add; then every block waits for the count with acquire loads
// and adds all blocks' partials itself, in block order (lane l: blocks l, l + 32, ..., then a
// shuffle tree), so all blocks get bitwise the same sums with no second round trip through a
// published result.  Partials alternate between two buffers: a block can post the partials of
// call k + 2 (same buffer as call k) only after every block has arrived at call k + 1, that is
// after every block has read the partials of call k.  Thread 0 of each block then evaluates
// post(v) (the scalar recurrence coefficients: FP64 divisions once per block, not per thread),
// which may rewrite v and returns one more value; every thread receives v and that value.  A
// wait gives up after timeout_ns and records SE_ETIMEOUT in status[0]; the function returns false
// once status[0] is set.
template <class Post>
__device__ bool grid_sum3(unsigned* count, unsigned call, int* status, unsigned nblocks,
                          long long timeout_ns, double* part, double (&v)[3], double& post_value,
                          double* red, Post post, unsigned blk) {
  __shared__ double s_out[4];
  block_sum3(v, red);
  double* buf = part + (size_t)(call & 1u) * 4 * nblocks;
  if (threadIdx.x == 0) {
    reinterpret_cast<double2*>(buf)[2 * blk] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(buf)[2 * blk + 1] = make_double2(v[2], 0.0);
    atomic_add_release(count, 1u);
    const unsigned target = (call + 1u) * nblocks;
    const long long t0 = global_ns();
    while ((int)(load_acquire(count) - target) < 0) {
      __nanosleep(32);
      if (*(volatile int*)status != 0) break;
      if (global_ns() - t0 > timeout_ns) {
        atomicExch(status, SE_ETIMEOUT);
        break;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    // all loads of the lane issued together: at most 10 blocks per lane in the first pass
    constexpr int UNR = 10;
    double2 lo[UNR], hi[UNR];
#pragma unroll
    for (int i = 0; i < UNR; ++i) {
      const unsigned k = threadIdx.x + 32u * i;
      lo[i] = k < nblocks ? __ldcg(reinterpret_cast<const double2*>(buf) + 2 * k) : make_double2(0.0, 0.0);
      hi[i] = k < nblocks ? __ldcg(reinterpret_cast<const double2*>(buf) + 2 * k + 1) : make_double2(0.0, 0.0);
    }
    // pairwise within the lane (absent blocks contribute exact zeros): short dependent chains
    double a0[UNR], a1[UNR], a2[UNR];
#pragma unroll
    for (int i = 0; i < UNR; ++i) {
      a0[i] = lo[i].x;
      a1[i] = lo[i].y;
      a2[i] = hi[i].x;
    }
    double s0 = pairwise_sum(a0), s1 = pairwise_sum(a1), s2 = pairwise_sum(a2);
    for (unsigned k = threadIdx.x + 32u * UNR; k < nblocks; k += 32) {
      const double2 l = __ldcg(reinterpret_cast<const double2*>(buf) + 2 * k);
      const double2 h = __ldcg(reinterpret_cast<const double2*>(buf) + 2 * k + 1);
      s0 += l.x;
      s1 += l.y;
      s2 += h.x;
    }
    if (threadIdx.x >= nblocks) s0 = s1 = s2 = 0.0;  // lanes without a block
    for (int o = 16; o > 0; o >>= 1) {
      s0 += __shfl_down_sync(0xffffffffu, s0, o);
      s1 += __shfl_down_sync(0xffffffffu, s1, o);
      s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if (threadIdx.x == 0) {
      double w[3] = {s0, s1, s2};
      const double pv = post(w);
      s_out[0] = w[0];
      s_out[1] = w[1];
      s_out[2] = w[2];
      s_out[3] = pv;
    }
  }
  __syncthreads();
  v[0] = s_out[0];
  v[1] = s_out[1];
  v[2] = s_out[2];
  post_value = s_out[3];
  const bool ok = *(volatile int*)status == 0;
  __syncthreads();
  return ok;
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

// Ahat = A D^-1 (column g' of row g scaled by dinv[g']): the pipelined iteration needs A applied
// only to D^-1-scaled vectors.  Slots whose neighbour lies outside the lattice hold 0 already.
__global__ void coarse_scale_columns_kernel(int NX, int NY, int64_t n, const double* __restrict__ dinv,
                                            double* __restrict__ A) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 27 * n) return;
  const int slot = (int)(t / n);
  const int64_t g = t - (int64_t)slot * n;
  const int dI = slot % 3 - 1, dJ = (slot / 3) % 3 - 1, dK = slot / 9 - 1;
  int64_t gc = g + dI + (int64_t)NX * (dJ + (int64_t)NY * dK);
  gc = gc < 0 ? 0 : (gc >= n ? n - 1 : gc);
  A[t] *= dinv[gc];
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
  coarse_scale_columns_kernel<<<grid_for(27 * n, 256), 256, 0, s>>>(lv.NX, lv.NY, n, lv.cdinv, lv.Ac);
  SE_LAUNCH_CHECK();
  return local_to_global(lv, lv.l2g, s);
}

// ------------------------------------------------------------------ persistent Jacobi-PCG
template <class T>
struct CoarseArgs {
  int n, L;
  int NX, NY;
  const double* Ah;    // A D^-1, [27][n]
  const double* dinv;
  const int* g2l;
  const int* l2g;
  const T* rin;
  T* xout;
  double *x, *r, *u, *p, *q, *s, *z, *w0, *w1, *part;
  unsigned* count;
  int* status;
  unsigned* flags;             // [nflags] w generations per block (register-resident solver)
  int nflags;
  unsigned long long* totals;  // iterations and solves, accumulated (null: not counted)
  double tol;
  int maxit;
  long long timeout_ns;
};

// (Ahat v)_g over the 27 lattice neighbours of g.  A slot whose neighbour lies outside the lattice
// holds 0 (assembly), so its index is only clamped into the array: the product adds exactly 0.
__device__ __forceinline__ double coarse_row(const double* __restrict__ Ah, const double* v, int n,
                                             int NX, int NXY, int g) {
  double acc = 0.0;
#pragma unroll
  for (int sl = 0; sl < 27; ++sl) {
    const int dI = sl % 3 - 1, dJ = (sl / 3) % 3 - 1, dK = sl / 9 - 1;
    const int gi = min(max(g + dI + NX * dJ + NXY * dK, 0), n - 1);
    acc = fma(Ah[(int64_t)sl * n + g], v[gi], acc);
  }
  return acc;
}

// Pipelined Jacobi-preconditioned CG (Ghysels and Vanroose, Parallel Computing 40, 2014,
// preconditioned pipelined CG), M^-1 = D^-1:
//   r = b, u = D^-1 r, w = A u
//   loop: gamma = (r, u), delta = (w, u)                         [one synchronisation]
//         beta = gamma / gamma_prev, alpha = gamma / (delta - beta gamma / alpha_prev)
//                                            (first pass: beta = 0, alpha = gamma / delta)
//         m = D^-1 w, n = A m (= Ahat w)
//         z = n + beta z, q = m + beta q, s = w + beta s, p = u + beta p
//         x += alpha p, r -= alpha s, u -= alpha q, w -= alpha z
// In exact arithmetic it produces the iterates of textbook PCG.  The synchronisation that sums
// (gamma, delta, (r, r)) also orders the neighbour reads of Ahat w: w alternates between two
// arrays (read one, write the other).  The stopping rule is that of the textbook loop: stop
// after the update that brings (r, r) to tol^2 (b, b) or below, or after maxit updates.
// Run by the nb blocks of one coarse problem; blk is this block's index among them.
template <class T>
__device__ __forceinline__ void coarse_pcg_run(const CoarseArgs<T>& c, unsigned blk, unsigned nb) {
  __shared__ double red[3 * CG_THREADS];
  const int stride = (int)nb * CG_THREADS;
  const int t0 = (int)blk * CG_THREADS + threadIdx.x;
  const int NXY = c.NX * c.NY;
  unsigned call = 0;
  double v[3] = {0.0, 0.0, 0.0}, unused;
  // r = b, u = D^-1 r, x = 0; (r, r)
  for (int g = t0; g < c.n; g += stride) {
    const double rv = (double)c.rin[c.g2l[g]];
    c.r[g] = rv;
    c.u[g] = c.dinv[g] * rv;
    c.x[g] = 0.0;
    v[2] = fma(rv, rv, v[2]);
  }
  bool ok = grid_sum3(c.count, call++, c.status, nb, c.timeout_ns, c.part, v, unused, red,
                      [](double (&)[3]) { return 0.0; }, blk);
  const double rr0 = v[2];
  const double tol2 = c.tol * c.tol * rr0;
  // w = A u = Ahat r; gamma = (r, u), delta = (w, u)
  v[0] = v[1] = v[2] = 0.0;
  if (ok) {
    for (int g = t0; g < c.n; g += stride) {
      const double wv = coarse_row(c.Ah, c.r, c.n, c.NX, NXY, g);
      const double uv = c.u[g], rv = c.r[g];
      c.w0[g] = wv;
      v[0] = fma(rv, uv, v[0]);
      v[1] = fma(wv, uv, v[1]);
    }
  }
  int it = 0;
  double gamma = 0.0, alpha = 0.0;
  while (ok && rr0 > 0.0) {
    // v = (gamma, delta, (r, r)) -> (alpha, beta, (r, r)); post returns gamma
    const double g_prev = gamma, a_prev = alpha;
    const bool first = it == 0;
    ok = grid_sum3(c.count, call++, c.status, nb, c.timeout_ns, c.part, v, gamma, red,
                   [=](double (&w)[3]) {
                     const double gm = w[0], dl = w[1];
                     const double be = first ? 0.0 : gm / g_prev;
                     w[0] = first ? gm / dl : gm / (dl - be * gm / a_prev);
                     w[1] = be;
                     return gm;
                   }, blk);
    if (!ok) break;
    // after a synchronisation, so x is complete whichever way the loop ends
    if (!first && v[2] <= tol2) break;  // (r, r) of the last update
    if (it >= c.maxit) break;
    alpha = v[0];
    const double beta = v[1];
    const double* wr = (it & 1) ? c.w1 : c.w0;
    double* ww = (it & 1) ? c.w0 : c.w1;
    v[0] = v[1] = v[2] = 0.0;
    for (int g = t0; g < c.n; g += stride) {
      const double wv = wr[g];
      const double mv = c.dinv[g] * wv;
      const double nv = coarse_row(c.Ah, wr, c.n, c.NX, NXY, g);
      const double zv = first ? nv : fma(beta, c.z[g], nv);
      const double qv = first ? mv : fma(beta, c.q[g], mv);
      const double sv = first ? wv : fma(beta, c.s[g], wv);
      const double pv = first ? c.u[g] : fma(beta, c.p[g], c.u[g]);
      c.z[g] = zv;
      c.q[g] = qv;
      c.s[g] = sv;
      c.p[g] = pv;
      c.x[g] = fma(alpha, pv, c.x[g]);
      const double rv = fma(-alpha, sv, c.r[g]);
      const double uv = fma(-alpha, qv, c.u[g]);
      const double wn = fma(-alpha, zv, wv);
      c.r[g] = rv;
      c.u[g] = uv;
      ww[g] = wn;
      v[0] = fma(rv, uv, v[0]);
      v[1] = fma(wn, uv, v[1]);
      v[2] = fma(rv, rv, v[2]);
    }
    ++it;
  }
  if (ok) {
    for (int l = t0; l < c.L; l += stride) c.xout[l] = (T)c.x[c.l2g[l]];
  }
  if (blk == 0 && threadIdx.x == 0) {
    c.status[1] = it;
    if (c.totals) {
      atomicAdd(c.totals, (unsigned long long)it);
      atomicAdd(c.totals + 1, 1ULL);
      if (!ok) atomicAdd(c.totals + 2, 1ULL);  // results of this solve are invalid
    }
  }
}

// ------------------------------------------------------------------ register-resident variant
// For a coarse problem with at most one node per thread of its grid.  Block blk owns the
// contiguous nodes [blk C, blk C + C), C = ceil(n / nb); each thread keeps its CG values in
// registers and its node's row of Ahat in shared memory (COARSE_ROW_SMEM bytes of dynamic shared
// memory per block), so per iteration only w travels through global memory.  The
// synchronisation is split in the way the pipelined method allows: the global sums of an
// iteration are posted as soon as its updates are done, and while they travel every block forms
// m = D^-1 w and n = Ahat w, which need only the w of the blocks within reach of the 27-point
// stencil (per-block flags, not the whole grid).  The iterates are those of coarse_pcg_run; only
// the order of the partial sums differs (block ranges instead of grid-strided loops).

constexpr size_t COARSE_ROW_SMEM = 27 * CG_THREADS * sizeof(double);

__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Block sums of three values in thread 0, one warp per value: the values go through shared
// memory, warp k adds value k (lane l: threads l, l + 32, ... pairwise, then a five-level
// shuffle tree).  Each warp-wide FP64 addition occupies the SM's 2-lane FP64 pipe for 16 cycles
// however many lanes are active, so three warps adding 12 times cost a third of the pipe time of
// eight warps' trees, at a similar depth of dependent additions.  A fixed order (deterministic).
__device__ __forceinline__ void block_sum3_split(double (&v)[3], double* red, double* out3) {
  static_assert(CG_THREADS % 32 == 0 && CG_THREADS >= 96, "three warps");
#pragma unroll
  for (int k = 0; k < 3; ++k) red[k * CG_THREADS + threadIdx.x] = v[k];
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (w < 3) {
    double a[CG_THREADS / 32];
#pragma unroll
    for (int i = 0; i < CG_THREADS / 32; ++i) a[i] = red[w * CG_THREADS + lane + 32 * i];
    double acc = pairwise_sum(a);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) out3[w] = acc;
  }
  __syncthreads();
}

// First half of a summing barrier: the block's sums of v are posted to part[call parity][blk];
// then (thread 0, release) this block's flag is set to flag_value and its arrival counted.
// Every write the block made before the call is visible to a block that observes either.
__device__ __forceinline__ void grid_post3(unsigned* count, unsigned call, unsigned nblocks,
                                           double* part, double (&v)[3], double* red, unsigned blk,
                                           unsigned* flag, unsigned flag_value) {
  __shared__ double s3[3];
  block_sum3_split(v, red, s3);
  if (threadIdx.x == 0) {
    double* buf = part + (size_t)(call & 1u) * 4 * nblocks;
    reinterpret_cast<double2*>(buf)[2 * blk] = make_double2(s3[0], s3[1]);
    reinterpret_cast<double2*>(buf)[2 * blk + 1] = make_double2(s3[2], 0.0);
    st_release(flag, flag_value);
    atomic_add_release(count, 1u);
  }
}

// Second half: waits until all nblocks blocks have posted call `call`, then adds their partials
// in a fixed order (warp k adds value k of the blocks in order, lane-sequentially, then a tree) and
// thread 0 evaluates post(v); every thread gets v and post's value.  False once status[0] is set
// (an expired wait here or elsewhere).
template <class Post>
__device__ bool grid_wait3(unsigned* count, unsigned call, int* status, unsigned nblocks,
                           long long timeout_ns, const double* part, double (&v)[3],
                           double& post_value, double* red, Post post) {
  __shared__ double s_out[4];
  const double* buf = part + (size_t)(call & 1u) * 4 * nblocks;
  if (threadIdx.x == 0) {
    const unsigned target = (call + 1u) * nblocks;
    const long long t0 = global_ns();
    while ((int)(load_acquire(count) - target) < 0) {
      if (*(volatile int*)status != 0) break;
      if (global_ns() - t0 > timeout_ns) {
        atomicExch(status, SE_ETIMEOUT);
        break;
      }
    }
  }
  __syncthreads();
  // warp k adds value k of every block (lane l: blocks l, l + 32, ..., all loads issued first),
  // then a shuffle tree; thread 0 gathers the three sums
  double w[3] = {0.0, 0.0, 0.0};
  {
    const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (wp < 3) {
      constexpr int UNR = 10;
      double t[UNR];
#pragma unroll
      for (int i = 0; i < UNR; ++i) {
        const unsigned k = lane + 32u * i;
        t[i] = k < nblocks ? __ldcg(buf + 4 * k + wp) : 0.0;
      }
      double acc = pairwise_sum(t);
      for (unsigned k = lane + 32u * UNR; k < nblocks; k += 32) acc += __ldcg(buf + 4 * k + wp);
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
      if (lane == 0) red[wp] = acc;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    w[0] = red[0];
    w[1] = red[1];
    w[2] = red[2];
    const double pv = post(w);
    s_out[0] = w[0];
    s_out[1] = w[1];
    s_out[2] = w[2];
    s_out[3] = pv;
  }
  __syncthreads();
  v[0] = s_out[0];
  v[1] = s_out[1];
  v[2] = s_out[2];
  post_value = s_out[3];
  return *(volatile int*)status == 0;
}

// Waits (bounded) until flags[b] >= want for every block b in [b0, b1]; warp 0 polls.
__device__ bool wait_flags(const unsigned* flags, int b0, int b1, unsigned want, int* status,
                           long long timeout_ns) {
  if (threadIdx.x < 32) {
    const long long t0 = global_ns();
    for (int b = b0 + (int)threadIdx.x; b <= b1; b += 32) {
      while ((int)(load_acquire(flags + b) - want) < 0) {
        if (*(volatile int*)status != 0) break;
        if (global_ns() - t0 > timeout_ns) {
          atomicExch(status, SE_ETIMEOUT);
          break;
        }
      }
    }
  }
  __syncthreads();
  return *(volatile int*)status == 0;
}

// Neighbour (slot sl of the 27-point row) of node g, clamped into [0, n): a slot outside the
// lattice holds 0 in Ahat, so the clamped read adds exactly 0.
__device__ __forceinline__ int coarse_nbr(int g, int sl, int n, int NX, int NXY) {
  const int dI = sl % 3 - 1, dJ = (sl / 3) % 3 - 1, dK = sl / 9 - 1;
  return min(max(g + dI + NX * dJ + NXY * dK, 0), n - 1);
}

template <class T>
__device__ __forceinline__ void coarse_pcg_reg(const CoarseArgs<T>& c, unsigned blk, unsigned nb) {
  __shared__ double red[3 * CG_THREADS];
  const int n = c.n, NX = c.NX, NXY = c.NX * c.NY;
  const int C = (int)((n + (int)nb - 1) / (int)nb);
  const int g0 = (int)blk * C;
  const int g = g0 + (int)threadIdx.x;
  const bool act = (int)threadIdx.x < C && g < n;
  // blocks whose nodes the rows of this block reach
  const int reach = NXY + NX + 1;
  const int glast = min(n, g0 + C) - 1;
  const int b0 = max(0, g0 - reach) / C;
  const int b1 = min((int)nb - 1, (glast + reach) / C);
  unsigned* myflag = c.flags + blk;
  extern __shared__ double row_sm[];  // [27][CG_THREADS]
  double* row = row_sm + threadIdx.x;
  double d = 0.0, r = 0.0, u = 0.0, x = 0.0, p = 0.0, q = 0.0, sv = 0.0, z = 0.0, w = 0.0;
  if (act) {
#pragma unroll
    for (int sl = 0; sl < 27; ++sl) row[sl * CG_THREADS] = c.Ah[(int64_t)sl * n + g];
    d = c.dinv[g];
    r = (double)c.rin[c.g2l[g]];
    u = d * r;
    // w = A u = Ahat r, the neighbours' r straight from the input
    double acc = 0.0;
#pragma unroll
    for (int sl = 0; sl < 27; ++sl)
      acc = fma(row[sl * CG_THREADS], (double)c.rin[c.g2l[coarse_nbr(g, sl, n, NX, NXY)]], acc);
    w = acc;
    c.w0[g] = w;
  }
  double v[3] = {r * u, w * u, r * r};
  unsigned call = 0;
  grid_post3(c.count, call, nb, c.part, v, red, blk, myflag, 1u);
  int it = 0;
  double gamma = 0.0, alpha = 0.0, tol2 = 0.0;
  double R = 0.0, K = 0.0;  // thread 0: 1 / gamma_prev, 1 / (gamma_prev alpha_prev)
  bool ok = true;
  for (;;) {
    // m = D^-1 w, n = Ahat w on this iteration's w (neighbours: generation it + 1 published)
    ok = wait_flags(c.flags, b0, b1, (unsigned)(it + 1), c.status, c.timeout_ns);
    if (!ok) break;
    const double* wr = (it & 1) ? c.w1 : c.w0;
    double m = 0.0, nv = 0.0;
    if (act) {
      m = d * w;
      double acc = 0.0;
#pragma unroll
      for (int sl = 0; sl < 27; ++sl)
        acc = fma(row[sl * CG_THREADS], wr[coarse_nbr(g, sl, n, NX, NXY)], acc);
      nv = acc;
    }
    // (gamma, delta, (r, r)) of the current iterate -> (alpha, beta, (r, r)); post returns gamma.
    // beta = gamma / gamma_prev and alpha = gamma / (delta - beta gamma / alpha_prev) with the
    // previous iteration's reciprocals, so one division is on the critical path (an FP64
    // division is a long chain of dependent FP64 operations on this part)
    const bool first = it == 0;
    ok = grid_wait3(c.count, call++, c.status, nb, c.timeout_ns, c.part, v, gamma, red,
                    [&](double (&s)[3]) {
                      const double gm = s[0], dl = s[1];
                      const double be = first ? 0.0 : gm * R;
                      const double al = gm / (first ? dl : fma(-gm * gm, K, dl));
                      s[0] = al;
                      s[1] = be;
                      return gm;
                    });
    if (!ok) break;
    if (first) {
      tol2 = c.tol * c.tol * v[2];
      if (!(v[2] > 0.0)) break;       // b = 0: x = 0
    } else if (v[2] <= tol2) {
      break;                          // (r, r) of the last update
    }
    if (it >= c.maxit) break;
    alpha = v[0];
    if (threadIdx.x == 0) {  // for the next iteration, while the other threads update
      R = 1.0 / gamma;
      K = R / alpha;
    }
    const double beta = v[1];
    if (act) {
      z = first ? nv : fma(beta, z, nv);
      q = first ? m : fma(beta, q, m);
      sv = first ? w : fma(beta, sv, w);
      p = first ? u : fma(beta, p, u);
      x = fma(alpha, p, x);
      r = fma(-alpha, sv, r);
      u = fma(-alpha, q, u);
      w = fma(-alpha, z, w);
      ((it & 1) ? c.w0 : c.w1)[g] = w;  // the buffer read one iteration ago
    }
    v[0] = r * u;
    v[1] = w * u;
    v[2] = r * r;
    ++it;
    grid_post3(c.count, call, nb, c.part, v, red, blk, myflag, (unsigned)(it + 1));
  }
  // x to memory, one more summing barrier (nothing summed), then each local copy takes its node
  if (ok) {
    if (act) c.x[g] = x;
    double zero[3] = {0.0, 0.0, 0.0}, unused;
    grid_post3(c.count, call, nb, c.part, zero, red, blk, myflag, 0xffffffffu);
    ok = grid_wait3(c.count, call++, c.status, nb, c.timeout_ns, c.part, zero, unused, red,
                    [](double (&)[3]) { return 0.0; });
  }
  if (ok) {
    const int stride = (int)nb * CG_THREADS;
    for (int l = (int)blk * CG_THREADS + (int)threadIdx.x; l < c.L; l += stride)
      c.xout[l] = (T)__ldcg(c.x + c.l2g[l]);
  }
  if (blk == 0 && threadIdx.x == 0) {
    c.status[1] = it;
    if (c.totals) {
      atomicAdd(c.totals, (unsigned long long)it);
      atomicAdd(c.totals + 1, 1ULL);
      if (!ok) atomicAdd(c.totals + 2, 1ULL);  // results of this solve are invalid
    }
  }
}

template <class T>
__global__ void __launch_bounds__(CG_THREADS) coarse_pcg_kernel(CoarseArgs<T> c) {
  coarse_pcg_run(c, blockIdx.x, gridDim.x);
}

// One node per thread (n <= gridDim.x * CG_THREADS); launched with COARSE_ROW_SMEM bytes of
// dynamic shared memory.
template <class T>
__global__ void __launch_bounds__(CG_THREADS) coarse_reg_kernel(CoarseArgs<T> c) {
  coarse_pcg_reg(c, blockIdx.x, gridDim.x);
}

// Many independent coarse problems in one cooperative launch: problem m runs on blocks
// [boff[m], boff[m + 1]) with its own arrival counter, partial sums, status and tolerance, so
// each iterates to its own stopping rule (the sub-grids never wait for one another).
template <class T>
__global__ void __launch_bounds__(CG_THREADS) coarse_group_kernel(const CoarseArgs<T>* __restrict__ args,
                                                                  const int* __restrict__ boff, int n) {
  int m = 0;
  while (m + 1 < n && boff[m + 1] <= (int)blockIdx.x) ++m;
  const CoarseArgs<T> c = args[m];
  const unsigned nb = (unsigned)(boff[m + 1] - boff[m]);
  if ((int64_t)c.n <= (int64_t)nb * CG_THREADS)  // uniform over the member's blocks
    coarse_pcg_reg(c, blockIdx.x - (unsigned)boff[m], nb);
  else
    coarse_pcg_run(c, blockIdx.x - (unsigned)boff[m], nb);
}

__global__ void coarse_group_reset_kernel(const CoarseArgs<double>* __restrict__ a64,
                                          const CoarseArgs<float>* __restrict__ a32, int n) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  unsigned* count = a64 ? a64[m].count : a32[m].count;
  int* status = a64 ? a64[m].status : a32[m].status;
  unsigned* flags = a64 ? a64[m].flags : a32[m].flags;
  const int nflags = a64 ? a64[m].nflags : a32[m].nflags;
  count[0] = count[1] = 0u;
  status[0] = status[1] = 0;
  for (int b = 0; b < nflags; ++b) flags[b] = 0u;
}

// The row-resident kernels take more than the default 48 KB of dynamic shared memory only if
// COARSE_ROW_SMEM grows past it; the attribute is set once per process (per device in use).
static int coarse_kernel_attrs() {
  static std::once_flag once;
  static cudaError_t err = cudaSuccess;
  std::call_once(once, [] {
    for (const void* k : {(const void*)coarse_reg_kernel<double>, (const void*)coarse_reg_kernel<float>,
                          (const void*)coarse_group_kernel<double>, (const void*)coarse_group_kernel<float>})
      if (err == cudaSuccess)
        err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)COARSE_ROW_SMEM);
  });
  SE_CUDA(err);
  return SE_OK;
}

// Partial sums of the summing barrier: two buffers of 4 doubles per block.
size_t coarse_partial_doubles(int nblocks) { return 8 * (size_t)nblocks; }

int coarse_alloc(const Level& lv, Allocs& allocs, CoarseWork* w) {
  const int64_t n = lv.n_global;
  SE_CHECK(lv.L < (int64_t)1 << 31 && 27 * n < (int64_t)1 << 40, SE_EINVAL,
           "coarse level with %lld points is too large for 32-bit node indices", (long long)lv.L);
  int dev = 0, sms = 0, per_sm = 0;
  SE_CUDA(cudaGetDevice(&dev));
  SE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  SE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coarse_pcg_kernel<double>, CG_THREADS, 0));
  // every coarse kernel must fit the grid chosen here (the solve picks one by the node count)
  SE_TRY(coarse_kernel_attrs());
  for (const void* k : {(const void*)coarse_pcg_kernel<float>, (const void*)coarse_reg_kernel<double>,
                        (const void*)coarse_reg_kernel<float>}) {
    int o = 0;
    const size_t dyn = k == (const void*)coarse_pcg_kernel<float> ? 0 : COARSE_ROW_SMEM;
    SE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k, CG_THREADS, dyn));
    if (o < per_sm) per_sm = o;
  }
  SE_CHECK(per_sm >= 1, SE_ECUDA, "coarse solver kernel cannot be resident");
  // one point per thread where possible; a grid of more than half the SMs is rounded up to a
  // multiple of the SM count so that the FP64 work spreads evenly
  int64_t want = (n + CG_THREADS - 1) / CG_THREADS;
  if (want > sms / 2) want = (want + sms - 1) / sms * sms;
  const int64_t cap = (int64_t)sms * (per_sm < 2 ? per_sm : 2);
  if (want > cap) want = cap;
  if (want < 1) want = 1;
  w->nblocks = (int)want;
  for (double** v : {&w->x, &w->r, &w->u, &w->p, &w->q, &w->s, &w->z, &w->w0, &w->w1})
    SE_TRY(dmalloc(allocs, v, n));
  SE_TRY(dmalloc(allocs, &w->partial, coarse_partial_doubles(w->nblocks)));
  SE_TRY(dmalloc(allocs, &w->bar, 2));
  SE_TRY(dmalloc(allocs, &w->status, 2));
  SE_TRY(dzero(w->bar, 2 * sizeof(unsigned), allocs.stream));
  SE_TRY(dzero(w->status, 2 * sizeof(int), allocs.stream));
  SE_TRY(dmalloc(allocs, &w->flags, (size_t)w->nblocks));
  SE_TRY(dzero(w->flags, (size_t)w->nblocks * sizeof(unsigned), allocs.stream));
  SE_TRY(dmalloc(allocs, &w->totals, 3));
  SE_TRY(dzero(w->totals, 3 * sizeof(unsigned long long), allocs.stream));
  return SE_OK;
}

template <class T>
int coarse_solve(const Level& lv, CoarseWork& w, const T* r_l, T* x_l, double tol, int maxit,
                 cudaStream_t s) {
  CoarseArgs<T> a;
  a.n = (int)lv.n_global;
  a.L = (int)lv.L;
  a.NX = lv.NX;
  a.NY = lv.NY;
  a.Ah = lv.Ac;
  a.dinv = lv.cdinv;
  a.g2l = lv.g2l;
  a.l2g = lv.l2g;
  a.rin = r_l;
  a.xout = x_l;
  a.x = w.x;
  a.r = w.r;
  a.u = w.u;
  a.p = w.p;
  a.q = w.q;
  a.s = w.s;
  a.z = w.z;
  a.w0 = w.w0;
  a.w1 = w.w1;
  a.part = w.partial;
  a.count = w.bar;
  a.status = w.status;
  a.flags = w.flags;
  a.nflags = w.nblocks;
  a.totals = w.totals;
  a.tol = tol;
  a.maxit = maxit;
  a.timeout_ns = BARRIER_TIMEOUT_NS;
  ProfScope prof(SE_K_COARSE, s, (double)lv.n_global, 0.0, 0.0);
  SE_CUDA(cudaMemsetAsync(w.bar, 0, 2 * sizeof(unsigned), s));
  SE_CUDA(cudaMemsetAsync(w.status, 0, 2 * sizeof(int), s));
  const bool reg = w.flags && lv.n_global <= (int64_t)w.nblocks * CG_THREADS;
  if (reg) SE_CUDA(cudaMemsetAsync(w.flags, 0, (size_t)w.nblocks * sizeof(unsigned), s));
  void* args[] = {&a};
  SE_TRY(coarse_kernel_attrs());
  SE_CUDA(cudaLaunchCooperativeKernel(reg ? (const void*)coarse_reg_kernel<T> : (const void*)coarse_pcg_kernel<T>,
                                      dim3(w.nblocks), dim3(CG_THREADS), args,
                                      reg ? COARSE_ROW_SMEM : 0, s));
  return SE_OK;
}

// ------------------------------------------------------------------ grouped coarse solves
template <class T>
static CoarseArgs<T> coarse_args(const Level& lv, const CoarseWork& w, const T* r_l, T* x_l,
                                 double tol, int maxit) {
  CoarseArgs<T> a;
  a.n = (int)lv.n_global;
  a.L = (int)lv.L;
  a.NX = lv.NX;
  a.NY = lv.NY;
  a.Ah = lv.Ac;
  a.dinv = lv.cdinv;
  a.g2l = lv.g2l;
  a.l2g = lv.l2g;
  a.rin = r_l;
  a.xout = x_l;
  a.x = w.x;
  a.r = w.r;
  a.u = w.u;
  a.p = w.p;
  a.q = w.q;
  a.s = w.s;
  a.z = w.z;
  a.w0 = w.w0;
  a.w1 = w.w1;
  a.part = w.partial;
  a.count = w.bar;
  a.status = w.status;
  a.flags = w.flags;
  a.nflags = w.nblocks;
  a.totals = w.totals;
  a.tol = tol;
  a.maxit = maxit;
  a.timeout_ns = BARRIER_TIMEOUT_NS;
  return a;
}

template <class T>
static int coarse_group_setup_t(CoarseGroup* g, const Level* const* lv, CoarseWork* const* w, int n,
                                const T* rin, T* xout, const int64_t* loff, double tol, int maxit,
                                Allocs& allocs, cudaStream_t s) {
  int dev = 0, sms = 0, per_sm = 0;
  SE_CUDA(cudaGetDevice(&dev));
  SE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  SE_TRY(coarse_kernel_attrs());
  SE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coarse_group_kernel<T>, CG_THREADS,
                                                        COARSE_ROW_SMEM));
  SE_CHECK(per_sm >= 1, SE_ECUDA, "grouped coarse solver kernel cannot be resident");
  const int cap = sms * per_sm;
  SE_CHECK(n <= cap, SE_EINVAL, "grouped coarse solve: %d problems above the %d resident blocks", n, cap);
  // blocks per problem: one node per thread where the co-resident capacity allows (the FP64
  // work of an iteration needs every SM), at most the problem's own work-space size; otherwise
  // proportional to the problem's nodes, at least one each (cooperative launch: the total must
  // be co-resident)
  std::vector<int> nb(n);
  int64_t want_total = 0;
  for (int m = 0; m < n; ++m) {
    const int64_t want = (lv[m]->n_global + CG_THREADS - 1) / CG_THREADS;
    nb[m] = (int)std::max<int64_t>(1, std::min<int64_t>(want, w[m]->nblocks));
    want_total += nb[m];
  }
  if (want_total > cap) {
    int64_t nodes_total = 0;
    for (int m = 0; m < n; ++m) nodes_total += lv[m]->n_global;
    for (int m = 0; m < n; ++m) {
      const int64_t share = (int64_t)((double)(cap - n) * (double)lv[m]->n_global / (double)nodes_total);
      nb[m] = (int)std::max<int64_t>(1, std::min<int64_t>(nb[m], 1 + share));
    }
  }
  int total = 0;
  for (int m = 0; m < n; ++m) total += nb[m];
  while (total > cap) {
    int big = 0;
    for (int m = 1; m < n; ++m)
      if (nb[m] > nb[big]) big = m;
    --nb[big];
    --total;
  }
  std::vector<CoarseArgs<T>> args(n);
  std::vector<int> boff(n + 1, 0);
  double nodes = 0.0;
  for (int m = 0; m < n; ++m) {
    args[m] = coarse_args<T>(*lv[m], *w[m], rin + loff[m], xout + loff[m], tol, maxit);
    boff[m + 1] = boff[m] + nb[m];
    nodes += (double)lv[m]->n_global;
  }
  SE_TRY(dmalloc_bytes(allocs, &g->args, n * sizeof(CoarseArgs<T>)));
  SE_TRY(dmalloc(allocs, &g->boff, n + 1));
  SE_CUDA(cudaMemcpyAsync(g->args, args.data(), n * sizeof(CoarseArgs<T>), cudaMemcpyHostToDevice, s));
  SE_CUDA(cudaMemcpyAsync(g->boff, boff.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  SE_CUDA(cudaStreamSynchronize(s));
  g->n = n;
  g->nblocks = total;
  g->fp32 = sizeof(T) == 4;
  g->nodes = nodes;
  return SE_OK;
}

int coarse_group_setup(CoarseGroup* g, const Level* const* lv, CoarseWork* const* w, int n, bool fp32,
                       const void* rin, void* xout, const int64_t* loff, double tol, int maxit,
                       Allocs& allocs, cudaStream_t s) {
  SE_CHECK(n >= 1, SE_EINVAL, "grouped coarse solve: no problem");
  if (fp32)
    return coarse_group_setup_t<float>(g, lv, w, n, static_cast<const float*>(rin),
                                       static_cast<float*>(xout), loff, tol, maxit, allocs, s);
  return coarse_group_setup_t<double>(g, lv, w, n, static_cast<const double*>(rin),
                                      static_cast<double*>(xout), loff, tol, maxit, allocs, s);
}

template <class T>
int coarse_group_solve(const CoarseGroup& g, cudaStream_t s) {
  SE_CHECK(g.fp32 == (sizeof(T) == 4), SE_EINVAL, "grouped coarse solve: precision mismatch");
  ProfScope prof(SE_K_COARSE, s, g.nodes, 0.0, 0.0);
  const CoarseArgs<T>* args = static_cast<const CoarseArgs<T>*>(g.args);
  coarse_group_reset_kernel<<<(g.n + 127) / 128, 128, 0, s>>>(
      sizeof(T) == 8 ? reinterpret_cast<const CoarseArgs<double>*>(args) : nullptr,
      sizeof(T) == 4 ? reinterpret_cast<const CoarseArgs<float>*>(args) : nullptr, g.n);
  SE_LAUNCH_CHECK();
  const int* boff = g.boff;
  int n = g.n;
  void* a[] = {(void*)&args, (void*)&boff, (void*)&n};
  SE_TRY(coarse_kernel_attrs());
  SE_CUDA(cudaLaunchCooperativeKernel((const void*)coarse_group_kernel<T>, dim3(g.nblocks),
                                      dim3(CG_THREADS), a, COARSE_ROW_SMEM, s));
  return SE_OK;
}
template int coarse_group_solve<double>(const CoarseGroup&, cudaStream_t);
template int coarse_group_solve<float>(const CoarseGroup&, cudaStream_t);

int coarse_fault_take(CoarseWork& w, cudaStream_t s) {
  if (!w.totals) return SE_OK;
  unsigned long long f = 0;
  SE_CUDA(cudaStreamSynchronize(s));
  SE_CUDA(cudaMemcpy(&f, w.totals + 2, sizeof(f), cudaMemcpyDeviceToHost));
  if (f == 0) return SE_OK;
  SE_TRY(dzero(w.totals + 2, sizeof(f), s));
  set_error("coarse solve: %llu solve(s) gave up a bounded grid-synchronisation wait (results invalid)", f);
  return SE_ETIMEOUT;
}

template int coarse_solve<double>(const Level&, CoarseWork&, const double*, double*, double, int, cudaStream_t);
template int coarse_solve<float>(const Level&, CoarseWork&, const float*, float*, double, int, cudaStream_t);

// ------------------------------------------------------------------ self-test of the wait limit
__global__ void barrier_timeout_kernel(unsigned* count, int* status, double* part, long long timeout_ns) {
  // one more arrival is expected than blocks exist: the count never reaches its target
  __shared__ double red[3 * 32];
  double v[3] = {1.0, 0.0, 0.0}, pv = 0.0;
  grid_sum3(count, 0u, status, gridDim.x + 1, timeout_ns, part, v, pv, red,
            [](double (&)[3]) { return 0.0; }, blockIdx.x);
}

}  // namespace se

using namespace se;

extern "C" int se_selftest_wait_timeout(double timeout_ms) {
  SE_CHECK(timeout_ms > 0 && timeout_ms <= 5000, SE_EINVAL, "timeout_ms must be in (0, 5000]");
  unsigned* bar = nullptr;
  int* status = nullptr;
  double* part = nullptr;
  constexpr int NB = 4;
  SE_CUDA(cudaMalloc(&bar, 2 * sizeof(unsigned)));
  SE_CUDA(cudaMalloc(&status, 2 * sizeof(int)));
  SE_CUDA(cudaMalloc(&part, coarse_partial_doubles(NB + 1) * sizeof(double)));
  // everything of this self-test on the legacy default stream (0), in order
  SE_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), 0));
  SE_CUDA(cudaMemsetAsync(status, 0, 2 * sizeof(int), 0));
  barrier_timeout_kernel<<<NB, 32, 0, 0>>>(bar, status, part, (long long)(timeout_ms * 1e6));
  cudaError_t e = cudaDeviceSynchronize();
  int h[2] = {0, 0};
  cudaMemcpy(h, status, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(bar);
  cudaFree(status);
  cudaFree(part);
  SE_CHECK(e == cudaSuccess, SE_ECUDA, "selftest kernel failed: %s", cudaGetErrorString(e));
  if (h[0] == SE_ETIMEOUT) {
    set_error("device wait gave up after %.1f ms (expected in this self-test)", timeout_ms);
    return SE_ETIMEOUT;
  }
  set_error("device wait did not report a timeout");
  return SE_ECUDA;
}

// ------------------------------------------------------------------ coarse solve, no allocation
// Scratch of se_pmg_coarse_solve_noalloc: the nine pipelined-CG vectors (x, r, u, p, q, s, z and
// the two alternating w) of at most NOALLOC_MAX_N coarse nodes, the per-block partial sums
// (two buffers of 4 doubles per block), and four 32-bit words at the end (barrier count and an
// unused word, status, iteration count).  It lives in the library's static device memory: every
// GPU that loads the library holds it until the process exits.
namespace se {
constexpr int64_t NOALLOC_MAX_N = 1 << 17;        // 131072 coarse (p = 1) global nodes
constexpr int NOALLOC_MAX_BLOCKS = 1024;
constexpr int NOALLOC_VECTORS = 9;
// vectors, partial sums, barrier and status words, per-block flags
constexpr int64_t NOALLOC_WORDS =
    NOALLOC_VECTORS * NOALLOC_MAX_N + 8 * NOALLOC_MAX_BLOCKS + 2 + NOALLOC_MAX_BLOCKS / 2;
static __device__ __align__(256) double g_coarse_scratch[NOALLOC_WORDS];

// Host code must not use g_coarse_scratch itself (that name is a host-side stand-in): the
// device address is looked up on every call, with the caller's device current (cheap, and never
// stale after a device reset).
static int noalloc_scratch(double** out) {
  void* p = nullptr;
  SE_CUDA(cudaGetSymbolAddress(&p, g_coarse_scratch));
  *out = static_cast<double*>(p);
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
  double** vecs[NOALLOC_VECTORS] = {&w.x, &w.r, &w.u, &w.p, &w.q, &w.s, &w.z, &w.w0, &w.w1};
  for (int k = 0; k < NOALLOC_VECTORS; ++k) *vecs[k] = base + k * NOALLOC_MAX_N;
  w.partial = base + NOALLOC_VECTORS * NOALLOC_MAX_N;  // coarse_partial_doubles(nblocks) <= 8 * 1024
  w.bar = reinterpret_cast<unsigned*>(base + NOALLOC_VECTORS * NOALLOC_MAX_N + 8 * NOALLOC_MAX_BLOCKS);
  w.status = reinterpret_cast<int*>(w.bar + 2);
  w.flags = reinterpret_cast<unsigned*>(base + NOALLOC_VECTORS * NOALLOC_MAX_N + 8 * NOALLOC_MAX_BLOCKS + 2);
  // coarse_solve zeroes the barrier, status and flag words before its launch; the vectors are fully
  // written before they are read
  SE_TRY(coarse_solve<double>(c, w, r, x, P->desc.coarse_tol, P->desc.coarse_maxit, s));
  int h[2] = {0, 0};
  SE_CUDA(cudaMemcpyAsync(h, w.status, sizeof(h), cudaMemcpyDeviceToHost, s));
  SE_CUDA(cudaStreamSynchronize(s));
  if (iters) *iters = h[1];
  SE_CHECK(h[0] == 0, SE_ETIMEOUT, "coarse solve: a grid barrier wait ran out");
  return SE_OK;
}
