// Batched solves (se_batch_*): many independent Poisson problems in one device-driven launch.
//
// Problems whose preconditioners share a configuration (schedule, smoother, Chebyshev orders,
// bounds multipliers, coarse tolerance, precision) form a group.  A group is solved as ONE union
// problem: every level's elements of all members are laid end to end (geometry, point flags,
// neighbour ids shifted by the member's first element, FDM factors, Jacobi diagonals), QQ^T of
// each union level runs from a sorted index map over the members' global ids shifted apart, and
// so each phase of the method (operator, QQ^T, smoother, Chebyshev update, transfers) is one
// launch over all members' elements.  The members' Chebyshev bounds differ (lambda-tilde of
// Sec. 2.2.3 per member and level); each member's smoother is scaled by 1/lambda-tilde (its FDM
// eigenvalues multiplied by lambda-tilde, its Jacobi diagonal divided by it), which leaves the
// Chebyshev polynomial of Algorithm 2 unchanged and gives every member the bounds
// (eig_lo, eig_hi), so one recurrence serves the whole group.  What stays per member:
//  * the outer flexible PCG's scalars: inner products over each member's point range
//    (deterministic per-member reductions), its own alpha, beta, residual and convergence; a
//    member that has converged keeps its iterate while the others continue;
//  * the coarsest level: the members' Jacobi-PCG solves run together in one cooperative launch,
//    each on its own blocks to its own tolerance.
// The solve loop is a CUDA graph: WHILE any member is active, the iteration's launches run once
// for the whole group.  Problems that do not fit a group (no preconditioner, ASM smoother,
// additive cycle, df64 V-cycle) run their own graph branch, as se_solve with graph_capture.
// With graph_capture = 0 the same launches run with the loops driven from the host.
#include <cmath>
#include <map>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "pmg_internal.h"
#include "reduce.h"

namespace se {

// ------------------------------------------------------------------ per-member reductions
// Block map of the per-member kernels: member m owns blocks [sboff[m], sboff[m + 1]) of a 1D grid,
// each block a chunk of `chunk` consecutive points of the member's range [off[m], off[m + 1]), so
// blocks are spread over the members in proportion to their sizes.
enum { SG_RZ = 0, SG_PW, SG_ALPHA, SG_BETA, SG_RR, SG_R0, SG_SLOTS = 8 };

struct SegMap {
  const int64_t* off;   // [n + 1] point offsets
  const int* sboff;     // [n + 1] block offsets
  int n;
  int64_t chunk;
};

// member of block b: the largest m with sboff[m] <= b
__device__ __forceinline__ int seg_member(const SegMap& g, int b) {
  int lo = 0, hi = g.n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (g.sboff[mid] <= b) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Fused elementwise + reduction per member: per-block partial sums, summed in block order by the
// member's last block (deterministic).  Members whose active flag is 0 are skipped entirely.
// Op: K, struct V (one point's loads), setup(m) (the member's scalars), load(i), apply(i, v, acc),
// finalize(m, sums).  A thread takes its points U at a time with all their loads issued before
// the first store (a store could alias a later load); the order of its sums is unchanged.
template <class Op>
__global__ void __launch_bounds__(RED_THREADS) seg_fused_kernel(Op op_in, SegMap g, const int* __restrict__ active,
                                                                double* __restrict__ partial,
                                                                unsigned* __restrict__ counter) {
  constexpr int K = Op::K;
  constexpr int U = sizeof(typename Op::V) <= 24 ? 4 : 2;
  const int m = seg_member(g, blockIdx.x);
  if (active && !active[m]) return;  // uniform over the member's blocks
  const int b0 = g.sboff[m], nb = g.sboff[m + 1] - b0, local = blockIdx.x - b0;
  Op op = op_in;
  op.setup(m);
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  const int64_t beg = g.off[m] + (int64_t)local * g.chunk;
  const int64_t end = min(beg + g.chunk, g.off[m + 1]);
  int64_t i = beg + threadIdx.x;
  for (; i + (U - 1) * RED_THREADS < end; i += U * RED_THREADS) {
    typename Op::V v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = op.load(i + u * RED_THREADS);
#pragma unroll
    for (int u = 0; u < U; ++u) op.apply(i + u * RED_THREADS, v[u], acc);
  }
  for (; i < end; i += RED_THREADS) op.apply(i, op.load(i), acc);
  __shared__ double sh[K][RED_THREADS / 32];
  __shared__ bool last;
  block_sum<K>(acc, sh);
  double* part = partial + (int64_t)b0 * K;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) part[(int64_t)local * K + k] = acc[k];
    __threadfence();
    const unsigned t = atomicAdd(counter + m, 1u);
    last = (t == (unsigned)nb - 1u);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double w[K];
#pragma unroll
  for (int k = 0; k < K; ++k) w[k] = 0.0;
  for (int b = threadIdx.x; b < nb; b += RED_THREADS)
#pragma unroll
    for (int k = 0; k < K; ++k) w[k] += __ldcg(part + (int64_t)b * K + k);
  block_sum<K>(w, sh);
  if (threadIdx.x == 0) {
    op.finalize(m, w);
    counter[m] = 0u;
  }
}

struct SegInitOp {  // rz = (r, z), rr = (r, r), r0 = rr
  static constexpr int K = 2;
  const double* r;
  const double* z;
  const uint8_t* pf;
  double* scal;
  struct V { double r, z; uint8_t f; };
  __device__ void setup(int) {}
  __device__ V load(int64_t i) const { return {r[i], z[i], pf[i]}; }
  __device__ void apply(int64_t, const V& v, double (&acc)[2]) const {
    const double rw = scale_pow2(v.r, mult_log2(v.f));
    acc[0] = fma(rw, v.z, acc[0]);
    acc[1] = fma(rw, v.r, acc[1]);
  }
  __device__ void finalize(int m, const double* s) const {
    double* q = scal + m * SG_SLOTS;
    q[SG_RZ] = s[0];
    q[SG_RR] = s[1];
    q[SG_R0] = s[1];
  }
};

struct SegNormOp {  // r0 = (b, b): the reference of the ||b||-relative stopping rule
  static constexpr int K = 1;
  const double* b;
  const uint8_t* pf;
  double* scal;
  struct V { double b; uint8_t f; };
  __device__ void setup(int) {}
  __device__ V load(int64_t i) const { return {b[i], pf[i]}; }
  __device__ void apply(int64_t, const V& v, double (&acc)[1]) const {
    acc[0] = fma(scale_pow2(v.b, mult_log2(v.f)), v.b, acc[0]);
  }
  __device__ void finalize(int m, const double* s) const { scal[m * SG_SLOTS + SG_R0] = s[0]; }
};

struct SegAlphaOp {  // pw = (p, w); alpha = rz / pw
  static constexpr int K = 1;
  const double* p;
  const double* w;
  const uint8_t* pf;
  double* scal;
  struct V { double p, w; uint8_t f; };
  __device__ void setup(int) {}
  __device__ V load(int64_t i) const { return {p[i], w[i], pf[i]}; }
  __device__ void apply(int64_t, const V& v, double (&acc)[1]) const {
    acc[0] = fma(scale_pow2(v.p, mult_log2(v.f)), v.w, acc[0]);
  }
  __device__ void finalize(int m, const double* s) const {
    double* q = scal + m * SG_SLOTS;
    q[SG_PW] = s[0];
    q[SG_ALPHA] = q[SG_RZ] / s[0];
  }
};

struct SegUpdateOp {  // x += alpha p; r_old = r; r -= alpha w; rr = (r, r)
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
  __device__ void setup(int m) { alpha = scal[m * SG_SLOTS + SG_ALPHA]; }
  __device__ V load(int64_t i) const { return {x[i], p[i], r[i], w[i], pf[i]}; }
  __device__ void apply(int64_t i, const V& v, double (&acc)[1]) const {
    x[i] = fma(alpha, v.p, v.x);
    r_old[i] = v.r;
    const double rv = fma(-alpha, v.w, v.r);
    r[i] = rv;
    acc[0] = fma(scale_pow2(rv, mult_log2(v.f)), rv, acc[0]);
  }
  __device__ void finalize(int m, const double* s) const { scal[m * SG_SLOTS + SG_RR] = s[0]; }
};

struct SegBetaOp {  // zr = (z, r); zro = (z, r_old); beta = (zr - zro) / rz; rz = zr
  static constexpr int K = 2;
  const double* z;
  const double* r;
  const double* r_old;
  const uint8_t* pf;
  double* scal;
  struct V { double z, r, ro; uint8_t f; };
  __device__ void setup(int) {}
  __device__ V load(int64_t i) const { return {z[i], r[i], r_old[i], pf[i]}; }
  __device__ void apply(int64_t, const V& v, double (&acc)[2]) const {
    const double zw = scale_pow2(v.z, mult_log2(v.f));
    acc[0] = fma(zw, v.r, acc[0]);
    acc[1] = fma(zw, v.ro, acc[1]);
  }
  __device__ void finalize(int m, const double* s) const {
    double* q = scal + m * SG_SLOTS;
    q[SG_BETA] = (s[0] - s[1]) / q[SG_RZ];
    q[SG_RZ] = s[0];
  }
};

__global__ void __launch_bounds__(RED_THREADS) seg_pupdate_kernel(double* __restrict__ p,
                                                                  const double* __restrict__ z,
                                                                  const double* __restrict__ scal, SegMap g,
                                                                  const int* __restrict__ active) {
  const int m = seg_member(g, blockIdx.x);
  if (!active[m]) return;
  const double beta = scal[m * SG_SLOTS + SG_BETA];
  const int64_t beg = g.off[m] + (int64_t)(blockIdx.x - g.sboff[m]) * g.chunk;
  const int64_t end = min(beg + g.chunk, g.off[m + 1]);
  int64_t i = beg + threadIdx.x;
  for (; i + 3 * RED_THREADS < end; i += 4 * RED_THREADS) {
    double pv[4], zv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      pv[u] = p[i + u * RED_THREADS];
      zv[u] = z[i + u * RED_THREADS];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) p[i + u * RED_THREADS] = fma(beta, pv[u], zv[u]);
  }
  for (; i < end; i += RED_THREADS) p[i] = fma(beta, p[i], z[i]);
}

// Members' vectors to and from the union vector: piece m of u is member m's vector.
__global__ void __launch_bounds__(RED_THREADS) seg_gather_kernel(double* __restrict__ u,
                                                                 const double* const* __restrict__ src, SegMap g) {
  const int m = seg_member(g, blockIdx.x);
  const double* a = src[m] - g.off[m];
  const int64_t beg = g.off[m] + (int64_t)(blockIdx.x - g.sboff[m]) * g.chunk;
  const int64_t end = min(beg + g.chunk, g.off[m + 1]);
  for (int64_t i = beg + threadIdx.x; i < end; i += RED_THREADS) u[i] = a[i];
}
__global__ void __launch_bounds__(RED_THREADS) seg_scatter_kernel(const double* __restrict__ u,
                                                                  double* const* __restrict__ dst, SegMap g) {
  const int m = seg_member(g, blockIdx.x);
  double* a = dst[m] - g.off[m];
  const int64_t beg = g.off[m] + (int64_t)(blockIdx.x - g.sboff[m]) * g.chunk;
  const int64_t end = min(beg + g.chunk, g.off[m + 1]);
  for (int64_t i = beg + threadIdx.x; i < end; i += RED_THREADS) a[i] = u[i];
}

struct SegStats {
  int iterations;
  int active;
  double rel;
};

// After the first residual: every member's relative residual, active flag, and the loop's
// condition (some member above tolerance).
__global__ void seg_init_check_kernel(const double* __restrict__ scal, SegStats* st, int* active,
                                      int n, double tol, int maxit, bool graph,
                                      cudaGraphConditionalHandle hw, int* any_out) {
  int any = 0;
  for (int m = threadIdx.x; m < n; m += blockDim.x) {
    const double ref = scal[m * SG_SLOTS + SG_R0];
    const double rel = ref > 0.0 ? sqrt(scal[m * SG_SLOTS + SG_RR] / ref) : 0.0;
    const int on = (ref > 0.0 && rel > tol && maxit > 0) ? 1 : 0;
    st[m].iterations = 0;
    st[m].rel = rel;
    st[m].active = on;
    active[m] = on;
    any |= on;
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    *any_out = any;
    if (graph) cudaGraphSetConditional(hw, any ? 1u : 0u);
  }
}

// After each update: the active members count the iteration and test their residual; the loop
// (and the preconditioner of this iteration) continues while any member stays active.
__global__ void seg_check_kernel(const double* __restrict__ scal, SegStats* st, int* active, int n,
                                 double tol, int maxit, bool graph, cudaGraphConditionalHandle hw,
                                 cudaGraphConditionalHandle hif, int* any_out) {
  int any = 0;
  for (int m = threadIdx.x; m < n; m += blockDim.x) {
    if (!active[m]) continue;
    const int it = st[m].iterations + 1;
    st[m].iterations = it;
    const double rel = sqrt(scal[m * SG_SLOTS + SG_RR] / scal[m * SG_SLOTS + SG_R0]);
    st[m].rel = rel;
    const int on = (rel > tol && it < maxit) ? 1 : 0;  // a NaN residual stops the member too
    st[m].active = on;
    active[m] = on;
    any |= on;
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    *any_out = any;
    if (graph) {
      cudaGraphSetConditional(hw, any ? 1u : 0u);
      cudaGraphSetConditional(hif, any ? 1u : 0u);
    }
  }
}

// Copy with a scale per member (piece m of dst = scale[m] x piece m of src).
template <class T>
__global__ void scaled_copy_kernel(T* __restrict__ dst, const T* __restrict__ src, int64_t n, double scale) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (T)((double)src[i] * scale);
}
__global__ void shifted_ids_kernel(int* __restrict__ dst, const int* __restrict__ src, int64_t n, int shift) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i] >= 0 ? src[i] + shift : -1;
}

// ------------------------------------------------------------------ one group
struct BatchGroup {
  std::vector<int> idx;        // the members' problem indices
  int n = 0;
  se_pmg_s* U = nullptr;       // union preconditioner: union levels, vectors, grouped coarse solve
  Level fine;                  // union level 0 as the outer operator uses it (FP64)
  std::vector<int64_t> hoff;   // level-0 point offsets of the members [n + 1]
  int64_t* off = nullptr;      // device copy
  double *b = nullptr, *x = nullptr, *r = nullptr, *r_old = nullptr, *z = nullptr, *p = nullptr,
         *w = nullptr;
  const double** bsrc = nullptr;  // device table of the members' b
  double** xdst = nullptr;        // device table of the members' x
  double* scal = nullptr;         // [n][SG_SLOTS]
  int* active = nullptr;          // [n]
  SegStats* stats = nullptr;      // [n]
  int* any = nullptr;             // [1]: some member still active (host-driven loop)
  int* hany = nullptr;            // pinned host mirror
  int* sboff = nullptr;           // [n + 1] block offsets of the per-member kernels
  int sblocks = 0;                // their grid
  int64_t chunk = 0;              // points per block
  double* partial = nullptr;      // [sblocks][2]
  unsigned* counter = nullptr;    // [n]
  CoarseGroup cg;
};

static SegMap seg_map(const BatchGroup& G) { return SegMap{G.off, G.sboff, G.n, G.chunk}; }

template <class Op>
static int run_seg(const BatchGroup& G, const Op& op, bool skip_inactive, cudaStream_t s, double bytes) {
  ProfScope prof(SE_K_KRYLOV, s, (double)G.fine.L, bytes, 2.0 * G.fine.L);
  seg_fused_kernel<Op><<<G.sblocks, RED_THREADS, 0, s>>>(op, seg_map(G), skip_inactive ? G.active : nullptr,
                                                         G.partial, G.counter);
  SE_LAUNCH_CHECK();
  return SE_OK;
}

// The union of the members' levels l (see the file comment).  lam_scale[m]: member m's smoother
// scale 1/lambda-tilde on this level (1 on the coarsest).
static int build_union_level(se_pmg_s* U, int l, const std::vector<se_pmg_s*>& Pm, bool fp32,
                             int smoother, cudaStream_t s) {
  const int n = (int)Pm.size();
  const bool coarsest = l == U->nlev - 1;
  const Level& a0 = *Pm[0]->lv[l];
  Level& u = U->owned[l];
  u = Level();
  u.p = a0.p;
  u.N = a0.N;
  u.basis = a0.basis;
  u.D64 = a0.D64;   // derivative tables depend on p only: shared with member 0
  u.D32 = a0.D32;
  u.eo64 = a0.eo64;
  for (int f = 0; f < 6; ++f) u.bc[f] = a0.bc[f];
  for (const se_pmg_s* P : Pm) {
    u.E += P->lv[l]->E;
    u.L += P->lv[l]->L;
    u.n_global += P->lv[l]->n_global;
  }
  SE_CHECK(u.L < ((int64_t)1 << 31), SE_EINVAL, "se_batch: a group's level %d has %lld points (limit 2^31)",
           l, (long long)u.L);
  Allocs& A = U->allocs;
  const int N3 = u.N * u.N * u.N, PB = u.p + 3;
  const bool want64 = l == 0 || (!fp32 && !coarsest);
  const bool want32 = fp32 && !coarsest;
  SE_TRY(dmalloc(A, &u.pflag, (size_t)u.L));
  SE_TRY(dmalloc(A, &u.pstatus, 1));
  SE_TRY(dzero(u.pstatus, sizeof(int), s));
  if (want64) SE_TRY(dmalloc(A, &u.G64, 6 * (size_t)u.L));
  if (want32) SE_TRY(dmalloc(A, &u.G32, 6 * (size_t)u.L));
  const bool ras = smoother == SE_SMOOTH_RAS && !coarsest;
  const bool jac = smoother == SE_SMOOTH_JACOBI && !coarsest;
  if (jac && !fp32) SE_TRY(dmalloc(A, &u.dinv64, (size_t)u.L));
  if (jac && fp32) SE_TRY(dmalloc(A, &u.dinv32, (size_t)u.L));
  int* nbr = nullptr;
  if (ras) {
    SE_TRY(dmalloc(A, &nbr, 27 * (size_t)u.E));
    u.nbr = nbr;
    if (fp32) {
      SE_TRY(dmalloc(A, &u.S32, 3 * (size_t)u.E * PB * PB));
      SE_TRY(dmalloc(A, &u.lam32, 3 * (size_t)u.E * PB));
    } else {
      SE_TRY(dmalloc(A, &u.S64, 3 * (size_t)u.E * PB * PB));
      SE_TRY(dmalloc(A, &u.lam64, 3 * (size_t)u.E * PB));
      SE_TRY(dmalloc(A, &u.fdm_dinv64, (size_t)u.E * PB * PB * PB));
    }
  }
  std::vector<int64_t> gid((size_t)u.L);
  std::vector<uint8_t> dir((size_t)u.L);
  int64_t eo = 0, lo = 0, go = 0;
  int* l2g = nullptr;
  int64_t maxL = 0;
  for (const se_pmg_s* P : Pm) maxL = std::max(maxL, P->lv[l]->L);
  SE_TRY(dmalloc_transient(reinterpret_cast<void**>(&l2g), (size_t)maxL * sizeof(int), s));
  std::vector<int> g32((size_t)maxL);
  std::vector<uint8_t> pf((size_t)maxL);
  int rc = SE_OK;
  for (int m = 0; m < n && rc == SE_OK; ++m) {
    const Level& a = *Pm[m]->lv[l];
    const double inv_lam = coarsest ? 1.0 : 1.0 / Pm[m]->lam[l];
    auto cp = [&](void* dst, const void* src, size_t bytes) {
      if (rc == SE_OK && cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
        set_error("se_batch: copy failed");
        rc = SE_ECUDA;
      }
    };
    cp(u.pflag + lo, a.pflag, (size_t)a.L);
    for (int c = 0; c < 6; ++c) {
      if (want64) cp(u.G64 + c * u.L + lo, a.G64 + c * a.L, (size_t)a.L * sizeof(double));
      if (want32) cp(u.G32 + c * u.L + lo, a.G32 + c * a.L, (size_t)a.L * sizeof(float));
    }
    if (jac && !fp32)
      scaled_copy_kernel<double><<<grid_for(a.L, 256), 256, 0, s>>>(u.dinv64 + lo, a.dinv64, a.L, inv_lam);
    if (jac && fp32)
      scaled_copy_kernel<float><<<grid_for(a.L, 256), 256, 0, s>>>(u.dinv32 + lo, a.dinv32, a.L, inv_lam);
    if (ras) {
      shifted_ids_kernel<<<grid_for(27 * a.E, 256), 256, 0, s>>>(nbr + 27 * eo, a.nbr, 27 * a.E, (int)eo);
      const int64_t ns = 3 * a.E * PB * PB, nl = 3 * a.E * PB;
      if (fp32) {
        cp(u.S32 + 3 * eo * PB * PB, a.S32, (size_t)ns * sizeof(float));
        scaled_copy_kernel<float><<<grid_for(nl, 256), 256, 0, s>>>(u.lam32 + 3 * eo * PB, a.lam32, nl,
                                                                   1.0 / inv_lam);
      } else {
        cp(u.S64 + 3 * eo * PB * PB, a.S64, (size_t)ns * sizeof(double));
        scaled_copy_kernel<double><<<grid_for(nl, 256), 256, 0, s>>>(u.lam64 + 3 * eo * PB, a.lam64, nl,
                                                                    1.0 / inv_lam);
        const int64_t nd = a.E * PB * PB * PB;
        scaled_copy_kernel<double><<<grid_for(nd, 256), 256, 0, s>>>(u.fdm_dinv64 + eo * PB * PB * PB,
                                                                    a.fdm_dinv64, nd, inv_lam);
      }
    }
    if (cudaGetLastError() != cudaSuccess && rc == SE_OK) {
      set_error("se_batch: union level kernel launch failed");
      rc = SE_ECUDA;
    }
    // global ids of the member's lattice, shifted past the previous members'
    if (rc == SE_OK) rc = local_to_global(a, l2g, s);
    if (rc == SE_OK &&
        (cudaMemcpyAsync(g32.data(), l2g, (size_t)a.L * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
         cudaMemcpyAsync(pf.data(), a.pflag, (size_t)a.L, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
         cudaStreamSynchronize(s) != cudaSuccess)) {
      set_error("se_batch: %s", cudaGetErrorString(cudaGetLastError()));
      rc = SE_ECUDA;
    }
    for (int64_t q = 0; q < a.L && rc == SE_OK; ++q) {
      gid[(size_t)(lo + q)] = go + g32[(size_t)q];
      dir[(size_t)(lo + q)] = (pf[(size_t)q] & PF_FREE) ? 0 : 1;
    }
    eo += a.E;
    lo += a.L;
    go += a.n_global;
    (void)N3;
  }
  cudaFreeAsync(l2g, s);
  SE_TRY(rc);
  SE_TRY(build_gsmap_from_gid(u, gid.data(), dir.data(), A, s));
  U->lv[l] = &U->owned[l];
  return SE_OK;
}

static void destroy_group(BatchGroup* G) {
  if (!G) return;
  if (G->hany) cudaFreeHost(G->hany);
  if (G->U) {
    cudaStreamSynchronize(G->U->stream);
    G->U->allocs.release();
    pinned_release(G->U->scratch.hscal);
    cudaStream_t st = G->U->stream;
    delete G->U;
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  delete G;
}

static int build_group(BatchGroup* G, const std::vector<se_problem>& probs, int op_df) {
  const int n = G->n = (int)G->idx.size();
  std::vector<se_pmg_s*> Pm(n);
  for (int m = 0; m < n; ++m) Pm[m] = probs[G->idx[m]].pmg;
  const se_pmg_desc& d = Pm[0]->desc;
  const bool fp32 = d.precision == SE_FP32;
  auto* U = new se_pmg_s();
  G->U = U;
  SE_CUDA(cudaStreamCreateWithFlags(&U->stream, cudaStreamNonBlocking));
  cudaStream_t s = U->stream;
  U->allocs.stream = s;
  U->desc = d;
  U->nlev = d.nlev;
  for (int m = 0; m < n; ++m)  // the members' set-up work must be complete
    SE_CUDA(cudaStreamSynchronize(Pm[m]->stream));
  SE_TRY(scratch_alloc(U->allocs, &U->scratch));
  for (int l = 0; l < U->nlev; ++l) {
    SE_TRY(build_union_level(U, l, Pm, fp32, d.smoother, s));
    U->lam[l] = 1.0;
    U->lmin[l] = d.eig_lo;
    U->lmax[l] = d.eig_hi;
    if (l + 1 < U->nlev) {
      U->J64[l] = Pm[0]->J64[l];  // interpolation matrices depend on the orders only
      U->J32[l] = Pm[0]->J32[l];
    }
    SE_TRY(pmg_alloc_vecs(U, l, fp32));
  }
  // coarse problems: the members' own coarse operators and work spaces, on the union vectors
  const int lc = U->nlev - 1;
  std::vector<const Level*> clv(n);
  std::vector<CoarseWork*> cwk(n);
  std::vector<int64_t> coff(n + 1, 0);
  for (int m = 0; m < n; ++m) {
    clv[m] = Pm[m]->lv[lc];
    cwk[m] = &Pm[m]->cw;
    coff[m + 1] = coff[m] + Pm[m]->lv[lc]->L;
  }
  const void* rin = fp32 ? (const void*)U->v32[lc].b : (const void*)U->v64[lc].b;
  void* xout = fp32 ? (void*)U->v32[lc].x : (void*)U->v64[lc].x;
  SE_TRY(coarse_group_setup(&G->cg, clv.data(), cwk.data(), n, fp32, rin, xout, coff.data(),
                            d.coarse_tol, d.coarse_maxit, U->allocs, s));
  U->cgroup = &G->cg;
  // outer solver state: level 0 in FP64, or in double-float arithmetic (operator_df64; the df64
  // geometry is made for the outer operator only, the V-cycle keeps its own arithmetic)
  if (op_df) SE_TRY(make_df_geometry(U->owned[0], U->allocs, s));
  G->fine = U->owned[0];
  G->fine.df = op_df != 0;
  const int64_t L = G->fine.L;
  Allocs& A = U->allocs;
  for (double** v : {&G->b, &G->x, &G->r, &G->r_old, &G->z, &G->p, &G->w}) SE_TRY(dmalloc(A, v, (size_t)L));
  G->hoff.assign(n + 1, 0);
  std::vector<const double*> bs(n);
  std::vector<double*> xs(n);
  for (int m = 0; m < n; ++m) {
    G->hoff[m + 1] = G->hoff[m] + Pm[m]->lv[0]->L;
    bs[m] = probs[G->idx[m]].b;
    xs[m] = probs[G->idx[m]].x;
  }
  SE_TRY(dmalloc(A, &G->off, (size_t)n + 1));
  SE_TRY(dmalloc(A, &G->bsrc, (size_t)n));
  SE_TRY(dmalloc(A, &G->xdst, (size_t)n));
  SE_TRY(dmalloc(A, &G->scal, (size_t)n * SG_SLOTS));
  SE_TRY(dmalloc(A, &G->active, (size_t)n));
  SE_TRY(dmalloc_bytes(A, reinterpret_cast<void**>(&G->stats), (size_t)n * sizeof(SegStats)));
  {  // block map: about 8 blocks per SM over the whole union, chunks of whole warps
    int dev = 0, sms = 0;
    SE_CUDA(cudaGetDevice(&dev));
    SE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t target = 8 * (int64_t)sms;
    int64_t chunk = (L + target - 1) / target;
    chunk = std::max<int64_t>(4 * RED_THREADS, (chunk + RED_THREADS - 1) / RED_THREADS * RED_THREADS);
    std::vector<int> sb(n + 1, 0);
    for (int m = 0; m < n; ++m) sb[m + 1] = sb[m] + (int)((G->hoff[m + 1] - G->hoff[m] + chunk - 1) / chunk);
    G->chunk = chunk;
    G->sblocks = sb[n];
    SE_TRY(dmalloc(A, &G->sboff, (size_t)n + 1));
    SE_CUDA(cudaMemcpyAsync(G->sboff, sb.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  }
  SE_TRY(dmalloc(A, &G->partial, (size_t)G->sblocks * 2));
  SE_TRY(dmalloc(A, &G->counter, (size_t)n));
  SE_TRY(dmalloc(A, &G->any, 1));
  SE_CUDA(cudaMallocHost(&G->hany, sizeof(int)));
  SE_CUDA(cudaMemcpyAsync(G->off, G->hoff.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  SE_CUDA(cudaMemcpyAsync(G->bsrc, bs.data(), n * sizeof(double*), cudaMemcpyHostToDevice, s));
  SE_CUDA(cudaMemcpyAsync(G->xdst, xs.data(), n * sizeof(double*), cudaMemcpyHostToDevice, s));
  SE_CUDA(cudaMemsetAsync(G->counter, 0, n * sizeof(unsigned), s));
  SE_CUDA(cudaMemsetAsync(G->scal, 0, n * SG_SLOTS * sizeof(double), s));
  SE_CUDA(cudaMemsetAsync(G->stats, 0, n * sizeof(SegStats), s));
  SE_CUDA(cudaStreamSynchronize(s));
  return SE_OK;
}

// The group's whole solve as one branch of G (x0 = the members' x at launch).
static int append_group_solve(cudaGraph_t Gr, cudaStream_t cs, BatchGroup* G, double tol, int maxit,
                              int tol_norm) {
  const Level& lv = G->fine;
  const int64_t L = lv.L;
  cudaGraphConditionalHandle hw, hif;
  SE_CUDA(cudaGraphConditionalHandleCreate(&hw, Gr, 0, 0));
  SE_CUDA(cudaStreamBeginCaptureToGraph(cs, Gr, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  int rc = SE_OK;
  cudaGraph_t wbody = nullptr, ifbody = nullptr;
  do {
    seg_gather_kernel<<<G->sblocks, RED_THREADS, 0, cs>>>(G->b, G->bsrc, seg_map(*G));
    seg_gather_kernel<<<G->sblocks, RED_THREADS, 0, cs>>>(G->x, const_cast<const double* const*>(G->xdst),
                                                          seg_map(*G));
    if ((rc = ax_apply<double>(lv, G->x, G->w, cs)) != SE_OK) break;
    if ((rc = axpby<double>(1.0, G->b, -1.0, G->w, G->r, L, cs)) != SE_OK) break;  // r = b - A x
    if ((rc = pmg_apply(G->U, G->r, G->z, cs)) != SE_OK) break;                    // z = M r
    if ((rc = run_seg(*G, SegInitOp{G->r, G->z, lv.pflag, G->scal}, false, cs, 17.0 * L)) != SE_OK) break;
    if (tol_norm == SE_TOL_B &&
        (rc = run_seg(*G, SegNormOp{G->b, lv.pflag, G->scal}, false, cs, 9.0 * L)) != SE_OK)
      break;
    if (cudaMemcpyAsync(G->p, G->z, L * sizeof(double), cudaMemcpyDeviceToDevice, cs) != cudaSuccess) {
      set_error("se_batch: copy capture failed");
      rc = SE_ECUDA;
      break;
    }
    seg_init_check_kernel<<<1, 256, 0, cs>>>(G->scal, G->stats, G->active, G->n, tol, maxit, true, hw,
                                             G->any);
    if ((rc = add_conditional(cs, hw, cudaGraphCondTypeWhile, &wbody)) != SE_OK) break;
    seg_scatter_kernel<<<G->sblocks, RED_THREADS, 0, cs>>>(G->x, G->xdst, seg_map(*G));  // after the loop
  } while (0);
  cudaGraph_t out = nullptr;
  cudaError_t ec = cudaStreamEndCapture(cs, &out);
  if (rc != SE_OK) return rc;
  SE_CHECK(ec == cudaSuccess, SE_ECUDA, "se_batch graph (init): %s", cudaGetErrorString(ec));
  // WHILE body: w = A p, per-member alpha, x / r update, convergence test
  SE_CUDA(cudaGraphConditionalHandleCreate(&hif, Gr, 0, 0));
  SE_CUDA(cudaStreamBeginCaptureToGraph(cs, wbody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  do {
    if ((rc = ax_apply<double>(lv, G->p, G->w, cs)) != SE_OK) break;
    if ((rc = run_seg(*G, SegAlphaOp{G->p, G->w, lv.pflag, G->scal}, true, cs, 17.0 * L)) != SE_OK) break;
    if ((rc = run_seg(*G, SegUpdateOp{G->x, G->p, G->r, G->w, G->r_old, lv.pflag, G->scal}, true, cs,
                      57.0 * L)) != SE_OK)
      break;
    seg_check_kernel<<<1, 256, 0, cs>>>(G->scal, G->stats, G->active, G->n, tol, maxit, true, hw, hif,
                                        G->any);
    rc = add_conditional(cs, hif, cudaGraphCondTypeIf, &ifbody);
  } while (0);
  ec = cudaStreamEndCapture(cs, &out);
  if (rc != SE_OK) return rc;
  SE_CHECK(ec == cudaSuccess, SE_ECUDA, "se_batch graph (loop): %s", cudaGetErrorString(ec));
  // IF body: z = M r for the union, per-member beta, p = z + beta p
  SE_CUDA(cudaStreamBeginCaptureToGraph(cs, ifbody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  do {
    if ((rc = pmg_apply(G->U, G->r, G->z, cs)) != SE_OK) break;
    if ((rc = run_seg(*G, SegBetaOp{G->z, G->r, G->r_old, lv.pflag, G->scal}, true, cs, 25.0 * L)) != SE_OK)
      break;
    {
      ProfScope prof(SE_K_KRYLOV, cs, (double)L, 24.0 * L, 2.0 * L);
      seg_pupdate_kernel<<<G->sblocks, RED_THREADS, 0, cs>>>(G->p, G->z, G->scal, seg_map(*G), G->active);
      if (cudaGetLastError() != cudaSuccess) {
        set_error("se_batch: launch failed");
        rc = SE_ECUDA;
      }
    }
  } while (0);
  ec = cudaStreamEndCapture(cs, &out);
  if (rc != SE_OK) return rc;
  SE_CHECK(ec == cudaSuccess, SE_ECUDA, "se_batch graph (preconditioner): %s", cudaGetErrorString(ec));
  return SE_OK;
}

// The same solve with the loop driven from the host (one read of the "any member active" flag per
// iteration): the launches of the graph, each one visible to the library's event profiler.
static int run_group_host(BatchGroup* G, double tol, int maxit, int tol_norm, cudaStream_t s) {
  const Level& lv = G->fine;
  const int64_t L = lv.L;
  cudaGraphConditionalHandle none{};
  auto any_left = [&](int* out) {
    if (cudaMemcpyAsync(G->hany, G->any, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      set_error("se_batch: %s", cudaGetErrorString(cudaGetLastError()));
      return SE_ECUDA;
    }
    *out = *G->hany;
    return SE_OK;
  };
  seg_gather_kernel<<<G->sblocks, RED_THREADS, 0, s>>>(G->b, G->bsrc, seg_map(*G));
  seg_gather_kernel<<<G->sblocks, RED_THREADS, 0, s>>>(G->x, const_cast<const double* const*>(G->xdst),
                                                       seg_map(*G));
  SE_LAUNCH_CHECK();
  SE_TRY(ax_apply<double>(lv, G->x, G->w, s));
  SE_TRY(axpby<double>(1.0, G->b, -1.0, G->w, G->r, L, s));
  SE_TRY(pmg_apply(G->U, G->r, G->z, s));
  SE_TRY(run_seg(*G, SegInitOp{G->r, G->z, lv.pflag, G->scal}, false, s, 17.0 * L));
  if (tol_norm == SE_TOL_B) SE_TRY(run_seg(*G, SegNormOp{G->b, lv.pflag, G->scal}, false, s, 9.0 * L));
  SE_CUDA(cudaMemcpyAsync(G->p, G->z, L * sizeof(double), cudaMemcpyDeviceToDevice, s));
  seg_init_check_kernel<<<1, 256, 0, s>>>(G->scal, G->stats, G->active, G->n, tol, maxit, false, none,
                                          G->any);
  SE_LAUNCH_CHECK();
  int go = 0;
  SE_TRY(any_left(&go));
  while (go) {
    SE_TRY(ax_apply<double>(lv, G->p, G->w, s));
    SE_TRY(run_seg(*G, SegAlphaOp{G->p, G->w, lv.pflag, G->scal}, true, s, 17.0 * L));
    SE_TRY(run_seg(*G, SegUpdateOp{G->x, G->p, G->r, G->w, G->r_old, lv.pflag, G->scal}, true, s, 57.0 * L));
    seg_check_kernel<<<1, 256, 0, s>>>(G->scal, G->stats, G->active, G->n, tol, maxit, false, none, none,
                                       G->any);
    SE_LAUNCH_CHECK();
    SE_TRY(any_left(&go));
    if (!go) break;
    SE_TRY(pmg_apply(G->U, G->r, G->z, s));
    SE_TRY(run_seg(*G, SegBetaOp{G->z, G->r, G->r_old, lv.pflag, G->scal}, true, s, 25.0 * L));
    {
      ProfScope prof(SE_K_KRYLOV, s, (double)L, 24.0 * L, 2.0 * L);
      seg_pupdate_kernel<<<G->sblocks, RED_THREADS, 0, s>>>(G->p, G->z, G->scal, seg_map(*G), G->active);
      SE_LAUNCH_CHECK();
    }
  }
  seg_scatter_kernel<<<G->sblocks, RED_THREADS, 0, s>>>(G->x, G->xdst, seg_map(*G));
  SE_LAUNCH_CHECK();
  return SE_OK;
}

// Problems that share a group: same preconditioner configuration, one of the supported kinds.
static bool groupable(const se_problem& q, const se_solve_opts&) {
  if (!q.pmg) return false;
  const se_pmg_desc& d = q.pmg->desc;
  return (d.precision == SE_FP64 || d.precision == SE_FP32) && d.cycle == SE_CYCLE_MULTIPLICATIVE &&
         (d.smoother == SE_SMOOTH_RAS || d.smoother == SE_SMOOTH_JACOBI);
}

// Size class of a problem of E elements: 0 below 4096 elements, then one class per factor 8.
// Problems of one configuration but different classes are solved as different groups: within a
// group every phase is one launch over all members and the grouped coarse solve lasts until its
// slowest member has converged, while different groups are independent branches of the graph,
// so small problems do not wait for large ones (the 64-problem batch of E in {8^3..24^3}: 291 ms
// as 4 groups, 277 ms as 8; splits into more or smaller groups measured no better).
static int size_class(int64_t E) {
  int c = 0;
  for (int64_t t = 4096; E >= t && c < 20; t *= 8) ++c;
  return c;
}

static std::string group_key(const se_pmg_desc& d) {
  std::string k = std::to_string(d.nlev) + ":" + std::to_string(d.smoother) + ":" +
                  std::to_string(d.precision) + ":";
  for (int l = 0; l < d.nlev; ++l) k += std::to_string(d.schedule[l]) + ",";
  k += ":";
  for (int l = 0; l + 1 < d.nlev; ++l) k += std::to_string(d.cheb_order[l]) + ",";
  char buf[96];
  snprintf(buf, sizeof(buf), ":%.17g:%.17g:%.17g:%d", d.eig_lo, d.eig_hi, d.coarse_tol, d.coarse_maxit);
  return k + buf;
}

}  // namespace se

using namespace se;

struct se_batch_s {
  std::vector<se_problem> probs;
  se_solve_opts opts;
  cudaGraphExec_t exec = nullptr;
  std::vector<BatchGroup*> groups;
  std::vector<int> alone;          // problems with their own graph branch
  std::vector<int> group_of, slot;  // per problem: group index (-1: alone) and member slot
  bool host = false;                // graph_capture == 0: loops driven from the host
  std::vector<se_solve_stats> alone_stats;
};

static void batch_free(se_batch_s* B) {
  if (!B) return;
  if (B->exec) cudaGraphExecDestroy(B->exec);
  for (BatchGroup* G : B->groups) destroy_group(G);
  delete B;
}

extern "C" {

int se_batch_create(int n, const se_problem* probs, const se_solve_opts* opts, se_batch_t* out) {
  SE_CHECK(n >= 1 && probs && opts && out, SE_EINVAL, "se_batch_create: bad argument");
  SE_CHECK(opts->method == SE_FPCG, SE_EINVAL, "se_batch_create: batched solves use SE_FPCG");
  SE_CHECK(opts->tol > 0 && opts->maxit >= 1, SE_EINVAL, "se_batch_create: bad tolerance or maxit");
  SE_CHECK(opts->tol_norm == SE_TOL_R0 || opts->tol_norm == SE_TOL_B, SE_EINVAL,
           "se_batch_create: bad tol_norm");
  for (int i = 0; i < n; ++i) {
    SE_CHECK(probs[i].mesh && probs[i].b && probs[i].x, SE_EINVAL, "se_batch_create: problem %d incomplete", i);
    SE_CHECK(!probs[i].pmg || probs[i].pmg->mesh == probs[i].mesh, SE_EINVAL,
             "se_batch_create: problem %d: preconditioner of another mesh", i);
    for (int j = 0; j < i; ++j) {
      SE_CHECK(probs[j].mesh != probs[i].mesh, SE_EINVAL,
               "se_batch_create: problems %d and %d share a mesh (its work space)", j, i);
      SE_CHECK(!probs[i].pmg || probs[j].pmg != probs[i].pmg, SE_EINVAL,
               "se_batch_create: problems %d and %d share a preconditioner", j, i);
    }
  }
  auto* B = new se_batch_s();
  B->probs.assign(probs, probs + n);
  B->opts = *opts;
  B->group_of.assign(n, -1);
  B->slot.assign(n, -1);
  std::map<std::string, int> keys;
  std::vector<std::vector<int>> members;
  for (int i = 0; i < n; ++i) {
    if (!groupable(probs[i], *opts)) {
      B->alone.push_back(i);
      continue;
    }
    const std::string k = group_key(probs[i].pmg->desc) + ":" + std::to_string(size_class(probs[i].mesh->fine.E));
    auto it = keys.find(k);
    if (it == keys.end()) {
      it = keys.emplace(k, (int)members.size()).first;
      members.emplace_back();
    }
    B->group_of[i] = it->second;
    B->slot[i] = (int)members[it->second].size();
    members[it->second].push_back(i);
  }
  int rc = SE_OK;
  for (size_t g = 0; g < members.size() && rc == SE_OK; ++g) {
    auto* G = new BatchGroup();
    G->idx = members[g];
    B->groups.push_back(G);
    rc = build_group(G, B->probs, opts->operator_df64);
  }
  for (int i : B->alone) {
    if (rc != SE_OK) break;
    rc = prepare_graph_solve(probs[i].mesh);
    if (rc == SE_OK && opts->operator_df64)
      rc = make_df_geometry(probs[i].mesh->fine, probs[i].mesh->allocs, probs[i].mesh->stream);
  }
  B->host = opts->graph_capture == 0;
  B->alone_stats.assign(n, se_solve_stats{});
  if (B->host) {
    if (rc != SE_OK) {
      batch_free(B);
      return rc;
    }
    *out = B;
    return SE_OK;
  }
  cudaGraph_t Gr = nullptr;
  if (rc == SE_OK && cudaGraphCreate(&Gr, 0) != cudaSuccess) {
    set_error("cudaGraphCreate failed");
    rc = SE_ECUDA;
  }
  cudaStream_t cs = nullptr;
  if (rc == SE_OK && cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    set_error("se_batch_create: stream creation failed");
    rc = SE_ECUDA;
  }
  for (BatchGroup* G : B->groups) {
    if (rc != SE_OK) break;
    rc = append_group_solve(Gr, cs, G, opts->tol, opts->maxit, opts->tol_norm);
  }
  for (int i : B->alone) {
    if (rc != SE_OK) break;
    rc = append_fpcg_solve(Gr, cs, probs[i].mesh, probs[i].pmg, probs[i].b, probs[i].x, opts->tol,
                           opts->maxit, opts->tol_norm, opts->operator_df64);
  }
  if (cs) cudaStreamDestroy(cs);
  if (rc == SE_OK && cudaGraphInstantiate(&B->exec, Gr, 0) != cudaSuccess) {
    set_error("se_batch_create: cudaGraphInstantiate: %s", cudaGetErrorString(cudaGetLastError()));
    rc = SE_ECUDA;
    B->exec = nullptr;
  }
  if (Gr) cudaGraphDestroy(Gr);
  if (rc != SE_OK) {
    batch_free(B);
    return rc;
  }
  *out = B;
  return SE_OK;
}

int se_batch_run(se_batch_t B, void* stream) {
  SE_CHECK(B, SE_EINVAL, "se_batch_run: null batch");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!B->host) {
    SE_CUDA(cudaGraphLaunch(B->exec, s));
    return SE_OK;
  }
  for (BatchGroup* G : B->groups)
    SE_TRY(run_group_host(G, B->opts.tol, B->opts.maxit, B->opts.tol_norm, s));
  for (int i : B->alone) {  // their own host-driven solve loops
    se_solve_opts o = B->opts;
    o.graph_capture = 0;
    o.stream = s;
    const int rc = se_solve(B->probs[i].mesh, B->probs[i].pmg, B->probs[i].b, B->probs[i].x, &o,
                            &B->alone_stats[i]);
    if (rc != SE_OK && rc != SE_ENOTCONV) return rc;
  }
  return SE_OK;
}

int se_batch_stats(se_batch_t B, void* stream, se_solve_stats* out) {
  SE_CHECK(B && out, SE_EINVAL, "se_batch_stats: null argument");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  SE_CUDA(cudaStreamSynchronize(s));
  int worst = SE_OK;
  std::vector<std::vector<SegStats>> gs(B->groups.size());
  for (size_t g = 0; g < B->groups.size(); ++g) {
    gs[g].resize(B->groups[g]->n);
    SE_CUDA(cudaMemcpy(gs[g].data(), B->groups[g]->stats, gs[g].size() * sizeof(SegStats),
                       cudaMemcpyDeviceToHost));
  }
  const double tol = B->opts.tol;
  for (size_t i = 0; i < B->probs.size(); ++i) {
    se_solve_stats st{};
    int rc = SE_OK;
    if (B->group_of[i] >= 0) {
      const SegStats& q = gs[B->group_of[i]][B->slot[i]];
      st.iterations = q.iterations;
      st.rel_residual = q.rel;
      if (std::isnan(q.rel)) {
        set_error("se_batch: problem %zu: residual became NaN", i);
        rc = SE_ENOTCONV;
      } else if (q.rel > tol) {
        set_error("se_batch: problem %zu: no convergence in %d iterations (rel. residual %.3e)", i,
                  B->opts.maxit, q.rel);
        rc = SE_ENOTCONV;
      }
    } else if (B->host) {
      st = B->alone_stats[i];
      rc = st.status;
    } else {
      rc = read_graph_stats(B->probs[i].mesh, s, &st, tol, B->opts.maxit);
    }
    st.status = rc;
    out[i] = st;
    if (rc != SE_OK) worst = rc;
  }
  // bounded device waits: a group's union levels count against all its members
  std::vector<bool> group_fault(B->groups.size(), false);
  for (size_t g = 0; g < B->groups.size(); ++g)
    group_fault[g] = pmg_faults_take(B->groups[g]->U, s) != SE_OK;
  for (size_t i = 0; i < B->probs.size(); ++i) {
    bool f = B->group_of[i] >= 0 && group_fault[B->group_of[i]];
    if (level_pipeline_take(B->probs[i].mesh->fine, s) != SE_OK) f = true;
    if (B->probs[i].pmg && pmg_faults_take(B->probs[i].pmg, s) != SE_OK) f = true;
    if (f) {
      out[i].status = SE_ETIMEOUT;
      worst = SE_ETIMEOUT;
    }
  }
  return worst;
}

int se_batch_destroy(se_batch_t B) {
  if (!B) return SE_OK;
  batch_free(B);
  return SE_OK;
}

int se_batch_solve(int n, const se_problem* probs, const se_solve_opts* opts, se_solve_stats* out) {
  se_batch_t B = nullptr;
  SE_TRY(se_batch_create(n, probs, opts, &B));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(opts->stream);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  int rc = se_batch_run(B, opts->stream);
  cudaEventRecord(e1, s);
  if (rc == SE_OK) rc = se_batch_stats(B, opts->stream, out);
  float ms = 0.f;
  cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms, e0, e1);
  for (int i = 0; i < n; ++i) out[i].ms_total = ms;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  se_batch_destroy(B);
  return rc;
}

int se_batch_info(se_batch_t B, int* groups, int* grouped_problems) {
  SE_CHECK(B, SE_EINVAL, "se_batch_info: null batch");
  if (groups) *groups = (int)B->groups.size();
  int k = 0;
  for (const BatchGroup* G : B->groups) k += G->n;
  if (grouped_problems) *grouped_problems = k;
  return SE_OK;
}

}  // extern "C"
