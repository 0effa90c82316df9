// Matrix-free spectral element operator (Sec. 2.1): local A_L u by tensor-product sum
// factorisation, and QQ^T direct stiffness summation with the Dirichlet mask.
#include "se_internal.h"

namespace se {

// ------------------------------------------------------------------ local Ax
// NE elements per block, N*N threads per element (thread (i,j) owns the column k = 0..N-1).
//   ur = D_r u, us = D_s u, ut = D_t u         (the t contraction runs in registers)
//   (wr, ws, wt) = G (ur, us, ut), G symmetric with 6 stored factors per point
//   y = D_r^T wr + D_s^T ws + D_t^T wt         (the t part accumulates in registers)
// 12N+15 flops per point; reads u and G (7 values) and writes y once.
template <int N, typename T>
__global__ void __launch_bounds__(512) ax_local_kernel(int64_t E, int NE, const T* __restrict__ u,
                                                       const T* __restrict__ G, int64_t L,
                                                       const T* __restrict__ Dg,
                                                       T* __restrict__ y,
                                                       const uint8_t* __restrict__ pflag) {
  constexpr int N2 = N * N, N3 = N * N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sD = reinterpret_cast<T*>(smem_raw);
  const int le = threadIdx.x / N2;
  const int ij = threadIdx.x - le * N2;
  const int i = ij % N, j = ij / N;
  T* su = sD + N2 + (size_t)le * 3 * N3;
  T* swr = su + N3;
  T* sws = swr + N3;
  for (int t = threadIdx.x; t < N2; t += blockDim.x) sD[t] = Dg[t];
  const int64_t e = (int64_t)blockIdx.x * NE + le;
  const bool valid = (le < NE) && (e < E);
  const int64_t eb = e * N3;
  T ru[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    T v = T(0);
    if (valid) {
      v = u[eb + ij + N2 * k];
      if (pflag && !(pflag[eb + ij + N2 * k] & PF_FREE)) v = T(0);
    }
    ru[k] = v;
    if (le < NE) su[ij + N2 * k] = v;
  }
  __syncthreads();
  T Dri[N], Drj[N];
#pragma unroll
  for (int l = 0; l < N; ++l) {
    Dri[l] = sD[i * N + l];
    Drj[l] = sD[j * N + l];
  }
  T ry[N];
#pragma unroll
  for (int l = 0; l < N; ++l) ry[l] = T(0);
  if (le < NE) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      T ur = T(0), us = T(0), ut = T(0);
#pragma unroll
      for (int l = 0; l < N; ++l) {
        ur += Dri[l] * su[l + N * j + N2 * k];
        us += Drj[l] * su[i + N * l + N2 * k];
        ut += sD[k * N + l] * ru[l];
      }
      T grr = T(0), grs = T(0), grt = T(0), gss = T(0), gst = T(0), gtt = T(0);
      if (valid) {
        const int64_t gi = eb + ij + N2 * k;
        grr = G[gi];
        grs = G[L + gi];
        grt = G[2 * L + gi];
        gss = G[3 * L + gi];
        gst = G[4 * L + gi];
        gtt = G[5 * L + gi];
      }
      const T wr = grr * ur + grs * us + grt * ut;
      const T ws = grs * ur + gss * us + gst * ut;
      const T wt = grt * ur + gst * us + gtt * ut;
      swr[ij + N2 * k] = wr;
      sws[ij + N2 * k] = ws;
#pragma unroll
      for (int l = 0; l < N; ++l) ry[l] += sD[k * N + l] * wt;
    }
  }
  __syncthreads();
  if (le >= NE) return;
  T Dci[N], Dcj[N];
#pragma unroll
  for (int l = 0; l < N; ++l) {
    Dci[l] = sD[l * N + i];
    Dcj[l] = sD[l * N + j];
  }
#pragma unroll
  for (int k = 0; k < N; ++k) {
    T acc = ry[k];
#pragma unroll
    for (int l = 0; l < N; ++l) {
      acc += Dci[l] * swr[l + N * j + N2 * k];
      acc += Dcj[l] * sws[i + N * l + N2 * k];
    }
    if (valid) y[eb + ij + N2 * k] = acc;
  }
}

// Elements per block for N*N threads per element: the tuned value if one is set and valid,
// else enough elements for about 256 threads.
int ax_elems_per_block(int p, bool fp32) {
  const int N = p + 1;
  const int t = tile_get(p, fp32).ax_ne;
  if (t >= 1 && t * N * N <= 512) return t;
  const int ne = 256 / (N * N);
  return ne < 1 ? 1 : ne;
}

template <int N, typename T>
static int launch_ax(const Level& lv, const T* u, T* y, const T* G, const T* D,
                     const uint8_t* pflag, cudaStream_t s) {
  const int NE = ax_elems_per_block(N - 1, sizeof(T) == 4);
  const int threads = NE * N * N;
  const size_t smem = (N * N + (size_t)NE * 3 * N * N * N) * sizeof(T);
  // set once per kernel (thread-safe static initialisation)
  static const cudaError_t attr = cudaFuncSetAttribute(
      ax_local_kernel<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  SE_CUDA(attr);
  const unsigned blocks = (unsigned)((lv.E + NE - 1) / NE);
  ax_local_kernel<N, T><<<blocks, threads, smem, s>>>(lv.E, NE, u, G, lv.L, D, y, pflag);
  SE_LAUNCH_CHECK();
  return SE_OK;
}

template <class T>
int ax_local(const Level& lv, const T* u, T* y, bool mask_in, cudaStream_t s) {
  const T* G;
  const T* D;
  if constexpr (sizeof(T) == 8) {
    G = lv.G64;
    D = lv.D64;
  } else {
    G = lv.G32;
    D = lv.D32;
  }
  SE_CHECK(G != nullptr, SE_EINVAL, "ax_local: geometric factors for this precision missing");
  const int N = lv.N;
  const double pts = (double)lv.L;
  ProfScope prof(SE_K_AX, s, pts, pts * 8.0 * sizeof(T), pts * (12.0 * N + 15.0),
                 prof_variant<T>(lv.p));
  const uint8_t* pf = mask_in ? lv.pflag : nullptr;
  if constexpr (sizeof(T) == 4) {
    if (!mask_in && ax_tma_supported(lv.p)) return ax_local_tma(lv, u, y, s);
  } else {
    if (!mask_in && ax_eo_supported(lv.p) && lv.eo64) return ax_local_eo(lv, u, y, s);
  }
  switch (N) {
    case 2: return launch_ax<2, T>(lv, u, y, G, D, pf, s);
    case 3: return launch_ax<3, T>(lv, u, y, G, D, pf, s);
    case 4: return launch_ax<4, T>(lv, u, y, G, D, pf, s);
    case 5: return launch_ax<5, T>(lv, u, y, G, D, pf, s);
    case 6: return launch_ax<6, T>(lv, u, y, G, D, pf, s);
    case 7: return launch_ax<7, T>(lv, u, y, G, D, pf, s);
    case 8: return launch_ax<8, T>(lv, u, y, G, D, pf, s);
    case 9: return launch_ax<9, T>(lv, u, y, G, D, pf, s);
    case 10: return launch_ax<10, T>(lv, u, y, G, D, pf, s);
    case 11: return launch_ax<11, T>(lv, u, y, G, D, pf, s);
    default: set_error("ax_local: unsupported N=%d", N); return SE_EINVAL;
  }
}

// ------------------------------------------------------------------ QQ^T + mask
// One thread per group of local copies of a global node; the copies are summed in index order
// (deterministic) and the sum written back to each.  Groups on Dirichlet faces (first id stored
// as ~id) are zeroed when masking; single-copy Dirichlet nodes follow the groups.
template <typename T, int M>
__device__ __forceinline__ void gs_group(const int* __restrict__ g, T* __restrict__ u, bool mask) {
  int id[M];
#pragma unroll
  for (int q = 0; q < M; ++q) id[q] = g[q];
  const bool msk = id[0] < 0;
  if (msk) id[0] = ~id[0];
  if (msk && mask) {
#pragma unroll
    for (int q = 0; q < M; ++q) u[id[q]] = T(0);
    return;
  }
  T v[M];
#pragma unroll
  for (int q = 0; q < M; ++q) v[q] = u[id[q]];
  T sacc = v[0];
#pragma unroll
  for (int q = 1; q < M; ++q) sacc += v[q];
#pragma unroll
  for (int q = 0; q < M; ++q) u[id[q]] = sacc;
}

// Pairs (the bulk of the groups) are processed four per thread, interleaved: thread t of T
// takes pairs t, t+T, t+2T, t+3T, so every load instruction of a warp still covers 32
// neighbouring pairs (shared sectors) while each thread keeps eight independent value loads in
// flight.  Quads, octets and single Dirichlet copies follow, one group per thread.
constexpr int GS_PAIRS_PER_THREAD = 4;

template <typename T>
__global__ void gs_kernel(int64_t n2, int64_t n4, int64_t n8, int64_t n1,
                          const int* __restrict__ ids, T* __restrict__ u, bool mask) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t T2 = (n2 + GS_PAIRS_PER_THREAD - 1) / GS_PAIRS_PER_THREAD;
  if (t < T2) {
    int a[GS_PAIRS_PER_THREAD], b[GS_PAIRS_PER_THREAD];
    bool m[GS_PAIRS_PER_THREAD], on[GS_PAIRS_PER_THREAD];
#pragma unroll
    for (int k = 0; k < GS_PAIRS_PER_THREAD; ++k) {
      const int64_t g = t + k * T2;
      on[k] = g < n2;
      const int2 q = on[k] ? *reinterpret_cast<const int2*>(ids + 2 * g) : make_int2(0, 0);
      m[k] = q.x < 0;
      a[k] = m[k] ? ~q.x : q.x;
      b[k] = q.y;
    }
    T va[GS_PAIRS_PER_THREAD], vb[GS_PAIRS_PER_THREAD];
#pragma unroll
    for (int k = 0; k < GS_PAIRS_PER_THREAD; ++k) {
      va[k] = on[k] ? u[a[k]] : T(0);
      vb[k] = on[k] ? u[b[k]] : T(0);
    }
#pragma unroll
    for (int k = 0; k < GS_PAIRS_PER_THREAD; ++k) {
      if (!on[k]) continue;
      const T sum = (m[k] && mask) ? T(0) : va[k] + vb[k];
      u[a[k]] = sum;
      u[b[k]] = sum;
    }
    return;
  }
  t -= T2;
  ids += 2 * n2;
  if (t < n4) {
    gs_group<T, 4>(ids + 4 * t, u, mask);
    return;
  }
  t -= n4;
  ids += 4 * n4;
  if (t < n8) {
    gs_group<T, 8>(ids + 8 * t, u, mask);
    return;
  }
  t -= n8;
  ids += 8 * n8;
  if (t < n1 && mask) u[ids[t]] = T(0);
}

template <class T>
int gs_apply(const Level& lv, T* u, bool mask, cudaStream_t s) {
  const int64_t n = (lv.n_pairs + GS_PAIRS_PER_THREAD - 1) / GS_PAIRS_PER_THREAD + lv.n_quads +
                    lv.n_octs + lv.n_masked;
  if (lv.n_pairs + n == 0) return SE_OK;
  const double entries = 2.0 * lv.n_pairs + 4.0 * lv.n_quads + 8.0 * lv.n_octs;
  ProfScope prof(SE_K_GS, s, entries, entries * (2.0 * sizeof(T) + 4.0) + lv.n_masked * (4.0 + sizeof(T)),
                 entries, prof_variant<T>(lv.p));
  gs_kernel<T><<<grid_for(n, 256), 256, 0, s>>>(lv.n_pairs, lv.n_quads, lv.n_octs, lv.n_masked,
                                                 lv.gs_ids, u, mask);
  SE_LAUNCH_CHECK();
  return SE_OK;
}

template <typename T>
__global__ void mask_kernel(int64_t L, const uint8_t* __restrict__ pflag, T* __restrict__ u) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < L && !(pflag[idx] & PF_FREE)) u[idx] = T(0);
}

template int ax_local<double>(const Level&, const double*, double*, bool, cudaStream_t);
template int ax_local<float>(const Level&, const float*, float*, bool, cudaStream_t);
template int gs_apply<double>(const Level&, double*, bool, cudaStream_t);
template int gs_apply<float>(const Level&, float*, bool, cudaStream_t);

int apply_mask64(const Level& lv, double* u, cudaStream_t s) {
  mask_kernel<double><<<grid_for(lv.L, 256), 256, 0, s>>>(lv.L, lv.pflag, u);
  SE_LAUNCH_CHECK();
  return SE_OK;
}

}  // namespace se

using namespace se;

extern "C" {

int se_ax(se_mesh_t m, const double* u, double* y, int flags, void* stream) {
  SE_CHECK(m && u && y, SE_EINVAL, "se_ax: null argument");
  SE_CHECK(u != y, SE_EINVAL, "se_ax: u and y must not overlap");
  cudaStream_t s = as_stream(stream, m->stream);
  Level& lv = m->fine;
  const bool mask = (flags & SE_AX_MASK) != 0;
  const bool assemble = (flags & SE_AX_ASSEMBLE) != 0;
  if (flags & SE_AX_FP32) {
    SE_TRY(make_fp32_geometry(lv, m->allocs, s));
    SE_TRY((convert<double, float>(u, m->tmpa32, lv.L, s)));
    SE_TRY(ax_local<float>(lv, m->tmpa32, m->tmpb32, mask, s));
    if (assemble) SE_TRY(gs_apply<float>(lv, m->tmpb32, mask, s));
    SE_TRY((convert<float, double>(m->tmpb32, y, lv.L, s)));
    if (!assemble && mask) SE_TRY(apply_mask64(lv, y, s));
    return SE_OK;
  }
  SE_TRY(ax_local<double>(lv, u, y, mask, s));
  if (assemble) return gs_apply<double>(lv, y, mask, s);
  if (mask) return apply_mask64(lv, y, s);
  return SE_OK;
}

int se_gs(se_mesh_t m, double* u, int mask, void* stream) {
  SE_CHECK(m && u, SE_EINVAL, "se_gs: null argument");
  return gs_apply<double>(m->fine, u, mask != 0, as_stream(stream, m->stream));
}

}  // extern "C"
