// Matrix-free spectral element operator (Sec. 2.1): local A_L u by tensor-product sum
// factorisation, and QQ^T direct stiffness summation with the Dirichlet mask.
#include "se_internal.h"

namespace se {

// ------------------------------------------------------------------ local Ax
// NE elements per block, N*N threads per element (thread (i,j) owns the column k = 0..N-1).
//   ur = D_r u, us = D_s u, ut = D_t u         (the t contraction runs in registers)
//   (wr, ws, wt) = G (ur, us, ut), G symmetric with 6 stored factors per point
//   y = D_r^T wr + D_s^T ws + D_t^T wt         (the t part accumulates in registers)
// 12N+15 flops per point; reads u and G (7 values) and writes y once.  T is the arithmetic type,
// IO the type of u, y and sub in memory (T, or double for T = df64).
template <int N, typename T, typename IO = T>
__global__ void __launch_bounds__(512) ax_local_kernel(int64_t E, int NE, const IO* __restrict__ u,
                                                       const T* __restrict__ G, int64_t L,
                                                       const T* __restrict__ Dg,
                                                       IO* __restrict__ y,
                                                       const uint8_t* __restrict__ pflag,
                                                       bool mask_in, const IO* __restrict__ sub) {
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
      v = from_io<T>(u[eb + ij + N2 * k]);
      if (mask_in && !(pflag[eb + ij + N2 * k] & PF_FREE)) v = T(0);
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
    if (valid) y[eb + ij + N2 * k] = ax_output(io_cast<IO>(acc), sub, pflag, eb + ij + N2 * k);
  }
}

// Elements per block for N*N threads per element: the tuned value if one is set and valid,
// else enough elements for about 256 threads.
int ax_elems_per_block(int p, bool fp32) {
  const int N = p + 1;
  const int t = tile_get(p, fp32).ax_ne;
  if (t >= 1 && t * N * N <= 512) return t;
  // FP64 even N (the folded kernel): measured on GB300 at 32^3 elements, elements per block
  // N = 4: 8 (16: 0.144 -> 0.138 ms), N = 6: 8 (7: 0.543 -> 0.525 ms), N = 10: 3 (2: 3.38 ->
  // 3.26 ms); N = 8 keeps 4 (1 to 4 within 0.5%)
  if (!fp32 && (N == 4 || N == 6)) return 8;
  if (!fp32 && N == 10) return 3;
  const int ne = 256 / (N * N);
  return ne < 1 ? 1 : ne;
}

template <int N, typename T>
static int launch_ax(const Level& lv, const T* u, T* y, const T* G, const T* D, bool mask_in,
                     const T* sub, cudaStream_t s) {
  const int NE = ax_elems_per_block(N - 1, sizeof(T) == 4);
  const int threads = NE * N * N;
  const size_t smem = (N * N + (size_t)NE * 3 * N * N * N) * sizeof(T);
  // set once per kernel (thread-safe static initialisation)
  static const cudaError_t attr = cudaFuncSetAttribute(
      ax_local_kernel<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  SE_CUDA(attr);
  const unsigned blocks = (unsigned)((lv.E + NE - 1) / NE);
  ax_local_kernel<N, T><<<blocks, threads, smem, s>>>(lv.E, NE, u, G, lv.L, D, y, lv.pflag, mask_in,
                                                       sub);
  SE_LAUNCH_CHECK();
  return SE_OK;
}

// df64 arithmetic on FP64 vectors, odd N (even orders; even N uses the folded kernel).
template <int N>
static int launch_ax_df(const Level& lv, const double* u, double* y, const double* sub,
                        cudaStream_t s) {
  const int NE = ax_elems_per_block(N - 1, false);
  const int threads = NE * N * N;
  const size_t smem = (N * N + (size_t)NE * 3 * N * N * N) * sizeof(df64);
  static const cudaError_t attr = cudaFuncSetAttribute(
      ax_local_kernel<N, df64, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  SE_CUDA(attr);
  const unsigned blocks = (unsigned)((lv.E + NE - 1) / NE);
  ax_local_kernel<N, df64, double><<<blocks, threads, smem, s>>>(lv.E, NE, u, lv.Gdf, lv.L, lv.Ddf, y,
                                                                  lv.pflag, false, sub);
  SE_LAUNCH_CHECK();
  return SE_OK;
}

static int ax_local_generic_df(const Level& lv, const double* u, double* y, const double* sub,
                               cudaStream_t s) {
  SE_CHECK(lv.Gdf != nullptr && lv.Ddf != nullptr, SE_EINVAL, "ax_df: df64 geometry missing");
  switch (lv.N) {
    case 3: return launch_ax_df<3>(lv, u, y, sub, s);
    case 5: return launch_ax_df<5>(lv, u, y, sub, s);
    case 7: return launch_ax_df<7>(lv, u, y, sub, s);
    case 9: return launch_ax_df<9>(lv, u, y, sub, s);
    case 11: return launch_ax_df<11>(lv, u, y, sub, s);
    default: set_error("ax_df: unsupported N=%d", lv.N); return SE_EINVAL;
  }
}

template <class T>
int ax_local(const Level& lv, const T* u, T* y, bool mask_in, cudaStream_t s, const T* sub) {
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
  bool use_df = false;
  if constexpr (sizeof(T) == 8) use_df = !mask_in && ax_df_route(lv);
  ProfScope prof(SE_K_AX, s, pts, pts * ((sub ? 9.0 : 8.0) * sizeof(T) + (sub ? 1.0 : 0.0)),
                 pts * (12.0 * N + 15.0), use_df ? lv.p + 64 : prof_variant<T>(lv.p));
  if constexpr (sizeof(T) == 4) {
    if (!mask_in && ax_tma_supported(lv.p)) return ax_local_tma(lv, u, y, s, sub);
  } else {
    if (use_df) {
      if (ax_eo_supported(lv.p)) return ax_local_eo_df(lv, u, y, s, sub);
      return ax_local_generic_df(lv, u, y, sub, s);
    }
    if (!mask_in && ax_eo_supported(lv.p) && lv.eo64) return ax_local_eo(lv, u, y, s, sub);
  }
  switch (N) {
    case 2: return launch_ax<2, T>(lv, u, y, G, D, mask_in, sub, s);
    case 3: return launch_ax<3, T>(lv, u, y, G, D, mask_in, sub, s);
    case 4: return launch_ax<4, T>(lv, u, y, G, D, mask_in, sub, s);
    case 5: return launch_ax<5, T>(lv, u, y, G, D, mask_in, sub, s);
    case 6: return launch_ax<6, T>(lv, u, y, G, D, mask_in, sub, s);
    case 7: return launch_ax<7, T>(lv, u, y, G, D, mask_in, sub, s);
    case 8: return launch_ax<8, T>(lv, u, y, G, D, mask_in, sub, s);
    case 9: return launch_ax<9, T>(lv, u, y, G, D, mask_in, sub, s);
    case 10: return launch_ax<10, T>(lv, u, y, G, D, mask_in, sub, s);
    case 11: return launch_ax<11, T>(lv, u, y, G, D, mask_in, sub, s);
    default: set_error("ax_local: unsupported N=%d", N); return SE_EINVAL;
  }
}

// ------------------------------------------------------------------ QQ^T + mask
// The mesh is a box lattice of elements, so the copies of a global node are the products of its
// per-direction copies, and QQ^T factors into three sweeps, one per direction: a sweep adds the
// two copies on either side of every element interface normal to its direction and writes the
// sum to both.  After the x sweep each copy holds the sum over its x-neighbours; the y sweep adds
// those partial sums across y-interfaces (edge nodes: 4 copies); the z sweep across z-interfaces
// (corners: 8).  Every copy ends with the sum over all copies of its node, and all copies of a
// node hold bitwise the same value (each pair writes one sum to both sides).  No index map is
// read, and every access is laid out for the element-major, i-fastest layout:
//   x: a warp holds whole rows of one k-plane for a run of elements along x and exchanges the
//      interface copies by shuffles (below);
//   y: lanes run along i: rows of N contiguous copies;
//   z: lanes run along (i, j): planes of N^2 contiguous copies.
// The y and z sweeps run as one launch (gs_sweep_yz): a node with copies across a y- and a
// z-interface is summed by one thread in the order of the two sweeps.
// Masking (Dirichlet) zeroes the copies on Dirichlet faces within the x sweep, before any sum (a
// node on such a face has all its copies there), so the sweeps then add zeros for masked nodes;
// a lattice one element wide in x has a separate mask kernel.
// x-interfaces per warp: 16 in FP32 (halves the per-warp index and mask work, which bounds the
// FP32 sweep), 8 in FP64
template <typename T>
__host__ __device__ constexpr int gs_x_seg() { return sizeof(T) == 4 ? 16 : 8; }

// x sweep: a warp holds R = 32/N consecutive rows (j, k) of an element (lane = (row, i); the
// element's N^2 rows are contiguous) for a run of consecutive elements along x, loaded coalesced
// (R N contiguous values per element), one value per lane per element kept in registers; the
// two copies of each x-interface (lane i = p of element m, lane i = 0 of element m + 1, same
// row) swap by one shuffle and both store their sum (a + b == b + a exactly: both copies get the
// same bits).  Every value of the vector
// is read once, in full sectors.  A warp takes a run of gs_x_seg<T>() interfaces (runs of one x-row
// overlap by one element, and no two runs write the same copy: a run writes the row ends of its
// interfaces only); it always loads gs_x_seg<T>() + 1 elements (indices clamped to the last element of
// the row) so that all loads are issued back to back.
// With Dirichlet bits (mask), the x sweep also applies the mask: a copy whose node lies on a
// Dirichlet face is zeroed before the sums and stored as zero (every copy of every element passes
// through some run, and a node's copies are all masked or none, so overlapping runs agree).
template <typename T, int N>
__global__ void __launch_bounds__(256) gs_sweep_x(int nx, int ny, int nz, int bits, T* __restrict__ u) {
  constexpr int N3 = N * N * N, R = 32 / N, NG = (N * N + R - 1) / R, SEG = gs_x_seg<T>();
  // index decomposition in 32-bit integers (every count here is below L < 2^31; a 64-bit
  // division by a run-time value costs an order of magnitude more instructions)
  const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  const int nseg = (nx - 1 + SEG - 1) / SEG;
  const int items = ny * nz * NG * nseg;               // (row group, run, element row along x)
  if (warp >= items) return;                           // whole warps
  const int grp = warp % NG;
  const int q = warp / NG;
  const int seg = q % nseg;
  const int row_e = q / nseg;                          // ey + ny ez
  const int r = lane / N, i = lane - r * N;
  const int jk = grp * R + r;                          // row j + N k of the element
  const bool on = r < R && jk < N * N;
  const int rowbase = r * N;                           // lane of (row r, i = 0)
  const int64_t off = on ? (int64_t)i + (int64_t)N * jk : 0;
  const int ex0 = seg * SEG;
  const int cnt = min(SEG, nx - 1 - ex0);              // interfaces of this run
  const int64_t e0 = (int64_t)nx * row_e + ex0;
  T v[SEG + 1];
#pragma unroll
  for (int m = 0; m <= SEG; ++m) v[m] = u[(e0 + min(m, cnt)) * N3 + off];
  if (bits) {
    const int j = jk % N, k = jk / N;
    const int ey = row_e % ny, ez = row_e / ny;
    // a lane's copies are masked in every element of the run (a Dirichlet y or z face), or only
    // in the run's first element (x = 0 face) or last one (x = 1 face): tested once per lane
    const bool myz = ((bits & 4) && j == 0 && ey == 0) || ((bits & 8) && j == N - 1 && ey == ny - 1) ||
                     ((bits & 16) && k == 0 && ez == 0) || ((bits & 32) && k == N - 1 && ez == nz - 1);
    const bool mx0 = (bits & 1) && i == 0 && ex0 == 0;
    const bool mx1 = (bits & 2) && i == N - 1 && ex0 + cnt == nx - 1;
    if (on && (myz || mx0 || mx1)) {
#pragma unroll
      for (int m = 0; m <= SEG; ++m) {
        if (m > cnt) break;
        if (myz || (m == 0 && mx0) || (m == cnt && mx1)) {
          v[m] = T(0);
          u[(e0 + m) * N3 + off] = T(0);
        }
      }
    }
  }
  // lane (r, p) holds the left copy (element m), lane (r, 0) the right copy (element m + 1):
  // one shuffle swaps them, one store writes both (each lane its own element)
  const bool left = i == N - 1, right = i == 0;
  const int partner = min(left ? rowbase : rowbase + N - 1, 31);
#pragma unroll
  for (int m = 0; m < SEG; ++m) {
    if (m >= cnt) break;
    const T mine = right ? v[m + 1] : v[m];
    const T other = __shfl_sync(0xffffffffu, mine, partner);
    if (on && (left || right)) u[(e0 + m + (right ? 1 : 0)) * N3 + off] = mine + other;
  }
}

// The y/z launch: each thread takes GS_YZ_PAIRS items, strided so that a warp's accesses stay
// contiguous, all loads issued before any store (these launches are bound by memory latency, not
// bandwidth).
constexpr int GS_YZ_PAIRS = 4;

// y and z directions in one launch (the x direction complete before it).  Items: y-pairs
// (element e, e + nx; copies (i, p, k), (i, 0, k)) and z-pairs (e, e + nx ny; (i, j, p), (i, j, 0)).
// A node on a y- and a z-interface has four copies; the y-item at k = p (ez < nz - 1) takes all
// four and sums them as the two sweeps would, (y-pair at k = p) + (y-pair of e + nx ny at k = 0),
// so every copy keeps the bits of the sweep order; the y-item at k = 0 of e + nx ny and the
// z-items at j = p (ey < ny - 1) and j = 0 (ey > 0) belong to such groups and do nothing.  Every
// interface copy is then read and written once, by one thread.
template <typename T, int N>
__global__ void gs_sweep_yz(int nx, int ny, int nz, T* __restrict__ u) {
  constexpr int N2 = N * N, N3 = N2 * N, K = GS_YZ_PAIRS;
  const int ny1 = ny - 1, nz1 = nz - 1;
  const int ty = N2 * nx * ny1 * nz;   // y-items, ordered (i, k, ex, ey, ez)
  const int total = ty + N2 * nx * ny * nz1;  // then z-items (ij, e), e over ez < nz - 1
  const int nthr = (total + K - 1) / K;
  const int t0 = (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (t0 >= nthr) return;
  const int exy = nx * ny;
  int ia[K], ib[K], ic[K], id[K];  // point indices < L < 2^31
  T a[K], b[K], c[K], d[K];
#pragma unroll
  for (int kk = 0; kk < K; ++kk) {
    const int t = t0 + kk * nthr;
    ia[kk] = -1;
    ic[kk] = -1;
    if (t < ty) {
      const int i = t % N;
      int q = t / N;
      const int k = q % N;
      q /= N;
      const int ex = q % nx;
      q /= nx;
      const int ey = q % ny1;
      const int ez = q / ny1;
      if (k == 0 && ez > 0) continue;                 // in the group of e - nx ny
      const int e = ex + nx * (ey + ny * ez);
      ia[kk] = e * N3 + i + N * ((N - 1) + N * k);     // element e, j = p
      ib[kk] = (e + nx) * N3 + i + N2 * k;             // element e + nx, j = 0
      a[kk] = u[ia[kk]];
      b[kk] = u[ib[kk]];
      if (k == N - 1 && ez < nz1) {                    // four copies: also k = 0 of e + nx ny
        ic[kk] = (e + exy) * N3 + i + N * (N - 1);
        id[kk] = (e + exy + nx) * N3 + i;
        c[kk] = u[ic[kk]];
        d[kk] = u[id[kk]];
      }
    } else if (t < total) {
      const int tz = t - ty;
      const int ij = tz % N2;
      const int e = tz / N2;                           // elements with ez < nz - 1, in order
      const int j = ij / N;
      const int ey = (e / nx) % ny;
      if ((j == N - 1 && ey < ny1) || (j == 0 && ey > 0)) continue;  // in a y-item's group
      ia[kk] = e * N3 + ij + N2 * (N - 1);             // element e, k = p
      ib[kk] = (e + exy) * N3 + ij;                    // element e + nx ny, k = 0
      a[kk] = u[ia[kk]];
      b[kk] = u[ib[kk]];
    }
  }
#pragma unroll
  for (int kk = 0; kk < K; ++kk) {
    if (ia[kk] < 0) continue;
    T sum = a[kk] + b[kk];
    if (ic[kk] >= 0) {
      sum = sum + (c[kk] + d[kk]);
      u[ic[kk]] = sum;
      u[id[kk]] = sum;
    }
    u[ia[kk]] = sum;
    u[ib[kk]] = sum;
  }
}

// Interface copies the fused y/z launch reads and writes once each.
template <int N>
static double yz_copies(int nx, int ny, int nz) {
  return 2.0 * N * N * ((double)nx * (ny - 1) * nz + (double)nx * ny * (nz - 1)) -
         4.0 * N * (double)nx * (ny - 1) * (nz - 1);
}

// The fused y/z launch with one profiling scope; `bytes` < 0: the interface copies' bytes.
template <typename T, int N>
static int gs_yz(int nx, int ny, int nz, T* u, int var, double bytes, cudaStream_t s) {
  if (ny <= 1 && nz <= 1) return SE_OK;
  const int64_t items = (int64_t)N * N * nx * ((int64_t)(ny - 1) * nz + (int64_t)ny * (nz - 1));
  const double copies = yz_copies<N>(nx, ny, nz);
  ProfScope prof(SE_K_GS, s, copies, bytes < 0 ? 2.0 * copies * sizeof(T) : bytes, (double)items, var);
  gs_sweep_yz<T, N><<<grid_for((items + GS_YZ_PAIRS - 1) / GS_YZ_PAIRS, 256), 256, 0, s>>>(nx, ny, nz, u);
  SE_LAUNCH_CHECK();
  return SE_OK;
}

// Zero the copies on the Dirichlet faces (bit f of `bits`: face f = x0, x1, y0, y1, z0, z1).
// Thread: (face, element on the face, point of the element's face).
template <typename T, int N>
__global__ void gs_mask_faces(int nx, int ny, int nz, int bits, T* __restrict__ u) {
  constexpr int N2 = N * N, N3 = N2 * N;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t fx = (int64_t)ny * nz * N2, fy = (int64_t)nx * nz * N2, fz = (int64_t)nx * ny * N2;
  int64_t r = t;
  int f;
  if (r < 2 * fx) {
    f = r < fx ? 0 : 1;
    r -= f * fx;
  } else if ((r -= 2 * fx) < 2 * fy) {
    f = r < fy ? 2 : 3;
    r -= (f - 2) * fy;
  } else if ((r -= 2 * fy) < 2 * fz) {
    f = r < fz ? 4 : 5;
    r -= (f - 4) * fz;
  } else {
    return;
  }
  if (!((bits >> f) & 1)) return;
  const int a = (int)(r % N), b = (int)((r / N) % N);
  const int64_t el = r / N2;  // element index along the face's two directions
  int ex, ey, ez, i, j, k;
  const int side = f & 1;
  if (f < 2) {
    ey = (int)(el % ny); ez = (int)(el / ny); ex = side ? nx - 1 : 0;
    i = side ? N - 1 : 0; j = a; k = b;
  } else if (f < 4) {
    ex = (int)(el % nx); ez = (int)(el / nx); ey = side ? ny - 1 : 0;
    j = side ? N - 1 : 0; i = a; k = b;
  } else {
    ex = (int)(el % nx); ey = (int)(el / nx); ez = side ? nz - 1 : 0;
    k = side ? N - 1 : 0; i = a; j = b;
  }
  const int64_t e = ex + (int64_t)nx * (ey + (int64_t)ny * ez);
  u[e * N3 + i + N * (j + N * k)] = T(0);
}

// One profiling scope per launch (so launch counts are exact); the algorithmic bytes of QQ^T
// (every interface copy read and written once) are attributed to the x sweep.
template <typename T, int N>
static int gs_sweeps(const Level& lv, T* u, bool mask, double bytes, double flops, cudaStream_t s) {
  const int nx = lv.nel[0], ny = lv.nel[1], nz = lv.nel[2];
  constexpr int N2 = N * N;
  const int var = prof_variant<T>(lv.p);
  int bits = 0;
  if (mask)
    for (int f = 0; f < 6; ++f)
      if (lv.bc[f] == SE_BC_DIRICHLET) bits |= 1 << f;
  if (bits && nx == 1) {  // no x sweep to carry the mask
    {
      const int64_t n = 2 * N2 * ((int64_t)ny * nz + (int64_t)nx * nz + (int64_t)nx * ny);
      ProfScope prof(SE_K_GS, s, (double)n, 0.0, 0.0, var);
      gs_mask_faces<T, N><<<grid_for(n, 256), 256, 0, s>>>(nx, ny, nz, bits, u);
      SE_LAUNCH_CHECK();
    }
  }
  if (nx > 1) {
    constexpr int R = 32 / N, NG = (N * N + R - 1) / R;
    constexpr int SEG = gs_x_seg<T>();
    const int64_t warps = (int64_t)ny * nz * NG * ((nx - 1 + SEG - 1) / SEG);
    ProfScope prof(SE_K_GS, s, (double)lv.L, bytes, flops, var);
    gs_sweep_x<T, N><<<grid_for(32 * warps, 256), 256, 0, s>>>(nx, ny, nz, bits, u);
    SE_LAUNCH_CHECK();
  }
  return gs_yz<T, N>(nx, ny, nz, u, var, 0.0, s);
}

// Copies on element interfaces (each is read and written once by the algorithm).
static double interface_copies(const Level& lv) {
  double inner = 1.0;  // local points on no interface: product over directions
  for (int d = 0; d < 3; ++d) inner *= (double)lv.nel[d] * lv.N - 2.0 * (lv.nel[d] - 1);
  return (double)lv.L - inner;
}

template <class T>
int gs_apply(const Level& lv, T* u, bool mask, cudaStream_t s) {
  if (lv.gsm_ids) return gsmap_apply<T>(lv, u, mask, s);
  const double shared = interface_copies(lv);
  const double bytes = shared * 2.0 * sizeof(T), flops = shared;
  switch (lv.N) {
#define SE_GS_CASE(NN) \
  case NN: return gs_sweeps<T, NN>(lv, u, mask, bytes, flops, s);
    SE_GS_CASE(2) SE_GS_CASE(3) SE_GS_CASE(4) SE_GS_CASE(5) SE_GS_CASE(6)
    SE_GS_CASE(7) SE_GS_CASE(8) SE_GS_CASE(9) SE_GS_CASE(10) SE_GS_CASE(11)
#undef SE_GS_CASE
    default: set_error("gs: unsupported N=%d", lv.N); return SE_EINVAL;
  }
}

// ------------------------------------------------------------------ folded FP64 operator
// The even-odd kernel sums the x-interfaces inside its blocks and masks (ax_local_eo_fold); the
// x-interfaces between blocks follow (gs_fold_fixup), then the fused y/z launch, so the x direction
// is complete before y and z start, as in the sweeps above, and every copy of a node gets the
// same bits.  This removes the x sweep, which
// reads and writes every sector of the vector (an x-interface copy is the first or last value of
// a row of N), from the operator applications of the solve.
bool ax_fold_ok(const Level& lv) {
  return !ax_df_route(lv) && lv.eo64 && ax_eo_supported(lv.p) && !lv.gsm_ids && lv.nel[0] >= 1 &&
         lv.nel[1] >= 1 && lv.nel[2] >= 1;
}

template <int N>
static int gs_after_fold(const Level& lv, double* y, int NE, cudaStream_t s) {
  const int nx = lv.nel[0], ny = lv.nel[1], nz = lv.nel[2];
  constexpr int N2 = N * N;
  const int var = prof_variant<double>(lv.p);
  // the x direction must be complete before the y sweep adds across y-interfaces: a copy summed
  // across a block-boundary x-interface after the y sweep would count its y-partner's x-neighbour
  // twice
  const int64_t nbnd = (lv.E + NE - 1) / NE - 1;
  if (nx > 1 && nbnd > 0) {
    const double n = (double)nbnd * N2;  // at most this many pairs
    ProfScope prof(SE_K_GS, s, n, 4.0 * n * sizeof(double), n, var);
    SE_TRY(gs_fold_fixup(lv, y, NE, s));
  }
  return gs_yz<double, N>(nx, ny, nz, y, var, -1.0, s);
}

int ax_apply_folded(const Level& lv, const double* u, double* y, const double* b, cudaStream_t s,
                    const double* dinv) {
  const int NE = ax_elems_per_block(lv.p, false);
  {
    const double pts = (double)lv.L;
    // u, y, 6 geometric factors, b (residual form) and D^-1 (scaled input) per point; the
    // folded kernel reads no point flags (mask and weights from the lattice position)
    ProfScope prof(SE_K_AX, s, pts,
                   pts * (8.0 + (b ? 1.0 : 0.0) + (dinv ? 1.0 : 0.0)) * sizeof(double),
                   pts * (12.0 * lv.N + 15.0), prof_variant<double>(lv.p));
    SE_TRY(ax_local_eo_fold(lv, u, y, b, NE, s, dinv));
  }
  switch (lv.N) {
    case 2: return gs_after_fold<2>(lv, y, NE, s);
    case 4: return gs_after_fold<4>(lv, y, NE, s);
    case 6: return gs_after_fold<6>(lv, y, NE, s);
    case 8: return gs_after_fold<8>(lv, y, NE, s);
    case 10: return gs_after_fold<10>(lv, y, NE, s);
    default: set_error("ax_apply_folded: unsupported N=%d", lv.N); return SE_EINVAL;
  }
}

template <typename T>
__global__ void mask_kernel(int64_t L, const uint8_t* __restrict__ pflag, T* __restrict__ u) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < L && !(pflag[idx] & PF_FREE)) u[idx] = T(0);
}

template int ax_local<double>(const Level&, const double*, double*, bool, cudaStream_t, const double*);
template int ax_local<float>(const Level&, const float*, float*, bool, cudaStream_t, const float*);
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
  if (flags & SE_AX_DF64) {
    SE_TRY(make_df_geometry(lv, m->allocs, s));
    Level ld = lv;
    ld.df = true;
    const double* in = u;
    if (mask) {  // masked input through the mesh's work vector
      SE_CUDA(cudaMemcpyAsync(m->tmp64, u, lv.L * sizeof(double), cudaMemcpyDeviceToDevice, s));
      SE_TRY(apply_mask64(lv, m->tmp64, s));
      in = m->tmp64;
    }
    SE_TRY(ax_local<double>(ld, in, y, false, s));
    if (assemble) return gs_apply<double>(ld, y, mask, s);
    if (mask) return apply_mask64(lv, y, s);
    return SE_OK;
  }
  SE_TRY(ax_local<double>(lv, u, y, mask, s));
  if (assemble) return gs_apply<double>(lv, y, mask, s);
  if (mask) return apply_mask64(lv, y, s);
  return SE_OK;
}

int se_residual(se_mesh_t m, const double* b, const double* u, double* r, int flags, void* stream) {
  SE_CHECK(m && b && u && r, SE_EINVAL, "se_residual: null argument");
  SE_CHECK(r != u && r != b, SE_EINVAL, "se_residual: r must not overlap b or u");
  SE_CHECK((flags & ~(SE_AX_FP32 | SE_AX_DF64)) == 0 && flags != (SE_AX_FP32 | SE_AX_DF64),
           SE_EINVAL, "se_residual: flags must be 0, SE_AX_FP32 or SE_AX_DF64");
  cudaStream_t s = as_stream(stream, m->stream);
  Level& lv = m->fine;
  if (flags & SE_AX_FP32) {
    SE_TRY(make_fp32_geometry(lv, m->allocs, s));
    if (!m->tmpc32) SE_TRY(dmalloc(m->allocs, &m->tmpc32, (size_t)lv.L));
    SE_TRY((convert<double, float>(u, m->tmpa32, lv.L, s)));
    SE_TRY((convert<double, float>(b, m->tmpc32, lv.L, s)));
    SE_TRY(residual_apply<float>(lv, m->tmpc32, m->tmpa32, m->tmpb32, s));
    return convert<float, double>(m->tmpb32, r, lv.L, s);
  }
  if (flags & SE_AX_DF64) {
    SE_TRY(make_df_geometry(lv, m->allocs, s));
    Level ld = lv;
    ld.df = true;
    return residual_apply<double>(ld, b, u, r, s);
  }
  return residual_apply<double>(lv, b, u, r, s);
}

int se_gs(se_mesh_t m, double* u, int mask, void* stream) {
  SE_CHECK(m && u, SE_EINVAL, "se_gs: null argument");
  return gs_apply<double>(m->fine, u, mask != 0, as_stream(stream, m->stream));
}

}  // extern "C"
