// FP64 local Ax with even-odd folded line contractions (even N).
//
// The GLL derivative matrix is centro-antisymmetric, D[N-1-k][N-1-l] = -D[k][l] (and so is its
// transpose).  For a line v of N values let e_l = v_l + v_{N-1-l}, o_l = v_l - v_{N-1-l}
// (l < H = N/2) and Ep[k][l] = (D[k][l] + D[k][N-1-l])/2, Om[k][l] = (D[k][l] - D[k][N-1-l])/2;
// then with E_k = sum_l Ep[k][l] e_l and O_k = sum_l Om[k][l] o_l (k < H):
//   (D v)_k = E_k + O_k,   (D v)_{N-1-k} = O_k - E_k.
// A line costs N^2/2 FMAs + 2N adds instead of N^2 FMAs.  GB300 runs FP64 at 2 FMA/clk/SM, so
// this kernel is bound by the FP64 pipe; shared memory (all lines and intermediates of the element
// are staged there) has ample headroom.  Same sum factorisation as ax_local_kernel:
//   (ur, us, ut) = (D_r u, D_s u, D_t u);  w = G (ur, us, ut);  y = D_r^T wr + D_s^T ws + D_t^T wt.
// The arithmetic type T is double, or df64 (double-float on the FP32 pipe, about 48 bits): u and
// y stay FP64 in memory either way; the df64 instance reads df64 copies of G and the tables.
#include "se_internal.h"

namespace se {

template <int N, typename T>
__device__ __forceinline__ void eo_line(const T* __restrict__ Ep, const T* __restrict__ Om,
                                        const T (&v)[N], T (&out)[N]) {
  constexpr int H = N / 2;
  T e[H], o[H];
#pragma unroll
  for (int l = 0; l < H; ++l) {
    e[l] = v[l] + v[N - 1 - l];
    o[l] = v[l] - v[N - 1 - l];
  }
#pragma unroll
  for (int k = 0; k < H; ++k) {
    T E = T(0.0), O = T(0.0);
#pragma unroll
    for (int l = 0; l < H; ++l) {
      E = fma(Ep[k * H + l], e[l], E);
      O = fma(Om[k * H + l], o[l], O);
    }
    out[k] = E + O;
    out[N - 1 - k] = O - E;
  }
}

// One line contraction from shared memory to shared memory: points base + stride * l.
// df64: the output index loop is not unrolled and each output pair goes straight to shared
// memory, so the folded tables are not held in registers across the six contractions (the
// unrolled form needs 128 registers in df64 and limits the SM to 16 warps).
template <int N, bool ACC, typename T>
__device__ __forceinline__ void eo_apply(const T* __restrict__ Ep, const T* __restrict__ Om,
                                         const T* src, T* dst, int base, int stride) {
  T v[N];
#pragma unroll
  for (int l = 0; l < N; ++l) v[l] = src[base + stride * l];
  if constexpr (is_df64<T>::value) {
    constexpr int H = N / 2;
    T e[H], o[H];
#pragma unroll
    for (int l = 0; l < H; ++l) {
      e[l] = v[l] + v[N - 1 - l];
      o[l] = v[l] - v[N - 1 - l];
    }
#pragma unroll 1
    for (int k = 0; k < H; ++k) {
      df_acc AE, AO;
#pragma unroll
      for (int l = 0; l < H; ++l) {
        df_acc_fma(AE, Ep[k * H + l], e[l]);
        df_acc_fma(AO, Om[k * H + l], o[l]);
      }
      const T E = df_acc_value(AE), O = df_acc_value(AO);
      T* d0 = dst + base + stride * k;
      T* d1 = dst + base + stride * (N - 1 - k);
      if constexpr (ACC) {
        *d0 = *d0 + (E + O);
        *d1 = *d1 + (O - E);
      } else {
        *d0 = E + O;
        *d1 = O - E;
      }
    }
  } else {
    T out[N];
    eo_line<N>(Ep, Om, v, out);
#pragma unroll
    for (int l = 0; l < N; ++l) {
      if constexpr (ACC) dst[base + stride * l] += out[l];
      else dst[base + stride * l] = out[l];
    }
  }
}

// tables: [0] Ep(D), [1] Om(D), [2] Ep(D^T), [3] Om(D^T), each H*H
// FOLD (T = double): the block's elements are consecutive in the element numbering, so
// neighbours along x (same row of the lattice, nx elements per row) are usually in the same
// block.  The kernel then also does the x part of QQ^T for them: both copies of each such
// x-interface node get left + right (the same bits on both sides), and it applies the Dirichlet
// mask (bit f of `bits`: face f = x0, x1, y0, y1, z0, z1 is Dirichlet); the x-interfaces between
// consecutive blocks are left to gs_fold_fixup_x.
// SCALE (with FOLD): the input is dinv .* u, formed as it is loaded (the first step of a
// Jacobi-Chebyshev smoother applies A to D^-1 r without storing D^-1 r).
template <int N, typename T, bool FOLD = false, bool SCALE = false>
__global__ void __launch_bounds__(512) ax_eo_kernel(int64_t E, int NE, const double* __restrict__ u,
                                                    const T* __restrict__ G, int64_t L,
                                                    const T* __restrict__ tables,
                                                    double* __restrict__ y,
                                                    const uint8_t* __restrict__ pflag,
                                                    const double* __restrict__ sub, int nx = 0,
                                                    int ny = 0, int nz = 0, int bits = 0,
                                                    const double* __restrict__ dinv = nullptr) {
  constexpr int N2 = N * N, N3 = N * N * N, H = N / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tab = reinterpret_cast<T*>(smem_raw);                    // 4 H^2
  const int le = threadIdx.x / N2;
  const int t = threadIdx.x - le * N2;
  T* su = tab + 4 * H * H + (size_t)le * 4 * N3;
  T* sr = su + N3;
  T* ss = sr + N3;
  T* st = ss + N3;
  T* sy = su;  // u is dead once the forward contractions are done
  for (int q = threadIdx.x; q < 4 * H * H; q += blockDim.x) tab[q] = tables[q];
  const int64_t e = (int64_t)blockIdx.x * NE + le;
  const bool valid = (le < NE) && (e < E);
  const int64_t eb = e * N3;
  if (valid) {
#pragma unroll
    for (int q = 0; q < N; ++q) {
      if constexpr (SCALE) su[t + N2 * q] = u[eb + t + N2 * q] * dinv[eb + t + N2 * q];
      else su[t + N2 * q] = from_io<T>(u[eb + t + N2 * q]);
    }
  }
  __syncthreads();
  const T* EpD = tab;
  const T* OmD = tab + H * H;
  const T* EpT = tab + 2 * H * H;
  const T* OmT = tab + 3 * H * H;
  const int a = t % N, b = t / N;
  if (valid) {
    eo_apply<N, false>(EpD, OmD, su, sr, N * a + N2 * b, 1);   // r-lines (j = a, k = b)
    eo_apply<N, false>(EpD, OmD, su, ss, a + N2 * b, N);       // s-lines (i = a, k = b)
    eo_apply<N, false>(EpD, OmD, su, st, a + N * b, N2);       // t-lines (i = a, j = b)
  }
  __syncthreads();
  // pointwise geometric factors: points t + N2 q
  if (valid) {
#pragma unroll
    for (int q = 0; q < N; ++q) {
      const int pt = t + N2 * q;
      const int64_t gi = eb + pt;
      const T ur = sr[pt], us = ss[pt], ut = st[pt];
      const T grr = G[gi], grs = G[L + gi], grt = G[2 * L + gi];
      const T gss = G[3 * L + gi], gst = G[4 * L + gi], gtt = G[5 * L + gi];
      sr[pt] = fma(grt, ut, fma(grs, us, grr * ur));
      ss[pt] = fma(gst, ut, fma(gss, us, grs * ur));
      st[pt] = fma(gtt, ut, fma(gst, us, grt * ur));
    }
  }
  __syncthreads();
  // transposed contractions: y = D_r^T wr (r-lines), then += D_s^T ws, then += D_t^T wt
  if (valid) eo_apply<N, false>(EpT, OmT, sr, sy, N * a + N2 * b, 1);
  __syncthreads();
  if (valid) eo_apply<N, true>(EpT, OmT, ss, sy, a + N2 * b, N);
  __syncthreads();
  if (valid) eo_apply<N, true>(EpT, OmT, st, sy, a + N * b, N2);
  __syncthreads();
  if constexpr (FOLD) {
    static_assert(sizeof(T) == sizeof(double), "the folded output is FP64");
    // the kernel is bound by the FP64 pipe, where a warp instruction costs the same with 2 or 32
    // lanes active: each interface pair is added once, by one lane of densely packed warps, and
    // the weights 2^-(interfaces) of the residual form are built from their exponent bits
    double* so0 = reinterpret_cast<double*>(tab + 4 * H * H);  // element 0 of the block
    double* so = reinterpret_cast<double*>(sy);
    // thread (le, t = i + N j) holds the points (i, j, k) of its element, k = 0..N-1; its place
    // in the lattice gives the multiplicity (a copy on an interior interface normal to a
    // direction has 2 copies along it) and the Dirichlet mask
    const int i = t % N, j = t / N;
    const int ei = (int)e;  // E < 2^31
    const int ex = ei % nx, ey = (ei / nx) % ny, ez = ei / (nx * ny);
    if (sub) {  // residual form: each copy's b / multiplicity - (A_L u), in place
      if (valid) {
        const int xy = (int)((i == 0 && ex > 0) || (i == N - 1 && ex < nx - 1)) +
                       (int)((j == 0 && ey > 0) || (j == N - 1 && ey < ny - 1));
#pragma unroll
        for (int q = 0; q < N; ++q) {
          const int pt = t + N2 * q;
          const int zin = (int)((q == 0 && ez > 0) || (q == N - 1 && ez < nz - 1));
          const double w = __longlong_as_double((long long)(1023 - xy - zin) << 52);
          so[pt] = sub[eb + pt] * w - so[pt];
        }
      }
      __syncthreads();
    }
    // x-interfaces inside the block: (N - 1, j, k) of element lp and (0, j, k) of lp + 1 when
    // both lie in one row; both copies get left + right
    const int64_t e0 = (int64_t)blockIdx.x * NE;
    for (int idx = threadIdx.x; idx < (NE - 1) * N2; idx += blockDim.x) {
      const int lp = idx / N2, jk = idx - lp * N2;
      const int el = (int)(e0 + lp);
      if (el + 1 < E && el % nx < nx - 1) {
        double* a = so0 + lp * 4 * N3 + (N - 1) + N * jk;
        double* b = a + 4 * N3 - (N - 1);
        const double v = *a + *b;
        *a = v;
        *b = v;
      }
    }
    __syncthreads();
    if (valid) {
      const bool dxy = ((bits & 1) && i == 0 && ex == 0) || ((bits & 2) && i == N - 1 && ex == nx - 1) ||
                       ((bits & 4) && j == 0 && ey == 0) || ((bits & 8) && j == N - 1 && ey == ny - 1);
#pragma unroll
      for (int q = 0; q < N; ++q) {
        const bool dz = ((bits & 16) && q == 0 && ez == 0) || ((bits & 32) && q == N - 1 && ez == nz - 1);
        y[eb + t + N2 * q] = (dxy || dz) ? 0.0 : so[t + N2 * q];
      }
    }
  } else {
    if (valid) {
#pragma unroll
      for (int q = 0; q < N; ++q)
        y[eb + t + N2 * q] = ax_output(io_cast<double>(sy[t + N2 * q]), sub, pflag, eb + t + N2 * q);
    }
  }
}

// The x-interfaces that ax_eo_kernel<FOLD> leaves: element e = (b + 1) NE - 1, the last of block b,
// and e + 1, the first of block b + 1, when both lie in one row.  Thread: (boundary, point (j, k)
// of the face).  Masked copies are zero on both sides (a node's copies are all masked or none).
template <int N>
__global__ void gs_fold_fixup_x(int64_t E, int NE, int nx, double* __restrict__ y) {
  constexpr int N2 = N * N, N3 = N2 * N;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nbnd = (E + NE - 1) / NE - 1;
  if (t >= nbnd * N2) return;
  const int64_t b = t / N2;
  const int jk = (int)(t - b * N2);
  const int64_t e = (b + 1) * NE - 1;
  if (e + 1 >= E || (int)(e % nx) == nx - 1) return;
  const int64_t ia = e * N3 + (N - 1) + (int64_t)N * jk;  // (N - 1, j, k) of e
  const int64_t ib = (e + 1) * N3 + (int64_t)N * jk;      // (0, j, k) of e + 1
  const double v = y[ia] + y[ib];
  y[ia] = v;
  y[ib] = v;
}

template <int N, bool SCALE>
static int launch_ax_eo_fold_t(const Level& lv, const double* u, double* y, const double* sub, int NE,
                               const double* dinv, cudaStream_t s) {
  constexpr int H = N / 2;
  const int threads = NE * N * N;
  const size_t smem = (4 * H * H + (size_t)NE * 4 * N * N * N) * sizeof(double);
  static const cudaError_t attr = cudaFuncSetAttribute(
      ax_eo_kernel<N, double, true, SCALE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  SE_CUDA(attr);
  const unsigned blocks = (unsigned)((lv.E + NE - 1) / NE);
  int bits = 0;
  for (int f = 0; f < 6; ++f)
    if (lv.bc[f] == SE_BC_DIRICHLET) bits |= 1 << f;
  ax_eo_kernel<N, double, true, SCALE><<<blocks, threads, smem, s>>>(
      lv.E, NE, u, lv.G64, lv.L, lv.eo64, y, lv.pflag, sub, lv.nel[0], lv.nel[1], lv.nel[2], bits, dinv);
  SE_LAUNCH_CHECK();
  return SE_OK;
}

template <int N>
static int launch_ax_eo_fold(const Level& lv, const double* u, double* y, const double* sub, int NE,
                             cudaStream_t s, const double* dinv) {
  return dinv ? launch_ax_eo_fold_t<N, true>(lv, u, y, sub, NE, dinv, s)
              : launch_ax_eo_fold_t<N, false>(lv, u, y, sub, NE, nullptr, s);
}

template <int N, typename T>
static int launch_ax_eo(const Level& lv, const double* u, double* y, const T* G, const T* tables,
                        const double* sub, cudaStream_t s) {
  constexpr int H = N / 2;
  const int NE = ax_elems_per_block(N - 1, false);
  const int threads = NE * N * N;
  const size_t smem = (4 * H * H + (size_t)NE * 4 * N * N * N) * sizeof(T);
  static const cudaError_t attr = cudaFuncSetAttribute(
      ax_eo_kernel<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  SE_CUDA(attr);
  const unsigned blocks = (unsigned)((lv.E + NE - 1) / NE);
  ax_eo_kernel<N, T><<<blocks, threads, smem, s>>>(lv.E, NE, u, G, lv.L, tables, y, lv.pflag, sub);
  SE_LAUNCH_CHECK();
  return SE_OK;
}

bool ax_eo_supported(int p) { return (p + 1) % 2 == 0 && p + 1 >= 2 && p + 1 <= 10; }

// Folded tables of D and D^T for even N (host, FP64).
void ax_eo_tables(const Basis1D& b, double* out) {
  const int N = b.p + 1, H = N / 2;
  for (int tr = 0; tr < 2; ++tr)
    for (int k = 0; k < H; ++k)
      for (int l = 0; l < H; ++l) {
        auto Dm = [&](int r, int c) { return tr ? b.D[c * N + r] : b.D[r * N + c]; };
        out[(2 * tr) * H * H + k * H + l] = 0.5 * (Dm(k, l) + Dm(k, N - 1 - l));
        out[(2 * tr + 1) * H * H + k * H + l] = 0.5 * (Dm(k, l) - Dm(k, N - 1 - l));
      }
}

template <typename T>
static int ax_eo_dispatch(const Level& lv, const double* u, double* y, const T* G, const T* tab,
                          cudaStream_t s, const double* sub) {
  switch (lv.N) {
    case 2: return launch_ax_eo<2, T>(lv, u, y, G, tab, sub, s);
    case 4: return launch_ax_eo<4, T>(lv, u, y, G, tab, sub, s);
    case 6: return launch_ax_eo<6, T>(lv, u, y, G, tab, sub, s);
    case 8: return launch_ax_eo<8, T>(lv, u, y, G, tab, sub, s);
    case 10: return launch_ax_eo<10, T>(lv, u, y, G, tab, sub, s);
    default: set_error("ax_eo: unsupported N=%d", lv.N); return SE_EINVAL;
  }
}

int ax_local_eo(const Level& lv, const double* u, double* y, cudaStream_t s, const double* sub) {
  SE_CHECK(lv.eo64 != nullptr, SE_EINVAL, "ax_eo: folded tables missing");
  return ax_eo_dispatch<double>(lv, u, y, lv.G64, lv.eo64, s, sub);
}

int ax_local_eo_fold(const Level& lv, const double* u, double* y, const double* sub, int NE,
                     cudaStream_t s, const double* dinv) {
  SE_CHECK(lv.eo64 != nullptr && lv.nel[0] >= 1, SE_EINVAL, "ax_eo_fold: folded tables or lattice missing");
  switch (lv.N) {
    case 2: return launch_ax_eo_fold<2>(lv, u, y, sub, NE, s, dinv);
    case 4: return launch_ax_eo_fold<4>(lv, u, y, sub, NE, s, dinv);
    case 6: return launch_ax_eo_fold<6>(lv, u, y, sub, NE, s, dinv);
    case 8: return launch_ax_eo_fold<8>(lv, u, y, sub, NE, s, dinv);
    case 10: return launch_ax_eo_fold<10>(lv, u, y, sub, NE, s, dinv);
    default: set_error("ax_eo_fold: unsupported N=%d", lv.N); return SE_EINVAL;
  }
}

int gs_fold_fixup(const Level& lv, double* y, int NE, cudaStream_t s) {
  const int64_t nbnd = (lv.E + NE - 1) / NE - 1;
  if (nbnd <= 0 || lv.nel[0] <= 1) return SE_OK;
  const int64_t n = nbnd * lv.N * lv.N;
  switch (lv.N) {
#define SE_FIX_CASE(NN)                                                                      \
  case NN:                                                                                   \
    gs_fold_fixup_x<NN><<<grid_for(n, 256), 256, 0, s>>>(lv.E, NE, lv.nel[0], y);            \
    break;
    SE_FIX_CASE(2) SE_FIX_CASE(4) SE_FIX_CASE(6) SE_FIX_CASE(8) SE_FIX_CASE(10)
#undef SE_FIX_CASE
    default: set_error("gs_fold_fixup: unsupported N=%d", lv.N); return SE_EINVAL;
  }
  SE_LAUNCH_CHECK();
  return SE_OK;
}

int ax_local_eo_df(const Level& lv, const double* u, double* y, cudaStream_t s, const double* sub) {
  SE_CHECK(lv.Gdf != nullptr && lv.eodf != nullptr, SE_EINVAL, "ax_eo_df: df64 geometry missing");
  return ax_eo_dispatch<df64>(lv, u, y, lv.Gdf, lv.eodf, s, sub);
}

__global__ void split_df_kernel(int64_t n, const double* __restrict__ a, df64* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = df64(a[i]);
}

int split_df(const double* a, df64* b, int64_t n, cudaStream_t s) {
  if (n <= 0) return SE_OK;
  split_df_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, a, b);
  SE_LAUNCH_CHECK();
  return SE_OK;
}

int make_df_geometry(Level& lv, Allocs& allocs, cudaStream_t s) {
  const bool eo = ax_eo_supported(lv.p) && lv.eo64;
  if (lv.Gdf && (eo ? lv.eodf != nullptr : lv.Ddf != nullptr)) return SE_OK;
  if (!lv.Gdf) {
    SE_TRY(dmalloc(allocs, &lv.Gdf, 6 * (size_t)lv.L));
    SE_TRY(split_df(lv.G64, lv.Gdf, 6 * lv.L, s));
  }
  if (eo && !lv.eodf) {
    const int H = lv.N / 2;
    SE_TRY(dmalloc(allocs, &lv.eodf, 4 * (size_t)H * H));
    SE_TRY(split_df(lv.eo64, lv.eodf, 4 * H * H, s));
  }
  if (!eo && !lv.Ddf) {
    SE_TRY(dmalloc(allocs, &lv.Ddf, (size_t)lv.N * lv.N));
    SE_TRY(split_df(lv.D64, lv.Ddf, (int64_t)lv.N * lv.N, s));
  }
  // made once and then read from any stream: complete before the first use
  SE_CUDA(cudaStreamSynchronize(s));
  return SE_OK;
}

}  // namespace se
