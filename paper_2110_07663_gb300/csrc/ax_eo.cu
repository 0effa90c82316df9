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
#include "se_internal.h"

namespace se {

template <int N>
__device__ __forceinline__ void eo_line(const double* __restrict__ Ep, const double* __restrict__ Om,
                                        const double (&v)[N], double (&out)[N]) {
  constexpr int H = N / 2;
  double e[H], o[H];
#pragma unroll
  for (int l = 0; l < H; ++l) {
    e[l] = v[l] + v[N - 1 - l];
    o[l] = v[l] - v[N - 1 - l];
  }
#pragma unroll
  for (int k = 0; k < H; ++k) {
    double E = 0.0, O = 0.0;
#pragma unroll
    for (int l = 0; l < H; ++l) {
      E = fma(Ep[k * H + l], e[l], E);
      O = fma(Om[k * H + l], o[l], O);
    }
    out[k] = E + O;
    out[N - 1 - k] = O - E;
  }
}

// tables: [0] Ep(D), [1] Om(D), [2] Ep(D^T), [3] Om(D^T), each H*H
template <int N>
__global__ void __launch_bounds__(512) ax_eo_kernel(int64_t E, int NE, const double* __restrict__ u,
                                                    const double* __restrict__ G, int64_t L,
                                                    const double* __restrict__ tables,
                                                    double* __restrict__ y,
                                                    const uint8_t* __restrict__ pflag,
                                                    const double* __restrict__ sub) {
  constexpr int N2 = N * N, N3 = N * N * N, H = N / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* tab = reinterpret_cast<double*>(smem_raw);          // 4 H^2
  const int le = threadIdx.x / N2;
  const int t = threadIdx.x - le * N2;
  double* su = tab + 4 * H * H + (size_t)le * 5 * N3;
  double* sr = su + N3;
  double* ss = sr + N3;
  double* st = ss + N3;
  double* sy = st + N3;
  for (int q = threadIdx.x; q < 4 * H * H; q += blockDim.x) tab[q] = tables[q];
  const int64_t e = (int64_t)blockIdx.x * NE + le;
  const bool valid = (le < NE) && (e < E);
  const int64_t eb = e * N3;
  if (valid) {
#pragma unroll
    for (int q = 0; q < N; ++q) su[t + N2 * q] = u[eb + t + N2 * q];
  }
  __syncthreads();
  const double* EpD = tab;
  const double* OmD = tab + H * H;
  const double* EpT = tab + 2 * H * H;
  const double* OmT = tab + 3 * H * H;
  const int a = t % N, b = t / N;
  double v[N], out[N];
  if (valid) {
    // r-lines (j = a, k = b)
#pragma unroll
    for (int l = 0; l < N; ++l) v[l] = su[l + N * a + N2 * b];
    eo_line<N>(EpD, OmD, v, out);
#pragma unroll
    for (int l = 0; l < N; ++l) sr[l + N * a + N2 * b] = out[l];
    // s-lines (i = a, k = b)
#pragma unroll
    for (int l = 0; l < N; ++l) v[l] = su[a + N * l + N2 * b];
    eo_line<N>(EpD, OmD, v, out);
#pragma unroll
    for (int l = 0; l < N; ++l) ss[a + N * l + N2 * b] = out[l];
    // t-lines (i = a, j = b)
#pragma unroll
    for (int l = 0; l < N; ++l) v[l] = su[a + N * b + N2 * l];
    eo_line<N>(EpD, OmD, v, out);
#pragma unroll
    for (int l = 0; l < N; ++l) st[a + N * b + N2 * l] = out[l];
  }
  __syncthreads();
  // pointwise geometric factors: points t + N2 q
  if (valid) {
#pragma unroll
    for (int q = 0; q < N; ++q) {
      const int pt = t + N2 * q;
      const int64_t gi = eb + pt;
      const double ur = sr[pt], us = ss[pt], ut = st[pt];
      const double grr = G[gi], grs = G[L + gi], grt = G[2 * L + gi];
      const double gss = G[3 * L + gi], gst = G[4 * L + gi], gtt = G[5 * L + gi];
      sr[pt] = grr * ur + grs * us + grt * ut;
      ss[pt] = grs * ur + gss * us + gst * ut;
      st[pt] = grt * ur + gst * us + gtt * ut;
    }
  }
  __syncthreads();
  // transposed contractions: y = D_r^T wr (r-lines), then += D_s^T ws, then += D_t^T wt
  if (valid) {
#pragma unroll
    for (int l = 0; l < N; ++l) v[l] = sr[l + N * a + N2 * b];
    eo_line<N>(EpT, OmT, v, out);
#pragma unroll
    for (int l = 0; l < N; ++l) sy[l + N * a + N2 * b] = out[l];
  }
  __syncthreads();
  if (valid) {
#pragma unroll
    for (int l = 0; l < N; ++l) v[l] = ss[a + N * l + N2 * b];
    eo_line<N>(EpT, OmT, v, out);
#pragma unroll
    for (int l = 0; l < N; ++l) sy[a + N * l + N2 * b] += out[l];
  }
  __syncthreads();
  if (valid) {
#pragma unroll
    for (int l = 0; l < N; ++l) v[l] = st[a + N * b + N2 * l];
    eo_line<N>(EpT, OmT, v, out);
#pragma unroll
    for (int l = 0; l < N; ++l) sy[a + N * b + N2 * l] += out[l];
  }
  __syncthreads();
  if (valid) {
#pragma unroll
    for (int q = 0; q < N; ++q) y[eb + t + N2 * q] = ax_output(sy[t + N2 * q], sub, pflag, eb + t + N2 * q);
  }
}

template <int N>
static int launch_ax_eo(const Level& lv, const double* u, double* y, const double* tables,
                        const double* sub, cudaStream_t s) {
  constexpr int H = N / 2;
  const int NE = ax_elems_per_block(N - 1, false);
  const int threads = NE * N * N;
  const size_t smem = (4 * H * H + (size_t)NE * 5 * N * N * N) * sizeof(double);
  static const cudaError_t attr =
      cudaFuncSetAttribute(ax_eo_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  SE_CUDA(attr);
  const unsigned blocks = (unsigned)((lv.E + NE - 1) / NE);
  ax_eo_kernel<N><<<blocks, threads, smem, s>>>(lv.E, NE, u, lv.G64, lv.L, tables, y, lv.pflag, sub);
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

int ax_local_eo(const Level& lv, const double* u, double* y, cudaStream_t s, const double* sub) {
  SE_CHECK(lv.eo64 != nullptr, SE_EINVAL, "ax_eo: folded tables missing");
  switch (lv.N) {
    case 2: return launch_ax_eo<2>(lv, u, y, lv.eo64, sub, s);
    case 4: return launch_ax_eo<4>(lv, u, y, lv.eo64, sub, s);
    case 6: return launch_ax_eo<6>(lv, u, y, lv.eo64, sub, s);
    case 8: return launch_ax_eo<8>(lv, u, y, lv.eo64, sub, s);
    case 10: return launch_ax_eo<10>(lv, u, y, lv.eo64, sub, s);
    default: set_error("ax_eo: unsupported N=%d", lv.N); return SE_EINVAL;
  }
}

}  // namespace se
