// Overlapping Schwarz smoother with fast-diagonalisation local solves (Sec. 2.2.2, eqs 4-9).
//
// Set-up: for every element and direction, the extended 1D stiffness/mass pair over
// [left neighbour, element, right neighbour] (box lengths from the mapped corners), restricted to
// the pbar = p+3 window points, is diagonalised on the GPU (one thread per problem, cyclic
// Jacobi rotations on B^-1/2 A B^-1/2): S^T A S = Lambda, S^T B S = I (eqs 6-7).
// Apply: each block gathers its element's pbar^3 window of the assembled residual (own nodes
// plus one layer from up to 26 neighbours, zero outside the domain), applies
// (S_z x S_y x S_x) D^-1 (S_z^T x S_y^T x S_x^T) (eqs 8-9) with the three tensor directions as
// line contractions in shared memory, and writes either the own nodes weighted by
// 1/multiplicity (restrictive additive Schwarz; QQ^T follows) or the whole window (additive
// Schwarz, combined by a gather over the covering windows).
#include <cmath>

#include "se_internal.h"

namespace se {

constexpr int PB_MAX = SE_MAX_ORDER + 3;

// ------------------------------------------------------------------ set-up
__device__ void jacobi_eigen(int n, double* A, double* V) {
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) V[a * n + b] = a == b ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, dg = 0.0;
    for (int a = 0; a < n; ++a) {
      dg += A[a * n + a] * A[a * n + a];
      for (int b = a + 1; b < n; ++b) off += A[a * n + b] * A[a * n + b];
    }
    if (off <= 1e-34 * dg) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[p * n + q];
        if (fabs(apq) < 1e-300) continue;
        // The angle needs no FP64 accuracy (a rotation that leaves a small a_pq is followed by
        // the next sweep's), only the rotation's orthogonality does: t from FP32 operations
        // (where the quotient of two doubles' difference underflows or overflows in FP32, the
        // FP64 form), then c = 1/sqrt(1 + t^2) and s = t c in FP64.  On this part FP64 division
        // and square root are long instruction sequences on the narrow FP64 pipe.
        const double dq = A[q * n + q] - A[p * n + p], e2 = 2.0 * apq;
        double t;
        float thf = 0.0f;
        const bool f32 = fabs(e2) >= 1e-30 && fabs(e2) <= 1e30 && fabs(dq) <= 1e30 &&
                         isfinite(thf = (float)dq / (float)e2);
        if (f32) {
          t = (double)(copysignf(1.0f, thf) / (fabsf(thf) + sqrtf(fmaf(thf, thf, 1.0f))));
        } else {
          const double theta = dq / e2;
          t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        }
        const double c = rsqrt(fma(t, t, 1.0)), s = t * c;
        for (int k = 0; k < n; ++k) {
          const double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          const double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
}

// One thread per (element, direction).  Window point q (0..p+2) is point p-1+q of the
// 3-element 1D assembly (left: 0..p, own: p..2p, right: 2p..3p).
__global__ void fdm_setup_kernel(int P, int64_t E, const int* __restrict__ nbr,
                                 const double* __restrict__ len, const double* __restrict__ Ke,
                                 const double* __restrict__ wq, int bcbits,
                                 double* __restrict__ S, double* __restrict__ lam) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * E) return;
  const int64_t e = t / 3;
  const int d = (int)(t - 3 * e);
  const int N = P + 1, PB = P + 3;
  const int stride = d == 0 ? 1 : (d == 1 ? 3 : 9);
  const int nl = nbr[27 * e + 13 - stride], nr = nbr[27 * e + 13 + stride];
  const bool hl = nl >= 0, hr = nr >= 0;
  const bool dl = (bcbits >> (2 * d)) & 1, dr = (bcbits >> (2 * d + 1)) & 1;
  const double lseg[3] = {hl ? len[3 * nl + d] : 0.0, len[3 * e + d], hr ? len[3 * nr + d] : 0.0};
  const bool seg_on[3] = {hl, true, hr};
  int act[PB_MAX];
  int n = 0;
  for (int q = 0; q < PB; ++q) {
    if (q == 0 && !hl) continue;
    if (q == PB - 1 && !hr) continue;
    if (q == 1 && !hl && dl) continue;
    if (q == PB - 2 && !hr && dr) continue;
    act[n++] = q;
  }
  double A[PB_MAX * PB_MAX], V[PB_MAX * PB_MAX], bi[PB_MAX];
  for (int a = 0; a < n; ++a) {
    const int wa = P - 1 + act[a];
    double bsum = 0.0;
    for (int sg = 0; sg < 3; ++sg) {
      const int o = sg * P;
      if (seg_on[sg] && wa >= o && wa <= o + P) bsum += 0.5 * lseg[sg] * wq[wa - o];
    }
    bi[a] = 1.0 / sqrt(bsum);
  }
  for (int a = 0; a < n; ++a) {
    const int wa = P - 1 + act[a];
    for (int b = 0; b < n; ++b) {
      const int wb = P - 1 + act[b];
      double v = 0.0;
      for (int sg = 0; sg < 3; ++sg) {
        const int o = sg * P;
        if (seg_on[sg] && wa >= o && wa <= o + P && wb >= o && wb <= o + P)
          v += (2.0 / lseg[sg]) * Ke[(wa - o) * N + (wb - o)];
      }
      A[a * n + b] = bi[a] * v * bi[b];
    }
  }
  jacobi_eigen(n, A, V);
  double* Se = S + (3 * e + d) * PB * PB;
  double* le = lam + (3 * e + d) * PB;
  for (int q = 0; q < PB * PB; ++q) Se[q] = 0.0;
  for (int m = 0; m < PB; ++m) le[m] = m < n ? A[m * n + m] : 1.0;
  for (int a = 0; a < n; ++a)
    for (int m = 0; m < n; ++m) Se[act[a] * PB + m] = bi[a] * V[a * n + m];
}

// 1/(lam_x[a] + lam_y[b] + lam_z[c]) per element window point (the paper's D^-1 storage).
__global__ void fdm_dinv_kernel(int PB, int64_t E, const double* __restrict__ lam,
                                double* __restrict__ dinv) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int PB3 = PB * PB * PB;
  if (t >= E * PB3) return;
  const int64_t e = t / PB3;
  const int q = (int)(t - e * PB3);
  const int a = q % PB, b = (q / PB) % PB, c = q / (PB * PB);
  const double* l = lam + 3 * e * PB;
  dinv[t] = 1.0 / (l[a] + l[PB + b] + l[2 * PB + c]);
}

template <class T>
__global__ void cast_kernel(int64_t n, const double* __restrict__ a, T* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (T)a[i];
}

int fdm_setup(const se_mesh_s* m, Level& lv, Allocs& allocs, bool want32, cudaStream_t s,
              bool want_df) {
  const int P = lv.p, N = P + 1, PB = P + 3;
  const int64_t E = lv.E;
  // 1D GLL stiffness D^T W D (reference element)
  double Ke[(SE_MAX_ORDER + 1) * (SE_MAX_ORDER + 1)];
  for (int a = 0; a < N; ++a)
    for (int b = 0; b < N; ++b) {
      double v = 0.0;
      for (int q = 0; q < N; ++q) v += lv.basis.D[q * N + a] * lv.basis.w[q] * lv.basis.D[q * N + b];
      Ke[a * N + b] = v;
    }
  double *dKe = nullptr, *dw = nullptr, *dlen = nullptr;
  SE_TRY(dmalloc(allocs, &dKe, N * N));
  SE_TRY(dmalloc(allocs, &dw, N));
  SE_TRY(dmalloc(allocs, &dlen, 3 * E));
  SE_TRY(h2d(dKe, Ke, N * N * sizeof(double), s));
  SE_TRY(h2d(dw, lv.basis.w, N * sizeof(double), s));
  SE_TRY(h2d(dlen, m->box_len.data(), 3 * E * sizeof(double), s));
  SE_TRY(dmalloc(allocs, &lv.S64, 3 * E * PB * PB));
  SE_TRY(dmalloc(allocs, &lv.lam64, 3 * E * PB));
  int bits = 0;
  for (int f = 0; f < 6; ++f)
    if (lv.bc[f] == SE_BC_DIRICHLET) bits |= 1 << f;
  fdm_setup_kernel<<<grid_for(3 * E, 64), 64, 0, s>>>(P, E, lv.nbr, dlen, dKe, dw, bits, lv.S64,
                                                      lv.lam64);
  SE_LAUNCH_CHECK();
  const int64_t n3 = E * PB * PB * PB;
  SE_TRY(dmalloc(allocs, &lv.fdm_dinv64, n3));
  fdm_dinv_kernel<<<grid_for(n3, 256), 256, 0, s>>>(PB, E, lv.lam64, lv.fdm_dinv64);
  SE_LAUNCH_CHECK();
  if (want32) {
    SE_TRY(dmalloc(allocs, &lv.S32, 3 * E * PB * PB));
    SE_TRY(dmalloc(allocs, &lv.lam32, 3 * E * PB));
    cast_kernel<float><<<grid_for(3 * E * PB * PB, 256), 256, 0, s>>>(3 * E * PB * PB, lv.S64, lv.S32);
    cast_kernel<float><<<grid_for(3 * E * PB, 256), 256, 0, s>>>(3 * E * PB, lv.lam64, lv.lam32);
    SE_LAUNCH_CHECK();
  }
  if (want_df) {
    SE_TRY(dmalloc(allocs, &lv.Sdf, 3 * E * PB * PB));
    SE_TRY(dmalloc(allocs, &lv.lamdf, 3 * E * PB));
    SE_TRY(split_df(lv.S64, lv.Sdf, 3 * E * PB * PB, s));
    SE_TRY(split_df(lv.lam64, lv.lamdf, 3 * E * PB, s));
  }
  return SE_OK;
}

// ------------------------------------------------------------------ apply
enum { FDM_RAS = 0, FDM_FULL = 1, FDM_EXT_IN = 2, FDM_GATHER = 3 };

// Window point (a, b, c) of element e: neighbour slot and local index in that element.
template <int P>
__device__ __forceinline__ int64_t window_source(const int* __restrict__ nb, int64_t e, int a,
                                                 int b, int c) {
  constexpr int N = P + 1, PB = P + 3;
  const int da = a == 0 ? -1 : (a == PB - 1 ? 1 : 0);
  const int db = b == 0 ? -1 : (b == PB - 1 ? 1 : 0);
  const int dc = c == 0 ? -1 : (c == PB - 1 ? 1 : 0);
  int64_t src = e;
  if (da | db | dc) {
    src = nb[(da + 1) + 3 * (db + 1) + 9 * (dc + 1)];
    if (src < 0) return -1;
  }
  const int ia = da < 0 ? P - 1 : (da > 0 ? 1 : a - 1);
  const int ib = db < 0 ? P - 1 : (db > 0 ? 1 : b - 1);
  const int ic = dc < 0 ? P - 1 : (dc > 0 ? 1 : c - 1);
  return src * (N * N * N) + ia + N * (ib + N * ic);
}

// NE elements per block.  Each contraction phase gives one thread per line of every element
// (lines numbered element-major), so active threads form a contiguous prefix and only the last
// warp of a phase can be partly idle (one element per 128-thread block left 28 of 128 lanes
// idle at p = 7).  S and S^T sit in shared memory with rows padded to a multiple of 4 entries
// and are read as 16-byte vectors (4 FP32 or 2 FP64 values per load) against register lines
// padded with zeros: the forward transform uses rows of S^T, the backward one rows of S.
template <int PB>
struct FdmDims {
  static constexpr int PBP = (PB + 3) / 4 * 4;            // padded row length
  static constexpr int PB3 = PB * PB * PB;
  static constexpr int PB3P = (PB3 + 3) / 4 * 4;           // buffer length, 16-byte multiple
  static constexpr int SROW = 3 * PB * PBP;                // S or S^T of 3 directions
};

// One FMA per multiply-add.  FP32: 16-byte loads of the padded row (the FP32 kernel is not
// ALU-bound; padding entries are zero).  FP64 (ALU-bound): scalar loads of the PB real entries.
template <int PB, int PBP, typename T>
__device__ __forceinline__ T dot_row(const T* __restrict__ row, const T (&v)[PBP]) {
  T acc = T(0);
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int a = 0; a < PBP; a += 4) {
      const float4 s = *reinterpret_cast<const float4*>(row + a);
      acc = fmaf(s.x, v[a], acc);
      acc = fmaf(s.y, v[a + 1], acc);
      acc = fmaf(s.z, v[a + 2], acc);
      acc = fmaf(s.w, v[a + 3], acc);
    }
  } else if constexpr (is_df64<T>::value) {
    // two independent accumulation chains (a df64 product-accumulate is a chain of about 10
    // dependent FP32 operations, so one chain per row would leave the FP32 pipe waiting on
    // latency), renormalised once at the end
    df_acc A0, A1;
#pragma unroll
    for (int a = 0; a + 1 < PB; a += 2) {
      // rows are padded to PBP (a multiple of 4) entries: two df64 values per 16-byte load
      const float4 q = *reinterpret_cast<const float4*>(row + a);
      df_acc_fma(A0, df64(q.x, q.y), v[a]);
      df_acc_fma(A1, df64(q.z, q.w), v[a + 1]);
    }
    if constexpr (PB % 2 == 1) df_acc_fma(A0, row[PB - 1], v[PB - 1]);
    acc = df_acc_merge(A0, A1);
  } else {
#pragma unroll
    for (int a = 0; a < PB; ++a) acc = fma(row[a], v[a], acc);
  }
  return acc;
}

// T is the arithmetic type (double, or df64: double-float on the FP32 pipe) and IO the type of
// the vectors in memory (T, or double for df64).
template <int P, typename T, int MODE, typename IO = T>
__global__ void __launch_bounds__(512) fdm_kernel(int64_t E, int NE, const int* __restrict__ nbr,
                                                  const IO* __restrict__ in,
                                                  const T* __restrict__ Sg,
                                                  const T* __restrict__ lamg,
                                                  const double* __restrict__ dinvg,
                                                  const uint8_t* __restrict__ pflag,
                                                  IO* __restrict__ out) {
  constexpr int N = P + 1, PB = P + 3, PB2 = PB * PB, PB3 = PB * PB * PB;
  using Dm = FdmDims<PB>;
  constexpr int PBP = Dm::PBP, PB3P = Dm::PB3P, SROW = Dm::SROW;
  constexpr int LAMP = (3 * PB + 3) / 4 * 4;
  constexpr int PER = 2 * PB3P + 2 * SROW + LAMP;  // shared values per element
  // output loops: fully unrolled in FP64; df64 unrolls them twice only (a df64 row dot product
  // is about 150 instructions, and the fully unrolled kernel overflows the instruction cache)
  constexpr int OUT_UNR = is_df64<T>::value ? 2 : PB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sbase = reinterpret_cast<T*>(smem_raw);
  int* snb = reinterpret_cast<int*>(sbase + (size_t)NE * PER);  // [NE][27]
  const int64_t e0 = (int64_t)blockIdx.x * NE;
  const int ne = (int)((E - e0) < NE ? (E - e0) : NE);             // elements in this block
  const int tid = threadIdx.x, nt = blockDim.x;
  auto B0 = [&](int le) { return sbase + (size_t)le * PER; };
  auto B1 = [&](int le) { return sbase + (size_t)le * PER + PB3P; };
  auto ST = [&](int le) { return sbase + (size_t)le * PER + 2 * PB3P; };          // S^T rows
  auto SR = [&](int le) { return sbase + (size_t)le * PER + 2 * PB3P + SROW; };   // S rows
  auto SL = [&](int le) { return sbase + (size_t)le * PER + 2 * PB3P + 2 * SROW; };
  if constexpr (MODE != FDM_GATHER) {
    // S[d][row][col] (row = window point, col = mode) -> S^T[d][col][row], S[d][row][col], padded
    for (int q = tid; q < ne * 3 * PB * PBP; q += nt) {
      const int le = q / (3 * PB * PBP), r = q - le * 3 * PB * PBP;
      const int d = r / (PB * PBP), rr = r - d * PB * PBP;
      const int i = rr / PBP, j = rr - i * PBP;
      const T* S = Sg + ((e0 + le) * 3 + d) * PB2;
      ST(le)[r] = j < PB ? S[j * PB + i] : T(0);
      SR(le)[r] = j < PB ? S[i * PB + j] : T(0);
    }
    for (int q = tid; q < ne * 3 * PB; q += nt) {
      const int le = q / (3 * PB), r = q - le * 3 * PB;
      SL(le)[r] = lamg[(e0 + le) * 3 * PB + r];
    }
  }
  for (int q = tid; q < ne * 27; q += nt) snb[q] = nbr[27 * e0 + q];
  __syncthreads();
  // ---- gather the extended window: one thread per (element, a, b), loop over c
  if constexpr (MODE == FDM_EXT_IN) {
    for (int q = tid; q < ne * PB3; q += nt) {
      const int le = q / PB3;
      B0(le)[q - le * PB3] = from_io<T>(in[e0 * PB3 + q]);
    }
  } else {
    if (tid < ne * PB2) {
      const int le = tid / PB2, ql = tid - le * PB2;
      const int a = ql % PB, b = ql / PB;
      T* b0 = B0(le);
      for (int c = 0; c < PB; ++c) {
        const int64_t src = window_source<P>(snb + 27 * le, e0 + le, a, b, c);
        b0[a + PB * (b + PB * c)] = src >= 0 ? from_io<T>(in[src]) : T(0);
      }
    }
  }
  if constexpr (MODE == FDM_GATHER) {
    __syncthreads();
    for (int q = tid; q < ne * PB3; q += nt) {
      const int le = q / PB3;
      out[e0 * PB3 + q] = io_cast<IO>(B0(le)[q - le * PB3]);
    }
    return;
  } else {
    __syncthreads();
    T v[PBP];
#pragma unroll
    for (int a = PB; a < PBP; ++a) v[a] = T(0);
    const bool full_line = tid < ne * PB2;
    const int le = full_line ? tid / PB2 : 0;
    const int ql = tid - le * PB2;
    const T* STx = ST(le);
    const T* STy = STx + PB * PBP;
    const T* STz = STx + 2 * PB * PBP;
    const T* SRz = SR(le) + 2 * PB * PBP;
    const T* sl = SL(le);
    T* b0 = B0(le);
    T* b1 = B1(le);
    // ---- forward: S_x^T along a (line (b, c))
    if (full_line) {
      const int b = ql % PB, c = ql / PB;
#pragma unroll
      for (int a = 0; a < PB; ++a) v[a] = b0[a + PB * (b + PB * c)];
#pragma unroll OUT_UNR
      for (int al = 0; al < PB; ++al) b1[al + PB * (b + PB * c)] = dot_row<PB, PBP>(STx + al * PBP, v);
    }
    __syncthreads();
    // ---- forward: S_y^T along b (line (alpha, c))
    if (full_line) {
      const int al = ql % PB, c = ql / PB;
#pragma unroll
      for (int b = 0; b < PB; ++b) v[b] = b1[al + PB * (b + PB * c)];
#pragma unroll OUT_UNR
      for (int be = 0; be < PB; ++be) b0[al + PB * (be + PB * c)] = dot_row<PB, PBP>(STy + be * PBP, v);
    }
    __syncthreads();
    // ---- forward: S_z^T along c, then D^-1 (line (alpha, beta))
    if (full_line) {
      const int al = ql % PB, be = ql / PB;
#pragma unroll
      for (int c = 0; c < PB; ++c) v[c] = b0[al + PB * (be + PB * c)];
      const T lxy = sl[al] + sl[PB + be];
#pragma unroll OUT_UNR
      for (int ga = 0; ga < PB; ++ga) {
        const T acc = dot_row<PB, PBP>(STz + ga * PBP, v);
        const int q = al + PB * (be + PB * ga);
        T dv;
        if constexpr (sizeof(T) == 8) dv = from_io<T>(dinvg[(e0 + le) * PB3 + q]);
        else dv = __frcp_rn(lxy + sl[2 * PB + ga]);
        b1[q] = acc * dv;
      }
    }
    __syncthreads();
    // ---- backward: S_z along gamma (own outputs c' = 1..N for RAS, all PB otherwise)
    constexpr int C0 = MODE == FDM_RAS ? 1 : 0;
    constexpr int NC = MODE == FDM_RAS ? N : PB;
    if (full_line) {
      const int al = ql % PB, be = ql / PB;
#pragma unroll
      for (int ga = 0; ga < PB; ++ga) v[ga] = b1[al + PB * (be + PB * ga)];
#pragma unroll OUT_UNR
      for (int cc = 0; cc < NC; ++cc) {
        const int c = C0 + cc;
        b0[al + PB * (be + PB * c)] = dot_row<PB, PBP>(SRz + c * PBP, v);
      }
    }
    __syncthreads();
    // ---- backward: S_y along beta (line (alpha, c'), PB*NC lines per element)
    if (tid < ne * PB * NC) {
      const int le2 = tid / (PB * NC), q2 = tid - le2 * PB * NC;
      const int al = q2 % PB, c = C0 + q2 / PB;
      const T* SRy = SR(le2) + PB * PBP;
      T* b0e = B0(le2);
      T* b1e = B1(le2);
#pragma unroll
      for (int be = 0; be < PB; ++be) v[be] = b0e[al + PB * (be + PB * c)];
#pragma unroll OUT_UNR
      for (int bb = 0; bb < NC; ++bb) {
        const int b = C0 + bb;
        b1e[al + PB * (b + PB * c)] = dot_row<PB, PBP>(SRy + b * PBP, v);
      }
    }
    __syncthreads();
    // ---- backward: S_x along alpha (line (b', c'), NC*NC lines per element), write out
    if (tid < ne * NC * NC) {
      const int le3 = tid / (NC * NC), q3 = tid - le3 * NC * NC;
      const int b = C0 + q3 % NC, c = C0 + q3 / NC;
      const T* SRx = SR(le3);
      const T* b1e = B1(le3);
      const int64_t e = e0 + le3;
#pragma unroll
      for (int al = 0; al < PB; ++al) v[al] = b1e[al + PB * (b + PB * c)];
#pragma unroll OUT_UNR
      for (int aa = 0; aa < NC; ++aa) {
        const int a = C0 + aa;
        const T acc = dot_row<PB, PBP>(SRx + a * PBP, v);
        if constexpr (MODE == FDM_RAS) {
          const int64_t li = e * (N * N * N) + (a - 1) + N * ((b - 1) + N * (c - 1));
          const int mlog = __ffs(pflag[li] & 0x0F) - 1;   // 1/multiplicity: exact power of 2
          const T wt = mlog == 0 ? T(1) : (mlog == 1 ? T(0.5) : (mlog == 2 ? T(0.25) : T(0.125)));
          out[li] = io_cast<IO>(acc * wt);
        } else {
          out[e * PB3 + a + PB * (b + PB * c)] = io_cast<IO>(acc);
        }
      }
    }
  }
}

// ------------------------------------------------------------------ FP32: one warp per element
// The FP32 solve is not bound by the FMA pipe but by instruction issue and shared-memory
// wavefronts, so its kernel is laid out to issue as few of both as possible:
//  * one warp owns one element, so phases are ordered by __syncwarp alone, and each row of S is
//    read once per warp (a broadcast) and applied to every line the lane holds (ceil(PB^2/32)
//    lines per lane) instead of once per line;
//  * one window buffer, updated in place: within a phase every lane reads its whole lines before
//    it writes them back, and no two lanes share a line (lanes past the last line read line 0
//    and discard what they compute);
//  * the forward z transform, D^-1 and the backward z transform run on the same lines, so the
//    eigen-space values stay in registers between them;
//  * layout a + PB b + PS c with the plane stride PS padded (PS >= PB^2) to the value with the
//    fewest bank conflicts over this kernel's access patterns, found by counting them for every
//    candidate PS in [PB^2, PB^2 + 32);
//  * where each window point comes from (neighbour slot, point in that element, buffer offset)
//    depends only on p: the block tabulates it once in shared memory, and every element's
//    gather is a table walk of cp.async copies, all in flight at once; the RAS outputs leave
//    through shared memory as contiguous, coalesced stores.
// Per output the arithmetic is one FMA chain over the contracted index in ascending order (the
// backward contractions: two, over even and odd indices, added at the end); D^-1
// is applied as a product with the hardware reciprocal of lambda_x + lambda_y + lambda_z (one
// rounding more than a division: far below the FP32 preconditioner's tolerance).
__host__ __device__ constexpr int fdm32_plane_stride(int PB) {
  return PB == 4 ? 19 : PB == 5 ? 25 : PB == 6 ? 37 : PB == 7 ? 52 : PB == 8 ? 79 : PB == 9 ? 81
       : PB == 10 ? 107 : PB == 11 ? 121 : PB == 12 ? 145 : PB * PB;
}

template <int PB>
struct Fdm32Dims {
  static constexpr int N = PB - 2;
  static constexpr int PS = fdm32_plane_stride(PB);
  static constexpr int BUF = (PS * PB + 3) / 4 * 4;       // window buffer (16-byte multiple)
  static constexpr int PBP = (PB + 3) / 4 * 4;             // padded row of S
  static constexpr int SMAT = PB * PBP;                    // S of one direction
  static constexpr int LAMP = (3 * PB + 3) / 4 * 4;
  static constexpr int PER = BUF + 3 * SMAT + LAMP + 28;   // floats per element (+27 neighbour ids)
  // block tables: window point -> buffer offset | slot << 12 | source point << 17 (PB^3 words),
  // own point -> buffer offset (N^3 half-words)
  static constexpr int TAB_BYTES = (PB * PB * PB * 4 + N * N * N * 2 + 15) / 16 * 16;
  static_assert(PS >= PB * PB, "plane stride below the plane size");
  static_assert(PS * PB <= 4096 && N * N * N <= 2048, "window table fields overflow");
};

// The row contractions below use Blackwell's packed FP32 FMA (two lanes per instruction,
// fma.rn.f32x2 through __ffma2_rn): this kernel is bound by instruction issue, not by the FMA
// pipe, so halving the FMA instruction count is what shortens it.

// acc[j][o] += S[r][o] x[j], o < PB: one padded row of S (float4 reads), NL lines; outputs in
// pairs (o, o + 1).
template <int PB, int PBP, int NL>
__device__ __forceinline__ void fdm32_axpy_row(const float* __restrict__ row, const float (&x)[NL],
                                               float (&acc)[NL][PB]) {
#pragma unroll
  for (int o4 = 0; o4 < PBP; o4 += 4) {
    const float4 s4 = *reinterpret_cast<const float4*>(row + o4);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int o = o4 + 2 * h;
      const float2 s2 = h ? make_float2(s4.z, s4.w) : make_float2(s4.x, s4.y);
      if (o + 1 < PB) {
#pragma unroll
        for (int j = 0; j < NL; ++j) {
          const float2 a = __ffma2_rn(s2, make_float2(x[j], x[j]), make_float2(acc[j][o], acc[j][o + 1]));
          acc[j][o] = a.x;
          acc[j][o + 1] = a.y;
        }
      } else if (o < PB) {
#pragma unroll
        for (int j = 0; j < NL; ++j) acc[j][o] = fmaf(s2.x, x[j], acc[j][o]);
      }
    }
  }
}

// out[j] = sum_o S[r][o] v[j][o]: one padded row of S, NL lines; even and odd o accumulate in
// the two lanes of a packed FMA (each in ascending o) and are added at the end.
template <int PB, int PBP, int NL>
__device__ __forceinline__ void fdm32_dot_row(const float* __restrict__ row, const float (&v)[NL][PB],
                                              float (&out)[NL]) {
  float2 acc[NL];
#pragma unroll
  for (int j = 0; j < NL; ++j) acc[j] = make_float2(0.f, 0.f);
  float tail[NL];
#pragma unroll
  for (int j = 0; j < NL; ++j) tail[j] = 0.f;
#pragma unroll
  for (int o4 = 0; o4 < PBP; o4 += 4) {
    const float4 s4 = *reinterpret_cast<const float4*>(row + o4);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int o = o4 + 2 * h;
      const float2 s2 = h ? make_float2(s4.z, s4.w) : make_float2(s4.x, s4.y);
      if (o + 1 < PB) {
#pragma unroll
        for (int j = 0; j < NL; ++j) acc[j] = __ffma2_rn(s2, make_float2(v[j][o], v[j][o + 1]), acc[j]);
      } else if (o < PB) {
#pragma unroll
        for (int j = 0; j < NL; ++j) tail[j] = s2.x * v[j][o];
      }
    }
  }
#pragma unroll
  for (int j = 0; j < NL; ++j) out[j] = (acc[j].x + acc[j].y) + tail[j];
}

// 4-byte asynchronous global -> shared copy; valid == false fills the word with zero and reads
// nothing (src must still be a mapped address).
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Lines of one phase: lane l holds lines l, l + 32, ..., l + 32 (NL - 1); the ones past `count`
// are read as line 0 and never written.
template <int NL>
struct LaneLines {
  int base[NL];
  bool ok[NL];
};

template <int P, int MODE>
__global__ void __launch_bounds__(256, P <= 6 ? 4 : (P <= 8 ? 3 : 2)) fdm32_warp_kernel(int64_t E, const int* __restrict__ nbr,
                                                         const float* __restrict__ in,
                                                         const float* __restrict__ Sg,
                                                         const float* __restrict__ lamg,
                                                         const uint8_t* __restrict__ pflag,
                                                         float* __restrict__ out) {
  static_assert(MODE == FDM_RAS || MODE == FDM_FULL, "FP32 warp kernel: RAS or full window");
  constexpr int N = P + 1, N2 = N * N, N3 = N2 * N, PB = P + 3, PB2 = PB * PB, PB3 = PB2 * PB;
  using Dm = Fdm32Dims<PB>;
  constexpr int RS = PB, PS = Dm::PS, PBP = Dm::PBP, SMAT = Dm::SMAT;
  constexpr int C0 = MODE == FDM_RAS ? 1 : 0;
  constexpr int NC = MODE == FDM_RAS ? N : PB;
  constexpr int NL = (PB2 + 31) / 32;         // lines per lane: PB^2 lines
  constexpr int NL2 = (PB * NC + 31) / 32;    // backward y: PB * NC lines
  constexpr int NL1 = (NC * NC + 31) / 32;    // backward x: NC^2 lines
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned* wtab = reinterpret_cast<unsigned*>(smem_raw);
  uint16_t* otab = reinterpret_cast<uint16_t*>(wtab + PB3);
  // ---- block tables (the same for every element of every block)
  for (int q = threadIdx.x; q < PB3; q += blockDim.x) {
    const int c = q / PB2, r2 = q - c * PB2, b = r2 / PB, a = r2 - b * PB;
    const int da = a == 0 ? -1 : (a == PB - 1 ? 1 : 0);
    const int db = b == 0 ? -1 : (b == PB - 1 ? 1 : 0);
    const int dc = c == 0 ? -1 : (c == PB - 1 ? 1 : 0);
    const int ia = da < 0 ? P - 1 : (da > 0 ? 1 : a - 1);
    const int ib = db < 0 ? P - 1 : (db > 0 ? 1 : b - 1);
    const int ic = dc < 0 ? P - 1 : (dc > 0 ? 1 : c - 1);
    const unsigned slot = (unsigned)((da + 1) + 3 * (db + 1) + 9 * (dc + 1));
    const unsigned src = (unsigned)(ia + N * (ib + N * ic));
    wtab[q] = (unsigned)(a + RS * b + PS * c) | (slot << 12) | (src << 17);
  }
  if constexpr (MODE == FDM_RAS) {
    for (int q = threadIdx.x; q < N3; q += blockDim.x) {
      const int k = q / N2, r2 = q - k * N2, j = r2 / N, i = r2 - j * N;
      otab[q] = (uint16_t)((i + 1) + RS * (j + 1) + PS * (k + 1));
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (e >= E) return;  // whole warps leave; nothing below synchronises beyond the warp
  float* buf = reinterpret_cast<float*>(smem_raw + Dm::TAB_BYTES) + (size_t)warp * Dm::PER;
  float* sS = buf + Dm::BUF;                  // [3][PB][PBP]: S[d][row = window point][mode]
  float* sl = sS + 3 * SMAT;                  // [3][PB] eigenvalues
  int* snb = reinterpret_cast<int*>(sl + Dm::LAMP);
  // All of the element's inputs move by cp.async, so that every copy of the warp is in flight at
  // once (one memory latency per element rather than one per loop trip).
  if (lane < 27) snb[lane] = nbr[27 * e + lane];
  for (int q = lane; q < 3 * SMAT; q += 32) {
    const int d = q / SMAT, rr = q - d * SMAT, i = rr / PBP, j = rr - i * PBP;
    if (j < PB) cp_async4(sS + q, Sg + (e * 3 + d) * PB2 + i * PB + j, true);
    else sS[q] = 0.f;
  }
  for (int q = lane; q < 3 * PB; q += 32) cp_async4(sl + q, lamg + e * 3 * PB + q, true);
  __syncwarp();
  // ---- gather the extended window (zero outside the domain; Dirichlet values are zero in r)
#pragma unroll 8
  for (int q = lane; q < PB3; q += 32) {
    const unsigned w = wtab[q];
    const int nb = snb[(w >> 12) & 31u];
    cp_async4(buf + (w & 4095u), nb >= 0 ? in + ((int64_t)nb * N3 + (w >> 17)) : in, nb >= 0);
  }
  cp_async_wait_all();
  __syncwarp();
  // ---- forward S_x^T along a: lines (b, c)
  {
    float acc[NL][PB];
    int base[NL];
    bool ok[NL];
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const int ql = lane + 32 * j;
      ok[j] = ql < PB2;
      const int c = ql / PB, b = ql - c * PB;
      base[j] = ok[j] ? RS * b + PS * c : 0;
#pragma unroll
      for (int o = 0; o < PB; ++o) acc[j][o] = 0.f;
    }
#pragma unroll 2
    for (int a = 0; a < PB; ++a) {
      float x[NL];
#pragma unroll
      for (int j = 0; j < NL; ++j) x[j] = buf[base[j] + a];
      fdm32_axpy_row<PB, PBP, NL>(sS + a * PBP, x, acc);
    }
#pragma unroll
    for (int j = 0; j < NL; ++j)
      if (ok[j]) {
#pragma unroll
        for (int o = 0; o < PB; ++o) buf[base[j] + o] = acc[j][o];
      }
  }
  __syncwarp();
  // ---- forward S_y^T along b: lines (alpha, c)
  {
    float acc[NL][PB];
    int base[NL];
    bool ok[NL];
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const int ql = lane + 32 * j;
      ok[j] = ql < PB2;
      const int c = ql / PB, al = ql - c * PB;
      base[j] = ok[j] ? al + PS * c : 0;
#pragma unroll
      for (int o = 0; o < PB; ++o) acc[j][o] = 0.f;
    }
#pragma unroll 2
    for (int b = 0; b < PB; ++b) {
      float x[NL];
#pragma unroll
      for (int j = 0; j < NL; ++j) x[j] = buf[base[j] + RS * b];
      fdm32_axpy_row<PB, PBP, NL>(sS + SMAT + b * PBP, x, acc);
    }
#pragma unroll
    for (int j = 0; j < NL; ++j)
      if (ok[j]) {
#pragma unroll
        for (int o = 0; o < PB; ++o) buf[base[j] + RS * o] = acc[j][o];
      }
  }
  __syncwarp();
  // ---- forward S_z^T along c, D^-1, backward S_z along gamma: lines (alpha, beta)
  {
    float acc[NL][PB];
    int base[NL];
    bool ok[NL];
    float lxy[NL];
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const int ql = lane + 32 * j;
      ok[j] = ql < PB2;
      const int be = ql / PB, al = ql - be * PB;
      base[j] = ok[j] ? al + RS * be : 0;
      lxy[j] = ok[j] ? sl[al] + sl[PB + be] : 1.f;
#pragma unroll
      for (int o = 0; o < PB; ++o) acc[j][o] = 0.f;
    }
#pragma unroll 2
    for (int c = 0; c < PB; ++c) {
      float x[NL];
#pragma unroll
      for (int j = 0; j < NL; ++j) x[j] = buf[base[j] + PS * c];
      fdm32_axpy_row<PB, PBP, NL>(sS + 2 * SMAT + c * PBP, x, acc);
    }
#pragma unroll
    for (int ga = 0; ga < PB; ++ga) {
      const float lz = sl[2 * PB + ga];
#pragma unroll
      for (int j = 0; j < NL; ++j) acc[j][ga] = acc[j][ga] * rcp_approx(lxy[j] + lz);
    }
#pragma unroll 2
    for (int cc = 0; cc < NC; ++cc) {
      const int c = C0 + cc;
      float o[NL];
      fdm32_dot_row<PB, PBP, NL>(sS + 2 * SMAT + c * PBP, acc, o);
#pragma unroll
      for (int j = 0; j < NL; ++j)
        if (ok[j]) buf[base[j] + PS * c] = o[j];
    }
  }
  __syncwarp();
  // ---- backward S_y along beta: lines (alpha, c) with c in the output range
  {
    float v[NL2][PB];
    int base[NL2];
    bool ok[NL2];
#pragma unroll
    for (int j = 0; j < NL2; ++j) {
      const int ql = lane + 32 * j;
      ok[j] = ql < PB * NC;
      const int cc = ql / PB, al = ql - cc * PB;
      base[j] = ok[j] ? al + PS * (C0 + cc) : 0;
#pragma unroll
      for (int be = 0; be < PB; ++be) v[j][be] = buf[base[j] + RS * be];
    }
#pragma unroll 2
    for (int bb = 0; bb < NC; ++bb) {
      const int b = C0 + bb;
      float o[NL2];
      fdm32_dot_row<PB, PBP, NL2>(sS + SMAT + b * PBP, v, o);
#pragma unroll
      for (int j = 0; j < NL2; ++j)
        if (ok[j]) buf[base[j] + RS * b] = o[j];
    }
  }
  __syncwarp();
  // RAS weights of the element's own points (four flag bytes per register), fetched before the
  // last contraction to hide their latency
  constexpr int NQ = MODE == FDM_RAS ? (N3 + 31) / 32 : 1;
  unsigned pf[(NQ + 3) / 4];
#pragma unroll
  for (int i = 0; i < (NQ + 3) / 4; ++i) pf[i] = 0u;
  if constexpr (MODE == FDM_RAS) {
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
      const int q = lane + 32 * i;
      const unsigned f = q < N3 ? pflag[e * N3 + q] : 0u;
      pf[i / 4] |= f << (8 * (i % 4));
    }
  }
  // ---- backward S_x along alpha: lines (b, c), both in the output range
  {
    float v[NL1][PB];
    int base[NL1];
    bool ok[NL1];
#pragma unroll
    for (int j = 0; j < NL1; ++j) {
      const int ql = lane + 32 * j;
      ok[j] = ql < NC * NC;
      const int cc = ql / NC, bb = ql - cc * NC;
      base[j] = ok[j] ? RS * (C0 + bb) + PS * (C0 + cc) : 0;
#pragma unroll
      for (int al = 0; al < PB; ++al) v[j][al] = buf[base[j] + al];
    }
#pragma unroll 2
    for (int aa = 0; aa < NC; ++aa) {
      const int a = C0 + aa;
      float o[NL1];
      fdm32_dot_row<PB, PBP, NL1>(sS + a * PBP, v, o);
#pragma unroll
      for (int j = 0; j < NL1; ++j)
        if (ok[j]) buf[base[j] + a] = o[j];
    }
  }
  __syncwarp();
  // ---- write out, contiguous
  if constexpr (MODE == FDM_RAS) {
#pragma unroll
    for (int n = 0; n < NQ; ++n) {
      const int q = lane + 32 * n;
      if (q < N3) {
        // 1/multiplicity = 2^-mlog, mlog = index of the lowest set bit of the flag's low nibble
        const int mlog = __ffs((pf[n / 4] >> (8 * (n % 4))) & 0x0F) - 1;
        const float wt = __int_as_float((127 - mlog) << 23);
        out[e * N3 + q] = buf[otab[q]] * wt;
      }
    }
  } else {
    for (int q = lane; q < PB3; q += 32) out[e * PB3 + q] = buf[wtab[q] & 4095u];
  }
}

// ------------------------------------------------------------------ FP32 RAS, plane/column per thread
// GB300's FP32 pipe reaches its FMA rate only with packed pairs (fma.rn.f32x2: one instruction,
// two lanes), and a warp alone cannot keep it busy (measured with independent chains per
// thread: one warp per scheduler reaches about 60% of the packed rate, three about 90%).  This
// kernel issues packed FMAs for every contraction and keeps as many warps per SM as its
// registers and one window per element allow:
//  * persistent blocks of independent warps; a warp owns EW = 32/pbar elements at a time (pbar
//    lanes each) and walks the elements in steps of the grid's warp count; one shared-memory
//    window per element and 8 warps per SM at p = 7, 12 at p = 3 and 5 (measured on GB300 at
//    32^3 elements: faster than two stages per warp with 6 warps per SM, 0.150 ms at p = 7, and
//    than 12 warps per SM at p = 7 with fewer registers per thread, 0.126 ms);
//  * the window gather (cp.async, 4-byte copies, zero fill outside the domain), S and Lambda of a
//    step are one cp.async group; the neighbour ids of the warp's next step are loaded into
//    registers during the current step;
//  * phase A, plane c = t per thread: the plane is read column by column into packed-pair
//    accumulators (S_x^T, pairs of output modes), then S_y^T is applied in registers and the
//    result written back in place;
//  * phase B, the pbar columns (a = t, b) per thread: S_z^T into registers, D^-1 (hardware
//    reciprocal of lambda_x + lambda_y + lambda_z), then S_z for the N own planes only;
//  * phase C, own plane t + 1 per thread (t < N): the plane as row pairs and the own rows of S_x
//    in registers; per own row, S_y then S_x (own columns), weights 1/multiplicity from the
//    element's place in the lattice, contiguous stores;
//  * outer loops stay rolled (small code), inner loops over registers are unrolled.
// Shared strides: the window plane stride PSN and the element stride TOT = pbar (mod 32) put the
// scalar accesses of every phase (plane rows, plane columns, columns across planes) of a warp's
// active lanes in distinct banks.
template <int PB>
struct Fdm32PipeDims {
  static_assert(PB == 6 || PB == 8 || PB == 10, "FP32 RAS plane/column kernel: pbar 6, 8 or 10");
  static constexpr int N = PB - 2, H = PB / 2, EW = 32 / PB;
  static constexpr int WARPS = 2;                                    // warps per block
  static constexpr int BLOCKS_PER_SM = PB == 10 ? 4 : 6;             // 8 / 12 warps per SM
  static constexpr int PSN = PB == 6 ? 47 : (PB == 8 ? 65 : 111);    // window plane stride
  static constexpr int OFF_S = (PB * PSN + 1) / 2 * 2;               // [3][PB][PB], 8-byte aligned
  static constexpr int OFF_L = OFF_S + 3 * PB * PB;                  // [3][PB]
  static constexpr int RAW = OFF_L + 3 * PB;
  static constexpr int TOT = RAW + ((PB - RAW % 32) % 32 + 32) % 32;  // = PB (mod 32), even
  static constexpr size_t SMEM = (size_t)WARPS * EW * TOT * sizeof(float);
  static_assert(TOT % 2 == 0 && OFF_S % 2 == 0 && OFF_L % 2 == 0, "8-byte copies need even offsets");
};

__device__ __forceinline__ void cp_async8(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}

template <int P>
__global__ void __launch_bounds__(64, Fdm32PipeDims<P + 3>::BLOCKS_PER_SM)
    fdm32_pipe_kernel(int64_t E, int nx, int ny, int nz, const int* __restrict__ nbr,
                      const float* __restrict__ in, const float* __restrict__ Sg,
                      const float* __restrict__ lamg, const uint8_t* __restrict__ pflag,
                      float* __restrict__ out) {
  constexpr int PB = P + 3, N = P + 1, N2 = N * N, N3 = N2 * N, PB2 = PB * PB, H = PB / 2;
  using D = Fdm32PipeDims<PB>;
  constexpr int PSN = D::PSN, EW = D::EW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane / PB, t = lane - g * PB;
  const bool lane_on = g < EW;
  float* const W = reinterpret_cast<float*>(smem_raw) + (size_t)(warp * EW + (lane_on ? g : 0)) * D::TOT;
  const float* const sS = W + D::OFF_S;
  const float* const sl = W + D::OFF_L;
  const int64_t nsteps = (E + EW - 1) / EW;
  const int64_t w0 = (int64_t)blockIdx.x * D::WARPS + warp, nw = (int64_t)gridDim.x * D::WARPS;

  // the column of the window this thread gathers: a = t (neighbour direction da)
  const int da = t == 0 ? -1 : (t == PB - 1 ? 1 : 0);
  const int ia = da < 0 ? P - 1 : (da > 0 ? 1 : t - 1);
  int nb9[3][3];
  auto load_nb = [&](int64_t q) {
    const int64_t e = q * EW + g;
    const bool on = lane_on && q < nsteps && e < E;
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int j = 0; j < 3; ++j) nb9[k][j] = on ? __ldg(nbr + 27 * e + (da + 1) + 3 * j + 9 * k) : -1;
  };
  load_nb(w0);
  for (int64_t q = w0; q < nsteps; q += nw) {
    const int64_t e = q * EW + g;
    const bool on = lane_on && e < E;
    // ---- gather: column a = t of every row (b, c) of the window; S and Lambda
    if (on) {
      const float* src_a = in + ia;
#pragma unroll
      for (int c = 0; c < PB; ++c) {
        const int dc = c == 0 ? -1 : (c == PB - 1 ? 1 : 0);
        const int ic = dc < 0 ? P - 1 : (dc > 0 ? 1 : c - 1);
#pragma unroll
        for (int b = 0; b < PB; ++b) {
          const int db = b == 0 ? -1 : (b == PB - 1 ? 1 : 0);
          const int ib = db < 0 ? P - 1 : (db > 0 ? 1 : b - 1);
          const int nb = nb9[dc + 1][db + 1];
          cp_async4(W + c * PSN + b * PB + t,
                    nb >= 0 ? src_a + (int64_t)nb * N3 + N * ib + N2 * ic : in, nb >= 0);
        }
      }
      const float* gS = Sg + e * 3 * PB2;
      for (int q2 = t; q2 < 3 * PB2 / 2; q2 += PB) cp_async8(W + D::OFF_S + 2 * q2, gS + 2 * q2);
      const float* gL = lamg + e * 3 * PB;
      for (int q2 = t; q2 < 3 * PB / 2; q2 += PB) cp_async8(W + D::OFF_L + 2 * q2, gL + 2 * q2);
    }
    load_nb(q + nw);     // ids of the next step, in flight during this one
    cp_async_wait_all();
    __syncwarp();
    // ---- phase A: plane c = t; S_x^T along a (output modes in pairs), then S_y^T along b
    if (on) {
      float* pl = W + t * PSN;
      float2 acc[PB][H];
#pragma unroll
      for (int b = 0; b < PB; ++b)
#pragma unroll
        for (int k = 0; k < H; ++k) acc[b][k] = make_float2(0.f, 0.f);
#pragma unroll 1
      for (int a = 0; a < PB; ++a) {
        float v[PB];
#pragma unroll
        for (int b = 0; b < PB; ++b) v[b] = pl[b * PB + a];
        float2 s2[H];
#pragma unroll
        for (int k = 0; k < H; ++k) s2[k] = *reinterpret_cast<const float2*>(sS + a * PB + 2 * k);
#pragma unroll
        for (int b = 0; b < PB; ++b) {
          const float2 vv = make_float2(v[b], v[b]);
#pragma unroll
          for (int k = 0; k < H; ++k) acc[b][k] = __ffma2_rn(s2[k], vv, acc[b][k]);
        }
      }
#pragma unroll 1
      for (int bq = 0; bq < PB; ++bq) {
        float2 w[H];
#pragma unroll
        for (int k = 0; k < H; ++k) w[k] = make_float2(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < PB; ++b) {
          const float s = sS[PB2 + b * PB + bq];
          const float2 ss = make_float2(s, s);
#pragma unroll
          for (int k = 0; k < H; ++k) w[k] = __ffma2_rn(ss, acc[b][k], w[k]);
        }
#pragma unroll
        for (int k = 0; k < H; ++k) {
          pl[bq * PB + 2 * k] = w[k].x;
          pl[bq * PB + 2 * k + 1] = w[k].y;
        }
      }
    }
    __syncwarp();
    // ---- phase B: columns (a = t, b = j): S_z^T, D^-1, S_z for the own planes
    if (on) {
      float* col = W + t;
      float2 acc[PB][H];
#pragma unroll
      for (int j = 0; j < PB; ++j)
#pragma unroll
        for (int k = 0; k < H; ++k) acc[j][k] = make_float2(0.f, 0.f);
#pragma unroll 1
      for (int c = 0; c < PB; ++c) {
        float v[PB];
#pragma unroll
        for (int j = 0; j < PB; ++j) v[j] = col[PB * j + PSN * c];
        float2 s2[H];
#pragma unroll
        for (int k = 0; k < H; ++k) s2[k] = *reinterpret_cast<const float2*>(sS + 2 * PB2 + c * PB + 2 * k);
#pragma unroll
        for (int j = 0; j < PB; ++j) {
          const float2 vv = make_float2(v[j], v[j]);
#pragma unroll
          for (int k = 0; k < H; ++k) acc[j][k] = __ffma2_rn(s2[k], vv, acc[j][k]);
        }
      }
      const float lx = sl[t];
      float lz[PB];
#pragma unroll
      for (int c = 0; c < PB; ++c) lz[c] = sl[2 * PB + c];
#pragma unroll
      for (int j = 0; j < PB; ++j) {
        const float lxy = lx + sl[PB + j];
#pragma unroll
        for (int k = 0; k < H; ++k) {
          acc[j][k].x *= rcp_approx(lxy + lz[2 * k]);
          acc[j][k].y *= rcp_approx(lxy + lz[2 * k + 1]);
        }
      }
#pragma unroll 1
      for (int cc = 1; cc <= N; ++cc) {
        float2 s2[H];
#pragma unroll
        for (int k = 0; k < H; ++k) s2[k] = *reinterpret_cast<const float2*>(sS + 2 * PB2 + cc * PB + 2 * k);
#pragma unroll
        for (int j = 0; j < PB; ++j) {
          float2 z = make_float2(0.f, 0.f);
#pragma unroll
          for (int k = 0; k < H; ++k) z = __ffma2_rn(s2[k], acc[j][k], z);
          col[PB * j + PSN * cc] = z.x + z.y;
        }
      }
    }
    __syncwarp();
    // ---- phase C: own plane t + 1: S_y (own rows), S_x (own columns), weights, stores
    if (on && t < N) {
      const float* pl = W + (t + 1) * PSN;
      float2 v2[H][PB];  // (v[2m][a], v[2m + 1][a])
#pragma unroll
      for (int m = 0; m < H; ++m)
#pragma unroll
        for (int a = 0; a < PB; ++a) v2[m][a] = make_float2(pl[2 * m * PB + a], pl[(2 * m + 1) * PB + a]);
      float2 sx[N][H];   // own rows of S_x as pairs
#pragma unroll
      for (int i = 0; i < N; ++i)
#pragma unroll
        for (int m = 0; m < H; ++m) sx[i][m] = *reinterpret_cast<const float2*>(sS + (1 + i) * PB + 2 * m);
      // weights from the element's place in the lattice, or (nx = 0: a level that is the union of
      // several lattices) from the point flags
      const bool lat = nx > 0;
      const int ex = lat ? (int)(e % nx) : 0, ey = lat ? (int)((e / nx) % ny) : 0;
      const int ez = lat ? (int)(e / ((int64_t)nx * ny)) : 0;
      const float wz = ((t == 0 && ez > 0) || (t == N - 1 && ez < nz - 1)) ? 0.5f : 1.f;
      const float wx0 = ex > 0 ? 0.5f : 1.f, wx1 = ex < nx - 1 ? 0.5f : 1.f;
      float* orow = out + e * N3 + (int64_t)N2 * t;
      const uint8_t* frow = pflag + e * N3 + (int64_t)N2 * t;
#pragma unroll 1
      for (int bb = 0; bb < N; ++bb) {
        float2 sy[H];
#pragma unroll
        for (int m = 0; m < H; ++m) sy[m] = *reinterpret_cast<const float2*>(sS + PB2 + (1 + bb) * PB + 2 * m);
        float y2[PB];    // this own row after S_y
#pragma unroll
        for (int a = 0; a < PB; ++a) {
          float2 z = make_float2(0.f, 0.f);
#pragma unroll
          for (int m = 0; m < H; ++m) z = __ffma2_rn(sy[m], v2[m][a], z);
          y2[a] = z.x + z.y;
        }
        const float wyz = wz * (((bb == 0 && ey > 0) || (bb == N - 1 && ey < ny - 1)) ? 0.5f : 1.f);
        float o[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
          float2 z = make_float2(0.f, 0.f);
#pragma unroll
          for (int m = 0; m < H; ++m) z = __ffma2_rn(sx[i][m], make_float2(y2[2 * m], y2[2 * m + 1]), z);
          const float wx = i == 0 ? wx0 : (i == N - 1 ? wx1 : 1.f);
          const float wf = lat ? wx * wyz : __int_as_float((127 - (__ffs(frow[N * bb + i] & 0x0F) - 1)) << 23);
          o[i] = (z.x + z.y) * wf;
        }
        float* dst = orow + N * bb;
        if constexpr (N % 4 == 0) {
#pragma unroll
          for (int q4 = 0; q4 < N / 4; ++q4)
            *reinterpret_cast<float4*>(dst + 4 * q4) = make_float4(o[4 * q4], o[4 * q4 + 1], o[4 * q4 + 2], o[4 * q4 + 3]);
        } else {
#pragma unroll
          for (int q2 = 0; q2 < N / 2; ++q2) *reinterpret_cast<float2*>(dst + 2 * q2) = make_float2(o[2 * q2], o[2 * q2 + 1]);
        }
      }
    }
    __syncwarp();  // the window is read completely before the next step's copies target it
  }
}

// Shared bytes per element: fdm_kernel<P, double, *> (two window buffers, S^T and S, the
// eigenvalues, 27 neighbour ids) or fdm32_warp_kernel<P, *> (Fdm32Dims<P + 3>::PER floats, and
// the block's window tables once per block).
template <int P, typename T>
constexpr size_t fdm_smem_per_element() {
  if constexpr (sizeof(T) == 4) {
    return Fdm32Dims<P + 3>::PER * sizeof(float);
  } else {
    using Dm = FdmDims<P + 3>;
    return (2 * Dm::PB3P + 2 * Dm::SROW + (3 * (P + 3) + 3) / 4 * 4) * sizeof(T) + 27 * sizeof(int);
  }
}

size_t fdm_smem_bytes(int p, bool fp32, int ne) {
  size_t per = 0, fixed = 0;  // per element; per block (the FP32 kernel's window tables)
  switch (p) {
#define SE_FDM_SM(PP)                                   \
  case PP:                                              \
    if (fp32) {                                         \
      per = fdm_smem_per_element<PP, float>();          \
      fixed = Fdm32Dims<PP + 3>::TAB_BYTES;             \
    } else {                                            \
      per = fdm_smem_per_element<PP, double>();         \
    }                                                   \
    break;
    SE_FDM_SM(1) SE_FDM_SM(2) SE_FDM_SM(3) SE_FDM_SM(4) SE_FDM_SM(5)
    SE_FDM_SM(6) SE_FDM_SM(7) SE_FDM_SM(8) SE_FDM_SM(9) SE_FDM_SM(10)
#undef SE_FDM_SM
    default: per = 0;
  }
  return per * ne + fixed;
}

// Largest block: 256 threads for fdm32_warp_kernel (its launch bounds), 512 for fdm_kernel.
int fdm_max_threads(bool fp32) { return fp32 ? 256 : 512; }

// Threads of a block with ne elements: FP32 one warp per element, FP64 one per line of a phase.
int fdm_block_threads(int p, bool fp32, int ne) {
  const int PB = p + 3;
  return fp32 ? 32 * ne : (ne * PB * PB + 31) / 32 * 32;
}

// Elements per block: the tuned value if one is set and valid; else FP32 8 (one warp each),
// FP64 about 400 lines per phase (at most 16 elements).
int fdm_elems_per_block(int p, bool fp32) {
  const int PB = p + 3;
  const int t = tile_get(p, fp32).fdm_ne;
  if (t >= 1 && t <= 16 && fdm_block_threads(p, fp32, t) <= fdm_max_threads(fp32) &&
      fdm_smem_bytes(p, fp32, t) <= 200 * 1024)
    return t;
  int ne = fp32 ? 8 : 400 / (PB * PB);
  ne = ne < 1 ? 1 : (ne > 16 ? 16 : ne);
  while (ne > 1 && fdm_smem_bytes(p, fp32, ne) > 200 * 1024) --ne;
  return ne;
}

template <int P, typename T, int MODE>
static int launch_fdm(const Level& lv, const T* in, const T* S, const T* lam, T* out,
                      cudaStream_t s) {
  const int NE = fdm_elems_per_block(P, sizeof(T) == 4);
  const int threads = fdm_block_threads(P, sizeof(T) == 4, NE);
  const size_t smem = fdm_smem_bytes(P, sizeof(T) == 4, NE);
  const unsigned blocks = (unsigned)((lv.E + NE - 1) / NE);
  if constexpr (sizeof(T) == 4) {
    static_assert(MODE == FDM_RAS || MODE == FDM_FULL, "FP32 FDM: RAS or full window only");
    if constexpr (MODE == FDM_RAS && (P == 3 || P == 5 || P == 7)) {
      using PD = Fdm32PipeDims<P + 3>;
      static const cudaError_t pattr = cudaFuncSetAttribute(
          fdm32_pipe_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PD::SMEM);
      SE_CUDA(pattr);
      int per_sm = 0, dev = 0, sms = 0;
      SE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fdm32_pipe_kernel<P>,
                                                            32 * PD::WARPS, PD::SMEM));
      SE_CHECK(per_sm >= 1, SE_ECUDA, "fdm32_pipe: no resident block fits");
      SE_CUDA(cudaGetDevice(&dev));
      SE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      const int64_t steps = (lv.E + PD::EW - 1) / PD::EW;
      int64_t pblocks = (int64_t)sms * per_sm;
      if (pblocks > (steps + PD::WARPS - 1) / PD::WARPS) pblocks = (steps + PD::WARPS - 1) / PD::WARPS;
      fdm32_pipe_kernel<P><<<(unsigned)pblocks, 32 * PD::WARPS, PD::SMEM, s>>>(
          lv.E, lv.nel[0], lv.nel[1], lv.nel[2], lv.nbr, in, S, lam, lv.pflag, out);
      SE_LAUNCH_CHECK();
      return SE_OK;
    }
    static const cudaError_t attr = cudaFuncSetAttribute(
        fdm32_warp_kernel<P, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    SE_CUDA(attr);
    fdm32_warp_kernel<P, MODE><<<blocks, threads, smem, s>>>(lv.E, lv.nbr, in, S, lam, lv.pflag, out);
  } else {
    static const cudaError_t attr = cudaFuncSetAttribute(
        fdm_kernel<P, T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    SE_CUDA(attr);
    fdm_kernel<P, T, MODE><<<blocks, threads, smem, s>>>(lv.E, NE, lv.nbr, in, S, lam,
                                                          lv.fdm_dinv64, lv.pflag, out);
  }
  SE_LAUNCH_CHECK();
  return SE_OK;
}

// df64 arithmetic on FP64 vectors: the FP64 kernel's layout (df64 values are 8 bytes, as FP64
// ones), its S and Lambda from the df64 copies.  Fewer elements per block than FP64 (measured
// on GB300 at 32^3 elements: p = 7 3 elements, 1.31 ms against 1.47 ms with FP64's 4; p = 5 3;
// p = 3 6), unless a tile is set for FP64.
static int fdm_df_elems_per_block(int p) {
  if (tile_get(p, false).fdm_ne > 0) return fdm_elems_per_block(p, false);
  switch (p) {
    case 1: return 16;
    case 2: return 10;
    case 3: return 6;
    case 4: return 5;
    case 5: return 3;
    case 6: return 3;
    case 7: return 3;
    default: return 2;
  }
}

template <int P, int MODE>
static int launch_fdm_df(const Level& lv, const double* in, double* out, cudaStream_t s) {
  const int NE = fdm_df_elems_per_block(P);
  const int threads = fdm_block_threads(P, false, NE);
  const size_t smem = fdm_smem_bytes(P, false, NE);
  const unsigned blocks = (unsigned)((lv.E + NE - 1) / NE);
  static const cudaError_t attr = cudaFuncSetAttribute(
      fdm_kernel<P, df64, MODE, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  SE_CUDA(attr);
  fdm_kernel<P, df64, MODE, double><<<blocks, threads, smem, s>>>(lv.E, NE, lv.nbr, in, lv.Sdf, lv.lamdf,
                                                                   lv.fdm_dinv64, lv.pflag, out);
  SE_LAUNCH_CHECK();
  return SE_OK;
}

template <typename T, int MODE>
static int dispatch_fdm(const Level& lv, const T* in, T* out, cudaStream_t s) {
  const T* S;
  const T* lam;
  if constexpr (sizeof(T) == 8) {
    S = lv.S64;
    lam = lv.lam64;
  } else {
    S = lv.S32;
    lam = lv.lam32;
  }
  SE_CHECK(MODE == FDM_GATHER || S != nullptr, SE_EINVAL, "FDM factors missing for this level/precision");
  const double PB = lv.p + 3.0, N = lv.N;
  const double fl = 2.0 * (3.0 * PB * PB * PB * PB + PB * PB * PB * N + PB * PB * N * N + PB * N * N * N) + PB * PB * PB;
  const double by = (PB * PB * PB + N * N * N + 3 * PB * PB + 3 * PB + (sizeof(T) == 8 ? PB * PB * PB : 0)) * sizeof(T);
  bool use_df = false;
  if constexpr (sizeof(T) == 8) use_df = MODE != FDM_GATHER && lv.df && lv.Sdf;
  ProfScope prof(SE_K_FDM, s, (double)lv.E, by * lv.E, fl * lv.E,
                 use_df ? lv.p + 64 : prof_variant<T>(lv.p));
  if constexpr (sizeof(T) == 8 && MODE != FDM_GATHER) {
    if (use_df) {
      switch (lv.p) {
#define SE_FDM_DF(PP) \
  case PP: return launch_fdm_df<PP, MODE>(lv, in, out, s);
        SE_FDM_DF(1) SE_FDM_DF(2) SE_FDM_DF(3) SE_FDM_DF(4) SE_FDM_DF(5)
        SE_FDM_DF(6) SE_FDM_DF(7) SE_FDM_DF(8) SE_FDM_DF(9) SE_FDM_DF(10)
#undef SE_FDM_DF
        default: break;
      }
    }
  }
  switch (lv.p) {
#define SE_FDM_CASE(PP) \
  case PP: return launch_fdm<PP, T, MODE>(lv, in, S, lam, out, s);
    SE_FDM_CASE(1) SE_FDM_CASE(2) SE_FDM_CASE(3) SE_FDM_CASE(4) SE_FDM_CASE(5)
    SE_FDM_CASE(6) SE_FDM_CASE(7) SE_FDM_CASE(8) SE_FDM_CASE(9) SE_FDM_CASE(10)
#undef SE_FDM_CASE
    default: set_error("fdm: unsupported p=%d", lv.p); return SE_EINVAL;
  }
}

// Additive Schwarz combine (eq 4 with post-multiplied W): for every local point, sum the
// full-window solutions of all elements whose window covers the node, divide by their count.
template <typename T>
__global__ void asm_combine_kernel(int P, int nx, int ny, int nz, int64_t L,
                                   const T* __restrict__ zbar, const uint8_t* __restrict__ pflag,
                                   T* __restrict__ out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= L) return;
  if (!(pflag[idx] & PF_FREE)) {
    out[idx] = T(0);
    return;
  }
  const int N = P + 1, N3 = N * N * N, PB = P + 3;
  const int64_t e = idx / N3;
  const int pt = (int)(idx - e * N3);
  const int i = pt % N, j = (pt / N) % N, k = pt / (N * N);
  const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
  const int I = ex * P + i, J = ey * P + j, K = ez * P + k;
  T acc = T(0);
  int cnt = 0;
  for (int cz = ez - 1; cz <= ez + 1; ++cz) {
    if (cz < 0 || cz >= nz) continue;
    const int c = K - (cz * P - 1);
    if (c < 0 || c >= PB) continue;
    for (int cy = ey - 1; cy <= ey + 1; ++cy) {
      if (cy < 0 || cy >= ny) continue;
      const int b = J - (cy * P - 1);
      if (b < 0 || b >= PB) continue;
      for (int cx = ex - 1; cx <= ex + 1; ++cx) {
        if (cx < 0 || cx >= nx) continue;
        const int a = I - (cx * P - 1);
        if (a < 0 || a >= PB) continue;
        const int64_t ee = cx + (int64_t)nx * (cy + (int64_t)ny * cz);
        acc += zbar[ee * PB * PB * PB + a + PB * (b + PB * c)];
        ++cnt;
      }
    }
  }
  out[idx] = acc / T(cnt);
}

template <class T>
int schwarz_apply(const Level& lv, int kind, const T* r, T* out, cudaStream_t s) {
  if (kind == SE_SMOOTH_RAS) {
    SE_TRY((dispatch_fdm<T, FDM_RAS>(lv, r, out, s)));
    return gs_apply<T>(lv, out, true, s);
  }
  T* ext;
  if constexpr (sizeof(T) == 8) ext = lv.ext64;
  else ext = lv.ext32;
  SE_CHECK(ext != nullptr, SE_EINVAL, "ASM window buffer missing");
  SE_TRY((dispatch_fdm<T, FDM_FULL>(lv, r, ext, s)));
  ProfScope prof(SE_K_GS, s, (double)lv.L, lv.L * (2.0 * sizeof(T) + 1.0), (double)lv.L);
  asm_combine_kernel<T><<<grid_for(lv.L, 256), 256, 0, s>>>(lv.p, lv.nel[0], lv.nel[1], lv.nel[2],
                                                            lv.L, ext, lv.pflag, out);
  SE_LAUNCH_CHECK();
  return SE_OK;
}

template <class T>
int gather_ext(const Level& lv, const T* r, T* rbar, cudaStream_t s) {
  return dispatch_fdm<T, FDM_GATHER>(lv, r, rbar, s);
}
template <class T>
int fdm_apply_ext(const Level& lv, const T* rbar, T* zbar, cudaStream_t s) {
  return dispatch_fdm<T, FDM_EXT_IN>(lv, rbar, zbar, s);
}

template int schwarz_apply<double>(const Level&, int, const double*, double*, cudaStream_t);
template int schwarz_apply<float>(const Level&, int, const float*, float*, cudaStream_t);
template int gather_ext<double>(const Level&, const double*, double*, cudaStream_t);
template int fdm_apply_ext<double>(const Level&, const double*, double*, cudaStream_t);

}  // namespace se

namespace se {
// RAS local solves only (own outputs weighted by 1/multiplicity, no QQ^T): used to time tiles.
template <class T>
int fdm_ras_local(const Level& lv, const T* r, T* out, cudaStream_t s) {
  return dispatch_fdm<T, FDM_RAS>(lv, r, out, s);
}
template int fdm_ras_local<double>(const Level&, const double*, double*, cudaStream_t);
template int fdm_ras_local<float>(const Level&, const float*, float*, cudaStream_t);
}  // namespace se
