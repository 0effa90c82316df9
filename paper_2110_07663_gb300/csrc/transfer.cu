// p-multigrid transfers between GLL bases (Algorithm 1, Sec. 2.2.2):
//   prolongation  e_f = (J x J x J) e_c            element by element
//   restriction   r_c = M_c QQ^T_c (J^T x J^T x J^T)(r_f / mult_f)
// with J_ij = h^c_j(xi^f_i).  For a continuous r_f the restriction is the transpose of the
// global prolongation.  The three directions are contracted in turn through shared memory (the
// folded kernel stores the last one straight from its lines).
//
// Both GLL node sets are symmetric about 0 and h^c_{Nc-1-j}(-x) = h^c_j(x), so J is
// centro-symmetric: J[Nf-1-i][Nc-1-j] = J[i][j] (and so is J^T).  For even Nf and Nc each line
// contraction runs folded (transfer_eo_kernel): with e_l = v_l + v_{n-1-l}, o_l = v_l - v_{n-1-l}
// over the input line v of n points and Ep = (M[o][l] + M[o][n-1-l])/2, Om = (M[o][l] -
// M[o][n-1-l])/2 for the line operator M (J or J^T), output o and its mirror are E_o + O_o and
// E_o - O_o: n/2 fewer FMAs per output pair at the cost of n + m adds per line (about 20% fewer
// FP64 instructions; GB300 runs this kernel on its FP64 pipe).  Several elements share a block.
// At N = 4 <-> 2 the fold costs more than it saves (10 instead of 8 FP64 instructions per line):
// transfer_small_kernel contracts densely, one thread per output value of each direction, several
// elements per block.  Odd N (even orders) use the plain kernel, one element per block.
// The restriction's 1/mult_f (1, 1/2, 1/4, 1/8) is applied by lowering the binary exponent with
// integer instructions (scale_pow2), not by an FP64 multiply: exact for every value above 2^-1019
// (2^-123 in FP32; smaller magnitudes, far below any residual a solve forms, become 0), and the
// FP64 pipe keeps only the contractions.
#include "se_internal.h"
#include "reduce.h"

namespace se {

constexpr int NMAX = SE_MAX_ORDER + 1;

template <typename T, bool RESTRICT>
__global__ void __launch_bounds__(128) transfer_kernel(int Nf, int Nc, const T* __restrict__ Jg,
                                                       const T* __restrict__ in,
                                                       const uint8_t* __restrict__ pflag_in,
                                                       T* __restrict__ out, bool accumulate) {
  __shared__ T sJ[NMAX * NMAX];
  __shared__ T t0[NMAX * NMAX * NMAX];
  __shared__ T t1[NMAX * NMAX * NMAX];
  const int64_t e = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int Ni = RESTRICT ? Nf : Nc;  // input points per direction
  const int No = RESTRICT ? Nc : Nf;  // output points per direction
  for (int q = tid; q < Nf * Nc; q += nt) sJ[q] = Jg[q];
  const int Ni3 = Ni * Ni * Ni, No3 = No * No * No;
  for (int q = tid; q < Ni3; q += nt) {
    T v = in[e * Ni3 + q];
    if (RESTRICT) v = scale_pow2(v, mult_log2(pflag_in[e * Ni3 + q]));
    t0[q] = v;
  }
  __syncthreads();
  // operator entry: prolong uses J[o][i] (Nf x Nc), restrict uses J^T: J[i][o]
  auto op = [&](int o, int i) -> T { return RESTRICT ? sJ[i * Nc + o] : sJ[o * Nc + i]; };
  // direction r: t1[k][j][a] = sum_i op(a, i) t0[k][j][i]      (k, j over Ni)
  for (int q = tid; q < No * Ni * Ni; q += nt) {
    const int a = q % No, j = (q / No) % Ni, k = q / (No * Ni);
    T acc = T(0);
    for (int i = 0; i < Ni; ++i) acc += op(a, i) * t0[i + Ni * (j + Ni * k)];
    t1[a + No * (j + Ni * k)] = acc;
  }
  __syncthreads();
  // direction s: t0[k][b][a] = sum_j op(b, j) t1[k][j][a]
  for (int q = tid; q < No * No * Ni; q += nt) {
    const int a = q % No, b = (q / No) % No, k = q / (No * No);
    T acc = T(0);
    for (int j = 0; j < Ni; ++j) acc += op(b, j) * t1[a + No * (j + Ni * k)];
    t0[a + No * (b + No * k)] = acc;
  }
  __syncthreads();
  // direction t: out[c][b][a] = sum_k op(c, k) t0[k][b][a]
  for (int q = tid; q < No3; q += nt) {
    const int a = q % No, b = (q / No) % No, c = q / (No * No);
    T acc = T(0);
    for (int k = 0; k < Ni; ++k) acc += op(c, k) * t0[a + No * (b + No * k)];
    const int64_t o = e * No3 + q;
    out[o] = accumulate ? out[o] + acc : acc;
  }
}

// Folded line contraction: NI inputs (stride si) -> NO outputs (stride so), tables [NO/2][NI/2].
template <typename T, int NI, int NO>
__device__ __forceinline__ void eo_transfer_line(const T* __restrict__ Ep, const T* __restrict__ Om,
                                                 const T* src, int si, T* dst, int so) {
  constexpr int HI = NI / 2, HO = NO / 2;
  T e[HI], o[HI];
#pragma unroll
  for (int l = 0; l < HI; ++l) {
    const T a = src[si * l], b = src[si * (NI - 1 - l)];
    e[l] = a + b;
    o[l] = a - b;
  }
#pragma unroll
  for (int k = 0; k < HO; ++k) {
    T E = T(0), O = T(0);
#pragma unroll
    for (int l = 0; l < HI; ++l) {
      E = fma(Ep[k * HI + l], e[l], E);
      O = fma(Om[k * HI + l], o[l], O);
    }
    dst[so * k] = E + O;
    dst[so * (NO - 1 - k)] = E - O;
  }
}

// The last direction's line, stored straight to memory: dst[so * o] = (M v)_o, or += with
// `accumulate`.
template <typename T, int NI, int NO>
__device__ __forceinline__ void eo_transfer_line_out(const T* __restrict__ Ep, const T* __restrict__ Om,
                                                     const T* src, int si, T* __restrict__ dst, int so,
                                                     bool accumulate) {
  constexpr int HI = NI / 2, HO = NO / 2;
  T e[HI], o[HI];
#pragma unroll
  for (int l = 0; l < HI; ++l) {
    const T a = src[si * l], b = src[si * (NI - 1 - l)];
    e[l] = a + b;
    o[l] = a - b;
  }
#pragma unroll
  for (int k = 0; k < HO; ++k) {
    T E = T(0), O = T(0);
#pragma unroll
    for (int l = 0; l < HI; ++l) {
      E = fma(Ep[k * HI + l], e[l], E);
      O = fma(Om[k * HI + l], o[l], O);
    }
    const T lo = E + O, hi = E - O;
    T* d0 = dst + so * k;
    T* d1 = dst + so * (NO - 1 - k);
    *d0 = accumulate ? *d0 + lo : lo;
    *d1 = accumulate ? *d1 + hi : hi;
  }
}

// NE elements per block; prolong: NI = NC -> NO = NF, restrict: NI = NF -> NO = NC.
template <typename T, int NF, int NC, bool RESTRICT>
__global__ void __launch_bounds__(256) transfer_eo_kernel(int64_t E, int NE, const T* __restrict__ Jg,
                                                          const T* __restrict__ in,
                                                          const uint8_t* __restrict__ pflag_in,
                                                          T* __restrict__ out, bool accumulate) {
  constexpr int NI = RESTRICT ? NF : NC, NO = RESTRICT ? NC : NF;
  constexpr int HI = NI / 2, HO = NO / 2;
  constexpr int NI3 = NI * NI * NI, NO3 = NO * NO * NO;
  constexpr int A = (NI3 > NO * NO * NI ? NI3 : NO * NO * NI);  // input, then direction-s output
  constexpr int B = NO * NI * NI;                                 // direction-r output
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ep = reinterpret_cast<T*>(smem_raw);
  T* Om = Ep + HO * HI;
  T* bufA = Om + HO * HI;
  T* bufB = bufA + (size_t)NE * A;
  const int tid = threadIdx.x, nt = blockDim.x;
  // line operator M[o][i]: prolong J[o][i] (NF x NC), restrict J^T: J[i][o]
  for (int q = tid; q < HO * HI; q += nt) {
    const int k = q / HI, l = q - k * HI;
    const T m0 = RESTRICT ? Jg[l * NC + k] : Jg[k * NC + l];
    const T m1 = RESTRICT ? Jg[(NI - 1 - l) * NC + k] : Jg[k * NC + (NI - 1 - l)];
    Ep[q] = T(0.5) * (m0 + m1);
    Om[q] = T(0.5) * (m0 - m1);
  }
  const int64_t e0 = (int64_t)blockIdx.x * NE;
  const int ne = (int)((E - e0) < NE ? (E - e0) : NE);
  for (int q = tid; q < ne * NI3; q += nt) {
    const int le = q / NI3, pt = q - le * NI3;
    T v = in[e0 * NI3 + q];
    if (RESTRICT) v = scale_pow2(v, mult_log2(pflag_in[e0 * NI3 + q]));
    bufA[le * A + pt] = v;
  }
  __syncthreads();
  // direction r: B[k][j][a] = sum_i M(a, i) A[k][j][i]      lines (j, k), NI^2 per element
  for (int q = tid; q < ne * NI * NI; q += nt) {
    const int le = q / (NI * NI), jk = q - le * (NI * NI);
    eo_transfer_line<T, NI, NO>(Ep, Om, bufA + le * A + NI * jk, 1, bufB + le * B + NO * jk, 1);
  }
  __syncthreads();
  // direction s: A[k][b][a] = sum_j M(b, j) B[k][j][a]      lines (a, k), NO NI per element
  for (int q = tid; q < ne * NO * NI; q += nt) {
    const int le = q / (NO * NI), r2 = q - le * (NO * NI), k = r2 / NO, a = r2 - k * NO;
    eo_transfer_line<T, NI, NO>(Ep, Om, bufB + le * B + a + NO * NI * k, NO,
                                bufA + le * A + a + NO * NO * k, NO);
  }
  __syncthreads();
  // direction t: out[c][b][a] = sum_k M(c, k) A[k][b][a]    lines (a, b), NO^2 per element,
  // stored to memory from the line (a warp's lanes hold consecutive (a, b): each plane c of an
  // element is a contiguous store)
  for (int q = tid; q < ne * NO * NO; q += nt) {
    const int le = q / (NO * NO), ab = q - le * (NO * NO);
    eo_transfer_line_out<T, NI, NO>(Ep, Om, bufA + le * A + ab, NO * NO,
                                    out + (e0 + le) * NO3 + ab, NO * NO, accumulate);
  }
}

// Small orders: each direction's outputs are computed one per thread (NI FMAs from shared
// memory), so every warp of a phase is full when NE x (outputs per element) is a multiple of 32.
// Buffers: A = input, then direction-s output; B = direction-r output, then direction-t output.
template <int NF, int NC, bool RESTRICT>
struct TransferSmallDims {
  static constexpr int NI = RESTRICT ? NF : NC, NO = RESTRICT ? NC : NF;
  static constexpr int R1 = NO * NI * NI, R2 = NO * NO * NI, NO3 = NO * NO * NO, NI3 = NI * NI * NI;
  static constexpr int MX = R1 > R2 ? (R1 > NO3 ? R1 : NO3) : (R2 > NO3 ? R2 : NO3);
  static constexpr int THREADS = 256, NE = THREADS / MX;
  static constexpr int A = NI3 > R2 ? NI3 : R2, B = R1 > NO3 ? R1 : NO3;
  static_assert(NE >= 1 && (NE * NO3) % 32 == 0 && (NE * R1) % 32 == 0 && (NE * R2) % 32 == 0,
                "every phase of a small transfer fills whole warps");
};

template <typename T, int NF, int NC, bool RESTRICT>
__global__ void __launch_bounds__(256) transfer_small_kernel(int64_t E, const T* __restrict__ Jg,
                                                             const T* __restrict__ in,
                                                             const uint8_t* __restrict__ pflag_in,
                                                             T* __restrict__ out, bool accumulate) {
  using D = TransferSmallDims<NF, NC, RESTRICT>;
  constexpr int NI = D::NI, NO = D::NO, NE = D::NE, NI3 = D::NI3, NO3 = D::NO3;
  __shared__ T sM[NO * NI];  // line operator M[o][i]: prolong J[o][i], restrict J^T: J[i][o]
  __shared__ T bufA[NE * D::A];
  __shared__ T bufB[NE * D::B];
  const int tid = threadIdx.x;
  for (int q = tid; q < NO * NI; q += D::THREADS) {
    const int o = q / NI, i = q - o * NI;
    sM[q] = RESTRICT ? Jg[i * NC + o] : Jg[o * NC + i];
  }
  const int64_t e0 = (int64_t)blockIdx.x * NE;
  const int ne = (int)((E - e0) < NE ? (E - e0) : NE);
  for (int q = tid; q < ne * NI3; q += D::THREADS) {
    const int le = q / NI3, pt = q - le * NI3;
    T v = in[e0 * NI3 + q];
    if (RESTRICT) v = scale_pow2(v, mult_log2(pflag_in[e0 * NI3 + q]));
    bufA[le * D::A + pt] = v;
  }
  __syncthreads();
  // direction r: B[k][j][a] = sum_i M(a, i) A[k][j][i]
  for (int q = tid; q < ne * D::R1; q += D::THREADS) {
    const int le = q / D::R1, r = q - le * D::R1, a = r % NO, jk = r / NO;
    const T* src = bufA + le * D::A + NI * jk;
    T acc = T(0);
#pragma unroll
    for (int i = 0; i < NI; ++i) acc = fma(sM[a * NI + i], src[i], acc);
    bufB[le * D::B + r] = acc;
  }
  __syncthreads();
  // direction s: A[k][b][a] = sum_j M(b, j) B[k][j][a]
  for (int q = tid; q < ne * D::R2; q += D::THREADS) {
    const int le = q / D::R2, r = q - le * D::R2, a = r % NO, b = (r / NO) % NO, k = r / (NO * NO);
    const T* src = bufB + le * D::B + a + NO * NI * k;
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < NI; ++j) acc = fma(sM[b * NI + j], src[NO * j], acc);
    bufA[le * D::A + r] = acc;
  }
  __syncthreads();
  // direction t: out[c][b][a] = sum_k M(c, k) A[k][b][a]
  for (int q = tid; q < ne * NO3; q += D::THREADS) {
    const int le = q / NO3, r = q - le * NO3, ab = r % (NO * NO), c = r / (NO * NO);
    const T* src = bufA + le * D::A + ab;
    T acc = T(0);
#pragma unroll
    for (int k = 0; k < NI; ++k) acc = fma(sM[c * NI + k], src[NO * NO * k], acc);
    const int64_t o = e0 * NO3 + q;
    out[o] = accumulate ? out[o] + acc : acc;
  }
}

template <typename T, int NF, int NC, bool RESTRICT>
static int launch_transfer_small(const Level& f, const T* J, const T* in, const uint8_t* pflag, T* out,
                                 bool accumulate, cudaStream_t s) {
  using D = TransferSmallDims<NF, NC, RESTRICT>;
  const unsigned blocks = (unsigned)((f.E + D::NE - 1) / D::NE);
  transfer_small_kernel<T, NF, NC, RESTRICT><<<blocks, D::THREADS, 0, s>>>(f.E, J, in, pflag, out, accumulate);
  SE_LAUNCH_CHECK();
  return SE_OK;
}

template <typename T, int NF, int NC, bool RESTRICT>
static int launch_transfer_eo(const Level& f, const T* J, const T* in, const uint8_t* pflag, T* out,
                              bool accumulate, cudaStream_t s) {
  constexpr int NI = RESTRICT ? NF : NC, NO = RESTRICT ? NC : NF;
  constexpr int A = (NI * NI * NI > NO * NO * NI ? NI * NI * NI : NO * NO * NI);
  constexpr int B = NO * NI * NI;
  // about 256 lines of the first direction per block, and at most 96 KB of shared memory (the
  // prolongation from N = 2 to 8 or 10 would need more than the 200 KB a block may have)
  constexpr int NE_LINES = (256 / (NI * NI)) < 1 ? 1 : (256 / (NI * NI));
  constexpr int NE_SMEM = (int)((96 * 1024) / ((A + B) * sizeof(T))) < 1 ? 1 : (int)((96 * 1024) / ((A + B) * sizeof(T)));
  constexpr int NE = NE_LINES < NE_SMEM ? NE_LINES : NE_SMEM;
  static_assert((2 * (NO / 2) * (NI / 2) + (size_t)NE * (A + B)) * sizeof(T) <= 200 * 1024,
                "transfer block exceeds the shared memory limit");
  const size_t smem = (2 * (NO / 2) * (NI / 2) + (size_t)NE * (A + B)) * sizeof(T);
  static const cudaError_t attr = cudaFuncSetAttribute(
      transfer_eo_kernel<T, NF, NC, RESTRICT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  SE_CUDA(attr);
  const unsigned blocks = (unsigned)((f.E + NE - 1) / NE);
  transfer_eo_kernel<T, NF, NC, RESTRICT><<<blocks, 256, smem, s>>>(f.E, NE, J, in, pflag, out, accumulate);
  SE_LAUNCH_CHECK();
  return SE_OK;
}

// Even-even pairs (Nf, Nc) with Nc < Nf <= SE_MAX_ORDER + 1: the folded kernel (the dense
// small-order kernel at 4 <-> 2); false otherwise.
template <typename T, bool RESTRICT>
static bool transfer_eo(const Level& f, const Level& c, const T* J, const T* in, const uint8_t* pflag,
                        T* out, bool accumulate, cudaStream_t s, int* st) {
  if (f.N == 4 && c.N == 2) {
    *st = launch_transfer_small<T, 4, 2, RESTRICT>(f, J, in, pflag, out, accumulate, s);
    return true;
  }
#define SE_TR(NF_, NC_)                                                                      \
  if (f.N == NF_ && c.N == NC_) {                                                            \
    *st = launch_transfer_eo<T, NF_, NC_, RESTRICT>(f, J, in, pflag, out, accumulate, s);    \
    return true;                                                                             \
  }
  SE_TR(6, 2) SE_TR(6, 4) SE_TR(8, 2) SE_TR(8, 4) SE_TR(8, 6)
  SE_TR(10, 2) SE_TR(10, 4) SE_TR(10, 6) SE_TR(10, 8)
#undef SE_TR
  return false;
}

template <class T>
int restrict_apply(const Level& f, const Level& c, const T* J, const T* rf, T* rc, cudaStream_t s) {
  const double Nf = f.N, Nc = c.N;
  {
    ProfScope prof(SE_K_RESTRICT, s, (double)f.E,
                   f.E * (Nf * Nf * Nf * (sizeof(T) + 1.0) + Nc * Nc * Nc * sizeof(T)),
                   2.0 * f.E * (Nf * Nf * Nf * Nc + Nf * Nf * Nc * Nc + Nf * Nc * Nc * Nc),
                   prof_variant<T>(f.p));
    int st = SE_OK;
    if (transfer_eo<T, true>(f, c, J, rf, f.pflag, rc, false, s, &st)) {
      SE_TRY(st);
    } else {
      transfer_kernel<T, true><<<(unsigned)f.E, 128, 0, s>>>(f.N, c.N, J, rf, f.pflag, rc, false);
      SE_LAUNCH_CHECK();
    }
  }
  return gs_apply<T>(c, rc, true, s);
}

template <class T>
int prolong_apply(const Level& f, const Level& c, const T* J, const T* ec, T* ef, bool accumulate,
                  cudaStream_t s) {
  const double Nf = f.N, Nc = c.N;
  ProfScope prof(SE_K_PROLONG, s, (double)f.E,
                 f.E * (Nf * Nf * Nf * (accumulate ? 2.0 : 1.0) + Nc * Nc * Nc) * sizeof(T),
                 2.0 * f.E * (Nc * Nc * Nc * Nf + Nc * Nc * Nf * Nf + Nc * Nf * Nf * Nf),
                 prof_variant<T>(f.p));
  int st = SE_OK;
  if (transfer_eo<T, false>(f, c, J, ec, nullptr, ef, accumulate, s, &st)) return st;
  transfer_kernel<T, false><<<(unsigned)f.E, 128, 0, s>>>(f.N, c.N, J, ec, nullptr, ef, accumulate);
  SE_LAUNCH_CHECK();
  return SE_OK;
}

template int restrict_apply<double>(const Level&, const Level&, const double*, const double*, double*, cudaStream_t);
template int restrict_apply<float>(const Level&, const Level&, const float*, const float*, float*, cudaStream_t);
template int prolong_apply<double>(const Level&, const Level&, const double*, const double*, double*, bool, cudaStream_t);
template int prolong_apply<float>(const Level&, const Level&, const float*, const float*, float*, bool, cudaStream_t);

}  // namespace se
