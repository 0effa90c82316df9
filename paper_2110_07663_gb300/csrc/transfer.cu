// p-multigrid transfers between GLL bases (Algorithm 1, Sec. 2.2.2):
//   prolongation  e_f = (J x J x J) e_c            element by element
//   restriction   r_c = M_c QQ^T_c (J^T x J^T x J^T)(r_f / mult_f)
// with J_ij = h^c_j(xi^f_i).  For a continuous r_f the restriction is the transpose of the
// global prolongation.  One element per block; the three directions are contracted in turn in
// shared memory.
#include "se_internal.h"

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
    if (RESTRICT) {
      const int mlog = __ffs(pflag_in[e * Ni3 + q] & 0x0F) - 1;
      v *= mlog == 0 ? T(1) : (mlog == 1 ? T(0.5) : (mlog == 2 ? T(0.25) : T(0.125)));
    }
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

template <class T>
int restrict_apply(const Level& f, const Level& c, const T* J, const T* rf, T* rc, cudaStream_t s) {
  const double Nf = f.N, Nc = c.N;
  {
    ProfScope prof(SE_K_RESTRICT, s, (double)f.E,
                   f.E * (Nf * Nf * Nf * (sizeof(T) + 1.0) + Nc * Nc * Nc * sizeof(T)),
                   2.0 * f.E * (Nf * Nf * Nf * Nc + Nf * Nf * Nc * Nc + Nf * Nc * Nc * Nc),
                   prof_variant<T>(f.p));
    transfer_kernel<T, true><<<(unsigned)f.E, 128, 0, s>>>(f.N, c.N, J, rf, f.pflag, rc, false);
    SE_LAUNCH_CHECK();
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
  transfer_kernel<T, false><<<(unsigned)f.E, 128, 0, s>>>(f.N, c.N, J, ec, nullptr, ef, accumulate);
  SE_LAUNCH_CHECK();
  return SE_OK;
}

template int restrict_apply<double>(const Level&, const Level&, const double*, const double*, double*, cudaStream_t);
template int restrict_apply<float>(const Level&, const Level&, const float*, const float*, float*, cudaStream_t);
template int prolong_apply<double>(const Level&, const Level&, const double*, const double*, double*, bool, cudaStream_t);
template int prolong_apply<float>(const Level&, const Level&, const float*, const float*, float*, bool, cudaStream_t);

}  // namespace se
