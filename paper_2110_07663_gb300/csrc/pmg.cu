// p-multigrid preconditioner (Sec. 2.2): level hierarchy, Chebyshev-accelerated smoothing
// (Algorithm 2), single-pass V-cycle (Algorithm 1), Chebyshev bounds from Arnoldi on S A.
#include <algorithm>
#include <cmath>
#include <atomic>
#include <complex>
#include <cstring>
#include <vector>

#include "pmg_internal.h"

namespace se {

// ------------------------------------------------------------------ eigenvalues of a small
// upper Hessenberg matrix: complex single-shift QR with Wilkinson shifts and deflation.
static void hessenberg_eigs(int n, const double* Hin, std::vector<std::complex<double>>& ev) {
  using cd = std::complex<double>;
  std::vector<cd> H(n * n);
  for (int q = 0; q < n * n; ++q) H[q] = Hin[q];
  ev.clear();
  int hi = n - 1, iter = 0, total = 0;
  while (hi >= 0) {
    if (hi == 0) {
      ev.push_back(H[0]);
      break;
    }
    int l = hi;
    while (l > 0) {
      double sc = std::abs(H[(l - 1) * n + l - 1]) + std::abs(H[l * n + l]);
      if (sc == 0.0) sc = 1.0;
      if (std::abs(H[l * n + l - 1]) <= 1e-15 * sc) break;
      --l;
    }
    if (l == hi || total > 200 * n) {
      ev.push_back(H[hi * n + hi]);
      --hi;
      iter = 0;
      continue;
    }
    if (l > 0) H[l * n + l - 1] = 0.0;
    const cd a = H[(hi - 1) * n + hi - 1], b = H[(hi - 1) * n + hi];
    const cd c = H[hi * n + hi - 1], d = H[hi * n + hi];
    const cd tr = a + d, det = a * d - b * c;
    const cd disc = std::sqrt(tr * tr / 4.0 - det);
    const cd m1 = tr / 2.0 + disc, m2 = tr / 2.0 - disc;
    cd mu = std::abs(m1 - d) < std::abs(m2 - d) ? m1 : m2;
    if (++iter % 11 == 0) mu = d + std::abs(c);  // exceptional shift
    ++total;
    for (int k = l; k <= hi; ++k) H[k * n + k] -= mu;
    std::vector<cd> cs(hi - l), sn(hi - l);
    for (int k = l; k < hi; ++k) {
      const cd x = H[k * n + k], y = H[(k + 1) * n + k];
      const double r = std::sqrt(std::norm(x) + std::norm(y));
      const cd cc = r == 0.0 ? cd(1.0) : x / r, ss = r == 0.0 ? cd(0.0) : y / r;
      cs[k - l] = cc;
      sn[k - l] = ss;
      for (int j = k; j <= hi; ++j) {
        const cd t1 = H[k * n + j], t2 = H[(k + 1) * n + j];
        H[k * n + j] = std::conj(cc) * t1 + std::conj(ss) * t2;
        H[(k + 1) * n + j] = -ss * t1 + cc * t2;
      }
    }
    for (int k = l; k < hi; ++k) {
      const cd cc = cs[k - l], ss = sn[k - l];
      const int iend = std::min(k + 2, hi);
      for (int i = l; i <= iend; ++i) {
        const cd t1 = H[i * n + k], t2 = H[i * n + k + 1];
        H[i * n + k] = t1 * cc + t2 * ss;
        H[i * n + k + 1] = -t1 * std::conj(ss) + t2 * std::conj(cc);
      }
    }
    for (int k = l; k <= hi; ++k) H[k * n + k] += mu;
  }
}

// Arnoldi start vector: 2U-1 of the level's global node id (SplitMix64 stream `seed`), masked.
__global__ void start_vector_kernel(int N, int nx, int ny, int64_t L, uint64_t seed,
                                    const uint8_t* __restrict__ pflag, double* __restrict__ v) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= L) return;
  const int N3 = N * N * N, p = N - 1;
  const int64_t e = idx / N3;
  const int pt = (int)(idx - e * N3);
  const int i = pt % N, j = (pt / N) % N, k = pt / (N * N);
  const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
  const int64_t NX = (int64_t)nx * p + 1, NY = (int64_t)ny * p + 1;
  const int64_t g = (ex * p + i) + NX * ((ey * p + j) + NY * (int64_t)(ez * p + k));
  const double u = (double)(splitmix64_hd(seed, (uint64_t)g) >> 11) * (1.0 / 9007199254740992.0);
  v[idx] = (pflag[idx] & PF_FREE) ? 2.0 * u - 1.0 : 0.0;
}

// ------------------------------------------------------------------ smoother and Chebyshev
template <class T>
const T* dinv_of(const Level& lv) {
  if constexpr (sizeof(T) == 8) return lv.dinv64;
  else return lv.dinv32;
}

template <class T>
int smooth(se_pmg_s* P, int l, const T* in, T* out, cudaStream_t s) {
  const Level& lv = *P->lv[l];
  if (P->desc.smoother == SE_SMOOTH_JACOBI) return scale_mul<T>(dinv_of<T>(lv), in, out, lv.L, s);
  return schwarz_apply<T>(lv, P->desc.smoother, in, out, s);
}

// Algorithm 2 for the residual `res`: x = correction (first) or x += correction.
template <class T>
int cheby(se_pmg_s* P, int l, const T* res, T* x, bool first, cudaStream_t s) {
  const Level& lv = *P->lv[l];
  LevelVecs<T>& V = P->vecs<T>(l);
  const double lmin = P->lmin[l], lmax = P->lmax[l];
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  const int order = P->desc.cheb_order[l];
  const bool jac = P->desc.smoother == SE_SMOOTH_JACOBI;
  // FP64 Jacobi on a folded-operator level: S res = D^-1 res is not stored; the first step's
  // operator scales its input as it loads it and the update forms D^-1 res itself
  bool fused = false;
  if constexpr (std::is_same<T, double>::value) fused = jac && order >= 1 && ax_fold_ok(lv);
  if (!fused) SE_TRY(smooth<T>(P, l, res, V.cr, s));             // r = S res
  const T inv_theta = T(1.0 / theta);
  if (order == 0) {                                              // x (+)= r / theta
    if (first) return axpby<T>(inv_theta, V.cr, T(0), V.cr, x, lv.L, s);
    return axpby<T>(inv_theta, V.cr, T(1), x, x, lv.L, s);
  }
  // d = r / theta is not stored: the first step applies A (and S) to r and scales by 1/theta
  for (int k = 0; k < order; ++k) {
    const bool from_r = k == 0, last = k == order - 1;
    if constexpr (std::is_same<T, double>::value) {
      if (fused && from_r) SE_TRY(ax_apply_folded(lv, res, V.w, nullptr, s, lv.dinv64));  // A D^-1 res
      else SE_TRY(ax_apply<T>(lv, from_r ? V.cr : V.cd, V.w, s));
    } else {
      SE_TRY(ax_apply<T>(lv, from_r ? V.cr : V.cd, V.w, s));     // A d  (A r for the first step)
    }
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    const T c1 = T(rho_new * rho), c2 = T(2.0 * rho_new / delta);
    const T* sa = V.w;                                           // Jacobi: dinv .* A d in the update
    if (!jac) {
      SE_TRY(smooth<T>(P, l, V.w, V.sv, s));                     // S A d
      sa = V.sv;
    }
    SE_TRY(cheb_update<T>(x, V.cd, V.cr, sa, jac ? dinv_of<T>(lv) : (const T*)nullptr, lv.L, c1, c2,
                          first && k == 0, s, inv_theta, from_r, last,
                          fused && from_r ? res : (const T*)nullptr, lv.p));  // last: also x += d
    rho = rho_new;
  }
  return SE_OK;
}

template <class T>
const T* jmat(se_pmg_s* P, int l) {
  if constexpr (sizeof(T) == 8) return P->J64[l];
  else return P->J32[l];
}

// Algorithm 1 on level l: vecs(l).b -> vecs(l).x
template <class T>
int vcycle(se_pmg_s* P, int l, cudaStream_t s) {
  LevelVecs<T>& V = P->vecs<T>(l);
  const Level& lv = *P->lv[l];
  if (l == P->nlev - 1) {
    if (P->cgroup) return coarse_group_solve<T>(*P->cgroup, s);  // reads V.b, writes V.x
    return coarse_solve<T>(lv, P->cw, V.b, V.x, P->desc.coarse_tol, P->desc.coarse_maxit, s);
  }
  LevelVecs<T>& C = P->vecs<T>(l + 1);
  const Level& lc = *P->lv[l + 1];
  SE_TRY(cheby<T>(P, l, V.b, V.x, true, s));                    // x = M b
  SE_TRY(residual_apply<T>(lv, V.b, V.x, V.r, s));               // r = b - A x
  SE_TRY(restrict_apply<T>(lv, lc, jmat<T>(P, l), V.r, C.b, s)); // r_C = P^T r
  SE_TRY(vcycle<T>(P, l + 1, s));                               // e_C
  SE_TRY(prolong_apply<T>(lv, lc, jmat<T>(P, l), C.x, V.x, true, s));  // x += P e_C
  SE_TRY(residual_apply<T>(lv, V.b, V.x, V.r, s));               // b - A x
  return cheby<T>(P, l, V.r, V.x, false, s);                    // x += M (b - A x)
}

// Additive V-cycle on level l (Sec. 2.2.2, Schwarz smoothers without Chebyshev acceleration):
// the smoother and the coarse correction act on the same right-hand side, x = S b + P V(P^T b),
// with no residual re-evaluation and no post-smoothing.
template <class T>
int vcycle_additive(se_pmg_s* P, int l, cudaStream_t s) {
  LevelVecs<T>& V = P->vecs<T>(l);
  const Level& lv = *P->lv[l];
  if (l == P->nlev - 1)
    return coarse_solve<T>(lv, P->cw, V.b, V.x, P->desc.coarse_tol, P->desc.coarse_maxit, s);
  LevelVecs<T>& C = P->vecs<T>(l + 1);
  const Level& lc = *P->lv[l + 1];
  SE_TRY(smooth<T>(P, l, V.b, V.x, s));                          // x = S b
  SE_TRY(restrict_apply<T>(lv, lc, jmat<T>(P, l), V.b, C.b, s)); // r_C = P^T b
  SE_TRY(vcycle_additive<T>(P, l + 1, s));                       // e_C
  return prolong_apply<T>(lv, lc, jmat<T>(P, l), C.x, V.x, true, s);  // x += P e_C
}

template <class T>
int cycle(se_pmg_s* P, cudaStream_t s) {
  return P->desc.cycle == SE_CYCLE_ADDITIVE ? vcycle_additive<T>(P, 0, s) : vcycle<T>(P, 0, s);
}

template <class T>
int apply_typed(se_pmg_s* P, const double* r, double* z, cudaStream_t s) {
  LevelVecs<T>& V = P->vecs<T>(0);
  const int64_t L = P->lv[0]->L;
  if constexpr (sizeof(T) == 8) {
    // FP64: the V-cycle reads the finest right-hand side without writing it and writes only its
    // result, so it runs on r and z themselves (no copies in or out) unless they are one vector
    if (r != z) {
      double* const b0 = V.b;
      double* const x0 = V.x;
      V.b = const_cast<double*>(r);
      V.x = z;
      const int st = cycle<T>(P, s);
      V.b = b0;
      V.x = x0;
      return st;
    }
  }
  SE_TRY((convert<double, T>(r, V.b, L, s)));
  SE_TRY(cycle<T>(P, s));
  return convert<T, double>(V.x, z, L, s);
}

int pmg_apply(se_pmg_s* P, const double* r, double* z, cudaStream_t s) {
  if (P->desc.precision == SE_FP32) return apply_typed<float>(P, r, z, s);
  return apply_typed<double>(P, r, z, s);
}

// ------------------------------------------------------------------ Arnoldi bound estimate
static int arnoldi_level(se_pmg_s* P, int l, cudaStream_t s, double* lam_out) {
  Level& lv = *P->lv[l];
  const int steps = P->desc.arnoldi_steps;
  const int64_t L = lv.L;
  std::vector<double*> Vv(steps + 1, nullptr);
  double *w = nullptr, *sv = nullptr;
  int st = SE_OK;
  // transient vectors, stream-ordered on s (freeing them does not wait for other streams)
  auto cleanup = [&]() {
    for (double* v : Vv)
      if (v) cudaFreeAsync(v, s);
    if (w) cudaFreeAsync(w, s);
    if (sv) cudaFreeAsync(sv, s);
  };
  for (auto& v : Vv)
    if (dmalloc_transient(reinterpret_cast<void**>(&v), L * sizeof(double), s) != SE_OK) {
      cleanup();
      set_error("Arnoldi: out of device memory");
      return SE_ENOMEM;
    }
  if (dmalloc_transient(reinterpret_cast<void**>(&w), L * sizeof(double), s) != SE_OK ||
      dmalloc_transient(reinterpret_cast<void**>(&sv), L * sizeof(double), s) != SE_OK) {
    cleanup();
    set_error("Arnoldi: out of device memory");
    return SE_ENOMEM;
  }
  Scratch& sc = P->scratch;
  const uint64_t seed = 1000ULL + (uint64_t)l + 7919ULL * P->desc.seed;
  start_vector_kernel<<<grid_for(L, 256), 256, 0, s>>>(lv.N, lv.nel[0], lv.nel[1], L, seed, lv.pflag, Vv[0]);
  std::vector<double> H((steps + 1) * steps, 0.0);  // H[i * steps + j]
  int m = steps;
  double hmax = 0.0;
  if ((st = dot_to_slot(lv, Vv[0], Vv[0], sc, SC_NORM, s)) != SE_OK ||
      (st = scale_inv_sqrt(Vv[0], Vv[0], sc.scal, SC_NORM, L, s)) != SE_OK) {
    cleanup();
    return st;
  }
  for (int j = 0; j < steps; ++j) {
    if ((st = ax_apply<double>(lv, Vv[j], w, s)) != SE_OK) break;
    if (P->desc.smoother == SE_SMOOTH_JACOBI) st = scale_mul<double>(lv.dinv64, w, sv, L, s);
    else st = schwarz_apply<double>(lv, P->desc.smoother, w, sv, s);
    if (st != SE_OK) break;
    if ((st = dot_to_slot(lv, sv, Vv[0], sc, SC_H, s)) != SE_OK) break;
    for (int i = 0; i <= j && st == SE_OK; ++i)
      st = axpy_dot(lv, sv, Vv[i], i < j ? Vv[i + 1] : nullptr, sc, SC_H + i,
                    i < j ? SC_H + i + 1 : SC_NORM, s);
    if (st != SE_OK) break;
    if (cudaMemcpyAsync(sc.hscal, sc.scal, SCAL_SLOTS * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      set_error("Arnoldi: %s", cudaGetErrorString(cudaGetLastError()));
      st = SE_ECUDA;
      break;
    }
    for (int i = 0; i <= j; ++i) {
      H[i * steps + j] = sc.hscal[SC_H + i];
      hmax = std::max(hmax, std::fabs(H[i * steps + j]));
    }
    const double sub = std::sqrt(std::max(sc.hscal[SC_NORM], 0.0));
    H[(j + 1) * steps + j] = sub;
    hmax = std::max(hmax, sub);
    if (sub <= 1e-12 * hmax) {  // Krylov space exhausted
      m = j + 1;
      break;
    }
    if (j + 1 <= steps && (st = scale_inv_sqrt(Vv[j + 1], sv, sc.scal, SC_NORM, L, s)) != SE_OK) break;
  }
  cudaStreamSynchronize(s);
  cleanup();
  if (st != SE_OK) return st;
  std::vector<double> Hm(m * m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) Hm[i * m + j] = H[i * steps + j];
  std::vector<std::complex<double>> ev;
  hessenberg_eigs(m, Hm.data(), ev);
  double lam = 0.0;
  for (auto& z : ev) lam = std::max(lam, std::abs(z));
  *lam_out = lam;
  return SE_OK;
}

// ------------------------------------------------------------------ set-up
// df64 arithmetic for the Arnoldi rounds of an FP64 or FP32 preconditioner: df64 copies of the
// smoothed levels' geometry and FDM factors live only while the bounds are estimated (copies
// the mesh already holds for its outer operator are used as they are).
static int df_transient(const double* src, df64** dst, int64_t n, cudaStream_t s,
                        std::vector<void*>& keep) {
  void* p = nullptr;
  SE_TRY(dmalloc_transient(&p, (size_t)n * sizeof(df64), s));
  keep.push_back(p);
  *dst = static_cast<df64*>(p);
  return split_df(src, *dst, n, s);
}

static int arnoldi_df_begin(se_pmg_s* P, cudaStream_t s, std::vector<void*>& keep) {
  for (int l = 0; l + 1 < P->nlev; ++l) {
    Level& lv = *P->lv[l];
    const int H = lv.N / 2, PB = lv.p + 3;
    const bool eo = ax_eo_supported(lv.p) && lv.eo64;
    if (!lv.Gdf) SE_TRY(df_transient(lv.G64, &lv.Gdf, 6 * lv.L, s, keep));
    if (eo && !lv.eodf) SE_TRY(df_transient(lv.eo64, &lv.eodf, 4 * H * H, s, keep));
    if (!eo && !lv.Ddf) SE_TRY(df_transient(lv.D64, &lv.Ddf, (int64_t)lv.N * lv.N, s, keep));
    if (lv.S64 && !lv.Sdf) {
      SE_TRY(df_transient(lv.S64, &lv.Sdf, 3 * lv.E * PB * PB, s, keep));
      SE_TRY(df_transient(lv.lam64, &lv.lamdf, 3 * lv.E * PB, s, keep));
    }
    lv.df = true;
  }
  return SE_OK;
}

static void arnoldi_df_end(se_pmg_s* P, cudaStream_t s, std::vector<void*>& keep) {
  auto owned = [&](void* p) { return std::find(keep.begin(), keep.end(), p) != keep.end(); };
  for (int l = 0; l + 1 < P->nlev; ++l) {
    Level& lv = *P->lv[l];
    lv.df = false;
    if (owned(lv.Gdf)) lv.Gdf = nullptr;
    if (owned(lv.eodf)) lv.eodf = nullptr;
    if (owned(lv.Ddf)) lv.Ddf = nullptr;
    if (owned(lv.Sdf)) lv.Sdf = nullptr;
    if (owned(lv.lamdf)) lv.lamdf = nullptr;
  }
  for (void* p : keep) cudaFreeAsync(p, s);
  keep.clear();
}

template <class T>
static int alloc_vecs(se_pmg_s* P, int l) {
  LevelVecs<T>& V = P->vecs<T>(l);
  const int64_t L = P->lv[l]->L;
  for (T** q : {&V.b, &V.x, &V.r, &V.cr, &V.cd, &V.w, &V.sv}) SE_TRY(dmalloc(P->allocs, q, L));
  return SE_OK;
}

int pmg_alloc_vecs(se_pmg_s* P, int l, bool fp32) {
  return fp32 ? alloc_vecs<float>(P, l) : alloc_vecs<double>(P, l);
}

static int pmg_build(se_pmg_s* P) {
  se_mesh_s* m = P->mesh;
  cudaStream_t s = P->stream;
  const se_pmg_desc& d = P->desc;
  const bool fp32 = d.precision == SE_FP32;
  const bool df = d.precision == SE_DF64;
  SE_TRY(scratch_alloc(P->allocs, &P->scratch));
  // df64 copies of the fine geometry belong to the mesh (the outer operator may use them too)
  if (df) SE_TRY(make_df_geometry(m->fine, m->allocs, s));
  P->owned[0] = m->fine;  // shallow copy: shares the mesh's geometry and maps
  P->owned[0].G32 = nullptr;
  P->lv[0] = &P->owned[0];
  for (int l = 1; l < P->nlev; ++l) {
    SE_TRY(build_level(m, d.schedule[l], &P->owned[l], P->allocs, s));
    SE_TRY(build_jacobi(P->owned[l], P->allocs, P->scratch, s));
    P->lv[l] = &P->owned[l];
  }
  for (int l = 0; l < P->nlev; ++l) {
    Level& lv = *P->lv[l];
    const bool coarsest = l == P->nlev - 1;
    if (fp32 && !coarsest) SE_TRY(make_fp32_geometry(lv, P->allocs, s));
    if (df && !coarsest) {
      SE_TRY(make_df_geometry(lv, P->allocs, s));
      lv.df = true;
    }
    if (!coarsest && d.smoother != SE_SMOOTH_JACOBI) {
      SE_TRY(fdm_setup(m, lv, P->allocs, fp32, s, df));
      if (d.smoother == SE_SMOOTH_ASM) {
        const int64_t n3 = lv.E * (int64_t)(lv.p + 3) * (lv.p + 3) * (lv.p + 3);
        SE_TRY(dmalloc(P->allocs, &lv.ext64, n3));
        if (fp32) SE_TRY(dmalloc(P->allocs, &lv.ext32, n3));
      }
    }
    if (coarsest) SE_TRY(coarse_setup(lv, P->allocs, s));
  }
  for (int l = 0; l + 1 < P->nlev; ++l) {
    const int Nf = d.schedule[l] + 1, Nc = d.schedule[l + 1] + 1;
    std::vector<double> J(Nf * Nc);
    std::vector<float> J32(Nf * Nc);
    interp_matrix(d.schedule[l], d.schedule[l + 1], J.data());
    for (int q = 0; q < Nf * Nc; ++q) J32[q] = (float)J[q];
    SE_TRY(dmalloc(P->allocs, &P->J64[l], Nf * Nc));
    SE_TRY(dmalloc(P->allocs, &P->J32[l], Nf * Nc));
    SE_TRY(h2d(P->J64[l], J.data(), Nf * Nc * sizeof(double), P->stream));
    SE_TRY(h2d(P->J32[l], J32.data(), Nf * Nc * sizeof(float), P->stream));
  }
  SE_TRY(coarse_alloc(*P->lv[P->nlev - 1], P->allocs, &P->cw));
  for (int l = 0; l < P->nlev; ++l) {
    if (fp32) SE_TRY(alloc_vecs<float>(P, l));
    else SE_TRY(alloc_vecs<double>(P, l));
  }
  // the coarse level always solves in FP64 from the V-cycle's precision; Arnoldi needs FP64
  // vectors (and FP64 or df64 arithmetic)
  std::vector<void*> transient;
  if (!df && d.arnoldi_df64) {
    const int rb = arnoldi_df_begin(P, s, transient);
    if (rb != SE_OK) {
      arnoldi_df_end(P, s, transient);
      return rb;
    }
  }
  SE_CUDA(cudaStreamSynchronize(s));
  int rc = SE_OK;
  for (int l = 0; l + 1 < P->nlev && rc == SE_OK; ++l) {
    double lam = 0.0;
    rc = arnoldi_level(P, l, s, &lam);
    P->lam[l] = lam;
    P->lmin[l] = d.eig_lo * lam;
    P->lmax[l] = d.eig_hi * lam;
  }
  if (!df && d.arnoldi_df64) arnoldi_df_end(P, s, transient);
  SE_TRY(rc);
  SE_CUDA(cudaStreamSynchronize(s));
  return SE_OK;
}

// Runs `fn` on level-lvl vectors of the pmg precision, converting FP64 in/out.
template <class F64, class F32>
static int precision_io(se_pmg_s* P, int lvl, const double* in, double* out, cudaStream_t s, F64 f64,
                        F32 f32) {
  const int64_t L = P->lv[lvl]->L;
  if (P->desc.precision == SE_FP32) {
    LevelVecs<float>& V = P->vecs<float>(lvl);
    SE_TRY((convert<double, float>(in, V.b, L, s)));
    SE_TRY(f32(V.b, V.x));
    return convert<float, double>(V.x, out, L, s);
  }
  return f64(in, out);
}

int pmg_faults_take(se_pmg_s* P, cudaStream_t s) {
  int rc = SE_OK;
  for (int l = 0; l < P->nlev; ++l)
    if (P->lv[l] && level_pipeline_take(*P->lv[l], s) != SE_OK) rc = SE_ETIMEOUT;
  if (coarse_fault_take(P->cw, s) != SE_OK) rc = SE_ETIMEOUT;
  return rc;
}

}  // namespace se

using namespace se;

extern "C" {

int se_pmg_setup(se_mesh_t m, const se_pmg_desc* desc, se_pmg_t* out) {
  SE_CHECK(m && desc && out, SE_EINVAL, "se_pmg_setup: null argument");
  const se_pmg_desc& d = *desc;
  SE_CHECK(d.nlev >= 2 && d.nlev <= SE_MAX_LEVELS, SE_EINVAL, "se_pmg_setup: nlev=%d not in 2..%d",
           d.nlev, SE_MAX_LEVELS);
  SE_CHECK(d.schedule[0] == m->fine.p, SE_EINVAL, "se_pmg_setup: schedule[0]=%d != mesh p=%d",
           d.schedule[0], m->fine.p);
  for (int l = 1; l < d.nlev; ++l)
    SE_CHECK(d.schedule[l] >= 1 && d.schedule[l] < d.schedule[l - 1], SE_EINVAL,
             "se_pmg_setup: schedule must decrease strictly (level %d)", l);
  SE_CHECK(d.schedule[d.nlev - 1] == 1, SE_EINVAL, "se_pmg_setup: the coarsest order must be 1");
  SE_CHECK(d.smoother == SE_SMOOTH_JACOBI || d.smoother == SE_SMOOTH_RAS || d.smoother == SE_SMOOTH_ASM,
           SE_EINVAL, "se_pmg_setup: bad smoother %d", d.smoother);
  for (int l = 0; l + 1 < d.nlev; ++l)
    SE_CHECK(d.cheb_order[l] >= 0 && d.cheb_order[l] <= 32, SE_EINVAL,
             "se_pmg_setup: Chebyshev order %d out of range", d.cheb_order[l]);
  // eig_lo = 0 is allowed (Table 1's first row): sigma = 1 and the Chebyshev polynomial no longer
  // damps, but the recurrence stays finite
  SE_CHECK(d.eig_hi > d.eig_lo && d.eig_lo >= 0, SE_EINVAL, "se_pmg_setup: need 0 <= eig_lo < eig_hi");
  SE_CHECK(d.arnoldi_steps >= 1 && d.arnoldi_steps <= 100, SE_EINVAL, "se_pmg_setup: arnoldi_steps");
  SE_CHECK(d.coarse_tol > 0 && d.coarse_maxit >= 1, SE_EINVAL, "se_pmg_setup: coarse tolerance");
  SE_CHECK(d.precision == SE_FP64 || d.precision == SE_FP32 || d.precision == SE_DF64, SE_EINVAL,
           "se_pmg_setup: precision");
  SE_CHECK(d.cycle == SE_CYCLE_MULTIPLICATIVE || d.cycle == SE_CYCLE_ADDITIVE, SE_EINVAL,
           "se_pmg_setup: cycle %d", d.cycle);
  SE_CHECK(d.arnoldi_df64 == 0 || d.arnoldi_df64 == 1, SE_EINVAL, "se_pmg_setup: arnoldi_df64");
  static std::atomic<uint64_t> next_uid{0};
  auto* P = new se_pmg_s();
  P->mesh = m;
  P->uid = ++next_uid;
  P->desc = d;
  P->nlev = d.nlev;
  P->stream = m->stream;
  P->allocs.stream = P->stream;
  int st = pmg_build(P);
  if (st != SE_OK) {
    cudaStreamSynchronize(P->stream);
    P->allocs.release();
    pinned_release(P->scratch.hscal);
    delete P;
    return st;
  }
  *out = P;
  return SE_OK;
}

int se_pmg_destroy(se_pmg_t P) {
  if (!P) return SE_OK;
  cudaStreamSynchronize(P->stream);
  se_mesh_s* m = P->mesh;
  if (m && m->gexec && m->gpmg_uid == P->uid) {  // the mesh's cached solve graph uses this handle
    cudaGraphExecDestroy(m->gexec);
    m->gexec = nullptr;
    m->gkey[0] = nullptr;
    m->gpmg_uid = 0;
  }
  P->release_graph();
  P->allocs.release();
  pinned_release(P->scratch.hscal);
  delete P;
  return SE_OK;
}

int se_pmg_coarse_stats(se_pmg_t P, int reset, int64_t* solves, int64_t* iterations) {
  SE_CHECK(P && P->cw.totals, SE_EINVAL, "se_pmg_coarse_stats: null argument");
  unsigned long long h[2] = {0, 0};
  SE_CUDA(cudaStreamSynchronize(P->stream));
  SE_CUDA(cudaMemcpy(h, P->cw.totals, sizeof(h), cudaMemcpyDeviceToHost));
  if (solves) *solves = (int64_t)h[1];
  if (iterations) *iterations = (int64_t)h[0];
  if (reset) SE_TRY(dzero(P->cw.totals, sizeof(h), P->stream));
  return SE_OK;
}

int se_pmg_apply(se_pmg_t P, const double* r, double* z, void* stream) {
  SE_CHECK(P && r && z, SE_EINVAL, "se_pmg_apply: null argument");
  return pmg_apply(P, r, z, as_stream(stream, P->stream));
}

int se_pmg_lambda(se_pmg_t P, int lvl, double* lam) {
  SE_CHECK(P && lam, SE_EINVAL, "se_pmg_lambda: null argument");
  SE_CHECK(lvl >= 0 && lvl + 1 < P->nlev, SE_EINVAL, "se_pmg_lambda: level %d has no smoother", lvl);
  *lam = P->lam[lvl];
  return SE_OK;
}

int se_pmg_level_info(se_pmg_t P, int lvl, se_mesh_info* info) {
  SE_CHECK(P && info && lvl >= 0 && lvl < P->nlev, SE_EINVAL, "se_pmg_level_info: bad argument");
  const Level& lv = *P->lv[lvl];
  info->E = lv.E;
  info->N = lv.N;
  info->L = lv.L;
  info->n_global = lv.n_global;
  info->n_dof = lv.E * (int64_t)lv.p * lv.p * lv.p;
  info->p = lv.p;
  for (int d = 0; d < 3; ++d) info->nel[d] = lv.nel[d];
  return SE_OK;
}

int se_pmg_level_ax(se_pmg_t P, int lvl, const double* u, double* y, void* stream) {
  SE_CHECK(P && u && y && lvl >= 0 && lvl < P->nlev, SE_EINVAL, "se_pmg_level_ax: bad argument");
  return ax_apply<double>(*P->lv[lvl], u, y, as_stream(stream, P->stream));
}

int se_pmg_smooth(se_pmg_t P, int lvl, const double* r, double* z, void* stream) {
  SE_CHECK(P && r && z && lvl >= 0 && lvl + 1 < P->nlev, SE_EINVAL, "se_pmg_smooth: bad argument");
  cudaStream_t s = as_stream(stream, P->stream);
  return precision_io(
      P, lvl, r, z, s, [&](const double* a, double* b) { return smooth<double>(P, lvl, a, b, s); },
      [&](const float* a, float* b) { return smooth<float>(P, lvl, a, b, s); });
}

int se_pmg_cheby(se_pmg_t P, int lvl, const double* r, double* x, void* stream) {
  SE_CHECK(P && r && x && lvl >= 0 && lvl + 1 < P->nlev, SE_EINVAL, "se_pmg_cheby: bad argument");
  SE_CHECK(r != x, SE_EINVAL, "se_pmg_cheby: r and x must differ");
  cudaStream_t s = as_stream(stream, P->stream);
  if (P->desc.precision != SE_FP32) {
    // the level's b vector holds a copy of r so that the caller's r is never written
    LevelVecs<double>& V = P->vecs<double>(lvl);
    SE_CUDA(cudaMemcpyAsync(V.b, r, P->lv[lvl]->L * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return cheby<double>(P, lvl, V.b, x, true, s);
  }
  return precision_io(
      P, lvl, r, x, s, [&](const double*, double*) { return SE_OK; },
      [&](const float* a, float* b) { return cheby<float>(P, lvl, a, b, true, s); });
}

int se_pmg_gather_ext(se_pmg_t P, int lvl, const double* r, double* rbar, void* stream) {
  SE_CHECK(P && r && rbar && lvl >= 0 && lvl < P->nlev, SE_EINVAL, "se_pmg_gather_ext: bad argument");
  return gather_ext<double>(*P->lv[lvl], r, rbar, as_stream(stream, P->stream));
}

int se_pmg_fdm(se_pmg_t P, int lvl, const double* rbar, double* zbar, void* stream) {
  SE_CHECK(P && rbar && zbar && lvl >= 0 && lvl + 1 < P->nlev, SE_EINVAL, "se_pmg_fdm: bad argument");
  SE_CHECK(P->lv[lvl]->S64 != nullptr, SE_EINVAL, "se_pmg_fdm: level %d has no FDM factors (Jacobi smoother)", lvl);
  return fdm_apply_ext<double>(*P->lv[lvl], rbar, zbar, as_stream(stream, P->stream));
}

int se_pmg_restrict(se_pmg_t P, int lvl, const double* rf, double* rc, void* stream) {
  SE_CHECK(P && rf && rc && lvl >= 0 && lvl + 1 < P->nlev, SE_EINVAL, "se_pmg_restrict: bad argument");
  cudaStream_t s = as_stream(stream, P->stream);
  const Level& f = *P->lv[lvl];
  const Level& c = *P->lv[lvl + 1];
  if (P->desc.precision == SE_FP32) {
    SE_TRY((convert<double, float>(rf, P->vecs<float>(lvl).b, f.L, s)));
    SE_TRY(restrict_apply<float>(f, c, P->J32[lvl], P->vecs<float>(lvl).b, P->vecs<float>(lvl + 1).b, s));
    return convert<float, double>(P->vecs<float>(lvl + 1).b, rc, c.L, s);
  }
  return restrict_apply<double>(f, c, P->J64[lvl], rf, rc, s);
}

int se_pmg_prolong(se_pmg_t P, int lvl, const double* ec, double* ef, void* stream) {
  SE_CHECK(P && ec && ef && lvl >= 0 && lvl + 1 < P->nlev, SE_EINVAL, "se_pmg_prolong: bad argument");
  cudaStream_t s = as_stream(stream, P->stream);
  const Level& f = *P->lv[lvl];
  const Level& c = *P->lv[lvl + 1];
  if (P->desc.precision == SE_FP32) {
    SE_TRY((convert<double, float>(ec, P->vecs<float>(lvl + 1).b, c.L, s)));
    SE_TRY(prolong_apply<float>(f, c, P->J32[lvl], P->vecs<float>(lvl + 1).b, P->vecs<float>(lvl).x, false, s));
    return convert<float, double>(P->vecs<float>(lvl).x, ef, f.L, s);
  }
  return prolong_apply<double>(f, c, P->J64[lvl], ec, ef, false, s);
}

int se_pmg_coarse_solve(se_pmg_t P, const double* r, double* x, int* iters, void* stream) {
  SE_CHECK(P && r && x, SE_EINVAL, "se_pmg_coarse_solve: null argument");
  cudaStream_t s = as_stream(stream, P->stream);
  const Level& c = *P->lv[P->nlev - 1];
  SE_TRY(coarse_solve<double>(c, P->cw, r, x, P->desc.coarse_tol, P->desc.coarse_maxit, s));
  int h[2] = {0, 0};
  SE_CUDA(cudaMemcpyAsync(h, P->cw.status, sizeof(h), cudaMemcpyDeviceToHost, s));
  SE_CUDA(cudaStreamSynchronize(s));
  if (iters) *iters = h[1];
  SE_CHECK(h[0] == 0, SE_ETIMEOUT, "coarse solve: a grid barrier wait ran out");
  return SE_OK;
}

}  // extern "C"
