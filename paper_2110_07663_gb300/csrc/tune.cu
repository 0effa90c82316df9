// Launch-tile autotuner: elements per block of the operator (Ax) and FDM kernels, measured per
// polynomial order and precision on a scratch problem of about two million points, fastest
// candidate stored in the process-wide tile table that the launchers consult.
#include <cmath>
#include <vector>

#include "pmg_internal.h"

namespace se {
template <class T>
int fdm_ras_local(const Level& lv, const T* r, T* out, cudaStream_t s);

template <class F>
static double time_launches(F&& launch, cudaStream_t s, int reps) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  for (int i = 0; i < 2; ++i) launch();
  cudaEventRecord(a, s);
  for (int i = 0; i < reps; ++i) launch();
  cudaEventRecord(b, s);
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms / reps;
}

template <class T>
static int tune_typed(se_pmg_s* P, int p, se_tile_cfg* out) {
  const bool fp32 = sizeof(T) == 4;
  Level& lv = *P->lv[0];
  cudaStream_t s = P->stream;
  const int64_t L = lv.L;
  T *u = nullptr, *y = nullptr;
  SE_CUDA(cudaMalloc(&u, L * sizeof(T)));
  if (cudaMalloc(&y, L * sizeof(T)) != cudaSuccess) {
    cudaFree(u);
    set_error("se_tune: out of device memory");
    return SE_ENOMEM;
  }
  int rc = convert<double, T>(lv.X, u, L, s);  // any smooth data of the right size
  const int N = p + 1;
  TileCfg best = tile_get(p, fp32);
  double best_ax = 1e30, best_fdm = 1e30;
  const int ax_cand[] = {1, 2, 3, 4, 6, 8, 12, 16};
  for (int ne : ax_cand) {
    if (rc != SE_OK) break;
    if (ne * N * N > 512 || (N * N + (size_t)ne * 3 * N * N * N) * sizeof(T) > 200 * 1024) continue;
    TileCfg c = best;
    c.ax_ne = ne;
    tile_set(p, fp32, c);
    const double ms = time_launches([&] { rc |= ax_local<T>(lv, u, y, false, s); }, s, 10);
    if (ms < best_ax) {
      best_ax = ms;
      best.ax_ne = ne;
    }
  }
  tile_set(p, fp32, best);
  const bool have_fdm = fp32 ? lv.S32 != nullptr : lv.S64 != nullptr;
  for (int ne = 1; ne <= 16 && have_fdm && rc == SE_OK; ++ne) {
    const size_t smem = fdm_smem_bytes(p, fp32, ne);
    if (fdm_block_threads(p, fp32, ne) > fdm_max_threads(fp32) || smem > 200 * 1024) continue;
    TileCfg c = best;
    c.fdm_ne = ne;
    tile_set(p, fp32, c);
    const double ms = time_launches([&] { rc |= fdm_ras_local<T>(lv, u, y, s); }, s, 10);
    if (ms < best_fdm) {
      best_fdm = ms;
      best.fdm_ne = ne;
    }
  }
  tile_set(p, fp32, best);
  cudaStreamSynchronize(s);
  cudaFree(u);
  cudaFree(y);
  if (rc != SE_OK) return rc;
  out->ax_elems_per_block = best.ax_ne;
  out->fdm_elems_per_block = have_fdm ? best.fdm_ne : 0;
  out->ax_ms = best_ax;
  out->fdm_ms = have_fdm ? best_fdm : 0.0;
  return SE_OK;
}

}  // namespace se

using namespace se;

extern "C" {

int se_tune(int p, int precision, se_tile_cfg* out) {
  SE_CHECK(out && p >= 2 && p <= SE_MAX_ORDER, SE_EINVAL, "se_tune: p=%d not in 2..%d", p, SE_MAX_ORDER);
  SE_CHECK(precision == SE_FP64 || precision == SE_FP32, SE_EINVAL, "se_tune: bad precision");
  const int N = p + 1;
  int n = (int)std::lround(std::cbrt(2.0e6 / (N * N * N)));
  if (n < 2) n = 2;
  se_mesh_desc d{};
  d.nel[0] = d.nel[1] = d.nel[2] = n;
  d.p = p;
  d.deform_amp = 0.05;
  d.perturb_frac = 0.05;
  d.seed = 1;
  se_mesh_t m = nullptr;
  SE_TRY(se_mesh_create(&d, &m));
  se_pmg_desc pd{};
  pd.nlev = 2;
  pd.schedule[0] = p;
  pd.schedule[1] = 1;
  pd.smoother = SE_SMOOTH_RAS;
  pd.cheb_order[0] = 1;
  pd.eig_lo = 0.1;
  pd.eig_hi = 1.1;
  pd.arnoldi_steps = 2;
  pd.coarse_tol = 1e-2;
  pd.coarse_maxit = 5;
  pd.precision = precision;
  se_pmg_t P = nullptr;
  int rc = se_pmg_setup(m, &pd, &P);
  if (rc == SE_OK) {
    out->p = p;
    out->precision = precision;
    rc = precision == SE_FP32 ? tune_typed<float>(P, p, out) : tune_typed<double>(P, p, out);
    se_pmg_destroy(P);
  }
  se_mesh_destroy(m);
  return rc;
}

int se_tune_get(int p, int precision, se_tile_cfg* out) {
  SE_CHECK(out && p >= 1 && p <= SE_MAX_ORDER, SE_EINVAL, "se_tune_get: bad argument");
  const bool fp32 = precision == SE_FP32;
  out->p = p;
  out->precision = precision;
  out->ax_elems_per_block = ax_elems_per_block(p, fp32);
  out->fdm_elems_per_block = fdm_elems_per_block(p, fp32);
  out->ax_ms = 0.0;
  out->fdm_ms = 0.0;
  return SE_OK;
}

int se_tune_set(const se_tile_cfg* cfg) {
  SE_CHECK(cfg && cfg->p >= 1 && cfg->p <= SE_MAX_ORDER, SE_EINVAL, "se_tune_set: bad argument");
  TileCfg c;
  c.ax_ne = cfg->ax_elems_per_block;
  c.fdm_ne = cfg->fdm_elems_per_block;
  tile_set(cfg->p, cfg->precision == SE_FP32, c);
  return SE_OK;
}

}  // extern "C"
