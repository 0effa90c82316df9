// Run-time preconditioner selection (the paper, Sec. 5 and Table 5): an exhaustive timed search
// on the first solve over a small space of p-multigrid preconditioners, keeping the one with the
// shortest time to solution.  The default space is Table 5 without SEMFEM: for p = 7,
// Cheby-ASM(2),(7,3,1), Cheby-RAS(2),(7,3,1), Cheby-Jac(2),(7,5,3,1); for p = 9 the same with
// (9,5,1), (9,5,1), (9,7,5,1).  Other orders get the analogous three: Schwarz through the
// largest odd order <= ceil(p/2) (the rule that gives 3 for p = 7 and 5 for p = 9), Jacobi in
// steps of two down to 1.
#include <chrono>
#include <cstring>
#include <vector>

#include "pmg_internal.h"

namespace se {

static void fill_desc_vec(se_pmg_desc* d, const std::vector<int>& sched, int smoother, int precision) {
  std::memset(d, 0, sizeof(*d));
  d->nlev = (int)sched.size();
  for (size_t i = 0; i < sched.size(); ++i) d->schedule[i] = sched[i];
  d->smoother = smoother;
  for (int l = 0; l < SE_MAX_LEVELS; ++l) d->cheb_order[l] = 2;
  d->eig_lo = 0.1;
  d->eig_hi = 1.1;
  d->arnoldi_steps = 10;
  d->seed = 0;
  d->coarse_tol = 1e-2;  // an inexact coarse solve, the size of one AMG cycle (Sec. 2.2.2)
  d->coarse_maxit = 500;
  d->precision = precision;
}

}  // namespace se

using namespace se;

extern "C" {

int se_pmg_autotune_space(int p, int precision, se_tune_candidate* out, int cap, int* n) {
  SE_CHECK(out && n && cap >= 3, SE_EINVAL, "se_pmg_autotune_space: need room for 3 candidates");
  SE_CHECK(p >= 2 && p <= SE_MAX_ORDER, SE_EINVAL, "se_pmg_autotune_space: p=%d not in 2..%d", p,
           SE_MAX_ORDER);
  SE_CHECK(precision == SE_FP64 || precision == SE_FP32 || precision == SE_DF64, SE_EINVAL,
           "se_pmg_autotune_space: precision");
  std::vector<int> schwarz{p}, jac;
  int mid = (p + 1) / 2;
  if (mid % 2 == 0) --mid;
  if (mid > 1) schwarz.push_back(mid);
  schwarz.push_back(1);
  if (p == 9) {
    jac = {9, 7, 5, 1};  // Table 5
  } else {
    for (int q = p; q > 1; q -= 2) jac.push_back(q);
    jac.push_back(1);
  }
  fill_desc_vec(&out[0].pmg, schwarz, SE_SMOOTH_ASM, precision);
  fill_desc_vec(&out[1].pmg, schwarz, SE_SMOOTH_RAS, precision);
  fill_desc_vec(&out[2].pmg, jac, SE_SMOOTH_JACOBI, precision);
  for (int i = 0; i < 3; ++i) {
    out[i].ms = 0.0;
    out[i].setup_ms = 0.0;
    out[i].iterations = 0;
    out[i].status = SE_OK;
  }
  *n = 3;
  return SE_OK;
}

int se_pmg_autotune(se_mesh_t m, const double* b, const se_solve_opts* opts, int repeats,
                    se_tune_candidate* cands, int n, int* best, se_pmg_t* out_pmg) {
  SE_CHECK(m && b && opts && cands && best && n >= 1, SE_EINVAL, "se_pmg_autotune: bad argument");
  SE_CHECK(repeats >= 1 && repeats <= 100, SE_EINVAL, "se_pmg_autotune: repeats");
  SE_CHECK(opts->method == SE_FPCG || opts->method == SE_FGMRES, SE_EINVAL, "se_pmg_autotune: method");
  cudaStream_t s = m->stream;
  const int64_t L = m->fine.L;
  double* x = nullptr;
  SE_TRY(dmalloc_transient(reinterpret_cast<void**>(&x), L * sizeof(double), s));
  cudaEvent_t e1 = nullptr, e2 = nullptr;
  cudaEventCreate(&e1);
  cudaEventCreate(&e2);
  se_solve_opts o = *opts;
  o.stream = s;
  se_pmg_t kept = nullptr;
  *best = -1;
  for (int i = 0; i < n; ++i) {
    se_tune_candidate& c = cands[i];
    se_pmg_t P = nullptr;
    const auto t0 = std::chrono::steady_clock::now();
    c.status = se_pmg_setup(m, &c.pmg, &P);  // synchronises
    c.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    c.ms = 0.0;
    c.iterations = 0;
    if (c.status != SE_OK) continue;
    se_solve_stats st{};
    int rc = SE_OK;
    // one untimed solve (captures the graph when graph_capture is set), then the timed ones
    if (cudaMemsetAsync(x, 0, L * sizeof(double), s) != cudaSuccess) rc = SE_ECUDA;
    if (rc == SE_OK) rc = se_solve(m, P, b, x, &o, &st);
    float total = 0.f;
    for (int r = 0; r < repeats && rc == SE_OK; ++r) {
      cudaMemsetAsync(x, 0, L * sizeof(double), s);
      cudaEventRecord(e1, s);
      rc = se_solve(m, P, b, x, &o, &st);
      cudaEventRecord(e2, s);
      cudaEventSynchronize(e2);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e1, e2);
      total += ms;
    }
    c.status = rc;
    c.iterations = st.iterations;
    c.ms = total / repeats;
    if (rc == SE_OK && (*best < 0 || c.ms < cands[*best].ms)) {
      if (kept) se_pmg_destroy(kept);
      kept = P;
      *best = i;
    } else {
      se_pmg_destroy(P);
    }
  }
  cudaFreeAsync(x, s);
  cudaStreamSynchronize(s);
  cudaEventDestroy(e1);
  cudaEventDestroy(e2);
  if (out_pmg) {
    *out_pmg = kept;
  } else if (kept) {
    se_pmg_destroy(kept);
  }
  SE_CHECK(*best >= 0, SE_ENOTCONV, "se_pmg_autotune: no candidate converged");
  return SE_OK;
}

}  // extern "C"
