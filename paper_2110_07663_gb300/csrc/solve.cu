// Outer Krylov solvers (Sec. 2.2), FP64: flexible preconditioned CG and right-preconditioned
// flexible GMRES(m) with modified Gram-Schmidt.  Scalars (alpha, beta, Gram-Schmidt
// coefficients) stay on the device; the host reads one residual norm per iteration.
#include <cmath>
#include <vector>

#include "pmg_internal.h"

namespace se {

static int ensure_solve_work(se_mesh_s* m, int restart, bool gmres) {
  const int64_t L = m->fine.L;
  if (!m->sr) {
    for (double** q : {&m->sr, &m->sr2, &m->sz, &m->sp, &m->sw}) SE_TRY(dmalloc(m->allocs, q, L));
    SE_CUDA(cudaEventCreate(&m->ev0));
    SE_CUDA(cudaEventCreate(&m->ev1));
  }
  if (gmres && m->gm_m < restart) {
    SE_TRY(dmalloc(m->allocs, &m->gmV, (size_t)(restart + 1) * L));
    SE_TRY(dmalloc(m->allocs, &m->gmZ, (size_t)restart * L));
    SE_TRY(dmalloc(m->allocs, &m->gm_zs, restart));
    SE_TRY(dmalloc(m->allocs, &m->gm_y, restart));
    std::vector<double*> zs(restart);
    for (int j = 0; j < restart; ++j) zs[j] = m->gmZ + (size_t)j * L;
    SE_CUDA(cudaMemcpy(m->gm_zs, zs.data(), restart * sizeof(double*), cudaMemcpyHostToDevice));
    m->gm_m = restart;
  }
  return SE_OK;
}

static int precondition(se_mesh_s* m, se_pmg_s* P, const double* r, double* z, cudaStream_t s) {
  if (P) return pmg_apply(P, r, z, s);
  return scale_mul<double>(m->fine.dinv64, r, z, m->fine.L, s);
}

static int read_scalars(se_mesh_s* m, cudaStream_t s, int count) {
  SE_CUDA(cudaMemcpyAsync(m->scratch.hscal, m->scratch.scal, count * sizeof(double),
                          cudaMemcpyDeviceToHost, s));
  SE_CUDA(cudaStreamSynchronize(s));
  return SE_OK;
}

// Flexible PCG: beta = (z_{k+1}, r_{k+1} - r_k) / (z_k, r_k).
static int fpcg(se_mesh_s* m, se_pmg_s* P, const double* b, double* x, const se_solve_opts& o,
                cudaStream_t s, se_solve_stats* st) {
  const Level& lv = m->fine;
  Scratch& sc = m->scratch;
  double *r = m->sr, *r2 = m->sr2, *z = m->sz, *p = m->sp, *w = m->sw;
  SE_TRY(ax_apply<double>(lv, x, w, s));
  SE_TRY(axpby<double>(1.0, b, -1.0, w, r, lv.L, s));         // r = b - A x
  SE_TRY(precondition(m, P, r, z, s));
  SE_TRY(fpcg_init(lv, r, z, sc, s));                           // rz, rr, r0
  SE_CUDA(cudaMemcpyAsync(p, z, lv.L * sizeof(double), cudaMemcpyDeviceToDevice, s));
  SE_TRY(read_scalars(m, s, SC_R0 + 1));
  const double r0 = std::sqrt(sc.hscal[SC_R0]);
  st->iterations = 0;
  st->rel_residual = r0 > 0 ? 1.0 : 0.0;
  if (r0 == 0.0) return SE_OK;
  for (int it = 1; it <= o.maxit; ++it) {
    SE_TRY(ax_apply<double>(lv, p, w, s));                      // w = A p
    SE_TRY(fpcg_alpha(lv, p, w, sc, s));                        // alpha = rz / (p, w)
    SE_TRY(fpcg_update(lv, x, p, r, w, r2, sc, s));             // x += a p; r2 = r - a w; rr
    SE_TRY(read_scalars(m, s, SC_RR + 1));
    const double rel = std::sqrt(sc.hscal[SC_RR]) / r0;
    st->iterations = it;
    st->rel_residual = rel;
    if (!(rel > o.tol)) {
      if (std::isnan(rel)) {
        set_error("se_solve: residual became NaN");
        return SE_ENOTCONV;
      }
      return SE_OK;
    }
    SE_TRY(precondition(m, P, r2, z, s));                       // z = M r2
    SE_TRY(fpcg_beta(lv, z, r2, r, sc, s));                     // beta, rz
    SE_TRY(fpcg_pupdate(lv, p, z, sc, s));                      // p = z + beta p
    std::swap(r, r2);
  }
  set_error("se_solve: no convergence in %d iterations (rel. residual %.3e)", o.maxit, st->rel_residual);
  return SE_ENOTCONV;
}

// Right-preconditioned flexible GMRES(m): Z_j = M V_j, w = A Z_j, modified Gram-Schmidt,
// Givens rotations on the host; x += Z y at the end of each cycle.
static int fgmres(se_mesh_s* m, se_pmg_s* P, const double* b, double* x, const se_solve_opts& o,
                  cudaStream_t s, se_solve_stats* st) {
  const Level& lv = m->fine;
  const int64_t L = lv.L;
  Scratch& sc = m->scratch;
  const int mr = o.restart;
  double* r = m->sr;
  double* w = m->sw;
  auto V = [&](int j) { return m->gmV + (size_t)j * L; };
  auto Z = [&](int j) { return m->gmZ + (size_t)j * L; };
  SE_TRY(ax_apply<double>(lv, x, w, s));
  SE_TRY(axpby<double>(1.0, b, -1.0, w, r, L, s));
  SE_TRY(dot_to_slot(lv, r, r, sc, SC_NORM, s));
  SE_TRY(read_scalars(m, s, SC_NORM + 1));
  const double r0 = std::sqrt(sc.hscal[SC_NORM]);
  double beta = r0;
  st->iterations = 0;
  st->rel_residual = r0 > 0 ? 1.0 : 0.0;
  if (r0 == 0.0) return SE_OK;
  std::vector<double> H((mr + 1) * mr), cs(mr), sn(mr), g(mr + 1), y(mr);
  int total = 0;
  while (total < o.maxit) {
    SE_TRY(axpby<double>(1.0 / beta, r, 0.0, r, V(0), L, s));
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int used = 0;
    bool done = false;
    for (int j = 0; j < mr; ++j) {
      SE_TRY(precondition(m, P, V(j), Z(j), s));
      SE_TRY(ax_apply<double>(lv, Z(j), w, s));
      SE_TRY(dot_to_slot(lv, w, V(0), sc, SC_H, s));
      for (int i = 0; i <= j; ++i)
        SE_TRY(axpy_dot(lv, w, V(i), i < j ? V(i + 1) : nullptr, sc, SC_H + i,
                        i < j ? SC_H + i + 1 : SC_NORM, s));
      SE_TRY(scale_inv_sqrt(V(j + 1), w, sc.scal, SC_NORM, L, s));
      SE_TRY(read_scalars(m, s, SC_H + j + 1));
      for (int i = 0; i <= j; ++i) H[i * mr + j] = sc.hscal[SC_H + i];
      double hsub = std::sqrt(std::max(sc.hscal[SC_NORM], 0.0));
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * H[i * mr + j] + sn[i] * H[(i + 1) * mr + j];
        H[(i + 1) * mr + j] = -sn[i] * H[i * mr + j] + cs[i] * H[(i + 1) * mr + j];
        H[i * mr + j] = t;
      }
      const double den = std::hypot(H[j * mr + j], hsub);
      cs[j] = H[j * mr + j] / den;
      sn[j] = hsub / den;
      H[j * mr + j] = den;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++total;
      used = j + 1;
      const double rel = std::fabs(g[j + 1]) / r0;
      st->iterations = total;
      st->rel_residual = rel;
      if (rel <= o.tol || total >= o.maxit) {
        done = rel <= o.tol;
        break;
      }
    }
    for (int i = used - 1; i >= 0; --i) {
      double acc = g[i];
      for (int k = i + 1; k < used; ++k) acc -= H[i * mr + k] * y[k];
      y[i] = acc / H[i * mr + i];
    }
    SE_CUDA(cudaMemcpyAsync(m->gm_y, y.data(), used * sizeof(double), cudaMemcpyHostToDevice, s));
    SE_TRY(lincomb(x, m->gm_zs, m->gm_y, used, L, s));
    SE_CUDA(cudaStreamSynchronize(s));  // y lives on the host stack until the copy completes
    if (done) return SE_OK;
    SE_TRY(ax_apply<double>(lv, x, w, s));
    SE_TRY(axpby<double>(1.0, b, -1.0, w, r, L, s));
    SE_TRY(dot_to_slot(lv, r, r, sc, SC_NORM, s));
    SE_TRY(read_scalars(m, s, SC_NORM + 1));
    beta = std::sqrt(sc.hscal[SC_NORM]);
    if (beta == 0.0) return SE_OK;
  }
  set_error("se_solve: no convergence in %d iterations (rel. residual %.3e)", o.maxit, st->rel_residual);
  return SE_ENOTCONV;
}

}  // namespace se

using namespace se;

extern "C" int se_solve(se_mesh_t m, se_pmg_t P, const double* b, double* x,
                        const se_solve_opts* opts, se_solve_stats* stats) {
  SE_CHECK(m && b && x && opts, SE_EINVAL, "se_solve: null argument");
  SE_CHECK(!P || P->mesh == m, SE_EINVAL, "se_solve: preconditioner built for another mesh");
  se_solve_opts o = *opts;
  SE_CHECK(o.method == SE_FPCG || o.method == SE_FGMRES, SE_EINVAL, "se_solve: bad method");
  SE_CHECK(o.tol > 0 && o.maxit >= 1, SE_EINVAL, "se_solve: bad tolerance or maxit");
  if (o.method == SE_FGMRES) SE_CHECK(o.restart >= 1 && o.restart <= 200, SE_EINVAL, "se_solve: restart");
  cudaStream_t s = as_stream(o.stream, m->stream);
  SE_TRY(ensure_solve_work(m, o.restart, o.method == SE_FGMRES));
  se_solve_stats st{};
  SE_CUDA(cudaEventRecord(m->ev0, s));
  int rc = o.method == SE_FPCG ? fpcg(m, P, b, x, o, s, &st) : fgmres(m, P, b, x, o, s, &st);
  cudaEventRecord(m->ev1, s);
  cudaEventSynchronize(m->ev1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, m->ev0, m->ev1);
  st.ms_total = ms;
  st.status = rc;
  if (stats) *stats = st;
  return rc;
}
