// Outer Krylov solvers (Sec. 2.2), FP64: flexible preconditioned CG and right-preconditioned
// flexible GMRES(m) with modified Gram-Schmidt.  Scalars (alpha, beta, Gram-Schmidt
// coefficients) stay on the device; the host reads one residual norm per iteration.
#include <cmath>
#include <vector>

#include <cuda_runtime.h>

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
    SE_TRY(h2d(m->gm_zs, zs.data(), restart * sizeof(double*), m->stream));
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

// The fine level as the outer operator sees it: FP64 arithmetic, or df64 (operator_df64) where
// the mesh holds df64 geometry.
static Level outer_level(const se_mesh_s* m, int op_df) {
  Level lv = m->fine;
  lv.df = op_df != 0;
  return lv;
}

// Flexible PCG: beta = (z_{k+1}, r_{k+1} - r_k) / (z_k, r_k).
static int fpcg(se_mesh_s* m, se_pmg_s* P, const double* b, double* x, const se_solve_opts& o,
                cudaStream_t s, se_solve_stats* st) {
  const Level lv = outer_level(m, o.operator_df64);
  Scratch& sc = m->scratch;
  double *r = m->sr, *r2 = m->sr2, *z = m->sz, *p = m->sp, *w = m->sw;
  SE_TRY(ax_apply<double>(lv, x, w, s));
  SE_TRY(axpby<double>(1.0, b, -1.0, w, r, lv.L, s));         // r = b - A x
  SE_TRY(precondition(m, P, r, z, s));
  SE_TRY(fpcg_init(lv, r, z, sc, s));                           // rz, rr, r0
  if (o.tol_norm == SE_TOL_B) SE_TRY(dot_to_slot(lv, b, b, sc, SC_R0, s));  // reference ||b||
  SE_CUDA(cudaMemcpyAsync(p, z, lv.L * sizeof(double), cudaMemcpyDeviceToDevice, s));
  SE_TRY(read_scalars(m, s, SC_R0 + 1));
  const double r0 = std::sqrt(sc.hscal[SC_R0]);
  st->iterations = 0;
  st->rel_residual = r0 > 0 ? std::sqrt(sc.hscal[SC_RR]) / r0 : 0.0;
  if (r0 == 0.0 || st->rel_residual <= o.tol) return SE_OK;
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
  const Level lv = outer_level(m, o.operator_df64);
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
  if (o.tol_norm == SE_TOL_B) SE_TRY(dot_to_slot(lv, b, b, sc, SC_TMP, s));
  SE_TRY(read_scalars(m, s, SC_NORM + 1));
  double beta = std::sqrt(sc.hscal[SC_NORM]);
  const double r0 = o.tol_norm == SE_TOL_B ? std::sqrt(sc.hscal[SC_TMP]) : beta;  // reference
  st->iterations = 0;
  st->rel_residual = r0 > 0 ? beta / r0 : 0.0;
  if (r0 == 0.0 || beta == 0.0 || st->rel_residual <= o.tol) return SE_OK;
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

int graph_solve(se_mesh_s* m, se_pmg_s* P, const double* b, double* x, const se_solve_opts& o,
                cudaStream_t s, se_solve_stats* st);

}  // namespace se

using namespace se;

extern "C" int se_solve(se_mesh_t m, se_pmg_t P, const double* b, double* x,
                        const se_solve_opts* opts, se_solve_stats* stats) {
  SE_CHECK(m && b && x && opts, SE_EINVAL, "se_solve: null argument");
  SE_CHECK(!P || P->mesh == m, SE_EINVAL, "se_solve: preconditioner built for another mesh");
  se_solve_opts o = *opts;
  SE_CHECK(o.method == SE_FPCG || o.method == SE_FGMRES, SE_EINVAL, "se_solve: bad method");
  SE_CHECK(o.tol > 0 && o.maxit >= 1, SE_EINVAL, "se_solve: bad tolerance or maxit");
  SE_CHECK(o.tol_norm == SE_TOL_R0 || o.tol_norm == SE_TOL_B, SE_EINVAL, "se_solve: bad tol_norm");
  if (o.method == SE_FGMRES) SE_CHECK(o.restart >= 1 && o.restart <= 200, SE_EINVAL, "se_solve: restart");
  SE_CHECK(o.operator_df64 == 0 || o.operator_df64 == 1, SE_EINVAL, "se_solve: operator_df64");
  cudaStream_t s = as_stream(o.stream, m->stream);
  SE_TRY(ensure_solve_work(m, o.restart, o.method == SE_FGMRES));
  if (o.operator_df64) SE_TRY(make_df_geometry(m->fine, m->allocs, s));
  se_solve_stats st{};
  SE_CUDA(cudaEventRecord(m->ev0, s));
  int rc;
  if (o.graph_capture && o.method == SE_FPCG) rc = graph_solve(m, P, b, x, o, s, &st);
  else rc = o.method == SE_FPCG ? fpcg(m, P, b, x, o, s, &st) : fgmres(m, P, b, x, o, s, &st);
  cudaEventRecord(m->ev1, s);
  cudaEventSynchronize(m->ev1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, m->ev0, m->ev1);
  if (level_pipeline_take(m->fine, s) != SE_OK) rc = SE_ETIMEOUT;
  if (P && pmg_faults_take(P, s) != SE_OK) rc = SE_ETIMEOUT;
  st.ms_total = ms;
  st.status = rc;
  if (stats) *stats = st;
  return rc;
}

extern "C" int se_solve_host(se_mesh_t m, se_pmg_t P, const double* b_host, const double* x0_host,
                             double* x_host, const se_solve_opts* opts, se_solve_stats* stats) {
  SE_CHECK(m && b_host && x_host && opts, SE_EINVAL, "se_solve_host: null argument");
  const int64_t L = m->fine.L;
  if (!m->hb) SE_TRY(dmalloc(m->allocs, &m->hb, (size_t)L));
  if (!m->hx) SE_TRY(dmalloc(m->allocs, &m->hx, (size_t)L));
  cudaStream_t s = as_stream(opts->stream, m->stream);
  SE_CUDA(cudaMemcpyAsync(m->hb, b_host, (size_t)L * sizeof(double), cudaMemcpyHostToDevice, s));
  if (x0_host) SE_CUDA(cudaMemcpyAsync(m->hx, x0_host, (size_t)L * sizeof(double), cudaMemcpyHostToDevice, s));
  else SE_CUDA(cudaMemsetAsync(m->hx, 0, (size_t)L * sizeof(double), s));
  const int rc = se_solve(m, P, m->hb, m->hx, opts, stats);
  if (rc != SE_OK && rc != SE_ENOTCONV) return rc;
  SE_CUDA(cudaMemcpyAsync(x_host, m->hx, (size_t)L * sizeof(double), cudaMemcpyDeviceToHost, s));
  SE_CUDA(cudaStreamSynchronize(s));
  return rc;
}

// =============================================================================================
// Device-driven flexible PCG as one CUDA graph: the iteration is a WHILE node whose condition a
// one-thread kernel sets from the device-resident residual norm; after convergence an IF node
// skips the preconditioner.  No host round trip per iteration: one graph launch per solve.
// Several solves become parallel branches of one graph (se_batch_*).
// =============================================================================================
namespace se {

struct DevStats {
  int iterations;
  int status;
  double rel;
};

__global__ void fpcg_graph_init_kernel(const double* __restrict__ scal, DevStats* st, double tol,
                                       int maxit, cudaGraphConditionalHandle hw) {
  const double ref = scal[SC_R0];  // ||r_0||^2, or ||b||^2 (SE_TOL_B)
  const double rel = ref > 0.0 ? sqrt(scal[SC_RR] / ref) : 0.0;
  st->iterations = 0;
  st->status = 0;
  st->rel = rel;
  cudaGraphSetConditional(hw, (ref > 0.0 && rel > tol && maxit > 0) ? 1u : 0u);
}

__global__ void fpcg_graph_check_kernel(const double* __restrict__ scal, DevStats* st, double tol,
                                        int maxit, cudaGraphConditionalHandle hw,
                                        cudaGraphConditionalHandle hif) {
  const int it = st->iterations + 1;
  st->iterations = it;
  const double rel = sqrt(scal[SC_RR] / scal[SC_R0]);
  st->rel = rel;
  const bool go = rel > tol && it < maxit;  // a NaN residual stops the loop too
  cudaGraphSetConditional(hw, go ? 1u : 0u);
  cudaGraphSetConditional(hif, go ? 1u : 0u);
}

// Adds a conditional node at the capture frontier of `cs` and moves the frontier after it.
int add_conditional(cudaStream_t cs, cudaGraphConditionalHandle h,
                           cudaGraphConditionalNodeType type, cudaGraph_t* body) {
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  SE_CUDA(cudaStreamGetCaptureInfo(cs, &st, nullptr, &g, &deps, nullptr, &ndeps));
  SE_CHECK(st == cudaStreamCaptureStatusActive, SE_ECUDA, "graph build: stream is not capturing");
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = type;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  SE_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &cp));
  *body = cp.conditional.phGraph_out[0];
  SE_CUDA(cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return SE_OK;
}

// Appends one whole FPCG solve (x0 = the content of x at launch) to graph G, independent of the
// rest of G.  All buffers must already exist: nothing is allocated while capturing.
int append_fpcg_solve(cudaGraph_t G, cudaStream_t cs, se_mesh_s* m, se_pmg_s* P,
                             const double* b, double* x, double tol, int maxit, int tol_norm,
                             int op_df) {
  const Level lv = outer_level(m, op_df);
  Scratch& sc = m->scratch;
  double *r = m->sr, *r_old = m->sr2, *z = m->sz, *p = m->sp, *w = m->sw;
  DevStats* st = static_cast<DevStats*>(m->gstats);
  cudaGraphConditionalHandle hw, hif;
  SE_CUDA(cudaGraphConditionalHandleCreate(&hw, G, 0, 0));
  // ---- initialisation
  SE_CUDA(cudaStreamBeginCaptureToGraph(cs, G, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  int rc = SE_OK;
  cudaGraph_t wbody = nullptr, ifbody = nullptr;
  do {
    if ((rc = ax_apply<double>(lv, x, w, cs)) != SE_OK) break;
    if ((rc = axpby<double>(1.0, b, -1.0, w, r, lv.L, cs)) != SE_OK) break;
    if ((rc = precondition(m, P, r, z, cs)) != SE_OK) break;
    if ((rc = fpcg_init(lv, r, z, sc, cs)) != SE_OK) break;
    if (tol_norm == SE_TOL_B && (rc = dot_to_slot(lv, b, b, sc, SC_R0, cs)) != SE_OK) break;
    if (cudaMemcpyAsync(p, z, lv.L * sizeof(double), cudaMemcpyDeviceToDevice, cs) != cudaSuccess) {
      set_error("graph build: copy capture failed");
      rc = SE_ECUDA;
      break;
    }
    fpcg_graph_init_kernel<<<1, 1, 0, cs>>>(sc.scal, st, tol, maxit, hw);
    rc = add_conditional(cs, hw, cudaGraphCondTypeWhile, &wbody);
  } while (0);
  cudaGraph_t out = nullptr;
  cudaError_t ec = cudaStreamEndCapture(cs, &out);
  if (rc != SE_OK) return rc;
  SE_CHECK(ec == cudaSuccess, SE_ECUDA, "graph build (init): %s", cudaGetErrorString(ec));
  // ---- WHILE body: w = A p, alpha, x/r update, convergence test
  SE_CUDA(cudaGraphConditionalHandleCreate(&hif, G, 0, 0));
  SE_CUDA(cudaStreamBeginCaptureToGraph(cs, wbody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  do {
    if ((rc = ax_apply<double>(lv, p, w, cs)) != SE_OK) break;
    if ((rc = fpcg_alpha(lv, p, w, sc, cs)) != SE_OK) break;
    if ((rc = fpcg_update_inplace(lv, x, p, r, w, r_old, sc, cs)) != SE_OK) break;
    fpcg_graph_check_kernel<<<1, 1, 0, cs>>>(sc.scal, st, tol, maxit, hw, hif);
    rc = add_conditional(cs, hif, cudaGraphCondTypeIf, &ifbody);
  } while (0);
  ec = cudaStreamEndCapture(cs, &out);
  if (rc != SE_OK) return rc;
  SE_CHECK(ec == cudaSuccess, SE_ECUDA, "graph build (loop): %s", cudaGetErrorString(ec));
  // ---- IF body: z = M r, beta, p = z + beta p
  SE_CUDA(cudaStreamBeginCaptureToGraph(cs, ifbody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  do {
    if ((rc = precondition(m, P, r, z, cs)) != SE_OK) break;
    if ((rc = fpcg_beta(lv, z, r, r_old, sc, cs)) != SE_OK) break;
    rc = fpcg_pupdate(lv, p, z, sc, cs);
  } while (0);
  ec = cudaStreamEndCapture(cs, &out);
  if (rc != SE_OK) return rc;
  SE_CHECK(ec == cudaSuccess, SE_ECUDA, "graph build (preconditioner): %s", cudaGetErrorString(ec));
  return SE_OK;
}

int prepare_graph_solve(se_mesh_s* m) {
  SE_TRY(ensure_solve_work(m, 0, false));
  if (!m->gstats) SE_TRY(dmalloc_bytes(m->allocs, &m->gstats, sizeof(DevStats)));
  return SE_OK;
}

int read_graph_stats(se_mesh_s* m, cudaStream_t s, se_solve_stats* out, double tol, int maxit) {
  DevStats h{};
  SE_CUDA(cudaMemcpyAsync(&h, m->gstats, sizeof(h), cudaMemcpyDeviceToHost, s));
  SE_CUDA(cudaStreamSynchronize(s));
  out->iterations = h.iterations;
  out->rel_residual = h.rel;
  if (std::isnan(h.rel)) {
    set_error("se_solve: residual became NaN");
    return SE_ENOTCONV;
  }
  if (h.rel > tol) {
    set_error("se_solve: no convergence in %d iterations (rel. residual %.3e)", maxit, h.rel);
    return SE_ENOTCONV;
  }
  return SE_OK;
}

// Builds (or reuses) this mesh's solve graph for (P, b, x, tol, maxit) and launches it on s
// without waiting.  read_graph_stats collects the result.
int graph_solve_launch(se_mesh_s* m, se_pmg_s* P, const double* b, double* x, double tol,
                       int maxit, cudaStream_t s, int tol_norm, int op_df) {
  SE_TRY(prepare_graph_solve(m));
  const uint64_t uid = P ? P->uid : 0;
  const bool same = m->gexec && m->gkey[0] == P && m->gpmg_uid == uid && m->gkey[1] == b && m->gkey[2] == x &&
                    m->gtol == tol && m->gmaxit == maxit && m->gtolnorm == tol_norm &&
                    m->gopdf == op_df;
  if (!same) {
    if (m->gexec) cudaGraphExecDestroy(m->gexec);
    m->gexec = nullptr;
    cudaGraph_t G;
    SE_CUDA(cudaGraphCreate(&G, 0));
    cudaStream_t cs;
    SE_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    int rc = append_fpcg_solve(G, cs, m, P, b, x, tol, maxit, tol_norm, op_df);
    cudaStreamDestroy(cs);
    if (rc == SE_OK) {
      cudaError_t e = cudaGraphInstantiate(&m->gexec, G, 0);
      if (e != cudaSuccess) {
        set_error("cudaGraphInstantiate: %s", cudaGetErrorString(e));
        rc = SE_ECUDA;
        m->gexec = nullptr;
      }
    }
    cudaGraphDestroy(G);
    if (rc != SE_OK) return rc;
    m->gkey[0] = P;
    m->gpmg_uid = uid;
    m->gkey[1] = b;
    m->gkey[2] = x;
    m->gtol = tol;
    m->gmaxit = maxit;
    m->gtolnorm = tol_norm;
    m->gopdf = op_df;
  }
  SE_CUDA(cudaGraphLaunch(m->gexec, s));
  return SE_OK;
}

int graph_solve_result(se_mesh_s* m, cudaStream_t s, double tol, int maxit, se_solve_stats* st) {
  return read_graph_stats(m, s, st, tol, maxit);
}

// se_solve with graph_capture: one launch of the cached graph, then its statistics.
int graph_solve(se_mesh_s* m, se_pmg_s* P, const double* b, double* x, const se_solve_opts& o,
                cudaStream_t s, se_solve_stats* st) {
  SE_TRY(graph_solve_launch(m, P, b, x, o.tol, o.maxit, s, o.tol_norm, o.operator_df64));
  return read_graph_stats(m, s, st, o.tol, o.maxit);
}

}  // namespace se

