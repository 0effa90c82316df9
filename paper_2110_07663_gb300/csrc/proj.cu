// Projection onto prior solutions (the paper, Secs. 3.2 and 4.2: every pressure solve starts from the
// projection of its right-hand side onto a space of up to 10 prior solutions, Fischer's method
// for successive right-hand sides).
//
// The space holds x_1..x_l with x_i^T A x_j = delta_ij and their images b_i = A x_i.  For a new
// b the A-norm-closest element of the space to A^-1 b is xbar = sum_i (x_i, b) x_i, since
// (x_i, b) = x_i^T A (A^-1 b): no operator application.  After the solve the new solution x is
// A-orthogonalised against the space by modified Gram-Schmidt in the A inner product (two passes;
// (x_i, A v) = (b_i, v)), its image is one operator application, and the pair is normalised.  A
// full space restarts from x alone.  Inner products are the unique-node products of the solver.
#include <cmath>
#include <vector>

#include "pmg_internal.h"

struct se_proj_s {
  se_mesh_s* m = nullptr;
  int maxv = 0;
  int l = 0;          // vectors held
  double* X = nullptr;   // [maxv][L]
  double* B = nullptr;   // [maxv][L]: B_i = A X_i
  double** xptr = nullptr;  // device array of the X_i (linear combinations)
  se::Allocs allocs;
};

namespace se {
constexpr int PROJ_MAX = 16;          // vectors at most (scalar slots of the Gram-Schmidt passes)
constexpr int PROJ_PASS2 = SC_H + 32;  // slots of the second pass
}  // namespace se

using namespace se;

extern "C" {

int se_proj_create(se_mesh_t m, int max_vectors, se_proj_t* out) {
  SE_CHECK(m && out, SE_EINVAL, "se_proj_create: null argument");
  SE_CHECK(max_vectors >= 1 && max_vectors <= PROJ_MAX, SE_EINVAL,
           "se_proj_create: max_vectors %d not in 1..%d", max_vectors, PROJ_MAX);
  auto* p = new se_proj_s();
  p->m = m;
  p->maxv = max_vectors;
  p->allocs.stream = m->stream;
  const int64_t L = m->fine.L;
  int rc = dmalloc(p->allocs, &p->X, (size_t)max_vectors * L);
  if (rc == SE_OK) rc = dmalloc(p->allocs, &p->B, (size_t)max_vectors * L);
  if (rc == SE_OK) rc = dmalloc(p->allocs, &p->xptr, (size_t)max_vectors);
  if (rc == SE_OK) {
    std::vector<double*> ptrs(max_vectors);
    for (int i = 0; i < max_vectors; ++i) ptrs[i] = p->X + (size_t)i * L;
    rc = h2d(p->xptr, ptrs.data(), max_vectors * sizeof(double*), m->stream);
  }
  if (rc != SE_OK) {
    cudaStreamSynchronize(m->stream);
    p->allocs.release();
    delete p;
    return rc;
  }
  *out = p;
  return SE_OK;
}

int se_proj_destroy(se_proj_t p) {
  if (!p) return SE_OK;
  cudaStreamSynchronize(p->m->stream);
  p->allocs.release();
  delete p;
  return SE_OK;
}

int se_proj_guess(se_proj_t p, const double* b, double* x, void* stream) {
  SE_CHECK(p && b && x, SE_EINVAL, "se_proj_guess: null argument");
  const Level& lv = p->m->fine;
  Scratch& sc = p->m->scratch;
  cudaStream_t s = as_stream(stream, p->m->stream);
  SE_TRY(fill_zero<double>(x, lv.L, s));
  if (p->l == 0) return SE_OK;
  for (int i = 0; i < p->l; ++i)
    SE_TRY(dot_to_slot(lv, p->X + (size_t)i * lv.L, b, sc, SC_H + i, s));  // alpha_i = (x_i, b)
  return lincomb(x, p->xptr, sc.scal + SC_H, p->l, lv.L, s);                // x = sum alpha_i x_i
}

int se_proj_update(se_proj_t p, const double* x, int* size, void* stream) {
  SE_CHECK(p && x, SE_EINVAL, "se_proj_update: null argument");
  const Level& lv = p->m->fine;
  Scratch& sc = p->m->scratch;
  cudaStream_t s = as_stream(stream, p->m->stream);
  const int64_t L = lv.L;
  if (p->l == p->maxv) p->l = 0;  // full: restart the space from this solution
  const int l = p->l;
  double* v = p->X + (size_t)l * L;
  double* w = p->B + (size_t)l * L;
  SE_CUDA(cudaMemcpyAsync(v, x, L * sizeof(double), cudaMemcpyDeviceToDevice, s));
  // v -= sum_i (b_i, v) x_i, twice (modified Gram-Schmidt in the A inner product); each pass
  // computes the next coefficient in the same sweep as the current update
  for (int pass = 0; pass < 2 && l > 0; ++pass) {
    const int base = pass == 0 ? SC_H : PROJ_PASS2;
    SE_TRY(dot_to_slot(lv, p->B, v, sc, base, s));
    for (int i = 0; i < l; ++i) {
      const bool more = i + 1 < l;
      SE_TRY(axpy_dot(lv, v, p->X + (size_t)i * L, more ? p->B + (size_t)(i + 1) * L : nullptr, sc,
                      base + i, more ? base + i + 1 : SC_TMP, s));
    }
  }
  SE_TRY(ax_apply<double>(lv, v, w, s));                // image of the remainder
  SE_TRY(dot_to_slot(lv, v, w, sc, SC_NORM, s));        // nu^2 = v^T A v
  SE_CUDA(cudaMemcpyAsync(sc.hscal, sc.scal, SCAL_SLOTS * sizeof(double), cudaMemcpyDeviceToHost, s));
  SE_CUDA(cudaStreamSynchronize(s));
  const double nu2 = sc.hscal[SC_NORM];
  double beta2 = 0.0;  // ||x||_A^2 = sum beta_i^2 + nu^2 (A-orthogonal split of the first pass)
  for (int i = 0; i < l; ++i) beta2 += sc.hscal[SC_H + i] * sc.hscal[SC_H + i];
  if (nu2 > 1e-14 * (beta2 + nu2) && nu2 > 0.0) {
    SE_TRY(scale_inv_sqrt(v, v, sc.scal, SC_NORM, L, s));
    SE_TRY(scale_inv_sqrt(w, w, sc.scal, SC_NORM, L, s));
    SE_CUDA(cudaStreamSynchronize(s));
    p->l = l + 1;
  }
  if (size) *size = p->l;
  return SE_OK;
}

}  // extern "C"
