// Internal declarations of the p-multigrid handle.
#pragma once

#include "se_internal.h"

namespace se {

template <class T>
struct LevelVecs {
  T *b = nullptr, *x = nullptr, *r = nullptr, *cr = nullptr, *cd = nullptr, *w = nullptr, *sv = nullptr;
};

int pmg_apply(se_pmg_s* P, const double* r, double* z, cudaStream_t s);
int graph_solve_launch(se_mesh_s* m, se_pmg_s* P, const double* b, double* x, double tol,
                       int maxit, cudaStream_t s, int tol_norm = SE_TOL_R0, int op_df = 0);
int graph_solve_result(se_mesh_s* m, cudaStream_t s, double tol, int maxit, se_solve_stats* st);
// Pieces of the device-driven FPCG graph (solve.cu), shared with the batched solves (batch.cu).
int prepare_graph_solve(se_mesh_s* m);
int read_graph_stats(se_mesh_s* m, cudaStream_t s, se_solve_stats* out, double tol, int maxit);
// Appends one whole FPCG solve of mesh m (x0 = the content of x at launch) to graph G as a branch
// independent of the rest of G.
int append_fpcg_solve(cudaGraph_t G, cudaStream_t cs, se_mesh_s* m, se_pmg_s* P, const double* b,
                      double* x, double tol, int maxit, int tol_norm, int op_df);
// Adds a conditional node at the capture frontier of cs and moves the frontier after it.
int add_conditional(cudaStream_t cs, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                    cudaGraph_t* body);
int pmg_alloc_vecs(se_pmg_s* P, int l, bool fp32);
// SE_ETIMEOUT if a bounded device wait in P's kernels (a pipelined operator of one of its levels,
// its coarse solve) expired since the last call; clears those records.  Synchronises s.
int pmg_faults_take(se_pmg_s* P, cudaStream_t s);
// b = M QQ^T B_L f for f = pi^2 (k1^2+k2^2+k3^2) a sin(k1 pi x) sin(k2 pi y) sin(k3 pi z), the
// right-hand side of the manufactured solution u* = a sin(k1 pi x) sin(k2 pi y) sin(k3 pi z).
int rhs_modes(se_mesh_s* m, const int k[3], double a, double* b, cudaStream_t s);

}  // namespace se

struct se_pmg_s {
  se_mesh_s* mesh = nullptr;
  uint64_t uid = 0;  // unique per handle: the mesh's cached solve graph is keyed by it, not by
                     // the address (a later handle may reuse a destroyed one's address)
  se_pmg_desc desc;
  int nlev = 0;
  cudaStream_t stream = nullptr;
  // level 0 is a shallow copy of the mesh level (shares its geometry and index maps); the
  // smoother data of every level belongs to this handle
  se::Level owned[SE_MAX_LEVELS];
  se::Level* lv[SE_MAX_LEVELS] = {};
  double lam[SE_MAX_LEVELS] = {};
  double lmin[SE_MAX_LEVELS] = {};
  double lmax[SE_MAX_LEVELS] = {};
  double* J64[SE_MAX_LEVELS] = {};
  float* J32[SE_MAX_LEVELS] = {};
  se::LevelVecs<double> v64[SE_MAX_LEVELS];
  se::LevelVecs<float> v32[SE_MAX_LEVELS];
  se::CoarseWork cw{};
  // set for the union preconditioner of a batch group: the coarsest level is solved as the
  // group's independent coarse problems (one cooperative launch)
  const se::CoarseGroup* cgroup = nullptr;
  se::Allocs allocs;
  se::Scratch scratch;
  cudaGraphExec_t graph = nullptr;
  const double* graph_r = nullptr;
  double* graph_z = nullptr;
  cudaStream_t graph_stream = nullptr;

  template <class T>
  se::LevelVecs<T>& vecs(int l) {
    if constexpr (sizeof(T) == 8) return v64[l];
    else return v32[l];
  }
  void release_graph() {
    if (graph) cudaGraphExecDestroy(graph);
    graph = nullptr;
    graph_r = nullptr;
    graph_z = nullptr;
  }
};
