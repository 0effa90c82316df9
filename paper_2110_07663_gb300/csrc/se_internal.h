// Internal declarations of libse.so: handles, level data, launch helpers, profiling.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "se.h"
#include "df64.h"

namespace se {

// ------------------------------------------------------------------ errors
void set_error(const char* fmt, ...);

#define SE_CUDA(call)                                                                         \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) {                                                                  \
      ::se::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,      \
                      __LINE__);                                                              \
      return SE_ECUDA;                                                                        \
    }                                                                                         \
  } while (0)

#define SE_CHECK(cond, code, ...)                                                             \
  do {                                                                                        \
    if (!(cond)) {                                                                            \
      ::se::set_error(__VA_ARGS__);                                                           \
      return code;                                                                            \
    }                                                                                         \
  } while (0)

#define SE_TRY(call)                                                                          \
  do {                                                                                        \
    int s_ = (call);                                                                          \
    if (s_ != SE_OK) return s_;                                                               \
  } while (0)

// Kernel launch check (launch-configuration errors are reported at once).
#define SE_LAUNCH_CHECK() SE_CUDA(cudaGetLastError())

// ------------------------------------------------------------------ device allocations
// Device allocations of one handle, stream-ordered on the handle's stream: allocating waits for
// that stream only, and freeing (release, dfree) is queued on it, so neither waits for the rest of
// the device (a plain cudaFree would wait for every stream, e.g. other requests' solves).
struct Allocs {
  std::vector<void*> ptrs;
  size_t bytes = 0;
  cudaStream_t stream = nullptr;  // owner's stream; set before the first allocation
  void release();
};

int dmalloc_bytes(Allocs& a, void** p, size_t bytes);
void dfree(Allocs& a, void* p, size_t bytes);
// Stream-ordered device buffer outside any handle (usable on every stream once this returns).
int dmalloc_transient(void** p, size_t bytes, cudaStream_t s);
// Upload and zero fill ordered on the owner's stream s, complete when they return.  Set-up code
// uses these, never the synchronous cudaMemcpy / cudaMemset: those run on the legacy default
// stream, which a non-blocking stream does not wait for, so a kernel on such a stream could read
// a table before its upload had landed.
int h2d(void* dst, const void* src, size_t bytes, cudaStream_t s);
int dzero(void* p, size_t bytes, cudaStream_t s);
// Pinned host scalars, recycled through a process-wide free list (cudaFreeHost may wait for the
// whole device).
int pinned_scalars(double** out);
void pinned_release(double* p);
template <class T>
inline int dmalloc(Allocs& a, T** p, size_t count) {
  return dmalloc_bytes(a, reinterpret_cast<void**>(p), count * sizeof(T) + (count == 0));
}

// ------------------------------------------------------------------ 1D GLL data (host)
struct Basis1D {
  int p = 0;
  double xi[SE_MAX_ORDER + 1];
  double w[SE_MAX_ORDER + 1];
  double D[(SE_MAX_ORDER + 1) * (SE_MAX_ORDER + 1)];  // D[i*N + j] = h_j'(xi_i)
};
void gll_basis(int p, Basis1D* b);
// J[i*Nc + j] = h^c_j(xi^f_i): coarse basis at fine points.
void interp_matrix(int pf, int pc, double* J);

// SplitMix64 (Steele, Lea, Flood 2014): value number c of stream `seed`.
__host__ __device__ inline uint64_t splitmix64_hd(uint64_t seed, uint64_t c) {
  uint64_t z = seed + (c + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
uint64_t splitmix64(uint64_t seed, uint64_t c);
double uniform01(uint64_t seed, uint64_t c);

// ------------------------------------------------------------------ per-point flags
// bits 0..3: multiplicity (number of local copies: 1, 2, 4, 8); bit 7: node is free (not on a
// Dirichlet face).
constexpr uint8_t PF_FREE = 0x80;

// ------------------------------------------------------------------ one discretisation level
struct Level {
  int p = 0, N = 0;
  int nel[3] = {0, 0, 0};
  int bc[6] = {0, 0, 0, 0, 0, 0};
  int64_t E = 0, L = 0, n_global = 0;
  int NX = 0, NY = 0, NZ = 0;
  Basis1D basis;
  double* X = nullptr;       // node coordinates [3][L]
  double* G64 = nullptr;     // geometric factors [6][L]: rr rs rt ss st tt
  float* G32 = nullptr;
  double* B = nullptr;       // diagonal mass w_i w_j w_k det J [L]
  double* dinv64 = nullptr;  // 1 / assembled diagonal, 0 on Dirichlet nodes [L]
  float* dinv32 = nullptr;
  uint8_t* pflag = nullptr;  // multiplicity and free bit [L]
  double* D64 = nullptr;     // derivative matrix on the device [N*N]
  double* eo64 = nullptr;    // even-odd folded D and D^T tables [4][N/2][N/2] (even N)
  // double-float copies for the operator and FDM kernels of SE_DF64 levels (FP64 vectors,
  // df64 arithmetic); `df` routes those two kernels of this level to them
  bool df = false;
  df64* Gdf = nullptr;       // [6][L]
  df64* eodf = nullptr;      // [4][N/2][N/2] (even N)
  df64* Ddf = nullptr;       // [N][N] (odd N)
  df64* Sdf = nullptr;       // [E][3][pb][pb]
  df64* lamdf = nullptr;     // [E][3][pb]
  float* D32 = nullptr;
  const int* nbr = nullptr;  // element neighbours [E][27] (owned by the mesh)
  // fast diagonalisation factors (all levels but the coarsest)
  double* S64 = nullptr;     // [E][3][pb][pb], S[row = window point][col = mode]
  double* lam64 = nullptr;   // [E][3][pb]
  float* S32 = nullptr;
  float* lam32 = nullptr;
  double* fdm_dinv64 = nullptr;  // 1/(lam_x + lam_y + lam_z) per window point [E][pb^3]
  double* ext64 = nullptr;   // full-window work buffer [E][pb^3] (additive Schwarz)
  float* ext32 = nullptr;
  // assembled operator of the coarsest level: 27-point rows over global nodes
  double* Ac = nullptr;      // [27][n_global]: A D^-1 (columns scaled by cdinv)
  double* cdinv = nullptr;   // [n_global]
  int* g2l = nullptr;        // first local copy of each global node [n_global]
  int* l2g = nullptr;        // global node of each local node [L]
  // QQ^T index map (SE_MESH_GS_MAP meshes, se_gsmap handles; gsmap.cu); null: QQ^T by sweeps
  int* gsm_ids = nullptr;    // buckets of local ids, bucket b starting at gsm_seg[b]
  int* gsm_goff = nullptr;   // CSR offsets of the groups of other multiplicities [gsm_n[3] + 1]
  int64_t gsm_n[5] = {0, 0, 0, 0, 0};    // groups of 2, 4, 8, other copies; masked single copies
  int64_t gsm_seg[5] = {0, 0, 0, 0, 0};
  int64_t gsm_entries = 0;   // local ids in groups of two or more
  // [1]: set to SE_ETIMEOUT by a pipelined kernel of this level whose bounded wait expired
  // (its output is then invalid); read and cleared by level_pipeline_take
  int* pstatus = nullptr;
};

// ------------------------------------------------------------------ reduction scratch
// Deterministic two-stage reductions: per-block partial sums, then the last block to finish
// sums them in block order.  Every handle owns one Scratch; calls on one handle are serialised.
constexpr int RED_THREADS = 256;
constexpr int RED_MAX_BLOCKS = 1216;   // 152 SMs x 8
constexpr int SCAL_SLOTS = 256;
struct Scratch {
  double* partial = nullptr;   // [RED_MAX_BLOCKS * 4]
  unsigned* counter = nullptr; // [1], returned to 0 by the last block
  double* scal = nullptr;      // device scalars [SCAL_SLOTS]
  double* hscal = nullptr;     // pinned host mirror [SCAL_SLOTS]
};
int scratch_alloc(Allocs& a, Scratch* s);

// Device scalar slots used by the solvers.
enum {
  SC_RZ = 0, SC_PW = 1, SC_ALPHA = 2, SC_BETA = 3, SC_RR = 4, SC_R0 = 5, SC_ZR = 6,
  SC_ZRO = 7, SC_TMP = 8, SC_NORM = 9,
  SC_H = 16      // SC_H + i: Gram-Schmidt coefficient i of the current column (i <= 200)

};

}  // namespace se

struct se_mesh_s {
  se_mesh_desc desc;
  std::vector<double> verts;     // host vertex lattice (interleaved xyz)
  std::vector<double> box_len;   // host box lengths [E][3]
  se::Level fine;
  int* nbr = nullptr;
  cudaStream_t stream = nullptr;
  se::Allocs allocs;
  se::Scratch scratch;
  double* tmp64 = nullptr;       // [L] work vector
  float* tmpa32 = nullptr;       // [L]
  float* tmpb32 = nullptr;       // [L]
  float* tmpc32 = nullptr;       // [L], allocated by the first FP32 se_residual
  // outer-solver work vectors, allocated on the first se_solve
  double *sr = nullptr, *sr2 = nullptr, *sz = nullptr, *sp = nullptr, *sw = nullptr;
  double *hb = nullptr, *hx = nullptr;  // device b and x of se_solve_host (first call)
  int gm_m = 0;                  // FGMRES restart length the V/Z blocks were sized for
  double* gmV = nullptr;         // [(m+1) L]
  double* gmZ = nullptr;         // [m L]
  double** gm_zs = nullptr;      // device array of the m Z pointers
  double* gm_y = nullptr;        // device [m]
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // device-driven (graph) solve of this mesh: statistics on the device and the cached graph
  void* gstats = nullptr;        // se::DevStats
  cudaGraphExec_t gexec = nullptr;
  const void* gkey[4] = {nullptr, nullptr, nullptr, nullptr};  // pmg, b, x, opts hash
  uint64_t gpmg_uid = 0;     // uid of the preconditioner the cached graph was built with
  double gtol = 0.0;
  int gmaxit = 0;
  int gtolnorm = 0;
  int gopdf = 0;
};

namespace se {

// ------------------------------------------------------------------ builders (mesh.cu)
int build_level(se_mesh_s* m, int p, Level* lv, Allocs& allocs, cudaStream_t s);
int build_jacobi(Level& lv, Allocs& allocs, Scratch& sc, cudaStream_t s);
int make_fp32_geometry(Level& lv, Allocs& allocs, cudaStream_t s);
int local_to_global(const Level& lv, int* l2g, cudaStream_t s);

// ------------------------------------------------------------------ kernels' host launchers
// Operator: y_L = A_L u (local), optionally followed by QQ^T + mask.  With `sub` (a continuous
// L-vector b), the local output is b / multiplicity - A_L u instead, so that QQ^T of it is the
// residual b - QQ^T A_L u (QQ^T (b / mult) = b for continuous b).
template <class T>
int ax_local(const Level& lv, const T* u, T* y, bool mask_in, cudaStream_t s,
             const T* sub = nullptr);
template <class T>
int gs_apply(const Level& lv, T* u, bool mask, cudaStream_t s);
// QQ^T by the index map of lv (gsm_ids set); gs_apply dispatches to it.
template <class T>
int gsmap_apply(const Level& lv, T* u, bool mask, cudaStream_t s);
// Builds lv's index map from its lattice numbering (SE_MESH_GS_MAP).
int build_level_gsmap(Level& lv, Allocs& allocs, cudaStream_t s);
// FP64 operator with the x part of QQ^T and the mask inside the even-odd kernel (even N, box
// lattice, sweeps): y = A u, or b - A u when b is given; the x-interfaces between the kernel's
// blocks, then the y/z launch follow (ax.cu).
bool ax_fold_ok(const Level& lv);
// dinv: y = A (dinv .* u) (the input scaled as it is loaded)
int ax_apply_folded(const Level& lv, const double* u, double* y, const double* b, cudaStream_t s,
                    const double* dinv = nullptr);
template <class T>
inline int ax_apply(const Level& lv, const T* u, T* y, cudaStream_t s) {
  if constexpr (sizeof(T) == 8)
    if (ax_fold_ok(lv)) return ax_apply_folded(lv, u, y, nullptr, s);
  SE_TRY(ax_local<T>(lv, u, y, false, s));
  return gs_apply<T>(lv, y, true, s);
}
// r = b - A u (masked), one operator pass: no separate subtraction over the vector.
template <class T>
inline int residual_apply(const Level& lv, const T* b, const T* u, T* r, cudaStream_t s) {
  if constexpr (sizeof(T) == 8)
    if (ax_fold_ok(lv)) return ax_apply_folded(lv, u, r, b, s);
  SE_TRY(ax_local<T>(lv, u, r, false, s, b));
  return gs_apply<T>(lv, r, true, s);
}

// Output of an operator kernel at local point idx: acc, or b / multiplicity - acc.
template <class T>
__device__ __forceinline__ T ax_output(T acc, const T* __restrict__ sub,
                                       const uint8_t* __restrict__ pflag, int64_t idx) {
  if (!sub) return acc;
  const int mlog = __ffs(pflag[idx] & 0x0F) - 1;  // 1/multiplicity = 2^-mlog, exact
  const T w = mlog == 0 ? T(1) : (mlog == 1 ? T(0.5) : (mlog == 2 ? T(0.25) : T(0.125)));
  return sub[idx] * w - acc;
}
// Elementwise and reduction kernels (blas.cu)
int dot_weighted(const Level& lv, const double* a, const double* b, double* dst_dev,
                 Scratch& sc, cudaStream_t s);
template <class Tin, class Tout>
int convert(const Tin* in, Tout* out, int64_t n, cudaStream_t s);
template <class T>
int fill_zero(T* x, int64_t n, cudaStream_t s);
template <class T>
int axpby(T a, const T* x, T b, const T* y, T* out, int64_t n, cudaStream_t s);  // out=a x+b y
template <class T>
// rin (first step of a Jacobi smoother, from_r): the smoothed residual is dinv .* rin, formed
// here instead of read from r (r is then only written, when the step is not the last)
int cheb_update(T* x, T* d, T* r, const T* sv, const T* dinv, int64_t n, T c1, T c2,
                bool first, cudaStream_t s, T scale = T(1), bool from_r = false, bool last = false,
                const T* rin = nullptr, int prof_p = 0);  // prof_p: the level's order, for profiles
template <class T>
int scale_mul(const T* a, const T* b, T* out, int64_t n, cudaStream_t s);  // out = a*b
// FP64 Krylov kernels with device scalars (slots of Scratch::scal)
int fpcg_init(const Level& lv, const double* r, const double* z, Scratch& sc, cudaStream_t s);
int fpcg_alpha(const Level& lv, const double* p, const double* w, Scratch& sc, cudaStream_t s);
int fpcg_update(const Level& lv, double* x, const double* p, const double* r, const double* w,
                double* r2, Scratch& sc, cudaStream_t s);
int fpcg_beta(const Level& lv, const double* z, const double* r2, const double* r, Scratch& sc,
              cudaStream_t s);
int fpcg_pupdate(const Level& lv, double* p, const double* z, Scratch& sc, cudaStream_t s);
int fpcg_update_inplace(const Level& lv, double* x, const double* p, double* r, const double* w,
                        double* r_old, Scratch& sc, cudaStream_t s);
int dot_to_slot(const Level& lv, const double* a, const double* b, Scratch& sc, int slot,
                cudaStream_t s);
int axpy_dot(const Level& lv, double* w, const double* v, const double* vnext, Scratch& sc,
             int hslot, int nslot, cudaStream_t s);
int scale_inv_sqrt(double* out, const double* in, double* scal, int slot, int64_t n, cudaStream_t s);
int lincomb(double* x, const double* const* zs_dev, const double* y_dev, int m, int64_t n,
            cudaStream_t s);
// Smoothers (fdm.cu)
template <class T>
int schwarz_apply(const Level& lv, int kind, const T* r, T* out, cudaStream_t s);
template <class T>
int gather_ext(const Level& lv, const T* r, T* rbar, cudaStream_t s);
template <class T>
int fdm_apply_ext(const Level& lv, const T* rbar, T* zbar, cudaStream_t s);
int fdm_setup(const se_mesh_s* m, Level& lv, Allocs& allocs, bool want32, cudaStream_t s,
              bool want_df = false);
int asm_weights(Level& lv, Allocs& allocs, cudaStream_t s);
// Transfers (transfer.cu): level f (fine) <-> level c (coarse)
template <class T>
int restrict_apply(const Level& f, const Level& c, const T* J, const T* rf, T* rc,
                   cudaStream_t s);
template <class T>
int prolong_apply(const Level& f, const Level& c, const T* J, const T* ec, T* ef, bool accumulate,
                  cudaStream_t s);
// Coarse solve (coarse.cu)
int coarse_setup(Level& lv, Allocs& allocs, cudaStream_t s);
struct CoarseWork {
  double *x, *r, *u, *p, *q, *s, *z, *w0, *w1;  // pipelined-CG vectors (w alternates)
  double* partial;  // coarse_partial_doubles(nblocks)
  unsigned* bar;    // [2]: arrival count (monotonic within a launch), unused
  int* status;      // [2]: error flag, iterations
  int nblocks;
  // [nblocks]: per block, how many w vectors it has published (register-resident solver; zeroed
  // before each launch)
  unsigned* flags = nullptr;
  // [3]: iterations and solves since the last reset, and solves whose bounded waits expired
  // (kept until read); may be null
  unsigned long long* totals = nullptr;
};
// SE_ETIMEOUT (and a cleared count) if a coarse solve of this work space gave up a bounded wait
// since the last call; synchronises `s` first.
int coarse_fault_take(CoarseWork& w, cudaStream_t s);
size_t coarse_partial_doubles(int nblocks);
int coarse_alloc(const Level& lv, Allocs& allocs, CoarseWork* w);
template <class T>
int coarse_solve(const Level& lv, CoarseWork& w, const T* r_l, T* x_l, double tol, int maxit,
                 cudaStream_t s);
// The coarse solves of several independent problems in one cooperative launch (batched solves):
// problem m's coarsest level lv[m] with work space w[m]; its right-hand side and solution are the
// L-vector pieces of rin / xout (FP32 when fp32) starting at loff[m] (host array).  Each problem
// iterates to its own tolerance on its own sub-grid of blocks.
struct CoarseGroup {
  int n = 0, nblocks = 0;
  bool fp32 = false;
  void* args = nullptr;  // device array of the n problems' kernel arguments
  int* boff = nullptr;   // device [n + 1]: first block of each problem
  double nodes = 0.0;    // global nodes of all problems (profiling units)
};
int coarse_group_setup(CoarseGroup* g, const Level* const* lv, CoarseWork* const* w, int n, bool fp32,
                       const void* rin, void* xout, const int64_t* loff, double tol, int maxit,
                       Allocs& allocs, cudaStream_t s);
template <class T>
int coarse_group_solve(const CoarseGroup& g, cudaStream_t s);
// QQ^T index map of a level from host global ids (any labels, int64) and Dirichlet bytes.
int build_gsmap_from_gid(Level& lv, const int64_t* gid, const uint8_t* dirichlet, Allocs& allocs,
                         cudaStream_t s);

// ------------------------------------------------------------------ profiling (common.cu)
// Profiling variant of a launch: polynomial order p (0..31) plus 32 for FP32 arithmetic, plus 64
// for double-float (df64) arithmetic on FP64 vectors.
constexpr int PROF_VARIANTS = 96;
template <class T>
inline int prof_variant(int p) {
  return (p & 31) + (sizeof(T) == 4 ? 32 : 0);
}
struct ProfScope {
  int kind;
  cudaStream_t s;
  double units, bytes, flops;
  int variant;
  bool on;
  cudaEvent_t a = nullptr, b = nullptr;
  ProfScope(int kind, cudaStream_t s, double units, double bytes, double flops, int variant = 0);
  ~ProfScope();
};

// ------------------------------------------------------------------ launch tiles (common.cu)
// Elements per block of the operator and FDM kernels for one (order, precision); 0 = the built-in
// heuristic.  se_tune measures the candidates and stores the fastest here.
struct TileCfg {
  int ax_ne = 0;
  int fdm_ne = 0;
};
TileCfg tile_get(int p, bool fp32);
void tile_set(int p, bool fp32, const TileCfg& c);
int ax_elems_per_block(int p, bool fp32);
// FP32 Ax pipelined with TMA bulk copies (even N only); device status of its bounded waits.
bool ax_tma_supported(int p);
int ax_tma_group(int p);
int ax_local_tma(const Level& lv, const float* u, float* y, cudaStream_t s, const float* sub);
// FP64 Ax with even-odd folded contractions (even N).
bool ax_eo_supported(int p);
void ax_eo_tables(const Basis1D& b, double* out);
int ax_local_eo(const Level& lv, const double* u, double* y, cudaStream_t s, const double* sub);
// The same with the x-interface sums of the block's elements and the mask (NE elements per block).
int ax_local_eo_fold(const Level& lv, const double* u, double* y, const double* sub, int NE,
                     cudaStream_t s, const double* dinv = nullptr);
// The x-interfaces between consecutive blocks of ax_local_eo_fold (NE elements per block).
int gs_fold_fixup(const Level& lv, double* y, int NE, cudaStream_t s);
// The same contractions in df64 arithmetic (FP64 in and out); needs lv.Gdf and lv.eodf.
int ax_local_eo_df(const Level& lv, const double* u, double* y, cudaStream_t s, const double* sub);
// b[i] = nearest df64 of a[i] (device arrays, stream-ordered).
int split_df(const double* a, df64* b, int64_t n, cudaStream_t s);
// df64 copies of a level's geometric factors and folded tables (no-op if present).
int make_df_geometry(Level& lv, Allocs& allocs, cudaStream_t s);
inline bool ax_df_route(const Level& lv) {
  return lv.df && lv.Gdf && (ax_eo_supported(lv.p) ? lv.eodf != nullptr : lv.Ddf != nullptr);
}
// SE_ETIMEOUT (and the record cleared) if a pipelined kernel of lv gave up a bounded wait since
// the last call; synchronises s first.
int level_pipeline_take(const Level& lv, cudaStream_t s);
int fdm_elems_per_block(int p, bool fp32);
size_t fdm_smem_bytes(int p, bool fp32, int ne);
int fdm_block_threads(int p, bool fp32, int ne);
int fdm_max_threads(bool fp32);

inline unsigned grid_for(int64_t n, int threads, int64_t max_blocks = 1 << 30) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (unsigned)b;
}

inline cudaStream_t as_stream(void* s, cudaStream_t dflt) {
  return s ? reinterpret_cast<cudaStream_t>(s) : dflt;
}

}  // namespace se
