/*
 * se.h -- C ABI of the GB300 spectral-element Poisson library (libse.so).
 *
 * The library implements the pressure-Poisson hot path of Phillips, Kerkemeier and Fischer,
 * "Tuning Spectral Element Preconditioners for Parallel Scalability on GPUs" (arXiv 2110.07663):
 * the matrix-free spectral element operator (Sec. 2.1), the p-multigrid V-cycle (Algorithm 1)
 * with Chebyshev acceleration (Algorithm 2) of restrictive/additive Schwarz smoothers built on
 * fast-diagonalisation local solves (Sec. 2.2.2, eqs 4-9) or of Jacobi smoothing, and flexible
 * Krylov outer solvers (Sec. 2.2).  One GPU, hand-written CUDA kernels for sm_103a.
 *
 * Conventions for every call:
 *  - Return value: SE_OK (0) or an se_status error code; se_last_error() gives a message
 *    (thread-local, valid until the next failing call on that thread).
 *  - Handles (se_mesh_t, se_pmg_t, se_server_t) are opaque, owned by the library, freed only by
 *    the matching *_destroy call.
 *  - Vectors are CALLER-OWNED device pointers (cudaMalloc or torch tensors) of FP64 values in
 *    L-vector layout unless stated: length L = E*N^3 with N = p+1, element-major, index
 *    i + N*(j + N*(k + N*e)) with i the fastest reference direction r; element
 *    e = ex + nx*(ey + ny*ez).  "Continuous" means all local copies of a global node hold the
 *    same value.  The library never frees caller memory and keeps no pointer to it after
 *    returning (except se_serve_submit, which copies the right-hand side).
 *  - Streams: `stream` is a cudaStream_t passed as void*; NULL means the handle's own stream,
 *    a blocking stream (ordered with the legacy default stream).  Calls enqueue work and return
 *    without synchronising unless they return host results (se_dot, se_solve statistics,
 *    se_pmg_coarse_solve iteration count, se_serve_*).
 */
#ifndef SE_H
#define SE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
enum se_status {
  SE_OK = 0,
  SE_EINVAL = 1,    /* invalid argument (null pointer, unsupported order, bad descriptor) */
  SE_ENOMEM = 2,    /* device or host allocation failed */
  SE_ENOTCONV = 3,  /* solver reached maxit without meeting the tolerance; stats are filled */
  SE_ECUDA = 4,     /* a CUDA runtime call failed; se_last_error() names it */
  SE_ETIMEOUT = 5,  /* a bounded device-side wait ran out (no hang: the kernel returned) */
  SE_EBUSY = 6,     /* served request still pending */
  SE_EREFUSED = 7,  /* served request can never fit the HBM budget */
  SE_ECANCELED = 8  /* served request removed from the queue by se_serve_cancel before it started */
};

enum { SE_BC_DIRICHLET = 0, SE_BC_NEUMANN = 1 };
/* Arithmetic of a preconditioner (se_pmg_desc.precision).  SE_DF64: FP64 vectors throughout, the
 * operator and FDM kernels of the smoothed levels compute in double-float arithmetic on the FP32
 * pipe (pairs of FP32 values, about 47-48 significant bits; odd orders use the even-odd folded
 * operator, even orders the plain sum factorisation).  Every df64 path (SE_DF64, SE_AX_DF64, operator_df64,
 * arnoldi_df64) takes operands of magnitude in [2^-103, 2^128) (about 1e-31 to 3e38) at that
 * accuracy; smaller values keep FP32 accuracy relative to themselves (below 2^-126 they are
 * zero) and larger ones overflow, so a problem scaled outside that range needs FP64. */
enum { SE_FP64 = 0, SE_FP32 = 1, SE_DF64 = 2 };
enum { SE_SMOOTH_JACOBI = 0, SE_SMOOTH_RAS = 1, SE_SMOOTH_ASM = 2 };
enum { SE_FPCG = 0, SE_FGMRES = 1 };
/* se_ax flags */
enum { SE_AX_ASSEMBLE = 1, SE_AX_MASK = 2, SE_AX_FP32 = 4, SE_AX_DF64 = 8 };

#define SE_MAX_LEVELS 8
#define SE_MAX_ORDER 10

typedef struct se_mesh_s* se_mesh_t;
typedef struct se_pmg_s* se_pmg_t;

const char* se_last_error(void);
int se_version(void);

/* ---------------------------------------------------------------- mesh (Sec. 2.1) */
/* Box-topology hexahedral mesh: nel[0]*nel[1]*nel[2] elements of a structured lattice of
 * (nel[0]+1)(nel[1]+1)(nel[2]+1) vertices.  Each element is mapped trilinearly from its 8
 * vertices to its GLL points, then every node x receives the smooth map
 * x_c <- x_c + deform_amp*sin(2 pi x)sin(2 pi y)sin(2 pi z) (same scalar for c = x, y, z).  The
 * isoparametric geometry of Sec. 2.1 is built from those node positions. */
typedef struct se_mesh_desc {
  int nel[3];              /* elements per direction, each >= 1 */
  int p;                   /* polynomial order, 1..SE_MAX_ORDER */
  const double* vertex_xyz;/* HOST, optional: vertex positions, xyz interleaved, vertex id
                              v = a + (nx+1)(b + (ny+1)c); NULL: unit box lattice whose interior
                              vertices move by perturb_frac*h*(2U-1) per direction, U the
                              SplitMix64 uniform number 3v+d of stream `seed` */
  double deform_amp;       /* amplitude of the smooth map (0.05 in the synthetic workloads) */
  double perturb_frac;     /* used only when vertex_xyz == NULL */
  uint64_t seed;
  int bc[6];               /* faces x-, x+, y-, y+, z-, z+: SE_BC_DIRICHLET or SE_BC_NEUMANN */
  int flags;               /* SE_MESH_NONBLOCKING_STREAM: the handle's stream is non-blocking;
                              SE_MESH_GS_MAP: QQ^T of this mesh and of every preconditioner level
                              built on it runs from a sorted index map (as se_gsmap_*) instead of
                              the direction sweeps over the box lattice (the default) */
} se_mesh_desc;
enum { SE_MESH_NONBLOCKING_STREAM = 1, SE_MESH_GS_MAP = 2 };

typedef struct se_mesh_info {
  int64_t E, N, L, n_global;  /* elements, points per direction, local points, global nodes */
  int64_t n_dof;              /* E*p^3, the paper's n (Sec. 1, Table 2) */
  int p;
  int nel[3];
} se_mesh_info;

/* Builds geometry, point flags (multiplicity, Dirichlet), element neighbours and the Jacobi
 * diagonal on the device (and the QQ^T index map with SE_MESH_GS_MAP). */
int se_mesh_create(const se_mesh_desc* desc, se_mesh_t* out);
int se_mesh_destroy(se_mesh_t m);
int se_mesh_get_info(se_mesh_t m, se_mesh_info* info);
/* Node coordinates: xyz_dev is a device array of 3*L doubles (x block, y block, z block). */
int se_mesh_nodes(se_mesh_t m, double* xyz_dev, void* stream);
/* Vertex lattice actually used (host array of 3*(nx+1)(ny+1)(nz+1) doubles, interleaved). */
int se_mesh_vertices(se_mesh_t m, double* xyz_host);
/* b = M QQ^T (B_L f) (Sec. 2.1, eq 3): f_dev holds f at the nodes (L-vector). */
int se_mesh_rhs(se_mesh_t m, const double* f_dev, double* b_dev, void* stream);

/* ---------------------------------------------------------------- operator (Sec. 2.1) */
/* y = [M] [QQ^T] A_L [M] u.  flags: SE_AX_ASSEMBLE applies QQ^T (direct stiffness
 * summation), SE_AX_MASK zeroes Dirichlet nodes of input and output, SE_AX_FP32 computes in
 * FP32, SE_AX_DF64 in double-float arithmetic (the first call
 * allocates df64 copies of the geometric factors, 6 L x 8 bytes, owned by the mesh); inputs and
 * outputs stay FP64.  A_L is applied by tensor-product sum factorisation
 * (Sec. 1: ~7E(p+1)^3 reads, 12E(p+1)^4 operations).  u and y must not overlap. */
int se_ax(se_mesh_t m, const double* u, double* y, int flags, void* stream);
/* Residual r = M (b - QQ^T A_L u), the step "r = b - A x" of Algorithm 1 (Sec. 2.2.2) in one
 * operator pass: the local kernel outputs b / multiplicity - A_L u, whose QQ^T is the residual.
 * b: continuous, masked L-vector; u: L-vector that is zero on Dirichlet nodes (it is used as
 * given).  flags: 0 (FP64), SE_AX_FP32 (computed in FP32; the first such call allocates one more
 * L-vector of floats, owned by the mesh) or SE_AX_DF64.  r must overlap neither b nor u;
 * SE_EINVAL otherwise. */
int se_residual(se_mesh_t m, const double* b, const double* u, double* r, int flags, void* stream);
/* In place u <- [M] QQ^T u (Sec. 2.1, gather-scatter); mask != 0 also zeroes Dirichlet nodes. */
int se_gs(se_mesh_t m, double* u, int mask, void* stream);
/* ---------------------------------------------------------------- QQ^T index map (Sec. 2.1) */
/* Direct stiffness summation QQ^T driven by a precomputed sorted index map, for ANY element
 * connectivity (se_gs uses direction sweeps that need the box lattice).  Q is given by the global
 * node id of every local point: (QQ^T u)_l = sum of u over the local copies of l's global node.
 *  gid:       HOST array of L int64 global ids, each >= 0 (any labels; compact labels below
 *             2L + 1024 are grouped by counting sort, others by sorting).
 *  dirichlet: HOST array of L bytes or NULL; a global node is Dirichlet when any of its copies
 *             has a non-zero byte; apply with mask != 0 sets all its copies to zero.
 * The map keeps, per global node with two or more copies, its local ids in ascending order
 * (int32, so L < 2^31), bucketed by multiplicity (2, 4, 8 and other counts), plus the single
 * copies of Dirichlet nodes; the copies are summed in ascending local id order from the first, so
 * the result equals the sequential sum in local-id order bitwise.  The handle owns its device
 * memory and its stream (blocking, like a mesh's: stream == NULL orders the call with the legacy
 * default stream).  Errors: SE_EINVAL for L outside [1, 2^31), a null gid or a
 * negative id (checked before any device work), SE_ENOMEM, SE_ECUDA. */
typedef struct se_gsmap_s* se_gsmap_t;
int se_gsmap_create(int64_t L, const int64_t* gid, const uint8_t* dirichlet, se_gsmap_t* out);
/* In place u <- [M] QQ^T u on a device vector of L values (FP64, or FP32 for _f32). */
int se_gsmap_apply(se_gsmap_t g, double* u, int mask, void* stream);
int se_gsmap_apply_f32(se_gsmap_t g, float* u, int mask, void* stream);
/* counts[5]: groups of 2, 4 and 8 copies, groups of other multiplicities (>= 2), single copies
 * of Dirichlet nodes. */
int se_gsmap_info(se_gsmap_t g, int64_t* counts);
/* Host only (no device call): the counts se_gsmap_create would produce for these arguments. */
int se_gsmap_count(int64_t L, const int64_t* gid, const uint8_t* dirichlet, int64_t* counts);
int se_gsmap_destroy(se_gsmap_t g);

/* Unique-node inner product sum_l a_l b_l / mult_l of two continuous L-vectors (FP64,
 * deterministic order).  Synchronises the stream; result written to *out_host. */
int se_dot(se_mesh_t m, const double* a, const double* b, double* out_host, void* stream);
/* Assembled, masked diagonal of A (Jacobi surrogate, Sec. 2.2.3) as an L-vector; Dirichlet
 * nodes get 1. */
int se_jacobi_diag(se_mesh_t m, double* d_dev, void* stream);

/* ---------------------------------------------------------------- p-multigrid (Sec. 2.2) */
typedef struct se_pmg_desc {
  int nlev;                      /* levels, 2..SE_MAX_LEVELS */
  int schedule[SE_MAX_LEVELS];   /* orders, schedule[0] == mesh p, strictly decreasing */
  int smoother;                  /* SE_SMOOTH_RAS, SE_SMOOTH_ASM or SE_SMOOTH_JACOBI */
  int cheb_order[SE_MAX_LEVELS]; /* Chebyshev order (loop count of Algorithm 2) per level */
  double eig_lo, eig_hi;         /* bounds (eig_lo, eig_hi)*lambda-tilde; paper: (0.1, 1.1);
                                    0 <= eig_lo < eig_hi */
  int arnoldi_steps;             /* Arnoldi rounds for lambda-tilde; paper: 10 */
  uint64_t seed;                 /* start-vector stream: level l uses 1000 + l + 7919*seed */
  double coarse_tol;             /* coarsest-level Jacobi-PCG relative tolerance (1e-2) */
  int coarse_maxit;              /* and iteration cap (500) */
  int precision;                 /* SE_FP64; SE_FP32 for the whole V-cycle except the coarse
                                    solve (Arnoldi and coarse solve stay FP64); SE_DF64: FP64
                                    vectors, operator and FDM kernels in double-float */
  int arnoldi_df64;              /* 1: the Arnoldi rounds of an SE_FP64 or SE_FP32 preconditioner
                                    apply the operator and FDM kernels in double-float (FP64
                                    vectors; df64 copies of the level data exist
                                    only during the set-up).  SE_DF64 always does. */
  int cycle;                     /* SE_CYCLE_MULTIPLICATIVE (0): Algorithm 1 with the Chebyshev
                                    smoother.  SE_CYCLE_ADDITIVE (1): the additive V-cycle the
                                    paper uses for Schwarz smoothers without Chebyshev
                                    acceleration (Sec. 2.2.2): on every level x = S b + P V(P^T b),
                                    S the smoother itself (cheb_order, eig_lo/hi unused), no
                                    residual re-evaluation, no post-smoothing. */
} se_pmg_desc;
enum { SE_CYCLE_MULTIPLICATIVE = 0, SE_CYCLE_ADDITIVE = 1 };

/* Builds the levels (each rediscretised on the same mapped mesh), Jacobi diagonals, FDM
 * factors S and Lambda (eqs 6-7), the assembled coarsest operator, and the Chebyshev bounds
 * from Arnoldi on S A at every level but the coarsest.  Synchronises. */
int se_pmg_setup(se_mesh_t m, const se_pmg_desc* desc, se_pmg_t* out);
int se_pmg_destroy(se_pmg_t pmg);
/* z = M r: one V-cycle (Algorithm 1) with x = 0 on entry.  r, z: fine-level L-vectors; r must be
 * continuous (all copies of a node equal, as every QQ^T output and every residual of an assembled
 * right-hand side is): the V-cycle forms its residuals b - A x in one operator pass that relies
 * on it. */
int se_pmg_apply(se_pmg_t pmg, const double* r, double* z, void* stream);
/* lambda-tilde of level lvl (largest |Ritz value| of Arnoldi on S A, Sec. 2.2.3). */
int se_pmg_lambda(se_pmg_t pmg, int lvl, double* lam);
int se_pmg_level_info(se_pmg_t pmg, int lvl, se_mesh_info* info);
/* Level-lvl building blocks, all on level-lvl L-vectors (FP64 in/out; computed in the pmg's
 * precision except where noted): */
/* y = M QQ^T A_L u (FP64 always). */
int se_pmg_level_ax(se_pmg_t pmg, int lvl, const double* u, double* y, void* stream);
/* s = S r: the surrogate smoother (RAS: eq 4 with own-node weights; ASM: eq 4; Jacobi). */
int se_pmg_smooth(se_pmg_t pmg, int lvl, const double* r, double* s, void* stream);
/* rbar = R_e r for all elements: E*(p+3)^3 values, element-major, window index
 * a + (p+3)*(b + (p+3)*c), window point (a,b,c) = lattice node (ex*p-1+a, ey*p-1+b, ez*p-1+c);
 * 0 outside the domain. */
int se_pmg_gather_ext(se_pmg_t pmg, int lvl, const double* r, double* rbar, void* stream);
/* zbar = Abar_e^-1 rbar per element by fast diagonalisation (eqs 8-9), E*(p+3)^3 values. */
int se_pmg_fdm(se_pmg_t pmg, int lvl, const double* rbar, double* zbar, void* stream);
/* x = Chebyshev correction of Algorithm 2 for residual res (order and bounds of the level). */
int se_pmg_cheby(se_pmg_t pmg, int lvl, const double* res, double* x, void* stream);
/* rc = P^T rf (level lvl -> lvl+1) and ef = P ec (level lvl+1 -> lvl). */
int se_pmg_restrict(se_pmg_t pmg, int lvl, const double* rf, double* rc, void* stream);
int se_pmg_prolong(se_pmg_t pmg, int lvl, const double* ec, double* ef, void* stream);
/* Coarsest level: x = A_c^-1 r by Jacobi-PCG to coarse_tol (FP64, one persistent cooperative
 * launch, pipelined form of the iteration: one grid synchronisation per iteration).  *iters
 * receives the iteration count (synchronises). */
int se_pmg_coarse_solve(se_pmg_t pmg, const double* r, double* x, int* iters, void* stream);
/* Coarse solves of this preconditioner since the last reset (every launch of its coarsest level,
 * inside V-cycles or by se_pmg_coarse_solve) and their total Jacobi-PCG iterations; reset != 0
 * starts a new count.  Synchronises the preconditioner's stream (the caller synchronises other
 * streams its solves ran on). */
int se_pmg_coarse_stats(se_pmg_t pmg, int reset, int64_t* solves, int64_t* iterations);
/* Same coarse solve as se_pmg_coarse_solve, for callers that must not allocate device memory
 * during the call: code running after its memory pool is fixed (an application or framework
 * that reserved the device memory up front and owns every later allocation), or a steady-state
 * loop whose allocations were all made at start-up.  The paper has no counterpart; this is a
 * library convenience.  It calls no cudaMalloc/cudaFree: the CG vectors, partial sums and
 * barrier words live in one static device array of the library (about 9.5 MB, held by every
 * GPU that loads the library until the process exits), so the coarsest level may have at most
 * 131072 global nodes; larger problems get SE_EINVAL.  The call synchronises its stream, so it
 * cannot be captured into a CUDA graph.  The first call on each device looks up the array's
 * device address with that device current and keeps it for the life of the process, so the entry
 * point must not be called again after cudaDeviceReset on that device.  The caller passes r and
 * x (coarse L-vectors) as for se_pmg_coarse_solve.  All calls
 * share the one array, which keeps the last call's contents (the call resets what must start at
 * zero): calls whose work overlaps on the GPU (other streams, other threads, other handles)
 * race and must be serialised by the caller.  Synchronises the stream. */
int se_pmg_coarse_solve_noalloc(se_pmg_t pmg, const double* r, double* x, int* iters,
                                void* stream);

/* ---------------------------------------------------------------- solve (Sec. 2.2) */
typedef struct se_solve_opts {
  int method;        /* SE_FPCG (flexible CG) or SE_FGMRES (right-preconditioned, flexible) */
  int restart;       /* FGMRES restart length m (paper: 20) */
  double tol;        /* stop when ||r_k||_2 / ||r_0||_2 <= tol (unique-node 2-norm; see tol_norm) */
  int maxit;
  int graph_capture; /* 1 (SE_FPCG only): the whole solve runs as one CUDA graph launch whose
                        iteration loop is a device-side WHILE node (no host round trip per
                        iteration); the graph is cached per mesh for the same pmg, b, x, tol,
                        maxit and rebuilt when one of them changes */
  void* stream;      /* NULL: the mesh's stream */
  int tol_norm;      /* SE_TOL_R0 (0): stop when ||r_k|| <= tol ||r_0||; SE_TOL_B (1): when
                        ||r_k|| <= tol ||b|| (for an initial guess from se_proj_guess: the same
                        accuracy whatever the guess; 0 iterations if the guess already meets it) */
  int operator_df64; /* 1: the outer operator A x computes in double-float arithmetic, as se_ax
                        with SE_AX_DF64 */
} se_solve_opts;
enum { SE_TOL_R0 = 0, SE_TOL_B = 1 };

typedef struct se_solve_stats {
  int iterations;
  int status;
  double rel_residual;   /* final ||r||/||r_0|| (SE_TOL_B: ||r||/||b||) as tracked by the method */
  double ms_total;       /* wall time of the solve (events on the stream) */
  double ms_precond;     /* time inside preconditioner applications */
  double ms_operator;    /* time inside outer operator applications */
} se_solve_stats;

/* x (in: initial guess, out: solution) of A x = b; pmg == NULL selects Jacobi preconditioning.
 * Returns SE_ENOTCONV (stats filled) if maxit is reached.  Synchronises. */
int se_solve(se_mesh_t m, se_pmg_t pmg, const double* b, double* x, const se_solve_opts* opts,
             se_solve_stats* stats);
/* se_solve with HOST buffers (L doubles each): b_host is copied to the device, the solve starts
 * from x0_host (copied too) or from zero (x0_host == NULL), and the solution is copied to x_host
 * (which may be x0_host).  The copies run on the solve's stream into device vectors the mesh
 * keeps from the first call (so a repeated graph solve reuses its graph); page-locked host
 * buffers give the copy engines' full rate, pageable ones are staged by the driver.  Returns as
 * se_solve; x_host holds the last iterate also when the status is SE_ENOTCONV.  Synchronises. */
int se_solve_host(se_mesh_t m, se_pmg_t pmg, const double* b_host, const double* x0_host,
                  double* x_host, const se_solve_opts* opts, se_solve_stats* stats);

/* ---------------------------------------------------------------- projection (Secs. 3.2 and 4.2) */
/* A space of up to max_vectors (1..16) prior solutions of A x = b on mesh m, for successive
 * right-hand sides (the paper projects each pressure solve onto up to 10 prior solutions,
 * Fischer's method): kept A-orthonormal, x_i^T A x_j = delta_ij, with the images A x_i.  Device
 * memory 2 * max_vectors * L doubles, owned by the handle.  The calls below use the mesh's
 * reduction scratch: do not overlap them with a solve on the same mesh. */
typedef struct se_proj_s* se_proj_t;
int se_proj_create(se_mesh_t m, int max_vectors, se_proj_t* out);
int se_proj_destroy(se_proj_t proj);
/* x = sum_i (x_i, b) x_i: the element of the space closest to A^-1 b in the A-norm (no operator
 * application); x = 0 for an empty space.  Solve from this x with tol_norm = SE_TOL_B. */
int se_proj_guess(se_proj_t proj, const double* b, double* x, void* stream);
/* Adds the solution x (FP64 L-vector, continuous): A-orthogonalised against the space by two
 * modified Gram-Schmidt passes, its image by one operator application, normalised.  A full space
 * restarts from x alone; a remainder below 1e-7 of ||x||_A (x already in the space) is not
 * added.  *size (optional) receives the vectors held.  Synchronises the stream. */
int se_proj_update(se_proj_t proj, const double* x, int* size, void* stream);

/* ---------------------------------------------------------------- batched solves */
/* Many independent problems solved together by flexible PCG in one device-driven CUDA graph.
 * Problems whose preconditioners share a configuration (schedule, smoother RAS or Jacobi,
 * Chebyshev orders, bounds multipliers, coarse tolerance, FP64 or FP32 V-cycle, multiplicative
 * cycle) and a size class (element counts below 4096, then one class per factor 8) form a group
 * that is solved as one union problem (groups are independent branches of the graph): each phase of an iteration (outer
 * operator, QQ^T, smoother, Chebyshev update, transfers, coarse solves) is one launch over all
 * members' elements, inner products and convergence stay per problem (a converged problem keeps
 * its iterate while the others continue), and each member's Chebyshev bounds (Sec. 2.2.3) are
 * folded into its smoother.  Other problems (no preconditioner, ASM, additive cycle, SE_DF64
 * V-cycle) run their own solve loop as a branch of the same graph.  Results of grouped problems agree with
 * se_solve of the same problem to within rounding (iteration counts can differ by one).  Each
 * problem needs its own mesh and preconditioner handles; pmg may be NULL (Jacobi).  b and x are
 * caller-owned device vectors of that mesh; x holds the initial guess at launch.  A group copies
 * its members' level data (geometry, factors, maps) into union arrays owned by the batch.
 * opts->graph_capture = 0 runs the same launches with the loops driven from the host (one read
 * per iteration; se_batch_run then synchronises), e.g. to time each kernel with se_prof_*. */
typedef struct se_problem {
  se_mesh_t mesh;
  se_pmg_t pmg;
  const double* b;
  double* x;
} se_problem;
typedef struct se_batch_s* se_batch_t;
/* Builds and instantiates the batch graph (the inputs are captured by pointer).  The batch uses
 * the problems' handles while it exists (a group's coarse solves run in its members'
 * preconditioner work space): destroy it before any of them, and do not solve a member on its
 * own while the batch runs. */
int se_batch_create(int n, const se_problem* probs, const se_solve_opts* opts, se_batch_t* out);
/* One graph launch on `stream` (NULL: legacy default stream); returns without waiting. */
int se_batch_run(se_batch_t batch, void* stream);
/* Waits for the stream and fills n statistics; returns SE_ENOTCONV if any problem missed tol. */
int se_batch_stats(se_batch_t batch, void* stream, se_solve_stats* out);
int se_batch_destroy(se_batch_t batch);
/* create + run + stats + destroy; ms_total of every entry is the wall time of the whole batch. */
int se_batch_solve(int n, const se_problem* probs, const se_solve_opts* opts, se_solve_stats* out);
/* Number of groups of the batch and of the problems they hold (the rest run alone). */
int se_batch_info(se_batch_t batch, int* groups, int* grouped_problems);

/* ---------------------------------------------------------------- launch-tile autotuner */
/* Elements per thread block of the operator (Ax) and FDM kernels for one polynomial order and
 * precision.  se_tune times every valid candidate on a scratch problem of about 2M points
 * (allocating its own buffers), keeps the fastest in the process-wide table used by all later
 * launches, and reports it with the measured per-launch times.  se_tune_get reports the
 * values in use (the built-in heuristic until tuned); se_tune_set installs given values
 * (0 = heuristic). */
typedef struct se_tile_cfg {
  int p;
  int precision;              /* SE_FP64 or SE_FP32 */
  int ax_elems_per_block;     /* elements * (p+1)^2 <= 512 threads */
  int fdm_elems_per_block;    /* FP64: elements * (p+3)^2 <= 512 threads (one per line);
                                 FP32: 1..8 elements, one warp each */
  double ax_ms, fdm_ms;       /* per launch on the tuning problem (se_tune only) */
} se_tile_cfg;
int se_tune(int p, int precision, se_tile_cfg* out);
int se_tune_get(int p, int precision, se_tile_cfg* out);
int se_tune_set(const se_tile_cfg* cfg);

/* ---------------------------------------------------------------- preconditioner autotuner */
/* The paper's run-time preconditioner selection (Sec. 5, Table 5 without SEMFEM): an exhaustive
 * timed search on the first solve.  A candidate is a preconditioner description; the search
 * fills its timings. */
typedef struct se_tune_candidate {
  se_pmg_desc pmg;
  double setup_ms;   /* se_pmg_setup */
  double ms;         /* mean time to solution over the timed solves */
  int iterations;
  int status;        /* SE_OK, or the error of its set-up or solve */
} se_tune_candidate;
/* The default space for order p: for p = 7 Cheby-ASM(2),(7,3,1), Cheby-RAS(2),(7,3,1),
 * Cheby-Jac(2),(7,5,3,1); for p = 9 (9,5,1), (9,5,1), (9,7,5,1); other orders the analogous
 * three.  Bounds, Arnoldi and coarse settings are the paper's defaults; precision as given.
 * Writes 3 candidates (cap >= 3). */
int se_pmg_autotune_space(int p, int precision, se_tune_candidate* out, int cap, int* n);
/* For each candidate: set up, one untimed solve of A x = b from x = 0 with `opts` (captures the
 * graph when opts->graph_capture), then `repeats` timed solves.  *best receives the index of the
 * fastest converged candidate; with out_pmg, the caller receives that candidate's preconditioner
 * (the others are destroyed).  Returns SE_ENOTCONV if none converged.  Synchronises. */
int se_pmg_autotune(se_mesh_t m, const double* b, const se_solve_opts* opts, int repeats,
                    se_tune_candidate* cands, int n, int* best, se_pmg_t* out_pmg);

/* ---------------------------------------------------------------- serving */
/* Estimated device bytes of a mesh with its preconditioner and solve work space (the sizes the
 * library allocates, plus the transient Arnoldi vectors of the set-up). */
int se_mesh_footprint_bytes(const se_mesh_desc* desc, const se_pmg_desc* pmg, size_t* out);

/* A solve server with continuous batching: submitted requests are admitted by a scheduler thread
 * as slots and device memory free up; resident meshes (keyed by the client) are reused with
 * their geometry, smoother data and captured solve graph; meshes that are not resident are built
 * by a pool of builder threads while the scheduler keeps admitting and completing; the
 * device-driven solves of admitted requests run concurrently on separate non-blocking streams.
 * Requests whose estimated footprint exceeds the whole budget are refused at submission
 * (SE_EREFUSED). */
enum { SE_RHS_MODES = 0, SE_RHS_HOST = 1 };
typedef struct se_request {
  se_mesh_desc mesh;       /* mesh to build when mesh_key is not resident (vertex_xyz unused) */
  uint64_t mesh_key;       /* client-chosen identity: requests with the same key share a mesh */
  se_pmg_desc pmg;         /* preconditioner of a newly built mesh */
  int rhs_kind;            /* SE_RHS_MODES: manufactured u* = amplitude prod_c sin(modes[c] pi x_c);
                              SE_RHS_HOST: b_host holds b (L-vector), copied at submission */
  int modes[3];
  double amplitude;
  const double* b_host;
  double* x_host;          /* optional host buffer (L doubles) that receives the solution */
  double tol;
  int maxit;
} se_request;
typedef struct se_result {
  int status;
  int iterations;
  double rel_residual;
  double latency_ms;       /* completion - submission */
  double queue_ms;         /* start of the solve - submission */
  int new_mesh;            /* 1 if the request built its mesh */
  double setup_ms;         /* time spent building the mesh and preconditioner (0 if reused) */
  double solve_ms;         /* completion - start of the solve */
} se_result;
typedef struct se_serve_cfg {
  size_t hbm_budget;       /* bytes of device memory the resident meshes may occupy */
  int max_slots;           /* requests in flight (being set up or solved) at once */
  int builders;            /* threads that build new meshes concurrently (0: min(4, max_slots)) */
  int proj_vectors;        /* 0: every solve starts from x = 0; 1..16: each resident mesh keeps a
                              projection space of that many prior solutions (se_proj_*), a
                              request on it starts from the projected guess and stops when
                              ||r|| <= tol ||b|| (counted in the footprint) */
  int operator_df64;       /* 1: outer operators of resident meshes compute in double-float
                              (df64 copies of the geometry, 48 bytes per point, counted) */
} se_serve_cfg;
typedef struct se_serve_stats {
  int64_t submitted, completed, refused, failed, pending;
  double solves_per_s;     /* completed / (last completion - first submission) */
  double p50_ms, p99_ms, mean_ms;
  int max_concurrent;
  int64_t meshes_created, mesh_reuses, evictions;
  size_t resident_bytes;
  int64_t projected;       /* requests that started from a non-zero projected guess */
  int64_t cancelled;       /* requests removed from the queue by se_serve_cancel */
} se_serve_summary;
typedef struct se_server_s* se_server_t;
int se_serve_create(const se_serve_cfg* cfg, se_server_t* out);
/* Queues a request; *ticket identifies it.  SE_EINVAL for a malformed request, SE_EREFUSED if it
 * can never fit the budget. */
int se_serve_submit(se_server_t s, const se_request* req, uint64_t* ticket);
/* SE_EBUSY while pending; otherwise the request's status with *res filled. */
int se_serve_poll(se_server_t s, uint64_t ticket, se_result* res);
/* Blocks up to timeout_ms (SE_ETIMEOUT if still pending). */
int se_serve_wait(se_server_t s, uint64_t ticket, double timeout_ms, se_result* res);
/* Cancels a request that is still queued (not yet admitted: no mesh set-up or solve of it has
 * started): SE_OK, and its result then carries status SE_ECANCELED.  A request whose set-up or
 * solve has started is not interrupted: SE_EBUSY, and it completes normally.  SE_EINVAL for an
 * unknown ticket or one that has finished. */
int se_serve_cancel(se_server_t s, uint64_t ticket);
int se_serve_stats(se_server_t s, se_serve_summary* out);
/* Stops the scheduler, waits for running solves, frees every resident mesh. */
int se_serve_destroy(se_server_t s);

/* ---------------------------------------------------------------- profiling */
/* Kernel classes timed with CUDA events on their launch stream while profiling is enabled. */
enum {
  SE_K_AX = 0, SE_K_GS = 1, SE_K_FDM = 2, SE_K_CHEBY_UPD = 3, SE_K_RESTRICT = 4,
  SE_K_PROLONG = 5, SE_K_COARSE = 6, SE_K_KRYLOV = 7, SE_K_JACOBI = 8, SE_K_COUNT = 9
};
int se_prof_enable(int on);
int se_prof_reset(void);
/* Totals since the last reset: summed event time (ms), launches, and the work units the
 * launches processed (points for AX/GS/KRYLOV, elements for FDM, ...; see each kernel). */
int se_prof_query(int kind, double* ms_total, int64_t* launches, double* units, double* bytes,
                  double* flops);
/* The same totals restricted to one variant: the level's polynomial order p (0..31) plus 32 for
 * FP32 arithmetic (e.g. 7 = FP64 kernels of p = 7 levels, 39 = FP32 kernels of p = 7 levels). */
int se_prof_query_variant(int kind, int variant, double* ms_total, int64_t* launches,
                          double* units, double* bytes, double* flops);

/* ALU roof of this GPU for the roofline of arithmetic-bound kernels (measurement only; the paper
 * has no counterpart): fused multiply-add throughput with independent chains on every SM,
 * kind 0 = FP64, 1 = FP32, 2 = FP32 in packed pairs (fma.rn.f32x2), 3 = TF32 tensor-core
 * multiply-adds with FP32 accumulation (warp-level mma.sync m16n8k8).  *tflops receives the best
 * of three timed launches (2 flops per FMA), *sms (may be NULL) the device's SM count.  The
 * launches go to `stream` (NULL: the legacy default stream); the call synchronises. */
int se_prof_fma_peak(int kind, double* tflops, int* sms, void* stream);

/* ---------------------------------------------------------------- self-test of bounded waits */
/* Runs the library's grid barrier with one more expected arrival than blocks launched, so no
 * block can ever pass it; each block gives up after timeout_ms and the call returns
 * SE_ETIMEOUT.  Checks the wait-limit path without hanging the GPU. */
int se_selftest_wait_timeout(double timeout_ms);
/* Host-side fault injection for the allocation failure paths: the n-th device allocation the
 * library makes after this call (n >= 1) fails with SE_ENOMEM before any CUDA call, as if the
 * device were out of memory; n = 0 disarms.  Process-wide, for tests. */
int se_selftest_fail_alloc(int n);

#ifdef __cplusplus
}
#endif
#endif /* SE_H */
