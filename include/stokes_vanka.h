/*
 * stokes_vanka.h -- C ABI of the GB300 (sm_103a) Q2-Q1 Stokes solver:
 * FGMRES right-preconditioned by a monolithic geometric-multigrid V-cycle
 * with additive Vanka relaxation.
 *
 * Paper: Spies, Olson, MacLachlan, "Exploiting mesh structure to improve
 * multigrid performance for saddle point problems".
 *   Section 2.1  -nu Lap u + grad p = f, div u = 0 on the unit square,
 *                Dirichlet velocity on every edge, pressure in L2/R.
 *   Section 2.2  Q2-Q1 Taylor-Hood on a uniform n x n grid,
 *                A = [[L, B^T], [B, 0]], L_ij = a(psi_j, psi_i),
 *                B_kj = b(psi_j, phi_k).
 *   Section 2.3  lexicographic numbering on the structured grid.
 *   Section 3    Algorithm 1 (MG): V-cycle, FE interpolation P, restriction P^T,
 *                exact solve on the coarsest level (level 0).
 *   Section 3.2  Algorithm 3 (additive Vanka): x += sum_i V_i^T W_i A_i^-1 V_i r.
 *   Section 6.3  25 distinct patch matrices on a uniform grid (shared inverses).
 *   Section 6.8  FGMRES preconditioned by the V-cycle.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Vectors are contiguous float64 DEVICE arrays owned by the caller, laid out
 *    as [u_x | u_y | p]: u_x and u_y on the (2n+1)^2 Q2 nodes, p on the (n+1)^2
 *    vertices, each row-major with the x index fastest; node (I, J) sits at
 *    (I/(2n), J/(2n)), vertex (i, j) at (i/n, j/n).  Length
 *    N(n) = 2 (2n+1)^2 + (n+1)^2.  Vectors of a level l use that level's n.
 *  - The operator A is the Dirichlet-eliminated one: rows and columns of
 *    boundary velocity nodes are identity rows/columns; it is symmetric and
 *    singular with kernel (0, 1_p).  b(v, p) = -int p div v.
 *  - Levels are numbered as in Algorithm 1: level 0 is the coarsest
 *    (coarse_n x coarse_n), level L-1 the finest (n x n).
 *  - Every call is stream-ordered on the stream given at creation and returns
 *    without a host synchronisation, except stokes_fgmres_solve, the adjoint
 *    and batched solves, which synchronise to read the convergence test.
 *  - Input and output arrays must not overlap unless a call says otherwise.
 *  - No C++ exception crosses this boundary.  Every call returns a
 *    stokes_status; on failure stokes_last_error() returns a message
 *    (thread-local, valid until the next call on the same thread).
 *  - The hierarchy owns its workspace (level vectors, patch inverses, the
 *    Krylov basis) and frees it in stokes_hierarchy_destroy.
 */
#ifndef STOKES_VANKA_H
#define STOKES_VANKA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  STOKES_OK = 0,
  STOKES_ERR_ARG = 1,        /* bad argument: size, null pointer, level index   */
  STOKES_ERR_OOM = 2,        /* device allocation failed                         */
  STOKES_ERR_CUDA = 3,       /* a CUDA runtime call or a kernel launch failed    */
  STOKES_ERR_NONFINITE = 4,  /* NaN/Inf met in the right-hand side or residual   */
  STOKES_NOT_CONVERGED = 5,  /* maxit reached; x holds the last iterate          */
  STOKES_ERR_TIMEOUT = 6     /* a bounded device wait expired                    */
} stokes_status;

/* Arithmetic of the preconditioner.  FGMRES (residuals, Arnoldi, Givens, the
 * update) and the coarse solve are FP64 in every mode. */
typedef enum {
  STOKES_FP64 = 0,        /* V-cycle entirely in FP64                              */
  STOKES_MIXED_FP32 = 1,  /* V-cycle vectors, residuals and patch solves in FP32   */
  STOKES_MIXED_BF16 = 2   /* as FP32, interior patch solves as BF16 tcgen05 GEMMs
                             with FP32 accumulation                                */
} stokes_precision;

typedef struct {
  int nu1;          /* pre-smoothing Vanka sweeps per level            (2)    */
  int nu2;          /* post-smoothing Vanka sweeps per level           (2)    */
  double omega;     /* Vanka damping: W_i = omega diag(1/m_j)          (0.7)  */
  int coarse_n;     /* coarsest grid, >= 4; n = coarse_n * 2^k         (4)    */
  int restart;      /* FGMRES restart length m, 1..64                  (30)   */
  int maxit;        /* FGMRES iteration cap                            (1000) */
  double rtol;      /* stop when ||b - A x|| <= rtol ||b - A x0||      (1e-8) */
  stokes_precision prec;  /*                                          (FP64) */
  int tile;         /* Vanka sweep configuration: -1 = chosen per level by
                       timing at creation; fused tiles of 0 = 8x8, 1 = 16x8,
                       2 = 16x16, 3 = 14x14 vertices (mixed forms: 3 = the
                       strip sweep of the interior tiles where they fit --
                       BF16 tensor-core patch GEMMs, or FP32 patch solves --
                       with a 14x14 SIMT ring); 4 = split sweep
                       (16x16 own-patch solves writing sums of their
                       corrections, then a separate update), 5 = the same
                       compiled for two CTAs
                       per SM, 6 = fused 4x4 tiles (small levels: more
                       CTAs)                                           (-1) */
  int smoother;     /* stokes_smoother below                             (0)  */
  /* Braess-Sarazin / Schur-Uzawa relaxation (smoothers 2, 3; Sections 3.1, 3.3): D =
   * diag(L) scaled by bs_t, S = -(1/bs_t) B D^-1 B^T relaxed by bs_jacobi_iters
   * weighted-Jacobi steps of weight bs_jacobi_weight from zero, the update
   * damped by bs_omega.  The paper leaves them to experiment.       */
  double bs_t;             /*                                       (1.0)  */
  double bs_omega;         /*                                       (1.0)  */
  double bs_jacobi_weight; /*                                       (1.0)  */
  int bs_jacobi_iters;     /* >= 1                                  (2)    */
  int cycle;        /* coarse-grid corrections per level (Algorithm 1): 1 =
                       V-cycle, 2 = W-cycle (the coarse problem is cycled twice;
                       the second time on the updated residual)           (1)  */
  int precond;      /* FGMRES preconditioner: 0 = monolithic multigrid (the
                       smoother above), 1 = block-triangular (Section 3.4,
                       Algorithm 5: M dp = -r_p, then L du = r_u - B^T dp, each
                       by bt_cycles V(bt_nu, bt_nu) cycles of scalar multigrid
                       with weighted Jacobi; FP64 only)                   (0)  */
  int bt_cycles;           /*                                       (3)    */
  int bt_nu;               /*                                       (3)    */
  double bt_omega_u;       /* Jacobi weight on L                    (1.0)  */
  double bt_omega_p;       /* Jacobi weight on M                    (0.6)  */
  int tail_n;       /* mixed forms with Vanka relaxation: the levels with n <=
                       tail_n below the finest one run the whole cycle there
                       (sweeps, residuals, transfers, coarse solve; V or W) as
                       one persistent cooperative launch with grid barriers,
                       with the 8 x 8 SIMT sweep tile; 0 = launch kernel by
                       kernel; negative (a test mode): the same kernel and steps
                       for n <= -tail_n, one launch per step.  Off by default:
                       on GB300 the coarse levels are bound by the latency of
                       a tile's patch solves, which the launch does not remove,
                       and the grid barriers cost more than the launches they
                       replace                                           (0)    */
  int orth;         /* Gram-Schmidt of the Arnoldi step (Section 6.8): 1 =
                       classical, two passes over the basis per iteration with
                       the second only where the first removed more than half
                       of ||w||^2 (DGKS test, taken on the device); 2 = modified,
                       one pass per basis vector in the textbook order; 0 = by
                       size: modified on grids of at least 2^20 dofs, where a
                       pass streams HBM faster than the FP64 units do the
                       classical passes' four FMAs per element and vector, and
                       classical below, where the modified form's one launch
                       per basis vector costs more than its arithmetic   (0)    */
} stokes_params;

/* How each Vanka patch solve A_i^-1 r_i is applied (Section 4, Section 6.2). */
typedef enum {
  /* "tuned" Vanka: patches of equal matrix share one factorisation (25
   * classes per level, Section 6.3); memory independent of n. */
  STOKES_SMOOTHER_SHARED = 0,
  /* "simple" Vanka: an explicit 51 x 51 inverse for every patch of every
   * level, computed at creation by Gauss-Jordan on the device and streamed
   * from HBM at every sweep (2601 doubles per vertex: 87 GB on the finest
   * 2048^2 level).  FP64 form only. */
  STOKES_SMOOTHER_PER_PATCH = 1,
  /* Braess-Sarazin relaxation instead of Vanka (Section 3.1, Algorithm 2, the
   * inexact variant), matrix-free, in the V-cycle's precision (FP64 or
   * STOKES_MIXED_FP32; not with STOKES_MIXED_BF16, whose tensor-core path is
   * Vanka's patch GEMM). */
  STOKES_SMOOTHER_BRAESS_SARAZIN = 2,
  /* Schur-Uzawa relaxation (Section 3.3, Algorithm 4): the block lower-
   * triangular step du = (1/t) D^-1 r_u, Jacobi on S dp = r_p - B du, with the
   * bs_* parameters (the paper's values: bs_t = 1, bs_jacobi_weight = 0.4 with
   * one Jacobi step, bs_omega = 1).  Same precisions as Braess-Sarazin. */
  STOKES_SMOOTHER_SCHUR_UZAWA = 3
} stokes_smoother;

typedef struct stokes_hierarchy stokes_hierarchy;

/* Fill *p with the defaults shown above. */
void stokes_default_params(stokes_params* p);

/* Build the multigrid hierarchy for an n x n grid (Section 3: rediscretised
 * levels n, n/2, ..., coarse_n), the 25 Vanka patch-class inverses per level
 * (Section 6.3) and the coarse-grid inverse.  n must be coarse_n * 2^k with
 * coarse_n >= 4.  viscosity > 0.  params may be NULL (defaults).  stream is a
 * cudaStream_t (NULL = legacy default stream).  The Krylov workspace
 * (2 restart + 1 vectors of N(n) doubles) is allocated here.  A mixed-
 * precision hierarchy also owns a second (non-blocking) stream and two events:
 * a strip sweep forks the SIMT ring of boundary tiles onto that stream and joins it
 * back, so every call stays ordered on `stream` (also under stream capture);
 * stokes_hierarchy_destroy synchronises and releases them. */
stokes_status stokes_hierarchy_create(int n, double viscosity, const stokes_params* params,
                                      void* stream, stokes_hierarchy** out);
stokes_status stokes_hierarchy_destroy(stokes_hierarchy* h);

/* Number of levels L and the grid size n_l of level l (0 = coarsest). */
stokes_status stokes_level_info(const stokes_hierarchy* h, int* num_levels, int* n_finest);
stokes_status stokes_level_n(const stokes_hierarchy* h, int level, int* n_level);
/* Sweep configuration used on a level (see stokes_params.tile).  In the mixed
 * forms, 3 on a level where the interior strips fit means the strip sweep
 * (tensor-core GEMMs in the BF16 form, FP32 patch solves in the FP32 form) with
 * its 14x14 SIMT ring; the autotuner may choose a SIMT shape (0..2, 6) there
 * instead. */
stokes_status stokes_level_tile(const stokes_hierarchy* h, int level, int* tile);

/* Right-hand side of the eliminated system (Section 2.2 with the boundary data
 * moved to the right): b = [M f - L_{.,D} u_D on free velocity rows ;
 * u_D on Dirichlet rows ; -B_{.,D} u_D on pressure rows].  f_nodal and
 * u_dirichlet are [2, 2n+1, 2n+1] (nodal values; only the boundary entries of
 * u_dirichlet are read), b has length N(n).  Finest level. */
stokes_status stokes_assemble_rhs(stokes_hierarchy* h, const double* f_nodal,
                                  const double* u_dirichlet, double* b);

/* y = A x on level `level` (Section 2.2, the block matrix A). */
stokes_status stokes_apply_operator(stokes_hierarchy* h, int level, const double* x, double* y);

/* r = b - A x on level `level` (the residual step of Algorithm 1). */
stokes_status stokes_residual(stokes_hierarchy* h, int level, const double* b, const double* x,
                              double* r);

/* One additive Vanka sweep on level `level` (Algorithm 3):
 * x_out = x + sum_i V_i^T W_i A_i^-1 V_i (b - A x), W_i = omega diag(1/m_j),
 * every patch using the same residual.  x == NULL means x = 0.  x_out must not
 * alias x or b.  Runs in the hierarchy's precision for levels of the
 * preconditioner; this entry point always uses FP64. */
stokes_status stokes_vanka_sweep(stokes_hierarchy* h, int level, const double* x,
                                 const double* b, double* x_out);

/* One relaxation sweep of the V-cycle's smoother on level `level`, in the
 * arithmetic the hierarchy's V-cycle uses (Algorithm 3 for Vanka; Algorithms 2
 * and 4 for the Braess-Sarazin and Schur-Uzawa smoothers): FP64 hierarchies as
 * stokes_vanka_sweep; STOKES_MIXED_FP32 rounds x and b to FP32, sweeps in FP32
 * (on the interior strips where the level's configuration is 3) and widens
 * x_out; STOKES_MIXED_BF16 does the same with the interior patch solves as BF16
 * tensor-core GEMMs on the strips (the tile configuration of the level,
 * stokes_level_tile).  This is the sweep the
 * V-cycle applies, exposed so that it can be compared dof by dof with an FP64
 * sweep.  x == NULL means x = 0; x_out must not alias x or b.  Uses the
 * level's FP32 work vectors, so it must not overlap a V-cycle of the same
 * hierarchy (it is ordered on the creation stream like every call). */
stokes_status stokes_relaxation_sweep(stokes_hierarchy* h, int level, const double* x,
                                      const double* b, double* x_out);

/* r_coarse = P^T r_fine, from level `level` (>= 1) to level-1 (Algorithm 1,
 * restriction).  P is the FE interpolation with Dirichlet rows/columns zero. */
stokes_status stokes_restrict(stokes_hierarchy* h, int level, const double* r_fine,
                              double* r_coarse);

/* x_fine += P e_coarse, from level-1 to level `level` (>= 1) (Algorithm 1,
 * correction). */
stokes_status stokes_prolong_add(stokes_hierarchy* h, int level, const double* e_coarse,
                                 double* x_fine);

/* e = A_0^-1 r on level 0 (Algorithm 1, exact coarse solve): the solution of
 * the bordered system [[A_0, e_p], [e_p^T, 0]] with e_p = (0, M_p 1), i.e. the
 * pressure has zero mean.  FP64. */
stokes_status stokes_coarse_solve(stokes_hierarchy* h, const double* r, double* e);

/* x0 for FGMRES: x0 = b on Dirichlet velocity rows and 0 elsewhere (finest
 * level; b and x0 of length N(n), may not alias). */
stokes_status stokes_initial_guess(stokes_hierarchy* h, const double* b, double* x0);

/* z = MG(r): one V(nu1, nu2) cycle on the finest level with zero initial
 * guess (Algorithm 1; a W-cycle with params.cycle = 2), or, with
 * params.precond = 1, one application of the block-triangular preconditioner
 * (Section 3.4, Algorithm 5) -- the preconditioner FGMRES applies.  r and z
 * have length N(n); they must not alias. */
stokes_status stokes_vcycle_apply(stokes_hierarchy* h, const double* r, double* z);

/* Solve A x = b by FGMRES(restart) right-preconditioned with the V-cycle
 * (Section 6.8).  x holds x0 on entry (its Dirichlet rows should equal b's)
 * and the solution on exit.  iters (may be NULL) receives the number of
 * preconditioned iterations, relres (may be NULL) the true relative residual
 * ||b - A x|| / ||b - A x0|| recomputed in FP64 at exit.  Returns
 * STOKES_NOT_CONVERGED after maxit iterations and STOKES_ERR_NONFINITE if b
 * or a residual is not finite.  Synchronises the stream. */
stokes_status stokes_fgmres_solve(stokes_hierarchy* h, const double* b, double* x, int* iters,
                                  double* relres);

/* Adjoint solve A^T lambda = g (A is symmetric, so the same FGMRES + MG solve),
 * then grad_f = R^T lambda where R maps nodal body forces to right-hand sides
 * (b = R f + lifting): grad_f[c, J, I] = sum over free velocity rows k of
 * M_(k),(I,J) lambda_k.  A is singular with kernel (0, 1_p), so the pressure
 * block of g is first shifted to zero mean (its component along the kernel of
 * A^T removed); losses that ignore the pressure constant have such g already.
 * lambda starts from g on Dirichlet rows and 0 elsewhere.  g has length N(n),
 * lambda length N(n), grad_f length 2 (2n+1)^2 (may be NULL).  Synchronises. */
stokes_status stokes_solve_adjoint(stokes_hierarchy* h, const double* g, double* lambda,
                                   double* grad_f, int* iters, double* relres);

/* grad_f = R^T lambda (see stokes_solve_adjoint), without a solve. */
stokes_status stokes_rhs_transpose(stokes_hierarchy* h, const double* lambda, double* grad_f);

/* Solve nprob independent systems hs[k] x_k = b_k (each an FGMRES solve as
 * above on its own hierarchy).  iters / relres are arrays of nprob entries
 * (may be NULL).  Returns the first non-OK status. */
stokes_status stokes_batched_solve(stokes_hierarchy* const* hs, int nprob, const double* const* b,
                                   double* const* x, int* iters, double* relres);

/* A batch of independent problems (grid sizes may differ), e.g. many
 * right-hand sides on one grid or a set of uneven grids, solved together:
 * FGMRES (Section 6.8) runs in lockstep over the problems, and iteration j of
 * all of them -- each problem's V-cycle (Algorithm 1, Algorithm 3), operator,
 * Arnoldi and Givens rotation -- is one CUDA graph with one independent branch
 * per problem, captured at the first solve and replayed (re-captured only when
 * the set of unconverged problems changes).  The host synchronises once per
 * iteration to read every residual estimate.  Each problem owns a hierarchy
 * (params shared; tile shapes tuned once per grid size) on a stream of its
 * own; stokes_batch_hierarchy gives access to it (e.g. for
 * stokes_assemble_rhs).  stream: the caller's stream, synchronised when a
 * solve starts.  n: nprob grid sizes. */
typedef struct stokes_batch stokes_batch;
stokes_status stokes_batch_create(int nprob, const int* n, double viscosity, const stokes_params* params,
                                  void* stream, stokes_batch** out);
stokes_status stokes_batch_destroy(stokes_batch* b);
stokes_status stokes_batch_hierarchy(stokes_batch* b, int k, stokes_hierarchy** out);
/* Solve problem k for rhs[k] into x[k] (x[k] holds x0 on entry, as in
 * stokes_fgmres_solve).  iters / relres: nprob entries each (may be NULL).
 * Returns STOKES_NOT_CONVERGED if any problem reached maxit.  Synchronises. */
stokes_status stokes_batch_solve(stokes_batch* b, const double* const* rhs, double* const* x, int* iters,
                                 double* relres);

/* Counters for measurement (the paper reports per-kernel runtimes, Section 6.2,
 * and roofline positions, Section 6.7).  When timing is enabled the library
 * records a CUDA-event pair on its stream around every finest-level Vanka
 * sweep it launches; stokes_stats_read synchronises the stream and returns the
 * summed event durations.  kernel_launches counts the CUDA kernels this
 * library launched (all hierarchies, since load). */
typedef struct {
  long long kernel_launches;
  long long vcycles;        /* V-cycles applied by this hierarchy since the last reset */
  long long sweeps_timed;   /* finest-level sweeps timed since the last reset          */
  double sweep_ms;          /* their summed durations (CUDA events)                    */
  long long tc_launches;    /* launches of the tensor-core (tcgen05) sweep kernel among
                               kernel_launches (all hierarchies, since load)           */
} stokes_stats;

/* The FP64 FMA throughput of the current device in GFLOP/s, measured: a kernel
 * of independent FMA chains on every SM, timed with CUDA events on `stream`
 * (best of three launches, about 10 ms each; synchronises).  The FP64 form is
 * bound by the FP64 pipe, and this is the peak its roofline fraction uses (the
 * paper's roofline, Section 6.7, likewise uses measured peaks).  gflops must
 * not be NULL. */
stokes_status stokes_measure_fp64_peak(void* stream, double* gflops);

stokes_status stokes_stats_enable_timing(stokes_hierarchy* h, int enable);
stokes_status stokes_stats_reset(stokes_hierarchy* h);
stokes_status stokes_stats_read(stokes_hierarchy* h, stokes_stats* out);

/* Device-side failures of asynchronous work: synchronises the creation
 * stream and returns STOKES_ERR_TIMEOUT if a bounded device wait (the
 * tensor-core sweep's mbarrier waits) expired in work queued since the last
 * report, else STOKES_OK.  The flag is cleared when reported, so the
 * hierarchy stays usable.  stokes_fgmres_solve and the other synchronising
 * solves check the same flag at every iteration. */
stokes_status stokes_device_status(stokes_hierarchy* h);

/* Test hooks: failures made on purpose, without faulting or hanging a GPU.
 *  - stokes_test_set_wait_limit: number of polls of the tensor-core sweep's
 *    first bounded wait (the mbarrier of the bulk copy of the patch inverse).
 *    0 makes that wait expire at once: the kernel sets the hierarchy's error
 *    flag, still waits for its copy with the full limit, frees its tensor
 *    memory and returns without writing x_out; the next synchronising call
 *    returns STOKES_ERR_TIMEOUT.  A negative value restores the default.
 *  - stokes_test_set_alloc_limit: cap on the device bytes one
 *    stokes_hierarchy_create (on any thread) may allocate; beyond it the
 *    creation frees what it holds and returns STOKES_ERR_OOM.  0 removes it. */
stokes_status stokes_test_set_wait_limit(stokes_hierarchy* h, int polls);
void stokes_test_set_alloc_limit(long long bytes);
/*  - stokes_test_set_grid_barrier: polls of each grid barrier of the persistent
 *    coarse-level launch before it gives up (negative: the default, about a
 *    quarter of a second), and a CTA that withholds its arrival at the first
 *    barrier (negative: none).  The other CTAs' waits then expire: they set
 *    the hierarchy's error flag and the kernel returns; the next synchronising
 *    call reports STOKES_ERR_TIMEOUT and resets the barrier. */
stokes_status stokes_test_set_grid_barrier(stokes_hierarchy* h, int polls, int withhold_cta);

/* The persistent coarse-level launch of a hierarchy (stokes_params.tail_n):
 * its top level (-1: none; the levels 0..top run in one launch), the number of
 * steps of one cycle there (sweeps, residuals, transfers, coarse solve; each
 * ends at a grid barrier) and the CTAs of the cooperative launch. */
stokes_status stokes_tail_info(const stokes_hierarchy* h, int* top_level, int* steps, int* ctas);

/* Largest grid accepted by stokes_residual_norm_noalloc. */
#define STOKES_NOALLOC_MAX_N 8192

/* ||b - A x||_2 on an n x n grid (1 <= n <= STOKES_NOALLOC_MAX_N) without
 * allocating any memory and without a hierarchy.  The paper has no
 * counterpart: this is a service for callers that cannot allocate device
 * memory -- code whose device memory is all owned by another allocator, or a
 * check that runs while another component records the stream into a CUDA
 * graph (cudaMalloc is not allowed then).  b and x are device vectors of
 * length N(n) in the layout above; *norm (device memory, one double) receives
 * the norm when the stream reaches this work; stream is a cudaStream_t.
 * Scratch: a fixed array of 3 * STOKES_NOALLOC_MAX_N + 2 doubles (196.6 KB)
 * that every GPU using this library keeps until the process exits.  The
 * first call on a device (and the first after a cudaDeviceReset, which makes a
 * new context) looks up that array's device address (cudaGetSymbolAddress),
 * so make one call per device before any stream capture.  Calls share the array: two calls whose kernels overlap on the
 * GPU (different streams or host threads) race.  Each call overwrites every
 * slot it later reads, so nothing is carried over from the previous call.
 * Returns STOKES_ERR_ARG for n out of range or null pointers. */
stokes_status stokes_residual_norm_noalloc(int n, double viscosity, const double* b,
                                           const double* x, double* norm, void* stream);

/* Message of the last failure on this thread ("" if none). */
const char* stokes_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* STOKES_VANKA_H */
