/*
 * biotmg.h -- C ABI of the GB300 (sm_103a) monolithic-multigrid solver for the
 * reduced-quadrature three-field Biot system of Adler, He, Hu, MacLachlan and Ohm,
 * "Monolithic multigrid for a reduced-quadrature discretization of poroelasticity"
 * (arXiv 2107.04060).
 *
 * Problem (Sec. 2.1 Eqs. discrete1-3, Sec. 2.3 Eq. block_form_rq): one backward-Euler step
 * of Biot's model on the unit square, discretised with P1-plus-face-bubble displacement,
 * lowest-order Raviart-Thomas Darcy velocity and P0 pressure on the uniform triangulation
 * of App. A (n x n squares, each cut along the diagonal from top-left to bottom-right),
 * with the reduced-quadrature grad-div term lambda (P_Q div u, P_Q div v):
 *
 *        | A_u^RQ      0          alpha B_u^T |
 *    A = | 0           tau M_w    tau B_w^T   |    A_u^RQ = 2 mu A_eps + lambda B_u^T M_p^{-1} B_u
 *        | alpha B_u   tau B_w    -(1/M) M_p  |
 *
 * Displacement is zero on the whole boundary; the pressure condition is natural (RT0
 * boundary fluxes are unknowns).  The solver is right-preconditioned FGMRES (Sec. 5.1)
 * with one monolithic V-cycle (Sec. 3, Eq. TG-Operator-Biot): additive Vanka on vertex
 * patches (Sec. 3.2.1) or inexact Braess-Sarazin (Sec. 3.2.2, App. D), the block
 * interpolation P = diag(P_u, P_w, P_p) with divergence-preserving P_u (Sec. 3.1), R = P^T,
 * rediscretised coarse operators and a direct solve on the coarsest grid (Sec. 5.1).
 *
 * ---------------------------------------------------------------------------------------
 * VECTOR LAYOUT (every vector argument).  A vector on an n-cell grid is 10 blocks, in the
 * order  ux, uy, bh, bv, bd, wh, wv, wd, pL, pU :
 *   ux, uy  P1 displacement at vertex (i, j)           0 <= i, j <= n
 *   bh, wh  bubble / RT0 on the edge (i,j)-(i+1,j)      0 <= i < n, 0 <= j <= n
 *   bv, wv  bubble / RT0 on the edge (i,j)-(i,j+1)      0 <= i <= n, 0 <= j < n
 *   bd, wd  bubble / RT0 on the diagonal of cell (i,j)  0 <= i, j < n
 *   pL, pU  P0 on the lower-left / upper-right triangle of cell (i, j)
 * Each block is (n+1) rows (j) of bmg_pitch(n) elements (i); element (i, j) of block k sits
 * at  k * bmg_block_len(n) + j * bmg_pitch(n) + i.  Slots outside the ranges above and the
 * constrained displacement slots (ux, uy on boundary vertices; bh on j = 0, n; bv on
 * i = 0, n) must hold 0 on input and are written as 0 on output.  Norms are Euclidean over
 * the whole vector (hence over the free DoFs).  Bubble coefficients are the normal
 * displacement at the edge midpoint (basis 4 l_a l_b n_e, n_h = (0,1), n_v = (1,0),
 * n_d = (1,1)/sqrt 2); RT0 coefficients are the normal flux density along the same normals.
 *
 * CONVENTIONS.  All pointers to vector or field data are DEVICE pointers unless the name
 * says _host.  Vectors are caller-owned; handles own every internal buffer.  `stream` is a
 * cudaStream_t (NULL = legacy default stream); every call is stream-ordered.  Calls return
 * BMG_OK (0) or a negative BMG_ERR_* code; bmg_status_string() describes a code.  A
 * non-converged solve is not an error: it is reported in bmg_solve_info.status.  Handles
 * are not thread-safe; distinct handles may be used concurrently on distinct streams.
 * There is no CPU fallback: without a usable CUDA device every call fails with
 * BMG_ERR_CUDA.
 */
#ifndef BIOTMG_H
#define BIOTMG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------------------ */
#define BMG_OK 0
#define BMG_ERR_ARG (-1)      /* invalid argument (size, pointer, option)              */
#define BMG_ERR_CUDA (-2)     /* CUDA runtime error (see bmg_last_error)               */
#define BMG_ERR_ALLOC (-3)    /* device or host allocation failed                      */
#define BMG_ERR_SINGULAR (-4) /* a patch or coarse-grid factorisation met a zero pivot */
#define BMG_ERR_NONFINITE (-5)/* non-finite input (right-hand side or coefficients)    */
#define BMG_ERR_NOCONV (-6)   /* an inner iterative solve missed its tolerance         */

/* ---- solve status (bmg_solve_info.status) ------------------------------------------ */
#define BMG_CONVERGED 0
#define BMG_MAXIT 1           /* iteration limit reached before the tolerance          */
#define BMG_BREAKDOWN 2       /* Arnoldi breakdown (h_{j+1,j} = 0) without convergence */
#define BMG_DIVERGED 3        /* non-finite residual                                   */

/* ---- options ----------------------------------------------------------------------- */
#define BMG_VANKA 0           /* additive Vanka, 20-DoF vertex patches (Sec. 3.2.1)     */
#define BMG_BSR 1             /* inexact Braess-Sarazin (Sec. 3.2.2, App. D)            */
#define BMG_BSR_EXACT 2       /* exact Braess-Sarazin: Eq. bsr_p solved with the fixed-stress
                                 S (CG to 1e-11 relative, preconditioned by a multigrid
                                 V-cycle on the coarser levels' S, FP64 only,
                                 V-cycles kernel by kernel; BMG_ERR_NOCONV if CG stalls)   */
#define BMG_FP64 0
#define BMG_FP32 1
#define BMG_PATCH_CYCLE 0     /* Vanka patch solves in the V-cycle's precision             */
#define BMG_PATCH_FP64 1      /* FP32 V-cycle with FP64 patch solves (FP64 inverses)       */
#define BMG_REDISC 0          /* coarse operators by rediscretisation (Sec. 3, the paper's) */
#define BMG_GALERKIN 1        /* coarse operators P^T A P (R = P^T, Eq. block_interp)      */

typedef struct bmg_system bmg_system;       /* one assembled operator (FP64)           */
typedef struct bmg_hierarchy bmg_hierarchy; /* multigrid preconditioner for a system   */

/* Layout helpers: row pitch (elements), block length, vector length, for n cells/side. */
int bmg_pitch(int n);
size_t bmg_block_len(int n);
size_t bmg_vector_len(int n);

/* Number of free (unconstrained) DoFs of an n-cell grid: 2(n-1)^2 displacement P1 values,
 * the bubbles on the 3n^2 - 2n interior edges, RT0 on all 3n^2 + 2n edges, 2n^2 pressures. */
size_t bmg_free_dofs(int n);

/*
 * bmg_assemble -- operator coefficients (Sec. 2.1 Eq. block_form; Sec. 2.3 a^RQ; App. A).
 *   n        cells per side, 1 <= n <= 16384 (multigrid needs n = n_coarse * 2^k).
 *   lambda, mu  Lame coefficients (> 0 and >= 0 respectively, finite).
 *   K        device pointer to per-triangle permeability, FP64, two blocks (L then U) of
 *            (n+1) x bmg_pitch(n) laid out like a vector block ([j][i], i, j < n used);
 *            may be NULL, then the permeability is K_const everywhere.  mu_f = 1.
 *   K_const  uniform permeability (> 0) used when K is NULL.
 *   tau      time step (> 0);  alpha  Biot-Willis constant;  inv_M  1/M (>= 0).
 * The permeability is read once (converted to K^{-1}); the caller keeps ownership.
 * On success *out receives a new system (free with bmg_destroy_system).
 * Errors: BMG_ERR_ARG (bad sizes/parameters), BMG_ERR_NONFINITE (K <= 0 or non-finite),
 * BMG_ERR_ALLOC, BMG_ERR_CUDA.
 */
int bmg_assemble(int n, double lambda, double mu, const double *K, double K_const,
                 double tau, double alpha, double inv_M, void *stream, bmg_system **out);

/*
 * bmg_assemble_divdiv -- as bmg_assemble, choosing the grad-div term: divdiv =
 * BMG_DIVDIV_REDUCED (0) gives the reduced-quadrature lambda (P_Q div u, P_Q div v) of Sec.
 * 2.3 (what bmg_assemble builds); BMG_DIVDIV_EXACT gives lambda (div u, div v) integrated
 * exactly, the original discretisation of Eq. block_form (Sec. 2.1), whose divergence-free
 * space has no local basis and with which Vanka and inexact Braess-Sarazin relaxation lose
 * their robustness as lambda / mu grows (Sec. 2.2, Table 1): a negative control.  Every other
 * call accepts such a system, except bmg_adjoint_gradient and the batched solver
 * (BMG_ERR_ARG).
 */
#define BMG_DIVDIV_REDUCED 0
#define BMG_DIVDIV_EXACT 1
int bmg_assemble_divdiv(int n, double lambda, double mu, const double *K, double K_const,
                        double tau, double alpha, double inv_M, int divdiv, void *stream,
                        bmg_system **out);

/*
 * bmg_assemble_logk -- as bmg_assemble with the permeability given as its logarithm:
 * logK is a device pointer to FP32 theta_T = log K_T per triangle in the layout of K
 * (K^{-1} = exp(-theta) is formed on the device).  Used by the adjoint gradient below.
 */
int bmg_assemble_logk(int n, double lambda, double mu, const float *logK, double tau,
                      double alpha, double inv_M, void *stream, bmg_system **out);

/*
 * bmg_apply -- y = A x (FP64, matrix-free).  bmg_residual -- r = b - A x.
 * x, y, b, r: device vectors of bmg_vector_len(n) doubles; y/r may not alias x.
 */
int bmg_apply(const bmg_system *s, const double *x, double *y, void *stream);
int bmg_residual(const bmg_system *s, const double *b, const double *x, double *r,
                 void *stream);

typedef struct {
  int smoother;     /* BMG_VANKA, BMG_BSR or BMG_BSR_EXACT                            */
  int nu1, nu2;     /* pre-/post-relaxation sweeps (>= 0)                             */
  double omega;     /* outer relaxation weight (Sec. 3.2: E_s = I - omega M^{-1} A)    */
  double omega_J;   /* Jacobi weight on the Schur complement (BSR only, App. D)        */
  int n_coarse;     /* coarsest grid (cells per side) for the direct solve, e.g. 8     */
  int precision;    /* BMG_FP64 or BMG_FP32 arithmetic inside the V-cycle             */
  double p_shift;   /* >= 0: -p_shift * |T| is added to every P0 diagonal entry of the
                       Vanka patch matrices (the regularisation of Sec. 5.3 for 1/M = 0;
                       0 = exact patch solves)                                          */
  int gamma;        /* coarse-grid cycles per level: 0 or 1 = V-cycle (Sec. 3), 2 = W-cycle
                       (the remedy the discussion of Table 4 suggests for multilevel inexact
                       BSR): the coarse problem is approximated by two cycles, the second on
                       the residual the first leaves; the coarsest solve is direct either way */
  int coarse_op;    /* BMG_REDISC (0) or BMG_GALERKIN: P^T A P on every coarse level.  P_u is
                       local to each coarse triangle, so P^T A P is an element assembly: the
                       coarse elasticity element matrices become dense 9 x 9 products, the
                       grad-div block is exactly 4 x its rediscretisation per level (the whole
                       divergence of a coarse triangle lands in its interior child), and the
                       RT0 and P0 blocks equal their rediscretisation (nested spaces)        */
  int patch_solve;  /* BMG_PATCH_CYCLE (0) or BMG_PATCH_FP64: with precision BMG_FP32 and the
                       Vanka smoother, the patch solves use the FP64 inverses and FP64 products
                       (vectors, residuals and transfers stay FP32); ignored otherwise        */
} bmg_mg_opts;

/*
 * bmg_setup_hierarchy -- multigrid hierarchy for system s (Sec. 3): levels n, n/2, ...,
 * n_coarse with rediscretised (or, with coarse_op = BMG_GALERKIN, Galerkin) operators (the
 * coarse RT0 mass is P_w^T M_w P_w, which is the rediscretisation with the fine-scale
 * K^{-1}); FP64 factorisation of every distinct
 * Vanka patch matrix (Gauss-Jordan with partial pivoting); FP64 inverse of the coarsest
 * operator.  The hierarchy keeps a pointer to s: s must outlive it.
 * Errors: BMG_ERR_ARG (n not n_coarse * 2^k, bad options), BMG_ERR_SINGULAR, BMG_ERR_ALLOC,
 * BMG_ERR_CUDA.
 */
int bmg_setup_hierarchy(const bmg_system *s, const bmg_mg_opts *o, void *stream,
                        bmg_hierarchy **out);

/*
 * bmg_vcycle -- z = M^{-1} r: one V(nu1, nu2) cycle (W-cycle if gamma = 2) from a zero
 * initial guess (Sec. 3).
 * r, z: device vectors (bmg_vector_len(n) doubles, FP64 whatever the V-cycle precision;
 * an FP32 hierarchy converts on entry and exit).  z may not alias r.
 */
int bmg_vcycle(bmg_hierarchy *h, const double *r, double *z, void *stream);

#define BMG_ARNOLDI_FP64 0   /* both Gram-Schmidt passes and updates in FP64 (default)    */
#define BMG_ARNOLDI_MIXED 1  /* first pass from an FP32 copy of the basis, second pass and
                                last correction in double-float arithmetic (see below)  */

typedef struct {
  double rtol;      /* stop when ||b - A x|| <= rtol ||b|| (true residual), e.g. 1e-8  */
  int restart;      /* FGMRES restart length m (1..200)                                */
  int maxit;        /* total iteration limit                                           */
  int x0_is_zero;   /* 1: ignore the contents of x on entry; 0: use x as initial guess */
  int arnoldi;      /* BMG_ARNOLDI_FP64 (0) or BMG_ARNOLDI_MIXED                        */
} bmg_krylov_opts;

typedef struct {
  int iters;        /* FGMRES iterations (preconditioner applications)                 */
  int restarts;     /* restart cycles started                                          */
  int status;       /* BMG_CONVERGED, BMG_MAXIT, BMG_BREAKDOWN or BMG_DIVERGED         */
  double relres;    /* final true relative residual ||b - A x|| / ||b||                */
  double relres_est;/* final Arnoldi estimate |g_{j+1}| / ||b||                        */
  double solve_ms;  /* wall time of the call (host clock, includes the final sync)     */
} bmg_solve_info;

/*
 * bmg_fgmres_solve -- x ~= A^{-1} b by right-preconditioned flexible GMRES(m) with one
 * V-cycle of h as the preconditioner (Sec. 5.1).  Arnoldi by classical Gram-Schmidt with
 * one re-orthogonalisation pass (CGS2): h1 = V^T w, w -= V h1, h2 = V^T w, w -= V h2, and the
 * Hessenberg column is h1 + h2.  With o->arnoldi = BMG_ARNOLDI_FP64 every product and update
 * is FP64.  With BMG_ARNOLDI_MIXED the first pass's coefficients come from an FP32 copy of the
 * basis, the update w -= V h1 is FP64, and the second pass's coefficients h2 and the last
 * correction w -= V h2 are formed in double-float arithmetic (pairs of FP32 values, about
 * 2^-46 relative) from the FP64 basis, which describes the subtracted combination to FP64
 * rounding; it moves most Gram-Schmidt work from the FP64 pipe to the FP32 pipe.  b, x:
 * device vectors.  The call returns after the solve has finished (it synchronises `stream`
 * once per iteration to read the Hessenberg column).  info may be NULL.
 */
int bmg_fgmres_solve(bmg_hierarchy *h, const double *b, double *x,
                     const bmg_krylov_opts *o, bmg_solve_info *info, void *stream);

/* Same with HOST vectors: copies b in, solves, copies x out (all on `stream`). */
int bmg_fgmres_solve_host(bmg_hierarchy *h, const double *b_host, double *x_host,
                          const bmg_krylov_opts *o, bmg_solve_info *info, void *stream);

/*
 * bmg_adjoint_gradient -- parameter gradients of a loss L on the solution of A x = b, given
 * x and the adjoint solution xi of A xi = dL/dx (A is symmetric, so xi comes from the same
 * bmg_fgmres_solve with right-hand side dL/dx).  dL/dq = -xi^T (dA/dq) x with the element
 * matrices of Sec. 2.3:
 *   dtheta[T] = dL/dtheta_T = K_T^{-1} xi_w,T^T (tau M_T) w_T   (theta_T = log K_T, M_T the
 *               unit-permeability RT0 mass), written per triangle in the layout of K (FP64,
 *               unused slots 0);
 *   dlame[0]  = dL/dlambda = -sum_T (g_T . xi_u,T)(g_T . u_T) / |T|;
 *   dlame[1]  = dL/dmu     = -sum_T xi_u,T^T 2 A_eps,T u_T.
 * All pointers are device pointers; the Lame sums are reduced in a fixed order.  The paper
 * has no adjoint; this entry point serves the differentiable solve of the Python binding.
 */
int bmg_adjoint_gradient(const bmg_system *s, const double *x, const double *xi,
                         double *dtheta, double *dlame, void *stream);

/*
 * bmg_backward_euler_rhs -- right-hand side of one backward-Euler step of Sec. 2.1 (Eqs.
 * discrete1-3, discrete3 scaled by -1): b = load + [0; 0; alpha B_u u_prev - (1/M) M_p p_prev],
 * i.e. the pressure rows of A applied to (u_prev, 0, p_prev) added to the step's loads, the
 * displacement and flux rows being the loads alone.  x_prev is the previous step's solution
 * (its flux blocks are not read; for the first step a vector holding the initial u and p);
 * load holds the step's loads in the vector layout, with the pressure rows already carrying
 * -tau (f, q); b receives the right-hand side (constrained and unused slots zero).  All
 * device vectors of bmg_vector_len(n) doubles; b may not alias x_prev or load.  A time loop
 * alternates this call with bmg_fgmres_solve (x_prev as the initial guess).
 */
int bmg_backward_euler_rhs(const bmg_system *s, const double *x_prev, const double *load,
                           double *b, void *stream);

/*
 * Kernel timing (tracing).  bmg_profile_start(kernel, n) makes every later launch of the
 * named kernel family on an n-cell grid (n = 0: any grid) bracket itself with a pair of CUDA
 * events on its own stream; bmg_profile_stop() synchronises those events and returns the
 * summed device time (ms), the number of launches and the number of grid cells the launches
 * processed (n*n per launch, times the batch).  Only one kernel family is timed at a time.
 * Timing adds two event records per timed launch and nothing else.
 */
#define BMG_PROF_APPLY 1      /* matrix-free operator application / residual           */
#define BMG_PROF_VANKA 2      /* additive Vanka sweep (20-DoF patches)                  */
#define BMG_PROF_VANKA_U 3    /* displacement Vanka + Jacobi step inside BSR            */
#define BMG_PROF_RESTRICT 4
#define BMG_PROF_PROLONG 5
#define BMG_PROF_COARSE 6     /* coarsest-grid solve                                   */
#define BMG_PROF_KRYLOV 7     /* FGMRES vector kernels (dots, updates, scaling)         */
#define BMG_PROF_SCHUR 8      /* exact BSR: the Schur-complement CG of one pressure step */
int bmg_profile_start(int kernel, int n);
/* Number of kernels this library has launched in the process so far (host-side count; a
 * replayed V-cycle graph counts its kernel nodes). */
long long bmg_launch_count(void);

/*
 * bmg_use_graphs -- V-cycles as CUDA graphs, process-wide (default on; the environment
 * variable BMG_NO_GRAPHS=1 starts with it off).  When on, the second and later V-cycles of a
 * hierarchy on a non-default stream are captured once per (input, output) vector pair and
 * replayed with one graph launch instead of a launch per kernel (the levels below about 128^2
 * cost more to launch than to run).  Results are identical either way.  Kernel timing
 * (bmg_profile_start) brackets only launches made kernel by kernel, so a caller that wants
 * the V-cycle's kernels timed turns graphs off.  Returns the previous setting.
 */
int bmg_use_graphs(int enable);
int bmg_profile_stop(double *total_ms, long long *launches, double *cells);

/*
 * bmg_fgmres_solve_noalloc -- the FGMRES solve of bmg_fgmres_solve with the FP64 Arnoldi
 * (same V-cycle, same CGS2 in FP64, o->arnoldi is ignored; the Gram-Schmidt passes run as
 * separate product and update kernels, so the rounding differs from bmg_fgmres_solve's fused
 * kernels: iteration counts agree within one for lambda/mu <= 1e4 and can differ by a
 * restart cycle's last few iterations at lambda/mu = 1e6, where the true residual near 1e-8
 * depends on rounding; both meet the tolerance)
 * for callers that cannot allocate device memory while they run: code that
 * works inside a fixed memory budget or a framework that owns every device allocation, or
 * that calls in from a context where cudaMalloc is not allowed.  bmg_fgmres_solve allocates
 * its Krylov workspace with cudaMalloc on its first call (and again when `restart` grows);
 * this variant allocates nothing.  The paper has no counterpart of this entry point.
 *   Workspace: one fixed array of bmg_noalloc_capacity() doubles (8 MiB) reserved on every
 *   device that loads the library and held until the process exits.  A call needs
 *   (2 * restart + 3) * bmg_vector_len(n) + 612 * (restart + 2) doubles of it and
 *   1 <= restart <= 64; a larger request fails with BMG_ERR_ARG and a message naming the
 *   limit (e.g. n = 32 allows restart <= 38, n = 64 allows restart <= 9).
 *   The first call on a device looks up the array's device address (once per device, with
 *   that device current); make that first call before any stream capture.
 *   Every call uses the same array, which keeps the last call's contents; the solve writes
 *   every part of it before reading it.  Calls that overlap on the GPU (different streams or
 *   threads at the same time) race on the array: serialise them.
 *   h, b, x, o, info, stream: as for bmg_fgmres_solve (h is set up beforehand by
 *   bmg_setup_hierarchy, which does allocate).  A bulk-copy wait of the FP32 operator that
 *   timed out during the solve is reported as BMG_ERR_CUDA, as by bmg_fgmres_solve.
 */
int bmg_fgmres_solve_noalloc(bmg_hierarchy *h, const double *b, double *x,
                             const bmg_krylov_opts *o, bmg_solve_info *info, void *stream);
size_t bmg_noalloc_capacity(void);

/*
 * Batched solves -- many independent systems A_i x_i = b_i, each with its own grid size,
 * coefficients and hierarchy, solved together by the FGMRES(m) + V-cycle iteration of Sec.
 * 5.1 (the iteration of bmg_fgmres_solve, run for every instance).  The paper solves one
 * system at a time; batching is this library's arrangement for many small problems.
 *
 * bmg_batch_create(hs, count, o, autotune, stream, out)
 *   hs[count]: distinct hierarchies from bmg_setup_hierarchy, all with smoother BMG_VANKA,
 *     precision BMG_FP64, V-cycles (gamma 0 or 1), rediscretised coarse operators, nu1 >= 1
 *     and the same nu1, nu2 and n_coarse (omega may differ).
 *     The batch borrows their level data and work vectors: keep them alive, and do not use
 *     them in other solves while a batch solve runs.  1 <= count <= 4096.
 *   o: rtol, restart, maxit, x0_is_zero and arnoldi for every instance (as for
 *     bmg_fgmres_solve).
 *   autotune != 0: time every candidate tile of the batched operator and Vanka kernels on
 *     this batch (per level size) and keep the fastest; 0: the single-instance rule.
 *   Allocates the Krylov workspace of every instance ((2m + 5) FP64 vectors of its size, and
 *   with BMG_ARNOLDI_MIXED an FP32 copy of its m + 1 basis vectors) and
 *   records the solve as one CUDA graph: a prologue (copy-in, ||b||), a device-side while
 *   loop whose body closes cycles and takes one Arnoldi step for every open instance, and
 *   an epilogue (copy-out).  Returns BMG_ERR_ARG on an invalid batch (message names why).
 * bmg_batch_solve(bt, b, x, infos, stream)
 *   b[count], x[count]: device vectors (bmg_vector_len(n_i) doubles) of the instances, x not
 *   aliasing b; x is the initial guess unless x0_is_zero.  One graph launch on `stream`,
 *   then a wait for it.  infos[count] (nullable): per-instance results as for
 *   bmg_fgmres_solve, solve_ms being the batch's wall time.  An instance whose b is not
 *   finite is left at status BMG_DIVERGED and the call returns BMG_ERR_NONFINITE after the
 *   others have been solved.
 * bmg_batch_tile(bt, kernel, n): tile chosen for BMG_PROF_APPLY or BMG_PROF_VANKA at level
 *   size n (index into the kernels' candidate list), -1 if none.
 * bmg_batch_trips(bt): while-loop trips of the last solve (Arnoldi steps of the slowest
 *   instance + 1).  bmg_batch_kernels_per_trip(bt): kernels in one trip.
 */
typedef struct bmg_batch bmg_batch;
int bmg_batch_create(bmg_hierarchy *const *hs, int count, const bmg_krylov_opts *o, int autotune,
                     void *stream, bmg_batch **out);
int bmg_batch_solve(bmg_batch *bt, const double *const *b, double *const *x,
                    bmg_solve_info *infos, void *stream);
int bmg_batch_tile(const bmg_batch *bt, int kernel, int n);
int bmg_batch_trips(const bmg_batch *bt);
long long bmg_batch_kernels_per_trip(const bmg_batch *bt);
void bmg_batch_destroy(bmg_batch *bt);

/* Grid size of a system / hierarchy (cells per side). */
int bmg_system_n(const bmg_system *s);
int bmg_hierarchy_levels(const bmg_hierarchy *h);

/*
 * bmg_hierarchy_tile -- tile chosen at setup (by timing the candidates on this device) for
 * the operator (BMG_PROF_APPLY), Vanka (BMG_PROF_VANKA) or displacement-Vanka
 * (BMG_PROF_VANKA_U) launches of level `level` (0 = finest): 0 = 32 x 8, 1 = 16 x 8,
 * 2 = 8 x 8, 3 = 8 x 4, 4 = 4 x 4 output positions (Vanka: patches),
 * 5 = FP32 operator, 32 x 8 with its input staged in shared memory by TMA bulk tensor
 * copies (FP64: the 32 x 8 tile), 6 = 32 x 8 and 7 = 16 x 8 operator tiles with registers
 * capped for 4 and 8 CTAs per SM, 8 = 32 x 8 and 9 = 16 x 8 FP64 operator tiles that load
 * the residual's b before the element products (the FP32 operator does so in every tile);
 * Vanka and displacement Vanka 5 = 32 x 8, 6 = 16 x 8,
 * 7 = 8 x 8 patches solved one patch per thread
 * (each packed inverse entry loaded once) instead of (row, patch) tasks.  -1: not tuned or
 * no such level.  The choice does not change any result.  Setting
 * the environment variable BMG_FORCE_APPLY_TILE to one of these indices before
 * bmg_setup_hierarchy fixes the operator's choice on every level; BMG_FORCE_SMOOTHER_TILE
 * (0-7) fixes the Vanka tile (Vanka hierarchies) or the displacement-Vanka tile (BSR) the
 * same way.  Out-of-range values select the built-in rule.  Both exist to test every
 * candidate.
 */
int bmg_hierarchy_tile(const bmg_hierarchy *h, int level, int kernel);

/*
 * bmg_hierarchy_schur_iters -- exact BSR (smoother BMG_BSR_EXACT): the most conjugate-gradient
 * iterations one pressure step (Eq. bsr_p) has taken on this hierarchy since setup; 0 before
 * the first V-cycle, -1 for other smoothers or h = NULL.
 */
int bmg_hierarchy_schur_iters(const bmg_hierarchy *h);

void bmg_destroy_system(bmg_system *s);
void bmg_destroy_hierarchy(bmg_hierarchy *h);

/* Text for a return code; bmg_last_error: detail of the last failure on this thread. */
const char *bmg_status_string(int code);
const char *bmg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* BIOTMG_H */
