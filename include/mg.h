/*
 * mg.h - C ABI of libmg.so, a B300 (sm_103a) learnable geometric multigrid.
 *
 * The library runs the learnable V-cycle of "A Learnable Multigrid Framework
 * via Graph Convolutions" (Algorithm 2): damped-Jacobi smoothing whose update
 * passes through a mean-aggregation SAGEConv (Sec. 3, Sec. 3.2), restriction
 * r_c = P^T Phi_R(r) and prolongation e = Phi_P(P e_c) (Sec. 3), Galerkin
 * coarse operators A_{l+1} = P^T A_l P (Sec. 2.2) and an exact Cholesky solve
 * on the coarsest level.  It is used as a solver, as an FP32 preconditioner
 * inside FP64 iterative refinement, and differentiated for training
 * (Algorithm 3).
 *
 * Conventions for every entry point
 *  - Level 0 is the finest level (the paper's l = 1); level J-1 the coarsest.
 *  - Vectors are node features X[n][nrhs]: row-major, right-hand-side index
 *    fastest, contiguous, on the device unless the name says host.
 *  - Host arrays passed in are copied; the caller keeps ownership.  A context
 *    owns every device buffer it allocates.  Caller-provided device buffers
 *    stay owned by the caller and must not alias one another unless stated.
 *  - Work is ordered on the CUDA stream passed in (NULL = the legacy default
 *    stream).  Only calls that return host results synchronise that stream.
 *  - Every call returns mg_status.  On failure mg_last_error() gives a
 *    message (per context, or global for calls without a context).
 *  - A context is not thread-safe: use one context per host thread.
 */
#ifndef MG_H
#define MG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MG_OK = 0,
  MG_NOT_CONVERGED = 1,       /* mg_solve hit max_iter before tol            */
  MG_ERR_INVALID = -1,        /* bad argument, size or layout                */
  MG_ERR_OOM = -2,            /* device or host allocation failed            */
  MG_ERR_NOT_SPD = -3,        /* Cholesky of the coarsest operator failed    */
  MG_ERR_CUDA = -4,           /* a CUDA runtime call failed                  */
  MG_ERR_TIMEOUT = -5,        /* a bounded device-side wait gave up          */
  MG_ERR_DIVERGED = -6,       /* non-finite residual in mg_solve             */
  MG_ERR_NOT_IMPLEMENTED = -7,
  MG_ERR_STATE = -8           /* call order violated (e.g. backward first)   */
} mg_status;

typedef struct mg_ctx mg_ctx;

/* Host CSR matrix, FP64 values, 32-bit indices (nnz < 2^31). */
typedef struct {
  int32_t n_rows;
  int32_t n_cols;
  int32_t nnz;
  const int32_t* rowptr;  /* [n_rows + 1] */
  const int32_t* col;     /* [nnz]        */
  const double* val;      /* [nnz]        */
} mg_csr;

/* CSR matrix whose arrays were allocated by the library (malloc); release
 * with mg_csr_owned_free(). */
typedef struct {
  int32_t n_rows;
  int32_t n_cols;
  int32_t nnz;
  int32_t* rowptr;
  int32_t* col;
  double* val;
} mg_csr_owned;

/* Transfer and graph data of a hierarchy with J levels (host). */
typedef struct {
  int32_t n_levels;                /* J >= 2                                       */
  const mg_csr* P;                 /* [J-1]; P[l] is n_l x n_{l+1}, <= 2 entries   */
                                   /* per row (natural inclusion, Sec. 2.2)        */
  const double* const* inv_deg;    /* [J]; inv_deg[l][i] = 1/|N(i)| on level l,    */
                                   /* the mean of the SAGEConv (Sec. 3.2)          */
} mg_hierarchy;

/* Learnable parameters Theta (Sec. 3): per level l = 0..J-2 the scalings
 * theta_l, eta_l and the scalar SAGEConv weights (w1, w2) of Phi_B, Phi_R,
 * Phi_P.  The identity initialisation of Sec. 3.4 is theta = omega, eta = 1,
 * w = (1, 0), which is the classical damped-Jacobi V-cycle. */
typedef struct {
  int32_t n_levels;      /* J, must match the hierarchy          */
  int32_t nu_pre;        /* pre-smoothing steps per level, >= 0  */
  int32_t nu_post;       /* post-smoothing steps per level, >= 0 */
  const double* theta;   /* [J-1]                                */
  const double* eta;     /* [J-1]                                */
  const double* wB;      /* [J-1][2] (w1, w2) of Phi_B           */
  const double* wR;      /* [J-1][2] of Phi_R                    */
  const double* wP;      /* [J-1][2] of Phi_P                    */
} mg_params;

/* ---------------------------------------------------------------------
 * Host set-up helpers (native, FP64).  They turn a nested mesh hierarchy
 * into the operators mg_setup takes; they do not touch the GPU.
 * ------------------------------------------------------------------- */

/* Galerkin coarsening A_c = P^T A P (Sec. 2.2, Eq. for A_{l+1}) over ALL
 * vertices of a nested P1 pair, with P the natural inclusion given by a
 * parent map: parent[2*i] = c, parent[2*i+1] = -1 when fine vertex i is
 * coarse vertex c; (a, b) when it is the midpoint of coarse edge a-b
 * (P_ia = P_ib = 1/2).  Off-diagonal results with
 * |a_IJ| <= drop_tol * max(|a_II|, |a_JJ|) are removed (round-off of the
 * product).  out is allocated by the library.  Errors: MG_ERR_INVALID for
 * out-of-range parents or non-square A, MG_ERR_OOM. */
mg_status mg_galerkin(const mg_csr* A_full, const int32_t* parent, int32_t nv_coarse,
                      double drop_tol, mg_csr_owned* out);

/* Dirichlet elimination of one level: keeps the rows and columns of the
 * vertices with boundary[i] == 0 (in vertex order; this is the DOF order),
 * dropping off-diagonal entries as in mg_galerkin.  inv_deg_out[k] (host,
 * [number of interior vertices]) receives 1/deg of interior vertex k, where
 * deg counts its neighbours in the algebraic graph {(i,j): A_ij != 0, i != j}
 * (Sec. 2.1) of the operator BEFORE elimination, so eliminated boundary
 * neighbours are counted and enter the mean as zeros. */
mg_status mg_eliminate(const mg_csr* A_full, const uint8_t* boundary, double drop_tol,
                       mg_csr_owned* A_int, double* inv_deg_out);

/* Complex-valued forms of mg_galerkin and mg_eliminate, for the complex
 * operators of two features per node (Sec. 3.2's W_1, W_2 acting on (Re u,
 * Im u); the Helmholtz experiment of Sec. 4.2): the val arrays of A_full and
 * of the result hold 2 * nnz doubles, (Re, Im) of each entry adjacent (C99
 * complex / numpy complex128 layout); the drop rule compares complex
 * moduli.  P is real, so the product sums each part exactly as the real
 * routine would. */
mg_status mg_galerkin_complex(const mg_csr* A_full, const int32_t* parent, int32_t nv_coarse,
                              double drop_tol, mg_csr_owned* out);
mg_status mg_eliminate_complex(const mg_csr* A_full, const uint8_t* boundary, double drop_tol,
                               mg_csr_owned* A_int, double* inv_deg_out);

/* Interior prolongation P (n_int_fine x n_int_coarse) from the parent map:
 * the natural inclusion (Sec. 2.2) restricted to interior vertices. */
mg_status mg_prolongation(const int32_t* parent, int32_t nv_fine, const uint8_t* boundary_fine,
                          int32_t nv_coarse, const uint8_t* boundary_coarse, mg_csr_owned* P_int);

void mg_csr_owned_free(mg_csr_owned* m);

/* ---------------------------------------------------------------------
 * Context
 * ------------------------------------------------------------------- */

/* Copies the hierarchy to the device and prepares the cycle.
 *  A_levels  [J] interior operators (SPD), A_levels[l] is n_l x n_l; its
 *            off-diagonal pattern is the convolution graph of level l.
 *  precision 64: the V-cycle runs in FP64 (plain / parity path);
 *            32: the V-cycle runs in FP32 (values, weights, accumulation)
 *            and mg_solve wraps it in FP64 iterative refinement.
 *  max_batch largest nrhs any later call will pass (sizes the workspace).
 * The coarsest operator is factorised by dense FP64 Cholesky here, on the
 * host before any device allocation (MG_ERR_NOT_SPD if that fails;
 * n_{J-1} <= 2048; a non-positive diagonal entry is MG_ERR_INVALID).  The
 * off-diagonals of each level are stored as DIA (values on at most 8
 * diagonals, no column indices) where they fit, else as SELL-32 slices
 * (mg_set_layout_policy), next to diagonal arrays.  *out is NULL on failure;
 * the message is then available from mg_last_error(NULL, ...). */
mg_status mg_setup(mg_ctx** out, const mg_hierarchy* h, const mg_csr* A_levels,
                   const mg_params* p, int32_t max_batch, int32_t precision, void* stream);

/* Matrix layout chosen by later mg_setup calls (process-wide):
 *   0 (default): per level, DIA (values on at most 8 diagonals, neighbour
 *      addresses computed, no column indices) when all off-diagonals lie on
 *      at most 8 diagonals and the CSR rows are sorted, else SELL-32;
 *   1: SELL-32 on every level.
 * Both layouts visit a row's entries in ascending column order, so results
 * do not depend on the layout. */
mg_status mg_set_layout_policy(int32_t policy);

/* Replaces Theta (same J); cheap: the device copy is updated on the next
 * call's stream.  Changing whether a w2 is zero switches kernels. */
mg_status mg_set_params(mg_ctx* ctx, const mg_params* p);

/* Highest degree mg_set_cheb accepts. */
#define MG_CHEB_MAX_DEGREE 8

/* ChebConv smoother (Sec. 3.3, remark on polynomial smoothers: a ChebConv
 * of order K in place of SAGEConv gives a degree-K polynomial smoother).
 * With K >= 1, every smoothing step of the cycle becomes
 *   delta = theta_l D_A^{-1} (f - A u),
 *   u <- u + eta_l sum_{k=0..K} c_{l,k} T_k(Lhat) delta,
 *   Lhat = D_g^{-1} L_g - I = -D_g^{-1} A_g   (T_0 = I, T_1 = Lhat,
 *   T_k = 2 Lhat T_{k-1} - T_{k-2}),
 * i.e. the random-walk normalised Laplacian of the SAGEConv mean, scaled by
 * lambda_max = 2; degree 1 is SAGEConv with w1 = c_0, w2 = -c_1.  W_B of
 * mg_params is then unused; theta, eta, Phi_R and Phi_P are kept.
 *  K     0 (back to the SAGEConv smoother; coef may be NULL) to
 *        MG_CHEB_MAX_DEGREE
 *  coef  host [J-1][K+1], level-major (level l's c_0..c_K), copied.
 * Costs K extra neighbour-mean passes per smoothing step; with K >= 1 all
 * levels run as grid kernels (the single-block small-level kernel
 * implements SAGEConv steps only).  Training (mg_forward_record) rejects a
 * context with K >= 1: the adjoint covers the SAGEConv smoother.
 * MG_ERR_INVALID for K out of range, a NULL or non-finite coef. */
mg_status mg_set_cheb(mg_ctx* ctx, int32_t K, const double* coef);

/* One learnable V-cycle (Algorithm 2) on level 0: u <- LMG(A, f, u, 1, Theta).
 * f_dev, u_dev: [n_0][nrhs] in the context precision (double for 64, float
 * for 32); u_dev is the initial guess and is overwritten; f_dev and u_dev
 * must not overlap.  1 <= nrhs <= max_batch. */
mg_status mg_vcycle(mg_ctx* ctx, const void* f_dev, void* u_dev, int32_t nrhs, void* stream);

/* One full multigrid (nested iteration) application, the preconditioner of
 * the paper's Krylov experiments (Sec. 4.2, tab:helmholtz-results-precond):
 * f is restricted to every level with
 * the cycle's restriction P^T Phi_R, the coarsest level is solved exactly,
 * and on each finer level the coarser solution, prolongated with the cycle's
 * Phi_P P, is the initial guess of one V-cycle (Algorithm 2 started on that
 * level).  u_dev receives the result (its input is not read); f_dev, u_dev:
 * [n_0][nrhs] in the context precision, not overlapping; 1 <= nrhs <=
 * max_batch.  Uses the context's level buffers (not thread-safe). */
mg_status mg_fmg(mg_ctx* ctx, const void* f_dev, void* u_dev, int32_t nrhs, void* stream);

/* Solves A u = f to ||f - A u||_2 / ||f||_2 < tol for every right-hand side.
 * f_dev, u_dev: FP64 [n_0][nrhs] on the device; u_dev holds the initial guess.
 * precision 64: u <- LMG(f, u) repeated (plain stationary multigrid);
 * precision 32: FP64 iterative refinement, r = f - A u in FP64, c = LMG_32(r,0)
 * in FP32, u += c in FP64.  A right-hand side stops changing as soon as it
 * meets tol, so its result does not depend on the others in the batch.
 * iters_out, relres_out: host arrays [nrhs] (may be NULL).  Synchronises the
 * stream.  Returns MG_NOT_CONVERGED if any right-hand side did not meet tol
 * within max_iter, MG_ERR_DIVERGED on a non-finite residual. */
mg_status mg_solve(mg_ctx* ctx, const double* f_dev, double* u_dev, int32_t nrhs, double tol,
                   int32_t max_iter, int32_t* iters_out, double* relres_out, void* stream);

/* Restarted flexible GMRES, FGMRES(restart) with right preconditioning
 * (Saad 1993), the outer Krylov method the paper uses with its V-cycle and
 * FMG preconditioners (Sec. 4.2, tab:helmholtz-results-precond).  The
 * preconditioner is one V-cycle from zero or one full multigrid
 * (MG_OPT_FCG_PRECOND).  Orthogonalisation is classical Gram-Schmidt applied
 * twice; the Hessenberg least-squares problem is FP64 with Givens rotations
 * per right-hand side.  The Arnoldi cycle runs in the context precision:
 *  - precision 64: FP64 basis, directions and K z = A z;
 *  - precision 32: an FP32 basis and FP32 directions (K z = -A z in FP32)
 *    within a restart cycle, and every restart recomputes r = f - A u and
 *    applies u += Z y in FP64 (GMRES-based iterative refinement).  A cycle
 *    also ends once its residual estimate falls below 10^-MG_OPT_FGMRES_FLOOR
 *    times its start, the accuracy an FP32 cycle resolves.
 * Arguments and results as mg_solve; u_dev is the initial guess;
 * 1 <= restart <= 64; max_iter counts Arnoldi steps (one preconditioner
 * application each, shared by the batch).  Each right-hand side stops
 * updating once its true residual meets tol at a restart.  The host reads
 * the convergence counts after every step (one synchronisation per step).
 * Workspace, allocated on first use with a given restart: restart + 1 basis
 * and restart direction vectors of [n_0][max_batch] in the context precision
 * (plus an FP32 zero vector in FP32 contexts). */
mg_status mg_solve_fgmres(mg_ctx* ctx, const double* f_dev, double* u_dev, int32_t nrhs,
                          double tol, int32_t max_iter, int32_t restart, int32_t* iters_out,
                          double* relres_out, void* stream);

/* Flexible conjugate gradients, FCG(1) of Notay (one stored direction), in
 * FP64 with the context's cycle as a variable preconditioner: z = LMG(A, r,
 * 0), or one full multigrid with MG_OPT_FCG_PRECOND = 1, in FP32 on a
 * power-of-two-scaled residual for precision-32 contexts.  Iteration:
 * u += alpha p, r -= alpha q, the test ||r||/||f|| < tol on this recurrence
 * residual, z = M(r), p = z - ((z, q)/(p, q)) p, q = A p,
 * alpha = (p, r)/(p, q).  The paper's preconditioner use (Sec. 4.2,
 * tab:helmholtz-results-precond) is FGMRES; flexible CG is its counterpart
 * for SPD operators.  Same arguments, stopping rule and batch independence
 * as mg_solve; max_iter counts iterations; the relres reported is that of
 * the true residual f - A u of the final iterate.  Synchronises the stream.
 * Workspace (four FP64 vectors [n_0][max_batch]) is allocated on first use. */
mg_status mg_solve_fcg(mg_ctx* ctx, const double* f_dev, double* u_dev, int32_t nrhs, double tol,
                       int32_t max_iter, int32_t* iters_out, double* relres_out, void* stream);

/* mg_solve with HOST f and u (pageable or pinned): copies f and the initial
 * u to the device, solves, copies u back.  Same semantics otherwise. */
mg_status mg_solve_host(mg_ctx* ctx, const double* f_host, double* u_host, int32_t nrhs,
                        double tol, int32_t max_iter, int32_t* iters_out, double* relres_out,
                        void* stream);

/* Single steps of Algorithm 2 on one level, for step-by-step checking.
 * All vectors device, context precision, [n][nrhs]; out must not alias inputs.
 *   MG_OP_SMOOTH    out = u + eta Phi_B(theta D^{-1}(f - A u))   x = f, y = u
 *   MG_OP_RESIDUAL  out = f - A u                                x = f, y = u
 *   MG_OP_RESTRICT  out = P^T Phi_R(x)  (out on level+1)         x = r
 *   MG_OP_PROLONG   out = y + Phi_P(P x) (x on level+1)          x = e_c, y = u
 *   MG_OP_COARSE    out = A^{-1} x (level must be J-1, FP64 Cholesky)
 *   MG_OP_OUTER_RESIDUAL  out = f - A u in FP64 on level 0 whatever the
 *                   context precision (the refinement residual); x = f,
 *                   y = u, out double
 *   MG_OP_REFINE_RESIDUAL the first residual step of mg_solve's FP64
 *                   refinement, as its kernels compute it: r = f - A u in
 *                   FP64 and its scaled FP32 copy, out[i][b] =
 *                   float(r[i][b] * 2^-s_b) with s_b = ilogb(||f_b||_2)
 *                   (0 when ||f_b|| is 0 or not finite), the input of the
 *                   FP32 cycle; x = f, y = u (FP64), out float, level 0
 */
typedef enum {
  MG_OP_SMOOTH = 0,
  MG_OP_RESIDUAL = 1,
  MG_OP_RESTRICT = 2,
  MG_OP_PROLONG = 3,
  MG_OP_COARSE = 4,
  MG_OP_OUTER_RESIDUAL = 5,
  MG_OP_REFINE_RESIDUAL = 6
} mg_op;

mg_status mg_level_apply(mg_ctx* ctx, int32_t level, int32_t op, const void* x, const void* y,
                         void* out, int32_t nrhs, void* stream);

/* Execution options of a context (they change launch shapes, never results
 * beyond rounding order: every option gives bitwise the same cycle).
 *   MG_OPT_TAIL_WORK  levels with rows * nrhs <= value, and all coarser ones,
 *                     run in one thread block with block barriers instead of
 *                     one grid kernel per step (default 2048; 0 disables)
 *   MG_OPT_TAIL_TEAMS k >= 1 (default 1): in that block each level runs on
 *                     the first W warps only (about k entries per thread, W
 *                     a power of two, no larger than the finer level's), whose
 *                     steps are separated by barriers among those W warps
 *                     (a named barrier, or a warp sync for one warp) instead
 *                     of all 512 threads; 0: every level on the whole block;
 *                     at most 64
 *   MG_OPT_PDL        1 (default): consecutive kernels use programmatic
 *                     dependent launch; 0: plain stream order
 *   MG_OPT_MULTI_RHS  with nrhs > 1, one thread owns a row and a tile of
 *                     right-hand sides (matrix read once per row, 16-byte
 *                     vector loads).  1 (default): the widest tile of at
 *                     most 8 dividing nrhs; 2, 4, 8 or 16 (FP32 only): at most
 *                     that many right-hand sides per thread; 0: one thread
 *                     per (row, rhs).  Other values: MG_ERR_INVALID.
 *   MG_OPT_DEVICE_LOOP 1 (default): mg_solve / mg_solve_fcg run their whole
 *                     iteration as one CUDA graph with a conditional while
 *                     node (one host synchronisation per solve); 0: the host
 *                     replays a plain graph of the same per-iteration kernels
 *                     and reads the convergence flag after each one (for
 *                     profilers that do not trace inside conditional nodes)
 *   MG_OPT_HALO_ROWS  rows per thread block of the halo-fused steps on DIA
 *                     levels (default 256; 0: unfused): each block evaluates
 *                     a step's first stage (delta, r or P e_c) on its rows
 *                     plus H = max|offset| halo rows on each side in shared
 *                     memory and applies the SAGEConv mean from there, one
 *                     kernel instead of two.  Used on a level when the tile
 *                     is at least H rows, tile plus halos fit in 48 KB for
 *                     the batch, and the first stage over all tiles fits in
 *                     one wave of the GPU; otherwise the two-kernel form.
 *                     Other values than [0, 2^30]: MG_ERR_INVALID.
 *   MG_OPT_SELL_HALO_ROWS rows per tile of the halo-fused steps on SELL
 *                     levels (default 0: unfused; else a multiple of 32 up
 *                     to 8192, else MG_ERR_INVALID).  At set-up (and when
 *                     this value changes) the host lists, per tile of
 *                     consecutive rows, the outside rows that neighbour it
 *                     and the local slot of every column; a block then
 *                     evaluates a step's first stage (delta, r or P e_c) on
 *                     its rows and that halo in shared memory and applies
 *                     the SAGEConv mean from there: one kernel per step, and
 *                     the first stage never written to device memory.  Used
 *                     on a level while (rows + halo) * nrhs values fit
 *                     160 KB.  Changing it synchronises the device.
 *   MG_OPT_SELL_HALO_THREADS threads per block of those steps (default 256;
 *                     a multiple of 32 up to 1024, else MG_ERR_INVALID)
 *   MG_OPT_SELL_HALO_MAX_BYTES the smoothing and restriction steps of a SELL
 *                     level use the halo form only while rows * nrhs * value
 *                     bytes is at most this (the prolongation: always); >= 0
 *   MG_OPT_FCG_PRECOND preconditioner of mg_solve_fcg and mg_solve_fgmres:
 *                     0 (default) one V-cycle from zero, 1 one full
 *                     multigrid (mg_fmg).
 *   MG_OPT_FGMRES_FLOOR FP32 contexts: an Arnoldi cycle of mg_solve_fgmres
 *                     ends (and an FP64 restart follows) once its residual
 *                     estimate is below 10^-value times the cycle's initial
 *                     residual; default 4, 0: no floor, at most 15.  FP64
 *                     contexts ignore it.  An FP32 cycle resolves about
 *                     1e-4..1e-7 of its start (CGS2 and K z in FP32);
 *                     a lower floor spends steps below that.
 *   MG_OPT_COARSE_INVERSE coarsest-level solve: 1 (default) a dense product
 *                     with the explicit FP64 inverse of A_J, one FP64 dot
 *                     per (row, rhs) spread over SMs, where set-up formed it
 *                     (32 <= n_{J-1} <= 512 and ||A_J||_1 ||A_J^{-1}||_1
 *                     <= 1e6; otherwise, and with 0, the two Cholesky
 *                     substitutions, whose 2 n_{J-1} dependent FP64 steps
 *                     run on one SM per right-hand side).  Both forms agree
 *                     to a few units of rounding times the condition number.
 *   MG_OPT_HALO2D_BYTES DIA levels (square meshes) whose vectors (rows *
 *                     nrhs * value bytes) are at least this large, and that
 *                     the one-wave rule of MG_OPT_HALO_ROWS leaves unfused,
 *                     run each smoothing step (and the restriction's residual
 *                     with Phi_R, and P e_c with Phi_P) as one kernel over 2D
 *                     tiles of 32 x 8 grid points plus a one-point ring,
 *                     where the tile fits 48 KB of shared memory for nrhs
 *                     right-hand sides.  0 (default): never.  Bitwise
 *                     neutral; measured slower than the two-kernel form on
 *                     the 8.4M-row stacked 1025^2 level (167 against 96 us
 *                     per smoothing step with one rhs), so it is off.
 *   MG_OPT_DIA_TWO_ROWS one right-hand side: 1 (default) the residual and
 *                     the mean-only steps (SAGEConv update, Phi_R, Phi_P with
 *                     the update) on DIA levels, and P e_c on every level,
 *                     take two consecutive rows per thread, sharing the
 *                     address arithmetic; 0: one row per thread.  Bitwise
 *                     neutral.
 *   MG_OPT_FCG_FP32   precision-32 contexts: mg_solve_fcg's vectors.  1:
 *                     FP32 vectors in phases of FCG(1) on the scaled
 *                     correction equation, each phase ended by an FP64
 *                     restart (u += 2^s e, the true residual f - A u in FP64,
 *                     the test, a fresh direction); 0: FP64 vectors
 *                     throughout, the FP32 cycle on the scaled residual; 2
 *                     (default): FP32 vectors when level 0 has at least 2^20
 *                     rows (there the FP64 vector work, bound by the FP64
 *                     pipe, dominates a step; measured 2.5x on the 3.1M-row
 *                     L-shape), else FP64 vectors (fewer steps: 17 against
 *                     23 on the 513^2 checkerboard).  The choice depends on
 *                     the operator, not the batch.  FP64 contexts ignore it.
 *   MG_OPT_FCG_FLOOR  the phase of a right-hand side ends once its
 *                     recurrence residual is below 10^-value times the
 *                     phase's first (default 2; 0: no floor; at most 15), or
 *                     once its scaled estimate is below tol ||f||, or at the
 *                     last iteration.  A phase solves the system of the FP32
 *                     operator, which differs from A by FP32 rounding: on
 *                     ill-conditioned operators its true residual stops
 *                     following the recurrence after a few digits, so deep
 *                     floors waste steps (measured: 10^-2 best on the 3.1M-row
 *                     anisotropic L-shape, 10^-1 .. 10^-3 within 10 % on the
 *                     513^2 checkerboard).
 * MG_OPT_FCG_PRECOND, MG_OPT_FGMRES_FLOOR, MG_OPT_COARSE_INVERSE,
 * MG_OPT_FCG_FP32 and MG_OPT_FCG_FLOOR change results (another
 * preconditioner, other restart points, other rounding of the coarsest
 * solve, other vector precision); the others only launch shapes. */
typedef enum {
  MG_OPT_TAIL_WORK = 0,
  MG_OPT_PDL = 1,
  MG_OPT_MULTI_RHS = 2,
  MG_OPT_DEVICE_LOOP = 3,
  MG_OPT_HALO_ROWS = 4,
  MG_OPT_FCG_PRECOND = 5,
  MG_OPT_FGMRES_FLOOR = 6,
  MG_OPT_SELL_HALO_ROWS = 7,
  MG_OPT_SELL_HALO_THREADS = 8,
  MG_OPT_SELL_HALO_MAX_BYTES = 9,
  MG_OPT_COARSE_INVERSE = 10,
  MG_OPT_TAIL_TEAMS = 11,
  MG_OPT_FCG_FP32 = 12,
  MG_OPT_FCG_FLOOR = 13,
  MG_OPT_HALO2D_BYTES = 14,
  MG_OPT_DIA_TWO_ROWS = 15
} mg_option;

mg_status mg_set_option(mg_ctx* ctx, int32_t option, int64_t value);

/* Kernel kinds reported by mg_vcycle_profile. */
typedef enum {
  MG_K_JACOBI = 0,          /* smoothing step with Phi_B = w1 I, one pass      */
  MG_K_RESIDUAL_SCALED = 1, /* delta = theta D^{-1} (f - A u)                  */
  MG_K_CONV_UPDATE = 2,     /* u += eta Phi_B(delta), mean over N(i)           */
  MG_K_RESIDUAL = 3,        /* r = f - A u before restriction                  */
  MG_K_RESTRICT = 4,        /* r_c = P^T Phi_R(r)                              */
  MG_K_PROLONG = 5,         /* u += Phi_P(P e_c)                               */
  MG_K_COARSE_CHOL = 6,     /* e_J = A_J^{-1} r_J                              */
  MG_K_OUTER_RESIDUAL = 7,  /* FP64 refinement residual                        */
  MG_K_TAIL = 8,            /* all small levels of a cycle in one thread block */
  MG_K_CONV_R = 9,          /* Phi_R(r) per fine row (then MG_K_RESTRICT gathers) */
  MG_K_PE = 10,             /* P e_c per fine row (then MG_K_PROLONG applies Phi_P) */
  MG_K_SMOOTH_HALO = 11,    /* smoothing step, both stages in one halo-tiled kernel */
  MG_K_RESTRICT_HALO = 12,  /* r and Phi_R(r) in one halo-tiled kernel            */
  MG_K_PROLONG_HALO = 13,   /* u += Phi_P(P e_c) in one halo-tiled kernel         */
  MG_K_CHEB_STEP = 14       /* one Chebyshev pass: T_k and u += eta c_k T_k       */
} mg_kernel_kind;

typedef struct {
  int32_t kernel;  /* mg_kernel_kind */
  int32_t level;
  float ms;        /* device time between CUDA events around the launch */
} mg_kernel_time;

/* One V-cycle exactly like mg_vcycle (same kernels, same result), but every
 * kernel is launched directly with a CUDA event pair around it on `stream`
 * instead of replaying a graph.  Writes up to max_out records (launch order)
 * to out and their count to *n_out.  Synchronises the stream. */
mg_status mg_vcycle_profile(mg_ctx* ctx, const void* f_dev, void* u_dev, int32_t nrhs,
                            mg_kernel_time* out, int32_t max_out, int32_t* n_out, void* stream);

/* Debug builds.  A library compiled with -DMG_BOUNDS_CHECK (python -m
 * paper_2608_29082_b300.build --debug: libmg_debug.so) checks every gathered
 * index that comes from a table (SELL columns, prolongation parents,
 * restriction children, fused-step halo rows and local columns) against its
 * range, skips an out-of-range access and records the first one; mg_vcycle,
 * mg_fmg and the solves then synchronise and return MG_ERR_INVALID with the
 * check site and index in the message.  mg_debug_bounds returns 1 in such a
 * build and writes (and clears) the raw record to *word (0: none; else
 * ((site << 32) | index) + 1), 0 in a release build (*word = 0), -1 on a CUDA
 * error.  word may be NULL. */
int32_t mg_debug_bounds(uint64_t* word);

/* Static name of a kernel kind ("unknown" if out of range). */
const char* mg_kernel_name(int32_t kind);

/* ---------------------------------------------------------------------
 * Training (Algorithm 3): K unrolled cycles, their hand-written adjoint and
 * the residual loss, all in the context precision.
 * ------------------------------------------------------------------- */

/* Runs K cycles u <- LMG(A, f, u) (Algorithm 2) in place and records, per
 * cycle, the level-0 input iterate and every coarse level's right-hand side
 * and output (per-level checkpoints; f is copied).  The checkpoints stay
 * valid until the next mg_forward_record or mg_set_params.  f, u: device
 * [n_0][nrhs] in the context precision; 1 <= K <= 1000. */
mg_status mg_forward_record(mg_ctx* ctx, const void* f_dev, void* u_dev, int32_t nrhs,
                            int32_t n_cycles, void* stream);

/* Reverse mode through the recorded cycles: given grad_u_out = dL/du_K,
 * writes grad_u_in = dL/du_0 (may be NULL), grad_f = dL/df summed over the
 * cycles (may be NULL) and grad_params = dL/dTheta, a DEVICE FP64 array
 * [J-1][8] in the order theta, eta, wB1, wB2, wR1, wR2, wP1, wP2 (per level,
 * not summed over shared parameters).  Each level's smoothing iterates are
 * recomputed from its checkpoint; reductions are deterministic.  n_cycles
 * must equal the recorded K; MG_ERR_STATE if nothing was recorded or the
 * parameters changed since. */
mg_status mg_vcycle_backward(mg_ctx* ctx, int32_t n_cycles, const void* grad_u_out_dev,
                             void* grad_u_in_dev, void* grad_f_dev, double* grad_params_dev,
                             void* stream);

/* Residual loss on level 0: s_b = ||f_b - A u_b||^2 per right-hand side.
 * per_rhs_dev [nrhs] (device FP64, may be NULL) receives s_b;
 * loss_dev (device FP64 scalar, may be NULL) receives sum_b w_b s_b and
 * grad_u_dev (context precision [n_0][nrhs], may be NULL) receives its
 * gradient -2 w_b A (f_b - A u_b); both need weights_dev [nrhs] (device).
 * With weights 1/(nrhs ||r_0,b||^2) this is the training loss
 * mean_b ||r_K||^2 / ||r_0||^2. */
mg_status mg_residual_loss(mg_ctx* ctx, const void* f_dev, const void* u_dev, int32_t nrhs,
                           const double* weights_dev, double* loss_dev, double* per_rhs_dev,
                           void* grad_u_dev, void* stream);

/* Sizes: n_rows_out[l] for l < J (host array of J). */
mg_status mg_level_sizes(const mg_ctx* ctx, int32_t* n_levels_out, int32_t* n_rows_out);

/* Device bytes mg_setup would allocate for this hierarchy and batch
 * (used for admission by memory footprint). */
mg_status mg_footprint_bytes(const mg_hierarchy* h, const mg_csr* A_levels, int32_t max_batch,
                             int32_t precision, size_t* bytes);

/* Copies the last error message of ctx (or the global one if ctx is NULL). */
mg_status mg_last_error(const mg_ctx* ctx, char* buf, size_t len);

/* Number of kernels this context has launched (graph replays counted by the
 * kernels they contain). */
int64_t mg_kernel_launches(const mg_ctx* ctx);

void mg_destroy(mg_ctx* ctx);

/* ---------------------------------------------------------------------
 * Stacked contexts: one operator per request on a structured square mesh
 * (serving).  A context holds `slots` independent systems -div(k grad u) = f
 * on the same N x N uniform right-triangle mesh of the unit square (every
 * cell split by its SW->NE diagonal, Dirichlet boundary), each with its own
 * element coefficients.  Every level stores the block-diagonal stack of the
 * slots' interior operators (block b = rows [b m_l, (b+1) m_l), m_l =
 * (N_l - 2)^2); the learnable cycle (Algorithm 2) runs on the stack, and a
 * block's rows only ever read their own block, so each system's result does
 * not depend on the others.  Vectors of the context: level-0 stacks, FP64
 * [slots * m_0].
 * ------------------------------------------------------------------- */

/* Creates a stacked context: N vertices per side (N - 1 divisible by
 * 2^(J-1)), J levels down to 3 x 3 vertices (one interior vertex, solved by
 * its explicit inverse), 1 <= slots <= 2048, Theta p, precision 64 or 32.
 * The transfers (natural inclusion between the nested grids, Sec. 2.2) and
 * the DIA layout are built here, once; the blocks' operators are placeholders
 * until mg_square_set_block writes them.  Errors as mg_setup, MG_ERR_INVALID
 * for sizes that do not coarsen to 3 x 3. */
mg_status mg_setup_square(mg_ctx** out, int32_t N, int32_t J, int32_t slots, const mg_params* p,
                          int32_t precision, void* stream);

/* Writes one request's operator into block `block` of a stacked context, on
 * the device (no host work, no allocation): the P1 stiffness of
 * -div(k grad u) from the element coefficients (Sec. 2.1's discretisation;
 * on these right isosceles triangles the element matrix is k_T/2 times the
 * reference one), Galerkin coarse operators A_{l+1} = P^T A_l P over all
 * vertices (Sec. 2.2), the drop of round-off couplings |a_ij| <= 1e-12
 * max(|a_ii|, |a_jj|), the graph degree before Dirichlet elimination, the
 * interior rows' DIA values, diagonals, 1/diagonals and 1/degrees, and the
 * coarsest vertex's inverse.  ke: DEVICE FP64 [2 (N-1)^2], element e =
 * 2 (cy (N-1) + cx) + t for cell (cx, cy) (x fastest), t = 0 the lower
 * triangle (SW, SE, NE), t = 1 the upper one (SW, NE, NW); it is read before
 * the call's work completes (stream order).  Queued on stream, not waited
 * for; uses the context's set-up scratch, so calls on one context must be
 * ordered on one stream. */
mg_status mg_square_set_block(mg_ctx* ctx, int32_t block, const double* ke_dev, void* stream);

/* Solves the leading nblocks blocks of a stacked context (blocks
 * 0 .. nblocks-1; 1 <= nblocks <= slots), each to its own tolerance:
 * ||f_b - A_b u_b||_2 / ||f_b||_2 < tol per block b, with mg_solve's methods
 * applied per block (precision 32: FP32 cycles inside FP64 refinement, the
 * residual of each block scaled by its own power of two; precision 64: the
 * stationary FP64 cycle), each block stopping as soon as it meets tol.  The
 * leading blocks are the leading rows of every level, so the work is that of
 * nblocks blocks, not of the whole context, and each block's result does not
 * depend on nblocks (bitwise).  One CUDA graph (a while node) per solve,
 * kept per (f, u, nblocks).  f_dev, u_dev: DEVICE FP64 level-0 stacks
 * [slots * m_0], of which the leading nblocks * m_0 entries are read and
 * written; u is the initial guess; a block whose f is zero is idle (relres 0,
 * no iterations).  iters_out, relres_out: host [nblocks] (may be NULL).
 * Synchronises the stream.  Returns MG_ERR_INVALID for an nblocks outside
 * 1 .. slots, MG_NOT_CONVERGED if a block missed tol within max_iter,
 * MG_ERR_DIVERGED on a non-finite residual. */
mg_status mg_solve_blocks(mg_ctx* ctx, int32_t nblocks, const double* f_dev, double* u_dev,
                          double tol, int32_t max_iter, int32_t* iters_out, double* relres_out,
                          void* stream);

/* ---------------------------------------------------------------------
 * Allocation-free entry point.  The paper has no counterpart: this is an
 * interface for callers that cannot call cudaMalloc (a host application
 * that owns all device memory and forbids plug-ins to allocate, or a
 * latency-critical loop that cannot take an allocation's implicit device
 * synchronisation).
 * ------------------------------------------------------------------- */

/* Size of the static device scratch used by mg_smooth_noalloc, in doubles
 * (4 MiB): n * nrhs must not exceed it. */
#define MG_NOALLOC_MAX_ELEMS 524288

/* nu learnable smoothing steps, delta = theta D^{-1} (f - A u),
 * u <- u + eta (w1 delta + w2 mean_{N(i)} delta), in FP64 on an operator
 * the caller holds in DEVICE memory: CSR rowptr[n+1], col[nnz], val[nnz]
 * (diagonal included; the off-diagonal nonzeros are the graph N(i)),
 * inv_deg[n] = 1/deg_i, f and u [n][nrhs].  u is updated in place; f and u
 * must not overlap.  Nothing is allocated: delta lives in a file-scope
 * __device__ array of MG_NOALLOC_MAX_ELEMS doubles that every GPU loading
 * the library holds until exit.  The first call on a device looks up that
 * array's device address (cudaGetSymbolAddress, with the device current);
 * make that first call before any stream capture.  All calls share the
 * array and it keeps the last call's contents (nothing needs clearing: each
 * step overwrites delta before reading it); calls that overlap on the GPU
 * race on it.  Returns MG_ERR_INVALID if n * nrhs exceeds
 * MG_NOALLOC_MAX_ELEMS or an argument is invalid (message via
 * mg_last_error(NULL, ...)); work is queued on stream and not waited for. */
mg_status mg_smooth_noalloc(int32_t n, const int32_t* rowptr_dev, const int32_t* col_dev,
                            const double* val_dev, const double* inv_deg_dev, const double* f_dev,
                            double* u_dev, int32_t nrhs, int32_t nu, double theta, double eta,
                            double w1, double w2, void* stream);

/* ---------------------------------------------------------------------
 * Two features per node (d = 2): complex systems
 *
 * The Helmholtz experiment (Sec. 4.2) solves a complex system and carries
 * (Re u, Im u) as two node features; every SAGEConv then holds
 * W_1, W_2 in R^{2x2} (the weight matrices of Sec. 3.2) and may mix them.  An mg2 context runs
 * that cycle (Algorithm 2):
 *   delta = theta_l D_A^{-1} (f - A u)       (complex arithmetic)
 *   u <- u + eta_l Phi_B(delta),  Phi(x)_i = W_1 x_i + W_2 mean_{N(i)} x_j
 *   r_c = P^T Phi_R(f - A u),  u <- u + Phi_P(P e_c)   (real P)
 *   coarsest level: e = A_J^{-1} r (A_J inverted in FP64 at set-up)
 * N(i) is the off-diagonal pattern of row i of A; the mean divides by
 * 1/inv_deg[i] (which may count eliminated neighbours, as in mg_eliminate).
 * Vectors: device, [n][nrhs] complex with (Re, Im) adjacent (C99 complex /
 * torch.complex64 or complex128 layout), in the context precision.
 * ------------------------------------------------------------------- */
typedef struct mg2_ctx mg2_ctx;

typedef struct {
  int32_t n;                /* rows (DOFs) of this level                      */
  const int32_t* A_indptr;  /* [n+1], CSR of the complex operator A_l          */
  const int32_t* A_indices; /* [nnz], diagonal included                        */
  const double* A_vals;     /* [2*nnz], (Re, Im) per entry                     */
  const double* inv_deg;    /* [n], 1/deg of the convolution graph             */
  const int32_t* P_indptr;  /* [n+1], real prolongation n x n_{l+1};           */
  const int32_t* P_indices; /*   all three NULL on the coarsest level          */
  const double* P_vals;
} mg2_level;

/* Copies a J-level complex hierarchy (host arrays, copied; the caller keeps
 * ownership) to the device: CSR operators, prolongations and their
 * transposes, per-level workspace for max_batch (1..65535) right-hand
 * sides, and the inverse of the coarsest operator (n_{J-1} <= 2048).
 * precision 64 or 32.  Parameters start at the classical cycle: W_1 = I,
 * W_2 = 0, theta = 2/3, eta = 1, one pre- and one post-smoothing step.
 * Every check below runs on the host before the first CUDA call.  Errors
 * (message via mg_last_error(NULL, ...)): MG_ERR_INVALID for missing arrays,
 * out-of-range indices or a zero diagonal entry; MG_ERR_NOT_SPD if the
 * coarsest operator is singular (an exactly zero pivot of its FP64
 * Gauss-Jordan inverse); MG_ERR_OOM / MG_ERR_CUDA. */
mg_status mg2_setup(mg2_ctx** out, int32_t J, const mg2_level* levels, int32_t max_batch,
                    int32_t precision);

/* Theta for J-1 levels (host, copied): theta[l], eta[l]; WB, WR, WP
 * [J-1][2][2][2] = per level (W_1, W_2), each row-major 2 x 2 acting on the
 * feature column (Re, Im).  MG_ERR_INVALID for NULL or non-finite values or
 * nu outside [0, 16]. */
mg_status mg2_set_params(mg2_ctx* ctx, const double* theta, const double* eta, const double* WB,
                         const double* WR, const double* WP, int32_t nu_pre, int32_t nu_post);

/* Launch shapes of the two-feature cycle (results are bitwise the same):
 *   MG_OPT_PDL        1 (default): consecutive kernels use programmatic
 *                     dependent launch; 0: plain launches.
 *   MG_OPT_MULTI_RHS  1 (default): a thread owns a row and a tile of the
 *                     widest of 4 (precision 32) or 2 (precision 64) complex
 *                     right-hand sides (32 bytes) that divides nrhs, so a
 *                     row's entries are read once per tile; 0: one thread
 *                     per (row, rhs).
 *   MG_OPT_TAIL_WORK  levels with rows * nrhs <= value, and every coarser
 *                     one but the coarsest, run in one thread block with block
 *                     barriers between the steps (two launches around the
 *                     coarsest product), when that covers a level above the
 *                     coarsest (at most 8 levels).  0 (default): never; at
 *                     257^2 with one rhs it measured no faster in precision
 *                     32 (0.102 ms per cycle either way) and slower in
 *                     precision 64 (0.31 against 0.23 ms).
 * Other options: MG_ERR_INVALID.  Drops the captured cycle graphs. */
mg_status mg2_set_option(mg2_ctx* ctx, int32_t option, int64_t value);

/* One cycle exactly like mg2_vcycle (same kernels, same result), launched
 * directly with a CUDA event pair around every kernel on `stream`.  Records
 * (launch order, up to max_out) use mg_kernel_kind: MG_K_RESIDUAL_SCALED and
 * MG_K_CONV_UPDATE (smoothing), MG_K_RESIDUAL and MG_K_CONV_R (restriction's
 * residual and Phi_R), MG_K_RESTRICT (the P^T product), MG_K_PE (P e_c),
 * MG_K_PROLONG (Phi_P added to u), MG_K_COARSE_CHOL (the coarsest product).
 * Synchronises the stream. */
mg_status mg2_vcycle_profile(mg2_ctx* ctx, const void* f_dev, void* u_dev, int32_t nrhs,
                             mg_kernel_time* out, int32_t max_out, int32_t* n_out, void* stream);

/* One cycle on level 0: u <- LMG(A, f, u) for nrhs complex right-hand sides
 * (device f and u, distinct; 1 <= nrhs <= max_batch).  Queued on stream,
 * not waited for.  The cycle is captured into a CUDA graph on first use
 * for each (f, u, nrhs) and replayed afterwards; mg2_set_params drops the
 * captured graphs (parameters are kernel arguments). */
mg_status mg2_vcycle(mg2_ctx* ctx, const void* f, void* u, int32_t nrhs, void* stream);

/* Restarted flexible GMRES on the complex system, with one two-feature
 * cycle from zero (precond 0) or one full multigrid (precond 1) as right
 * preconditioner: the pairing of the paper's Helmholtz preconditioner
 * table (Sec. 4.2, tab:helmholtz-results-precond).  W_1, W_2 mix Re and
 * Im, so the preconditioner is
 * real-linear, not complex-linear: the Krylov method runs on the equivalent
 * real system of size 2n, [[Re A, -Im A], [Im A, Re A]], with real inner
 * products sum_i (Re x_i Re y_i + Im x_i Im y_i) per right-hand side.
 * Classical Gram-Schmidt twice, FP64 Hessenberg with Givens rotations; the
 * host drives the restarts (restart = m, 1..64).  f and u: device, FP64
 * complex [n][nrhs] whatever the context precision (the preconditioner runs
 * in the context precision); u is the initial guess and receives the
 * iterate.  iters_out / relres_out (host, [nrhs], may be NULL): Arnoldi
 * steps and the true final relative residual per right-hand side.  Returns
 * MG_OK, MG_NOT_CONVERGED (max_iter steps without meeting tol),
 * MG_ERR_DIVERGED (non-finite residual) or an error; synchronises stream. */
mg_status mg2_solve_fgmres(mg2_ctx* ctx, const void* f, void* u, int32_t nrhs, double tol,
                           int32_t max_iter, int32_t restart, int32_t precond,
                           int32_t* iters_out, double* relres_out, void* stream);

/* Frees every device buffer of the context (synchronises the device). */
void mg2_destroy(mg2_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* MG_H */
