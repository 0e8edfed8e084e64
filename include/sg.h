/*
 * sg.h -- C ABI of the GB300 stochastic Galerkin (SG) solver for the diffusion equation with a
 * lognormal coefficient (arXiv 1910.11505).
 *
 * The problem (Sec. 2, Eq. Strong_PS): -div(a grad u) = f on [0,1]^2, u = 0 on the boundary,
 * a = a_min + exp(gamma), gamma a Gaussian field with the separable exponential covariance of
 * Eq. standard_deviation, truncated to M Karhunen-Loeve terms (Eq. aKL).  The SG discretisation
 * (Eqs. u_discrete, dataProjection, A_q, stochastic_matrix) on a uniform n x n mesh of bilinear
 * (Q1) elements gives K u = F with K = sum_k G_k (x) A_k.
 *
 * Layout shared by every entry point:
 *   - a nodal field over the chaos basis is an N x P array, row-major, chaos index fastest:
 *     X[j*P + b] = coefficient of psi_b at node j.  N = (n+1)^2 nodes including the Dirichlet
 *     boundary (boundary rows are identity rows, their values are 0 in every solution);
 *     node id j = i1 + (n+1)*i2 for the grid point (i1/n, i2/n).
 *   - P = |J(p)| = (M+p)!/(M! p!) chaos terms of the solution, L = |J(q)| terms of the
 *     coefficient (q = 2p by default), multi-indices in lexicographic order, last index fastest.
 *   - Every device pointer is owned by the caller and must stay valid until the work queued on
 *     the given stream has finished.  ``stream`` is a cudaStream_t (NULL = legacy default stream).
 *
 * Errors: every int-returning call gives SG_OK (0) or a negative SG_ERR_* code; sg_last_error()
 * then returns a message (per host thread).  No call aborts the process.
 */
#ifndef SG_GB300_H
#define SG_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SG_OK 0
#define SG_ERR_ARG (-1)            /* invalid argument or unsupported size                     */
#define SG_ERR_CUDA (-2)           /* a CUDA runtime call failed                               */
#define SG_ERR_OOM (-3)            /* device allocation failed                                 */
#define SG_ERR_NAN (-4)            /* NaN or Inf met in a residual norm                        */
#define SG_ERR_NOT_CONVERGED (-5)  /* GMRES stopped at max_iters above tolerance               */

#define SG_PC_NONE 0       /* identity                                                          */
#define SG_PC_MEAN 1       /* mean-based block diagonal I (x) ILU0(A_0) (Sec. 1, cited there)   */
#define SG_PC_FS_GS 2      /* field split, block lower triangular P of Eq. P_preconditioner     */
#define SG_PC_FS_JACOBI 3  /* field split, block diagonal of K                                  */
#define SG_PC_MG 4         /* geometric multigrid V-cycle (Sec. 3): on every level one pre- and */
                           /* one post-smoothing step of Eq. level_solver with the block        */
                           /* preconditioner mg_smoother, a direct solve on the coarsest mesh   */
#define SG_PC_FG 5         /* grouped field split (Sec. 3, Eq. P_group): block Gauss-Seidel over */
                           /* the splits that fg_rule forms, the diagonal block of each split   */
                           /* approximated by its ILU(0) on the node-major block pattern (every */
                           /* field of a node coupled to every field of its 9-point neighbours; */
                           /* nodes in the four-colour order).  fg_rule SG_FG_WHOLE (one split) */
                           /* is the ILU(0) of K: G-I alone, G-M-I as the multigrid smoother     */

#define SG_FP64 0          /* every step in FP64                                                */
#define SG_MIXED_FP32 1    /* FP32 operator / preconditioner inside FP64 flexible GMRES + IR    */
#define SG_MIXED_BF16 2    /* BF16-stored operator, FP32 arithmetic, inside FP64 FGMRES + IR    */

typedef struct sg_handle sg_handle;

/* Parameters of one SG system.  a = a_min + exp(mu + sum_n sqrt(lambda_n) b_n(x) y_n). */
typedef struct {
  int n;             /* cells per side of the Q1 mesh of [0,1]^2: 2..1024, with ILU(0) 2..769  */
  int M;             /* KL terms kept, 1 <= M <= 8                                             */
  int p;             /* total degree of the solution chaos, 0 <= p <= 6                        */
  int q;             /* total degree of the coefficient chaos; <= 0 selects 2p                 */
  double sigma;      /* standard deviation of gamma (Eq. standard_deviation), >= 0             */
  double ell;        /* correlation length L_c, > 0                                            */
  double a_min;      /* lower bound of a (Assumption 1), >= 0                                  */
  double mu;         /* mean of gamma                                                          */
  double f;          /* constant forcing                                                       */
  int precond;       /* SG_PC_*                                                                 */
  int inner_iters;   /* ILU(0)-Richardson steps per diagonal block, >= 1                       */
  int outer_sweeps;  /* steps of the level solver, Eq. level_solver (i_max), >= 1              */
  int restart;       /* GMRES restart length m, 1 <= m <= 1024                                 */
  int max_iters;     /* cap on GMRES iterations (inner iterations summed over restarts)       */
  double rtol;       /* stop when ||F - K x||_2 <= max(rtol ||F||_2, atol)                     */
  double atol;
  int precision;     /* SG_FP64 | SG_MIXED_FP32 | SG_MIXED_BF16                                */
  double inner_rtol; /* mixed precision: each inner FGMRES cycle stops once its residual       */
                     /* estimate drops below inner_rtol times the current true residual        */
  int graphs;        /* 1: capture each GMRES cycle of this system once as a CUDA graph (keyed  */
                     /* by cycle length and the F, X pointers) and replay it; 0: plain launches */
  int mg_smoother;   /* SG_PC_MG: smoother of every level, SG_PC_MEAN | SG_PC_FS_GS |           */
                     /* SG_PC_FS_JACOBI | SG_PC_FG (G-M-F-I of the paper is SG_PC_FS_GS,        */
                     /* G-M-Fg-I SG_PC_FG with SG_FG_PAPER, G-M-I SG_PC_FG with SG_FG_WHOLE)    */
  int mg_coarse;     /* SG_PC_MG: cells per side of the coarsest mesh (the paper: 2); n must be  */
                     /* mg_coarse times a power of two, and the coarsest interior system of     */
                     /* (mg_coarse - 1)^2 P unknowns is solved with its dense inverse (<= 4096)  */
  int op_kernel;     /* SG operator kernel: SG_OP_AUTO (time the candidates on this system at   */
                     /* setup, keep the fastest; the choice is cached per N, P, L and precision */
                     /* for the process), SG_OP_PAIRS or SG_OP_TILE                             */
  int op_kappa;      /* SG_OP_TILE: k per register group, 1, 2 or 4 (0: 2 in FP64, 4 in FP32)   */
  int op_ctas;       /* SG_OP_TILE: CTAs per SM the shared memory is planned for, 1 or 2 (0: 1) */
  int ilu_order;     /* ILU(0) node ordering: SG_ILU_NATURAL, or SG_ILU_COLOR4 (colour           */
                     /* (x mod 2) + 2 (y mod 2), colours in turn: every triangular sweep runs   */
                     /* in 4 fully parallel phases; requires inner_iters = 1)                   */
  int coupling_bf16; /* SG_MIXED_FP32 with a field-split Gauss-Seidel sweep (alone or as the    */
                     /* smoother): 1 = the sweep's coupling sum_{b<a} K_ab z_b reads a BF16     */
                     /* copy of the stiffness values (FP32 arithmetic), half the bytes of the   */
                     /* sweep's dominant traffic; the operator keeps its FP32 copy              */
  int fg_rule;       /* SG_PC_FG (alone or as mg_smoother): how fields form splits, one of      */
                     /* SG_FG_PAPER, SG_FG_GROUPS, SG_FG_WHOLE; a split holds at most 96 fields; */
                     /* requires ilu_order SG_ILU_COLOR4                                        */
  int fg_bf16;       /* SG_MIXED_FP32 with SG_PC_FG: 1 = the block ILU(0) factors (computed in   */
                     /* FP32) are stored in BF16 and applied in FP32 arithmetic: half the bytes  */
                     /* of the smoother's traffic; the preconditioner changes, the solution not  */
} sg_params;

/* Splits of SG_PC_FG.  Fields are grouped by the first index of their multi-index (the groups
 * are consecutive ranges of the chaos basis, lexicographic with the last index fastest). */
#define SG_FG_PAPER 0   /* in order, a group holding a multi-index with all indices equal opens */
                        /* a new split, any other group joins the preceding split (Sec. 3)      */
#define SG_FG_GROUPS 1  /* every group is a split                                               */
#define SG_FG_WHOLE 2   /* one split of all fields: the ILU(0) of K (G-I, G-M-I)                */

#define SG_ILU_NATURAL 0
#define SG_ILU_COLOR4 1

#define SG_OP_AUTO 0   /* choose by timing (see op_kernel)                                      */
#define SG_OP_PAIRS 1  /* one CTA per 4 rows, (k, b) pairs over threads, operands in shared mem */
#define SG_OP_TILE 2   /* 32 rows of a grid line per CTA, one per lane, k groups in registers  */

typedef struct {
  int iters;         /* GMRES iterations (all cycles; inner FGMRES iterations in mixed mode)  */
  int restarts;      /* GMRES cycles (mixed mode: refinement steps, one inner cycle each)      */
  int status;        /* SG_OK, SG_ERR_NOT_CONVERGED or SG_ERR_NAN                              */
  double rel_resid;  /* final true FP64 residual ||F - K x|| / ||F||                           */
  double seconds;    /* wall time of the solve of this batch                                   */
} sg_solve_info;

/* Fill ``prm`` with defaults: n=16, M=2, p=2, q=2p, sigma=0.5, ell=1, a_min=0, mu=0, f=1,
 * mean preconditioner, 1 inner / 1 outer step, restart 30, max_iters 2000, rtol 1e-10,
 * atol 0, FP64, inner_rtol 1e-4, graphs 0, mg_smoother SG_PC_FS_GS, mg_coarse 2,
 * op_kernel SG_OP_AUTO, op_kappa 0, op_ctas 0, ilu_order SG_ILU_NATURAL, coupling_bf16 0,
 * fg_rule SG_FG_PAPER, fg_bf16 0. */
void sg_default_params(sg_params* prm);

/* Build ``nsys`` independent SG systems (Sec. 2: KL modes of Eq. gen_eigen in closed form,
 * chaos coefficients of Eq. dataProjection, stiffness stack of Eq. A_q on the shared 9-point
 * pattern, triple products G_k of Sec. 2.2, Dirichlet rows, ILU(0) factors for the chosen
 * preconditioner) on the current CUDA device.  ``prm`` points to nsys parameter sets (host).
 * All device memory of the systems is owned by the handle.  Work is queued on ``stream`` and
 * the call synchronises it before returning.  On error *out is NULL. */
int sg_setup(const sg_params* prm, int nsys, void* stream, sg_handle** out);

/* Sizes of system ``sys``: N nodes, P solution chaos terms, L coefficient chaos terms. */
int sg_dims(const sg_handle* h, int sys, int* N, int* P, int* L);

/* Number of stored nonzeros of the 9-point pattern and of the triple-product tensor G. */
int sg_nnz(const sg_handle* h, int sys, long long* nnz_A, long long* nnz_G);

/* Y = K X = sum_k A_k X G_k^T (Eqs. stochastic_matrix, K_matrix); X, Y device, N x P FP64,
 * must not overlap.  Asynchronous on ``stream``. */
int sg_matvec(sg_handle* h, int sys, const double* X, double* Y, void* stream);

/* Same operator with the FP32 (precision SG_MIXED_FP32) or BF16 (SG_MIXED_BF16) copy of the
 * stiffness stack and FP32 arithmetic; X, Y device N x P FP32.  SG_ERR_ARG for an FP64 system. */
int sg_matvec_lowp(sg_handle* h, int sys, const float* X, float* Y, void* stream);

/* Z = P^{-1} R for the system's preconditioner, with ``outer_sweeps`` steps of Eq. level_solver
 * from zero and ``inner_iters`` ILU(0)-Richardson steps per diagonal block; mean-based
 * (I (x) ILU0(A_0)), field-split Gauss-Seidel (Eq. P_preconditioner), block Jacobi or the
 * multigrid V-cycle.  R, Z device N x P FP64, must not overlap.  Asynchronous on ``stream``.
 * SG_ERR_ARG for a field-split Gauss-Seidel sweep (alone or as a smoother) of a mixed-precision
 * system, whose FP64 coupling copy is not kept (use sg_precond_apply_lowp). */
int sg_precond_apply(sg_handle* h, int sys, const double* R, double* Z, void* stream);

/* The same preconditioner application in FP32 arithmetic with the FP32 ILU(0) factors and the
 * FP32 (SG_MIXED_FP32) or BF16 (SG_MIXED_BF16) stack copy used by the inner solver of the mixed
 * forms; R, Z device N x P FP32, must not overlap.  SG_ERR_ARG for an FP64 system.
 * Asynchronous on ``stream``. */
int sg_precond_apply_lowp(sg_handle* h, int sys, const float* R, float* Z, void* stream);

/* No counterpart in the paper: the same field-split Gauss-Seidel application as
 * sg_precond_apply (outer_sweeps = 1), for callers that must not allocate device memory, such as
 * a process whose device memory is already reserved by another allocator (a framework's caching
 * pool) or code with a fixed memory budget that may not grow.  Its scratch, the P right-hand
 * sides of the block solves as columns of ldN = N rounded up to a multiple of 4 entries, is a
 * fixed array of SG_NOALLOC_MAX_ENTRIES doubles (8 MiB) inside this library, which every GPU that
 * loads the library holds until the process exits; the call itself allocates nothing and
 * overwrites the part it uses from R before reading it.  Every call looks up that array's device
 * address on the current device (the lookup allocates nothing); the first lookup on a device
 * loads the library's module there, so make that first call before any stream capture.  All calls share the one array: calls whose
 * work overlaps on the GPU (other streams, other threads) race and give wrong results.
 * SG_ERR_ARG if the system does not use SG_PC_FS_GS with outer_sweeps = 1, if P x ldN exceeds
 * SG_NOALLOC_MAX_ENTRIES, or if the handle's device is not current.  R, Z as for sg_precond_apply.  Asynchronous on ``stream``. */
#define SG_NOALLOC_MAX_ENTRIES (1 << 20)
int sg_precond_apply_noalloc(sg_handle* h, int sys, const double* R, double* Z, void* stream);

/* F of Eq. stochastic_matrix: F[j*P + 0] = int f phi_j, other chaos terms 0, boundary rows 0.
 * F device N x P FP64.  Asynchronous on ``stream``. */
int sg_rhs(sg_handle* h, int sys, double* F, void* stream);

/* Solve K x = F for every system of the handle with restarted right-preconditioned GMRES
 * (Sec. 3), CGS2 Arnoldi and Givens rotations on the device.  F[s], X[s] are device N x P FP64
 * arrays; X[s] holds the initial guess on entry (zeros for a cold start) and the solution on
 * return.  In mixed precision (SG_MIXED_*) the solve is FP64 iterative refinement around an
 * inner flexible GMRES whose operator and preconditioner run in FP32 arithmetic; the FP64 true
 * residual decides convergence.  ``info`` (host, nsys entries) is filled; the call returns
 * SG_OK if every system converged, else the first failing status.  Synchronises ``stream``. */
int sg_gmres_solve(sg_handle* h, const double* const* F, double* const* X, sg_solve_info* info,
                   void* stream);

/* Copy an internal array of system ``sys`` to host memory ``dst`` of ``bytes`` bytes, for
 * tests: what = 0 stack values (nnz_A x L doubles, entry e and chaos k at e*L + k),
 * 1 CSR row pointers (N+1 ints), 2 CSR columns (nnz_A ints), 3 KL eigenvalues (M doubles),
 * 4 ILU(0) factor values of the first factor set (nnz_A doubles on the CSR pattern: the unit
 * lower factor at entries of nodes before the row's node in the ILU ordering, the upper factor
 * at the others), 5 triple products as (k, a, b, value) records sorted by k then a then b
 * (nnz_G x 4 doubles).  Synchronous.  SG_ERR_ARG if ``bytes`` is too small. */
int sg_export(const sg_handle* h, int sys, int what, void* dst, size_t bytes);

/* Which SG operator kernel system ``sys`` runs: info[0..3] for the FP64 operator and info[4..7]
 * for the FP32 one, each {kernel (0 none, 1 pair kernel, 2 row-tiled kernel), kappa, shared
 * memory bytes, chunks}; ``msg`` (msg_len bytes, may be NULL) receives why a row-tiled operator
 * was not built ("" if it was). */
int sg_op_info(const sg_handle* h, int sys, long long* info, char* msg, int msg_len);

/* For tests, host only (no device work): plan the row-tiled operator of a system with these sizes
 * in FP64 (precision SG_FP64) or FP32 (any other precision) for the six variants kappa in {1, 2, 4}
 * k per register group x 1 or 2 CTAs per SM (rows 0..5, CTAs outer), under a shared-memory budget
 * of smem_max bytes per SM (halved per CTA for two CTAs).  Row r is out[16 r .. 16 r + 15] =
 * {kappa, CTAs, fits, shared-memory bytes, chunks, largest chunk's T slots, (k, b) pairs placed,
 * stage-2 entries placed, k kept, k groups, tables verified by decoding them as the kernel does,
 * budget, union entries, stage-1 steps and stage-2 steps of the slowest warp summed over the
 * chunks, 0}; ``out`` holds 96 values.  SG_ERR_ARG for invalid sizes. */
int sg_tune_plan(int n, int M, int p, int q, int precision, long long smem_max, long long* out);

/* Host only, no device use: the splits of SG_PC_FG for the chaos basis of total degree p in M
 * variables under fg_rule ``rule`` (Sec. 3, the rule before Eq. P_group), as field ranges
 * [out[2s], out[2s+1]) in basis order; ``out`` holds room for 2 (M+p)!/(M! p!) ints (host),
 * *count receives the number of splits.  SG_ERR_ARG for M, p or rule out of range. */
int sg_fg_splits(int M, int p, int rule, int* out, int* count);

/* Measure the device's FMA throughput (independent FMA chains on every SM, CUDA events) in FP64
 * (precision SG_FP64) or FP32 (any other), in GFLOP/s (2 flops per FMA), on the legacy default
 * stream of the current device; synchronous.  The ALU roofline of the FP64 operator divides by it. */
int sg_probe_fma(int precision, double* gflops);

/* Count of kernel launches this library has queued since load (all handles, all threads); each
 * replay of a captured GMRES segment counts the kernel nodes of its graph. */
long long sg_launch_count(void);

/* Live kernel timing.  Kernel classes: */
#define SG_K_APPLY_F64 0   /* SG operator, FP64                                             */
#define SG_K_APPLY_LOWP 1  /* SG operator, FP32 arithmetic on the FP32 / BF16 stack          */
#define SG_K_ILU_SOLVE 2   /* ILU(0) block solves of the preconditioners                    */
#define SG_K_GS_SCATTER 3  /* field-split Gauss-Seidel off-diagonal push                   */
#define SG_K_ARNOLDI 4     /* CGS2 dot products, updates, Givens step, normalisation        */
#define SG_K_OTHER 5       /* norms, cycle start and end, casts, preconditioner transposes  */
#define SG_K_NCLASS 6
/* Start timing: from now on every ``stride``-th launch of each class queued through handle h is
 * bracketed by CUDA events recorded on the stream it is launched on (up to 2^15 timed launches).
 * Allocates the events; call it outside a timed region.  Resets previous counts. */
int sg_timing_start(sg_handle* h, int stride);
/* Stop timing, wait for the recorded events and report per class (host arrays of SG_K_NCLASS):
 * ms = summed duration of the timed launches, timed = how many were timed, launches = how many
 * were queued.  Any pointer may be NULL. */
int sg_timing_stop(sg_handle* h, double* ms, long long* timed, long long* launches);

/* Free every device array of the handle (after synchronising its streams).  NULL is a no-op. */
void sg_free(sg_handle* h);

/* Message of the last failing call on this host thread ("" if none). */
const char* sg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SG_GB300_H */
