/*
 * plam.h -- C ABI of the GB300 (sm_103a) PLAM / PCAL hot path.
 *
 * Method: Gao, Liu, Yuan, "Parallelizable algorithms for optimization problems
 * with orthogonality constraints" (arXiv:1810.03930).  The problem is
 *
 *     min f(X)  subject to  X^T X = I_p,   X in R^{n x p},  2p <= n      (Section 1, eq. prob)
 *
 * and one iteration at X = X^k, with G = grad f(X), B = X^T X, is
 *
 *     Lambda0 = Psi(G^T X),  Psi(A) = (A + A^T)/2                        (eq. Lambda1)
 *     Lambda  = Lambda0 [+ Phi(X^T grad_X L_beta(X, Lambda0)) for PCAL]  (eq. lambda2)
 *     R       = G - X Lambda + beta X (B - I)  = grad_X L_beta(X, Lambda) (eq. S1)
 *     PLAM:  X <- X - R / eta                                            (eq. PLAM-main)
 *     PCAL:  X_i <- (X_i - R_i/eta) / ||X_i - R_i/eta||_2 for every column (Algorithm 3)
 *
 * with eta from the rules of Section 5.1 (alternating Barzilai-Borwein by
 * default), the stopping test ||G - X Psi(G^T X)||_F / (same at X^0) < tol
 * (Section 5.1 with the Section 3.3 shortcut) and one final orthonormalisation
 * (Section 5.3, Table "orth step").
 *
 * Conventions for every entry point
 *   - Matrices are column-major.  X is n x p with leading dimension ldx >= n;
 *     column i starts at X + i*ldx.  Device pointers must be aligned to their
 *     element size (misaligned pointers are rejected with PLAM_ERR_INVALID).
 *   - "storage type" is double for PLAM_PREC_FP64 and float for every other
 *     precision mode.  X, G and dense operators are passed in the storage type.
 *   - The caller owns every pointer it passes and keeps it alive until the call
 *     (and, for device work, the stream) completes.  A handle owns its own
 *     device workspace (allocated in plam_create, freed in plam_destroy) and
 *     never frees caller memory.
 *   - All device work is ordered on the handle's stream (a cudaStream_t passed
 *     as void*; NULL selects the legacy default stream).  Calls that return
 *     host-side results (info, f) synchronise that stream before returning.
 *   - Every call returns a plam_status_t and never aborts the process.  On
 *     PLAM_ERR_INVALID nothing was launched.  On PLAM_ERR_CUDA the CUDA error
 *     string is available from plam_last_error().
 */
#ifndef PLAM_H_
#define PLAM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PLAM_OK = 0,
  PLAM_ERR_INVALID = 1,        /* null pointer, 2p > n, ld < n, bad enum, misalignment */
  PLAM_ERR_NOT_CONVERGED = 2,  /* maxit iterations performed without meeting tol */
  PLAM_ERR_DIVERGED = 3,       /* non-finite KKT value, step size or column norm */
  PLAM_ERR_CHOLESKY = 4,       /* X^T X not numerically positive definite */
  PLAM_ERR_TIMEOUT = 5,        /* a bounded device-side wait (grid barrier, tensor-core pipeline) expired */
  PLAM_ERR_CUDA = 6,           /* a CUDA runtime call failed */
  PLAM_ERR_NOMEM = 7,          /* device or pinned host allocation failed */
  PLAM_ERR_UNSUPPORTED = 8     /* valid request that this build does not implement */
} plam_status_t;

/* MOPTQR: the comparison solver of Sections 5.3-5.4 (plam_solve only): a Riemannian gradient
 * step on the projected gradient D = G - X G^T X with the same Barzilai-Borwein rules, then
 * the Cholesky retraction X <- V L^{-T}, V = X - D/eta, V^T V = L L^T, every iteration
 * (Table "cost"); the retraction's Gram, Cholesky and product run in FP64 arithmetic. */
enum { PLAM_VARIANT_PLAM = 0, PLAM_VARIANT_PCAL = 1, PLAM_VARIANT_MOPTQR = 2 };
/* Multiplier rule: eq. (Lambda1), eq. (lambda2) (PCAL only), or the dual
 * ascent step of Algorithm 1, Lambda^k = Lambda^{k-1} - beta ((X^k)^T X^k - I)
 * from Lambda^0 = Psi(grad f(X^0)^T X^0) (PLAM-DA / PCAL-DA, Section 5.3's
 * comparison; graph engine only). */
enum { PLAM_LAMBDA1 = 0, PLAM_LAMBDA2 = 1, PLAM_LAMBDA_DA = 2 };
/* Proximal parameter rules of Section 5.1: alternating BB (default), BB1, BB2,
 * constant gamma, differential ||Y||_F/||S||_F. */
enum { PLAM_ETA_ABB = 0, PLAM_ETA_BB1 = 1, PLAM_ETA_BB2 = 2, PLAM_ETA_CONST = 3, PLAM_ETA_DIFF = 4 };
/* Arithmetic of the iteration.  FP64: everything in double.  FP32: float
 * storage, products and partial sums (Kahan-compensated across row chunks),
 * the O(p^2) multiplier algebra and the scalars in double; the final
 * orthonormalisation forms its Gram in double (exact products of floats) and
 * writes a double result. */
enum { PLAM_PREC_FP64 = 0, PLAM_PREC_FP32 = 1 };
/* Built-in objectives (Section 5.2):
 *   DENSE      f = 1/2 tr(X^T A X), A symmetric n x n              (Problem 3)
 *   HARTREE1D  f = q tr(X^T L X) + (alpha/4) rho^T L^{-1} rho     (Problem 1, KS form eq. KS-energy;
 *                  - (3 xc / 4) sum rho^{4/3}                      with xc: Problem 6's exchange)
 *                  + tr(G_lin^T X)                                 (with lin: Problem 2's linear term)
 *              rho = diag(X X^T), L = tridiag(-1,2,-1) Dirichlet, or with block = b > 0 the
 *              block-diagonal Diag(L_1, ..., L_s) of such matrices on b consecutive rows each
 *              (the last on the n - (s-1) b rows left): Section 5.4 runs Problem 1 with b = 5
 *              and Problem 2 as q = 1/2, alpha = 0, A = L with a random G_lin
 *   STENCIL3D  f = 1/2 tr(X^T (L3 + Diag(V)) X), L3 the 7-point Dirichlet
 *              Laplacian on nx*ny*nz points, index i = x + nx*(y + ny*z);
 *              nx*ny*nz must equal n and stay below 2^31.
 *   QAP        f = 1/2 tr(A^T X B X^T), A n x n and B p x p symmetric          (Problem 4, eq. QAP)
 *              (A in A / lda, B in Bq / ldbq); grad f = A X B.
 * and a user objective (the problem statement of Section 2 admits any f with
 * a gradient):
 *   CALLBACK   f and grad f from plam_objective_t.grad, called on the host
 *              once per gradient evaluation (see plam_grad_fn).  plam_solve
 *              then launches each iteration directly (no CUDA graph; the
 *              resident engine does not apply). */
enum { PLAM_OBJ_DENSE = 0, PLAM_OBJ_HARTREE1D = 1, PLAM_OBJ_STENCIL3D = 2, PLAM_OBJ_CALLBACK = 3,
       PLAM_OBJ_QAP = 4 };

/* User gradient of PLAM_OBJ_CALLBACK: reads X (device, storage type, n x p,
 * leading dimension ldx), writes G = grad f(X) (device, storage type, leading
 * dimension ldg) and the value f(X) into *f (a device double), all as work
 * ordered on `stream` (the handle's cudaStream_t); it may return before that
 * work completes.  Returns 0 on success; any other value stops the calling
 * entry point with PLAM_ERR_CUDA and the message "objective callback failed". */
typedef int (*plam_grad_fn)(void* ctx, const void* X, int64_t ldx, void* G, int64_t ldg, double* f,
                            void* stream);
/* How plam_solve runs the loop.  GRAPH: the kernel sequence of one iteration,
 * replayed from a captured CUDA graph (any size).  RESIDENT: one cooperative
 * persistent launch for the whole solve, each SM keeping its rows of X, G/R
 * and the previous R in shared memory (FP32 mode, p <= 64, HARTREE1D or
 * DENSE, and the rows per SM must fit; otherwise PLAM_ERR_UNSUPPORTED).
 * AUTO: RESIDENT when it applies, else GRAPH. */
enum { PLAM_ENGINE_AUTO = 0, PLAM_ENGINE_GRAPH = 1, PLAM_ENGINE_RESIDENT = 2 };
/* Flag or-ed into plam_params_t.tensor_cores (with 1 or 2): the tensor-core Grams and update
   use one CTA per tile for every p instead of CTA pairs for p >= 256. */
enum { PLAM_TC_SINGLE_CTA = 8 };

typedef struct {
  int variant;          /* PLAM_VARIANT_* used by plam_solve (plam_step/pcal_step choose their own;
                           MOPTQR: plam_solve and plam_time_kernels only, not row-sharded) */
  int lambda_rule;      /* PLAM_LAMBDA1 / PLAM_LAMBDA2 / PLAM_LAMBDA_DA; PCAL default LAMBDA2;
                           PLAM uses LAMBDA1 unless DA is asked for */
  double beta;          /* penalty parameter beta > = 0 */
  int eta_rule;         /* PLAM_ETA_* */
  double eta0;          /* eta at k = 0; <= 0 selects ||G^0||_F/||X^0||_F + beta */
  double eta_gamma;     /* constant for PLAM_ETA_CONST (<= 0: use eta0) */
  double tol;           /* relative KKT tolerance, Section 5.1 (1e-8 in the paper) */
  int maxit;            /* iteration limit (3000 in the paper) */
  int precision;        /* PLAM_PREC_* */
  int final_orth;       /* 0: none, 1: one Cholesky-QR pass, 2: two passes (CholQR2) */
  int graph_iters;      /* iterations per captured CUDA graph in plam_solve; 0 = plain launches */
  int engine;           /* plam_solve engine: PLAM_ENGINE_AUTO, _GRAPH or _RESIDENT */
  int tensor_cores;     /* FP32 mode Grams on tcgen05 (kind::tf32, operands rounded to nearest TF32):
                           0 off; 1 TF32, switching for the rest of the run to compensated 3xTF32
                           (hi*hi + hi*lo + lo*hi) once the relative KKT value is below refine_switch
                           or has not halved its best value for 100 iterations (TF32 rounding can
                           floor it above refine_switch); 2 always 3xTF32; -1 auto (= 1 when
                           p >= 128).  For p >= 256 the Grams (256 x 256 tiles) and the update
                           (256-row tiles) run on CTA pairs; 1 or 2 or-ed with PLAM_TC_SINGLE_CTA
                           keeps one CTA per tile.  Needs 16-byte aligned X and G with leading
                           dimensions that are multiples of 4, otherwise the CUDA-core Grams run */
  double refine_switch; /* relative KKT value below which the tensor-core kernels are compensated
                           (0: neither rule switches, plain TF32 throughout) */
  double feas_max;      /* > 0: the run stops with PLAM_ERR_DIVERGED once ||X^T X - I||_F exceeds it
                           (a penalty too small for PLAM lets X grow without bound; default 1e6);
                           0: only non-finite values stop it */
  int orth_metrics;     /* 1 (default): plam_solve also evaluates f, the relative KKT value and the
                           feasibility ||Q^T Q - I||_F of the orthonormalised output Q
                           (plam_info_t.f_orth, kkt_orth, feas_orth); 0: skipped (NaN) — the
                           feasibility alone is one more FP64 Gram of Q, n p^2 / 2 multiply-adds */
  double eta_min;       /* > 0: lower bound of every step-size parameter eta^k (eta0 included); 0: 1e-10 eta0.
                           The convergence analysis asks eta^k in an interval [eta_low, eta_up];
                           a lower bound caps the step 1/eta^k that the BB rules may take */
  double eta_max;       /* > 0: upper bound of eta^k; 0: 1e10 eta0.  eta_min <= eta_max when both > 0 */
} plam_params_t;

typedef struct {
  int kind;             /* PLAM_OBJ_* */
  const void* A;        /* DENSE, QAP: device, n x n symmetric, storage type, column-major */
  int64_t lda;          /* DENSE, QAP: leading dimension >= n */
  double alpha;         /* HARTREE1D: Hartree coupling alpha */
  double quad_scale;    /* HARTREE1D: q, the coefficient of tr(X^T L X) (1/4 Kohn-Sham, 1/2 Problem 1) */
  int nx, ny, nz;       /* STENCIL3D: grid, nx*ny*nz == n */
  const void* V;        /* STENCIL3D: device n-vector potential, storage type (may be NULL: V = 0) */
  plam_grad_fn grad;    /* CALLBACK: the user gradient (required) */
  void* grad_ctx;       /* CALLBACK: passed to grad unchanged */
  double xc;            /* HARTREE1D: exchange coefficient gamma of Problem 6, adding
                           -(3 gamma / 4) sum_i rho_i^{4/3} (0: none; the resident engine needs 0) */
  int64_t block;        /* HARTREE1D: rows per Dirichlet block of L; 0 (or >= n): one block of n rows.
                           With alpha or xc nonzero a block must have 1..64 rows (PLAM_ERR_INVALID
                           otherwise: L^{-1} rho is then formed block by block in shared memory) */
  const void* lin;      /* HARTREE1D: device n x p linear term G_lin (storage type, column-major,
                           leading dimension ldlin >= n, referenced like A), or NULL.  block != 0 or
                           lin != NULL selects the row-tile x column-group gradient kernels and
                           rules out the resident engine */
  int64_t ldlin;        /* HARTREE1D: leading dimension of lin */
  const void* Bq;       /* QAP: device, p x p symmetric, storage type, column-major */
  int64_t ldbq;         /* QAP: leading dimension of Bq (>= p) */
} plam_objective_t;

typedef struct {
  int iters;            /* updates performed so far (k) */
  int status;           /* plam_status_t of the run / step */
  int converged;        /* 1 when the relative KKT value fell below tol */
  int pad_;
  double f;             /* f(X^k) at the last evaluated iterate */
  double kkt_rel;       /* ||G - X Psi(G^T X)||_F / K0 at that iterate */
  double feas;          /* ||X^T X - I||_F at that iterate */
  double eta;           /* last eta used for an update */
  double K0;            /* ||G^0 - X^0 Psi(G^0^T X^0)||_F */
  double eta0;          /* eta at k = 0 */
  double f_orth;        /* f after the final orthonormalisation (NaN if not run; evaluated in the
                           storage precision: FP32 mode rounds the FP64 output to float first) */
  double kkt_orth;      /* relative KKT after the final orthonormalisation (likewise; NaN when
                           p x 16 storage-type values exceed 227 KB of shared memory) */
  double feas_orth;     /* ||Q^T Q - I||_F of the orthonormalised output (NaN with orth_metrics off) */
  double ms_iterations; /* plam_solve: device time of the iterations in ms (CUDA events on the handle's
                           stream; the kernel groups inside them: plam_time_kernels); NaN elsewhere */
  double ms_orth;       /* plam_solve: device time of the final orthonormalisation and its metrics in
                           ms (the paper's "Orth" category; 0 without one); NaN elsewhere */
} plam_info_t;

typedef struct plam_handle_s* plam_handle_t;

/* Fills *prm with the paper's defaults: PCAL, eq. (lambda2), beta = 1, ABB,
 * eta0 automatic, tol = 1e-8, maxit = 3000 (Section 5.1), FP64, one final
 * orthonormalisation, 16 iterations per graph. */
plam_status_t plam_default_params(plam_params_t* prm);

/* Creates a solver for problem size n x p (2p <= n, p >= 1) with the given
 * objective and parameters.  Allocates all device workspace (gradient,
 * residual history, split-K partials, p x p buffers, state) on the current
 * device.  The objective's device arrays are referenced, not copied: keep them
 * alive until plam_destroy.  `stream` is a cudaStream_t (NULL: default stream).
 * Errors: PLAM_ERR_INVALID, PLAM_ERR_NOMEM, PLAM_ERR_CUDA; *h is NULL then. */
plam_status_t plam_create(plam_handle_t* h, int64_t n, int64_t p, const plam_objective_t* obj,
                          const plam_params_t* prm, void* stream);

/* ---- Row-sharded solves (Section 5.4's parallel structure): the rows of X, G and R are
 * split into contiguous blocks over `size` ranks (processes, usually one per GPU).  Every
 * O(np) and O(np^2) kernel works on a rank's own rows; per iteration the ranks exchange the
 * reduced Grams [X^T X | X^T G] (2 p^2 doubles) and the column and Barzilai-Borwein dots
 * (3p + 7 doubles) through the caller's all-gather, each rank adds the gathered buffers in
 * rank order (so every rank holds the same sums bit for bit and takes the same step size
 * and stop decision), and the 3D stencil exchanges one z-plane of halo rows per neighbour.
 * The final orthonormalisation gathers X^T X the same way.
 *
 * allgather: recv (device, size * count doubles) receives every rank's send (device, count
 *            doubles) in rank order; all device work ordered on `stream`; returns 0 on success.
 * exchange:  (STENCIL3D only) sends send_lo (the first `count` halo values: this rank's first
 *            z-plane of every column, contiguous, storage type) to rank - 1 and send_hi (its
 *            last plane) to rank + 1, and receives rank - 1's last plane into recv_lo and
 *            rank + 1's first plane into recv_hi (the library leaves the buffers of a
 *            missing neighbour alone and uses zeros, the Dirichlet boundary, there).
 * A nonzero return of a callback stops the entry point with PLAM_ERR_CUDA. */
typedef int (*plam_allgather_fn)(void* ctx, const double* send, double* recv, int64_t count,
                                 void* stream);
typedef int (*plam_exchange_fn)(void* ctx, const void* send_lo, const void* send_hi, void* recv_lo,
                                void* recv_hi, int64_t count, void* stream);
typedef struct {
  int rank, size;                 /* this rank, number of ranks (>= 1) */
  int64_t row0;                   /* first global row of this rank's block */
  int64_t n_global;               /* rows of the whole problem (2p <= n_global) */
  plam_allgather_fn allgather;    /* required when size > 1 */
  plam_exchange_fn exchange;      /* required for STENCIL3D when size > 1 */
  void* ctx;                      /* passed to the callbacks unchanged */
} plam_comm_t;

/* A handle on this rank's n_local rows of a row-sharded problem (n_local >= 1; the objective
 * describes the rank's own rows).  Supported objectives:
 *   STENCIL3D  nx * ny * nz = n_local: the rank's z-slab of the global nx x ny grid, row0 a
 *              multiple of nx * ny.  X passed to the calls must have halo rows: for every
 *              column, the nx * ny rows before X and after X + n_local are valid memory that
 *              the library overwrites with the neighbours' planes (ldx >= n_local + 2 nx ny).
 *   HARTREE1D  with block b >= 1 (block-diagonal L, as Section 5.4 runs Problem 1; the blocks
 *              never cross ranks: row0 a multiple of b, and n_local a multiple of b on every
 *              rank but the last).
 * Others return PLAM_ERR_UNSUPPORTED.  The handle runs plain launches (graph_iters and the
 * resident engine do not apply: the callbacks run on the host between kernels) and skips
 * the output's f / KKT / feasibility report (orth_metrics is taken as 0).  plam_step,
 * pcal_step, plam_solve, plam_orthonormalize and plam_last_iteration apply (on local rows);
 * every rank must make the same sequence of calls. */
plam_status_t plam_create_sharded(plam_handle_t* h, int64_t n_local, int64_t p,
                                  const plam_objective_t* obj, const plam_params_t* prm,
                                  const plam_comm_t* comm, void* stream);

/* The engine plam_solve runs on this handle: PLAM_ENGINE_RESIDENT or
 * PLAM_ENGINE_GRAPH (graph_iters > 0), or 0 for direct launches. */
int plam_solve_engine(plam_handle_t h);

/* Releases every resource of the handle (synchronises its stream first). */
plam_status_t plam_destroy(plam_handle_t h);

/* Forgets the iteration history (k = 0, no Barzilai-Borwein pair, K0 and eta0
 * recomputed by the next step). */
plam_status_t plam_reset(plam_handle_t h);

/* One PLAM iteration (Algorithm 2): evaluates G, B, C = X^T G, the KKT value
 * and feasibility at X = X^k; if the KKT test passes (or k = maxit) X is left
 * unchanged and info->converged says why, else X is overwritten by X^{k+1}
 * (eq. PLAM-main) with Lambda from eq. (Lambda1).  X: device, storage type,
 * n x p, leading dimension ldx.  info may be NULL.  Returns PLAM_OK,
 * PLAM_ERR_DIVERGED (X keeps the last finite iterate) or an error. */
plam_status_t plam_step(plam_handle_t h, void* X, int64_t ldx, plam_info_t* info);

/* One PCAL iteration (Algorithm 3 with its column-wise closed form): as
 * plam_step, but Lambda from the handle's lambda_rule and every column of
 * X - R/eta scaled to unit 2-norm. */
plam_status_t pcal_step(plam_handle_t h, void* X, int64_t ldx, plam_info_t* info);

/* Runs the handle's variant from X (in place, storage type) until the relative
 * KKT value is below tol or maxit updates were made (Section 5.1), then, if
 * final_orth > 0 and Xout != NULL, writes the orthonormalised FP64 result
 * Q = X R^{-1}, X^T X = R^T R, to Xout (device, n x p, leading dimension ldo)
 * (Section 5.3).  X keeps the last iterate.  The loop runs without host
 * synchronisation inside a captured graph of graph_iters iterations; the
 * host reads the device stop flag once per graph launch.
 * Returns PLAM_OK, PLAM_ERR_NOT_CONVERGED (Xout still written), PLAM_ERR_DIVERGED,
 * PLAM_ERR_CHOLESKY or an error. */
plam_status_t plam_solve(plam_handle_t h, void* X, int64_t ldx, double* Xout, int64_t ldo,
                         plam_info_t* info);

/* Final orthonormalisation (Section 5.3; Eigen LLT in Section 5.4): B = X^T X
 * in FP64, Cholesky B = R^T R with diag(R) > 0, Xout = X R^{-1} in FP64;
 * `passes` = 2 repeats it on Xout (CholQR2).  X: device, storage type, n x p;
 * Xout: device FP64 n x p (may alias X only in FP64 mode).  If feas is not NULL
 * the host receives ||Xout^T Xout - I||_F.  Returns PLAM_ERR_CHOLESKY when a
 * pivot is not positive and finite (Xout is then undefined). */
plam_status_t plam_orthonormalize(plam_handle_t h, const void* X, int64_t ldx, double* Xout,
                                  int64_t ldo, int passes, double* feas);

/* Objective evaluation: G = grad f(X) (device, storage type, leading
 * dimension ldg) and, if f is not NULL, the host value f(X) (Section 5.2, Table
 * "cost" rows "evaluate function").  Used by the autograd wrapper and tests. */
plam_status_t plam_energy_grad(plam_handle_t h, const void* X, int64_t ldx, void* G, int64_t ldg,
                               double* f);

/* The energy as a forward / backward pair (Section 5.2 objectives), for an
 * automatic-differentiation wrapper.  No call synchronises the stream.
 *   plam_energy          *f_dev = f(X), f_dev a device double.
 *   plam_energy_backward G = s grad f(X), s = *scale_dev (a device double) or
 *                        1 when scale_dev is NULL; G: device, storage type,
 *                        leading dimension ldg (rows >= n are not written).
 * Both use the handle's workspace: calls on one handle must not overlap. */
plam_status_t plam_energy(plam_handle_t h, const void* X, int64_t ldx, double* f_dev);
plam_status_t plam_energy_backward(plam_handle_t h, const void* X, int64_t ldx,
                                   const double* scale_dev, void* G, int64_t ldg);

/* ---- Batched solves: many independent dense trace problems
 * f_b = 1/2 tr(X_b^T A_b X_b) (Problem 3, Section 5.2) of uneven sizes in ONE
 * persistent launch.  Each CTA takes problems from a device work queue (largest
 * n^2 p first) and runs the whole PLAM / PCAL loop of one problem with
 * block-level synchronisation; FP32 storage and products, FP64 p x p algebra,
 * and the FP64 Cholesky-QR of each final iterate.  The launch, the queue reset
 * and the copy of the results are captured once in a CUDA graph and replayed. */
typedef struct {
  int64_t n, p;         /* 1 <= p <= 64, 2p <= n */
  const void* A;        /* device float, n x n symmetric, column-major */
  int64_t lda;          /* >= n */
  void* X;              /* device float, n x p: the start on entry, the last iterate on return */
  int64_t ldx;          /* >= n */
  double* Q;            /* device FP64 n x p: orthonormalised output (NULL: not formed) */
  int64_t ldq;          /* >= n when Q is given */
} plam_batch_problem_t;

typedef struct plam_batch_s* plam_batch_t;

/* prm: precision must be PLAM_PREC_FP32; variant, lambda_rule, beta, eta rule,
 * eta_min, eta_max, tol and maxit apply to every problem (the other fields,
 * feas_max among them, are not used: a problem stops as diverged only on
 * non-finite values).  The problem array is copied; A, X and
 * Q stay owned by the caller and must outlive the batch.  The workspace (three
 * n x p float buffers per problem) is allocated here. */
plam_status_t plam_batch_create(plam_batch_t* b, const plam_batch_problem_t* probs, int count,
                                const plam_params_t* prm, void* stream);
/* Solves every problem; infos (host, count entries, may be NULL) receives each
 * problem's result in the layout of plam_info_t (status PLAM_OK when it
 * converged; f_orth, kkt_orth and the timings are NaN).  Returns PLAM_OK unless
 * a CUDA call failed. */
plam_status_t plam_batch_solve(plam_batch_t b, plam_info_t* infos);
/* The autotuner: times `iters` iterations of every problem for each row-block
 * height of the kernel's tiles (64, 128, 256) from the current X (restored
 * after each trial) and keeps the fastest; *tile_rows and *ms (may be NULL)
 * receive the choice and its time. */
plam_status_t plam_batch_autotune(plam_batch_t b, int iters, int* tile_rows, double* ms);
/* Fixes the row-block height (64, 128 or 256; default 128). */
plam_status_t plam_batch_set_tile(plam_batch_t b, int tile_rows);
plam_status_t plam_batch_destroy(plam_batch_t b);

/* The split-K tall-skinny Grams of one iteration (Table "cost": X^T X and
 * grad f^T X): B = X^T X and C = X^T G as FP64 p x p column-major device
 * matrices with leading dimension p.  Partial sums over row chunks go through
 * the handle's workspace and are reduced in a fixed order (bitwise
 * reproducible).  G may be NULL, then only B is formed. */
plam_status_t plam_grams(plam_handle_t h, const void* X, int64_t ldx, const void* G, int64_t ldg,
                         double* B, double* C);

/* Kernel attribution: runs up to `iters` iterations of the handle's variant on
 * X (in place, continuing the current run; call plam_reset for a fresh start)
 * without a graph, recording CUDA events on the handle's stream between the
 * kernel groups of each iteration.  ms[0..5] receive the average duration in
 * milliseconds of: the objective gradient, gram_partial, gram_finalize
 * (reduction and p x p multiplier step), update (R = G - XM with the column
 * dots), step_size, primal_update.  *done receives the iterations run (fewer
 * when the run stops).  The solver semantics are those of plam_solve. */
plam_status_t plam_time_kernels(plam_handle_t h, void* X, int64_t ldx, int iters, double* ms,
                                int* done);

/* The Grams of plam_grams (B = X^T X, and C = X^T G when G is not NULL; FP64
 * p x p column-major device outputs, leading dimension p) without a handle and
 * without allocating any device memory.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate -- applications whose
 * device memory belongs to another memory manager with a fixed budget, or
 * latency-critical loops where cudaMalloc's implicit device synchronisation is
 * not acceptable.  The split-K partial sums use an 8 MiB array that the
 * library reserves statically on every device that loads it, until the
 * process exits; requests with 2 p^2 partial sums of one chunk above that
 * (p > 1024 in FP32 mode, p > 724 in FP64 mode) return PLAM_ERR_INVALID.
 * precision: PLAM_PREC_FP64 (X, G double) or PLAM_PREC_FP32 (float).  The
 * first call in each CUDA context looks up the array's device address and
 * caches it under the context's id (do that first call before any stream
 * capture; after cudaDeviceReset the next call looks it up again).  The work
 * is ordered on `stream` and the call returns without synchronising.  All
 * calls share the one array: calls whose kernels overlap on the GPU race and
 * must be serialised by the caller.  Every error return leaves a message for
 * plam_last_error(). */
plam_status_t plam_grams_noalloc(int64_t n, int64_t p, int precision, const void* X, int64_t ldx,
                                 const void* G, int64_t ldg, double* B, double* C, void* stream);

/* Internals of the latest evaluated iterate X^k of the handle's current run,
 * for checking the kernels one by one (plam_step / pcal_step / the graph
 * engine; after a resident-engine solve the contents are unspecified):
 *   R        device, storage type, n x p, leading dimension ldr: the residual
 *            R^k = G - X M = grad_X L_beta(X^k, Lambda) of eq. S1 that the
 *            update kernel wrote (NULL: not copied);
 *   M        device, storage type, p x p column-major (leading dimension p):
 *            M = Lambda - beta (B - I) as the update consumed it (eqs.
 *            Lambda1 / lambda2, S1; NULL: not copied);
 *   colsums  host, 3p doubles: ||X_i||^2 (p), <X_i, R_i> (p), ||R_i||^2 (p),
 *            the reduced column dots that give PCAL's column norms (Algorithm 3);
 *   bb       host, 3 doubles: <S,S>, <S,Y>, <Y,Y> with S = X^k - X^{k-1},
 *            Y = R^k - R^{k-1} (Section 5.1; zeros at k = 0).
 * Synchronises the handle's stream.  PLAM_ERR_INVALID before any iterate was
 * evaluated (after plam_create or plam_reset). */
plam_status_t plam_last_iteration(plam_handle_t h, void* R, int64_t ldr, void* M, double* colsums,
                                  double* bb);

/* Checkpoint and resume of a run's iteration state (everything the next iteration reads besides
 * X: the iteration counter and stop state, K0, eta0, the step size, the previous residual
 * R^{k-1} and the previous column scales for the Barzilai-Borwein differences, the latched
 * compensated phase, the dual-ascent multiplier).  plam_state_bytes gives the size of the
 * host buffer; plam_get_state copies the state to it (synchronising the stream);
 * plam_set_state loads one taken from a handle of the same n, p, precision and variant (the
 * buffer's header is checked: PLAM_ERR_INVALID otherwise).  With the X of the checkpointed
 * iterate, plam_step / pcal_step then continue the run exactly (bit for bit) where it stood;
 * plam_solve always starts a fresh run.  The history records are not part of the state. */
size_t plam_state_bytes(plam_handle_t h);
plam_status_t plam_get_state(plam_handle_t h, void* buf, size_t bytes);
plam_status_t plam_set_state(plam_handle_t h, const void* buf, size_t bytes);

/* Copies up to `cap` per-iteration records (k, f, kkt_rel, feas, eta as 5
 * doubles each, in that order) of the current run to host memory `out`;
 * *count receives the number written. */
plam_status_t plam_history(plam_handle_t h, double* out, int cap, int* count);

/* Number of kernels this handle launched since creation (each graph replay
 * counts its kernel nodes). */
int64_t plam_kernel_launches(plam_handle_t h);

/* Message of the last PLAM_ERR_CUDA on this thread, and of any error returned by
 * plam_grams_noalloc (static storage; not cleared by successful calls). */
const char* plam_last_error(void);

/* Library version as major*10000 + minor*100 + patch. */
int plam_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PLAM_H_ */
