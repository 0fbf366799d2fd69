/*
 * rbicgstab.h -- C ABI of the GB300 recycling-BiCGSTAB library (librbicgstab.so).
 *
 * The library solves sequences of sparse non-symmetric systems
 *     A^(iota) x^(iota,kappa) = b^(iota,kappa)                      (Sec. 1, eq. (1.1))
 * with Alg. 2 (RBiCGSTAB, Sec. 4) on one CUDA device, carrying a recycle space
 * U (and U~) from one system to the next (Sec. 3, definition of C = A U,
 * C~ = A^T U~).  Plain BiCGSTAB is the same solver with an empty recycle space.
 *
 * Conventions for every entry point
 *   - Return value: RB_OK (0) on success, a warning (> 0) or an error (< 0);
 *     rbicgstab_error_string() names it.  On an error nothing the caller owns
 *     is modified except where stated.
 *   - `where` says where caller pointers live: RB_HOST (pageable or pinned host
 *     memory) or RB_DEVICE (device memory on the handle's device).
 *   - Every setter COPIES its inputs into library-owned device memory; no
 *     caller pointer is retained after the call returns.
 *   - Calls are ordered on opts.cuda_stream (NULL = the legacy default stream)
 *     and synchronise that stream before returning.
 *   - A handle is not thread-safe; separate handles are independent.
 *   - Matrices are CSR with int32 row pointers and column indices (0-based;
 *     column indices need not be sorted) and float64 values; n, nnz < 2^31.
 *   - Dense n x k blocks (U, U~) are column-major with leading dimension
 *     ld >= n.
 */
#ifndef RBICGSTAB_H
#define RBICGSTAB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define RB_OK                 0
#define RB_WRECYCLE_RANK      1   /* warning: C~^T C numerically singular, k reduced */
#define RB_EINVAL            -1   /* bad argument (NULL pointer, bad enum, k too large) */
#define RB_EDIM              -2   /* dimension mismatch / no matrix set */
#define RB_EBADCSR           -3   /* malformed CSR (row_ptr not monotone, column out of range) */
#define RB_ENONFINITE        -4   /* NaN or Inf in an input */
#define RB_ENOMEM            -5   /* device allocation failed */
#define RB_ECUDA             -6   /* a CUDA runtime call failed */
#define RB_ENOTCONV          -7   /* max_itn reached; x holds the last iterate */
#define RB_EBREAKDOWN_RHO    -8   /* (r~_0, r) = 0 or (r~_0, q) = 0 after redraws (Alg. 2) */
#define RB_EBREAKDOWN_OMEGA  -9   /* (t, t) = 0 with s != 0, or omega = 0 */
#define RB_ETIMEOUT         -10   /* a bounded device-side wait expired */

/* ---- enums --------------------------------------------------------------- */
#define RB_HOST    0
#define RB_DEVICE  1

#define RB_FP64    0   /* FP64 storage and arithmetic throughout */
#define RB_MIXED   1   /* FP32 inner RBiCGSTAB with FP64 residual replacement; a solve
                         whose FP32 iteration stalls, breaks down or overflows is
                         finished in FP64 from its current x */

#define RB_RECYCLE_NONE          0  /* plain BiCGSTAB (U ignored) */
#define RB_RECYCLE_FIXED         1  /* use U, U~ as given; never change them */
#define RB_RECYCLE_UPDATE_FIRST  2  /* update U during the first solve after each set_matrix */
#define RB_RECYCLE_UPDATE_ALL    3  /* update U during every solve */

#define RB_KMAX  64   /* largest supported recycle dimension */

typedef struct rb_ctx* rb_handle;

/* Options (copied at create).  Zero fields take the stated defaults. */
typedef struct {
  int32_t  k_max;          /* recycle dimension k (Sec. 6.2 uses 20); 0..RB_KMAX       */
  int32_t  cycle_s;        /* cycle length s of the recycle update (Sec. 6.2: 25); 0->25 */
  int32_t  max_itn;        /* iteration cap (Alg. 2); 0 -> min(n, 20000)               */
  int32_t  precision;      /* RB_FP64 or RB_MIXED                                      */
  int32_t  recycle_mode;   /* RB_RECYCLE_*                                             */
  int32_t  update_cycles;  /* cycles per solve that update U; 0 = every cycle          */
  int32_t  poll;           /* iterations per host convergence check; 0 = automatic     */
  int32_t  reserved;
  double   tol;            /* relative residual tolerance ||r|| <= tol ||b||; 0->1e-8  */
  uint64_t shadow_seed;    /* SplitMix64 seed of r~_{-1} (Alg. 2); 0 -> 0x5EED         */
  void*    cuda_stream;    /* cudaStream_t the calls are ordered on (NULL = default)   */
} rb_opts;

/* Per-solve statistics. */
typedef struct {
  int32_t iters;           /* Alg. 2 iterations (a half step counts as one)            */
  int32_t status;          /* same code the call returned                              */
  int32_t k_used;          /* recycle columns in use after biorthogonalisation         */
  int32_t seeds_used;      /* shadow draws (1 unless (r_0, r~_0) = 0 forced a redraw)  */
  int64_t matvecs;         /* A-products inside the iteration (2 per iteration)        */
  int64_t matvecs_setup;   /* columns of C = A U and C~ = A^T U~ formed for this solve */
  int64_t matvecs_check;   /* true-residual products                                   */
  int32_t cycles;          /* recycle-update cycles performed                          */
  int32_t outer;           /* RB_MIXED: FP64 true-residual checks (residual            */
                           /* replacements and restarts); else 1                       */
  double  relres_rec;      /* ||r_i|| / ||b|| of the recursive residual                */
  double  relres_true;     /* ||b - A x|| / ||b|| recomputed in FP64 after x - U x_c   */
  double  ms_total;        /* wall time of the call (CUDA events)                      */
  double  bytes_model;     /* algorithmic HBM bytes of the iterations                  */
  double  ms_update;       /* host wall time spent in recycle-space updates (cycle
                              Gram/eig/rebuild and the new space's recycle setup)      */
} rb_stats;

/* Create a solver handle on the current CUDA device.  *h receives the handle.
 * Errors: RB_EINVAL (NULL or out-of-range option), RB_ECUDA, RB_ENOMEM. */
int rbicgstab_create(rb_handle* h, const rb_opts* opts);

/* Release every device resource of the handle.  NULL is accepted. */
int rbicgstab_destroy(rb_handle h);

/* Set the system matrix A^(iota) (Sec. 1, eq. (1.1)): CSR, n rows, nnz entries.
 * The matrix is validated on the device (monotone row_ptr, 0 <= col < n,
 * finite values), re-laid out as SELL-32 slices, and its transpose is built
 * (needed for C~ = A^T U~).  An existing recycle space U, U~ is kept and its
 * C, C~, D_c are recomputed for the new matrix (Sec. 3).
 * Errors: RB_EINVAL, RB_EBADCSR, RB_ENONFINITE, RB_ENOMEM, RB_ECUDA. */
int rbicgstab_set_matrix(rb_handle h, int64_t n, int64_t nnz, const int32_t* row_ptr,
                         const int32_t* col, const double* val, int where);

/* Replace only the values of the current matrix (same pattern, same order as
 * the last set_matrix call).  Cheaper than set_matrix for sequences such as
 * A^(i) = A0 + sigma_i A1 (Sec. 6.1).  Errors: RB_EDIM (no matrix), RB_ENONFINITE. */
int rbicgstab_set_values(rb_handle h, const double* val, int where);

/* Set the recycle space (Sec. 3): U (n x k) and U~ (n x k; NULL means U~ = U,
 * the right-only variant of Sec. 5), column-major with leading dimension ld.
 * Forms C = A U, C~ = A^T U~, biorthogonalises them by an SVD of C~^T C
 * (so D_c = C~^T C is diagonal and positive) and forms C-hat = C~ D_c^{-1}
 * (Sec. 3, eq. (3.4)).  k = 0 clears the space.  Needs a matrix.
 * Returns RB_WRECYCLE_RANK when columns were dropped (k_used < k).
 * Errors: RB_EINVAL (k > k_max), RB_EDIM, RB_ENONFINITE. */
int rbicgstab_set_recycle(rb_handle h, int32_t k, const double* U, const double* Ut,
                          int64_t ld, int where);

/* Copy the current (biorthogonalised) recycle space out: *k receives k_used;
 * U and Ut (either may be NULL) receive n x k_used column-major blocks with
 * leading dimension ld.  Errors: RB_EINVAL. */
int rbicgstab_get_recycle(rb_handle h, int32_t* k, double* U, double* Ut, int64_t ld,
                          int where);

/* Solve A x = b with Alg. 2 using the current recycle space.  x holds the
 * initial guess x_{-1} on entry (eq. (3.5)) and the solution on return
 * (after the final correction x = x - U x_c).  In the RB_RECYCLE_UPDATE_* modes the recycle
 * space is replaced by the harmonic-Ritz update built from this solve.
 * st may be NULL.  On RB_ENOTCONV / RB_EBREAKDOWN_* x holds the last iterate.
 * Errors: RB_EDIM (no matrix), RB_ENONFINITE (NaN/Inf in b or x), RB_ECUDA. */
int rbicgstab_solve(rb_handle h, const double* b, double* x, int where, rb_stats* st);

/* Maximum number of right-hand sides of one blocked solve. */
#define RB_MAX_RHS 4

/* Blocked solve of A X = B for 1 <= nrhs <= RB_MAX_RHS right-hand sides of
 * the same matrix (a practical extension: the paper solves one system at a
 * time).  Column i of B and X (column-major, leading dimension ld >= n when
 * nrhs > 1) is one system; X holds the initial guesses on entry and the
 * solutions on return.  Every system runs Alg. 2 with its own iterates and
 * scalars, the same recycle space and the same shadow vector r~_0; their
 * iterations share each pass over A, C and C-hat, and a system that has
 * converged stops updating while the others go on.  Each system's iterates
 * are those rbicgstab_solve would compute for it alone, up to the rounding
 * of the dot products and of a reseeded shadow (when (r~_0, r_0) = 0 for one
 * system, all take the next seed).  In the RB_RECYCLE_UPDATE_* modes the
 * update is built from the first system's Krylov vectors.  st, if not NULL,
 * receives nrhs records (cycles, matvecs_setup and ms_update describe the
 * whole call; ms_total is the call's duration).  Returns RB_OK when every
 * system converged, else the first system's non-OK status.  Errors as
 * rbicgstab_solve, plus RB_EINVAL for nrhs outside 1..RB_MAX_RHS or ld < n. */
int rbicgstab_solve_block(rb_handle h, int32_t nrhs, const double* B, double* X, int64_t ld,
                          int where, rb_stats* st);

/* Alg. 1 (RBiCG, Sec. 4): the primary system A x = b and the dual system
 * A^T x~ = b~ solved together with the handle's recycle space (U, U~ as given
 * to rbicgstab_set_recycle, or U~ = U; C = A U and C~ = A^T U~ biorthogonal,
 * C-hat = C~ D_c^{-1}, C-check = C D_c^{-1}, eq. (3.4)), in FP64 whatever the
 * handle's precision.  b, b~ and x, x~ are n-vectors (host or device per
 * `where`); bt may be NULL, and then the shadow vector r~_{-1} of Alg. 2
 * (seed opts.shadow_seed) is the dual right-hand side.  x and xt hold the
 * initial guesses x_{-1}, x~_{-1} on entry (eq. (3.5) forms x_0, r_0, x~_0,
 * r~_0) and the solutions after the final correction on return.  When (r_0, r~_0) = 0,
 * x~_{-1} is replaced by the shadow vector (seed + 0, 1, 2) and the dual start
 * formed again.  Converged when ||r_i|| <= tol ||b|| and
 * ||r~_i|| <= tol ||b~|| on the recursive residuals.  st and st_dual, if not
 * NULL, receive the primary and the dual system's records (iters, status and
 * matvecs are shared; relres_* are each system's own; seeds_used counts the
 * dual starts drawn).  The recycle space is not updated.  Returns RB_OK, or
 * RB_EBREAKDOWN_RHO ((p~_i, q_i) = 0 or (r~_i, r_i) = 0), RB_ENOTCONV,
 * RB_ENONFINITE (NaN/Inf in b, b~, x, x~ or during the iteration), with the
 * last iterates in x, xt.  Errors: RB_EDIM (no matrix), RB_EINVAL, RB_ECUDA. */
int rbicg_solve(rb_handle h, const double* b, const double* bt, double* x, double* xt, int where,
                rb_stats* st, rb_stats* st_dual);

/* y = A v (transpose = 0) or y = A^T v (transpose = 1) with the library's
 * FP64 SpMV kernels; v and y have n entries.  Errors: RB_EDIM, RB_EINVAL. */
int rbicgstab_apply(rb_handle h, const double* v, double* y, int transpose, int where);

/* out_e = scale * u_i * v_j for every entry e = (i, j) of the matrix's
 * sparsity pattern, in the CSR order given to rbicgstab_set_matrix (nnz
 * values).  With u = lam, v = x and scale = -1 this is the gradient
 * dL/dA_ij = -lam_i x_j of a functional L of the solution of A x = b, lam the
 * solution of the dual system A^T lam = dL/dx (Sec. 2's A^* x~ = b~; solve
 * it with rbicg_solve).  u, v (n entries) and out (nnz entries) are device
 * pointers (where = RB_DEVICE; RB_HOST is rejected with RB_EINVAL).
 * Errors: RB_EINVAL (null pointer, host memory, non-finite scale), RB_EDIM
 * (no matrix), RB_ECUDA. */
int rbicgstab_pattern_outer(rb_handle h, const double* u, const double* v, double scale, double* out,
                            int where);

/* The singular value decomposition used to biorthogonalise C and C~ (the
 * host step of the recycle setup; Sec. 3 requires C~^T C diagonal with positive
 * entries): M = C~^T C (k x k, column-major) = P diag(sigma) Q^T with P, Q
 * orthogonal (k x k, column-major) and sigma descending (k entries); the
 * library then rotates U <- U Q, C <- C Q, U~ <- U~ P, C~ <- C~ P.  One-sided
 * Jacobi; pure host code, needs no device.  Errors: RB_EINVAL (k < 1 or
 * k > 256, null pointer), RB_ENONFINITE (non-finite entry of M). */
int rbicgstab_svd_small(int32_t k, const double* M, double* P, double* sigma, double* Q);

/* Harmonic-Ritz selection on the host (the small dense step of the recycle
 * update, run between cycles of s iterations, Sec. 6.2): given G = Z^T Z and
 * H = Z^T W (m x m, column-major) for a subspace W with Z = A W, return in Y
 * (m x k, column-major, ld = m) the coefficients of the k harmonic Ritz
 * vectors of smallest |theta| (G y = theta H y), a complex pair as
 * [Re y, Im y], and their values in theta_re/theta_im (k each, may be NULL).
 * *k_used receives the number of columns written.  Pure host code; needs no
 * device.  Errors: RB_EINVAL. */
int rbicgstab_harmonic_ritz(int32_t m, const double* G, const double* H, int32_t k,
                            double* Y, double* theta_re, double* theta_im, int32_t* k_used);

/* Benchmark helper: run `reps` iterations of the fused passes from a fresh
 * start on the nrhs right-hand sides in B (column-major, leading dimension
 * ld; x_{-1} = 0, convergence test disabled), each pass launched on its own
 * between CUDA events on the handle's stream, and write the average duration
 * in milliseconds of passes P1..P5 to ms[0..4] (ms[3] = 0 when k = 0: plain
 * BiCGSTAB has no separate P4).  The iterates are left in an unspecified
 * state; call rbicgstab_solve afterwards as usual.  Returns a breakdown code
 * if the iteration broke down during timing.  Errors: RB_EINVAL (reps
 * outside 1..1000, nrhs outside 1..RB_MAX_RHS, ld < n), RB_EDIM. */
int rbicgstab_time_passes(rb_handle h, int32_t nrhs, const double* B, int64_t ld, int where,
                          int32_t reps, double* ms);

/* Residual without allocation: r = b - A x and *rnorm2 = ||r||^2 for an n x n
 * CSR matrix given by device pointers (row_ptr[n+1], col[nnz], val[nnz]), with
 * x, b, r (n entries each) and rnorm2 (one double) also in device memory.
 * The paper has no counterpart: this is for callers that cannot allocate
 * device memory (a framework that owns the allocator and forbids cudaMalloc,
 * work about to be captured into a CUDA graph, a service whose device memory
 * is sized once at start-up).  Nothing is allocated and no handle is needed:
 * the kernel's scratch (1024 block and 65 group partial sums and the
 * completion tickets, about 9 KB) is a fixed device array that every GPU loading the library
 * keeps until the process exits.  The first call on a device looks up that
 * array's address (which can load the module): make it before any stream
 * capture.  The call is ordered on `cuda_stream` (NULL = legacy default
 * stream) and does not synchronise; outputs are ready when the stream gets
 * there.  All calls share the one scratch array, so calls whose kernels can
 * overlap on the GPU (different streams, or different host threads) race;
 * serialise them.  The CSR is not validated (pass a matrix that
 * rbicgstab_set_matrix accepts).  Errors: RB_EINVAL (n <= 0, n > 2^31 - 1,
 * or a NULL pointer), RB_ECUDA. */
int rbicgstab_residual_noalloc(int64_t n, const int32_t* row_ptr, const int32_t* col,
                               const double* val, const double* x, const double* b, double* r,
                               double* rnorm2, void* cuda_stream);

/* ---- batched solves of many independent systems ------------------------
 * A batch holds S independent systems A_i x_i = b_i of uneven sizes n_i (the
 * sequence of Sec. 1 for many parameter samples at once), each with its own
 * optional fixed recycle space U_i of k <= 16 columns (U~_i = U_i, the
 * right-only variant of Sec. 5; Sec. 3 setup per system).  One solve runs
 * Alg. 2 for all systems together: every pass of an iteration is one
 * persistent kernel over a work list of tiles (slice ranges inside one
 * system) with per-system dot products, scalars and convergence; iterations
 * are captured as a CUDA graph; the tile size and CTAs per SM are chosen by
 * an autotuner at the first solve after a matrix or space change.
 * opts: tol, max_itn, poll, shadow_seed, cuda_stream, precision (RB_FP64, or
 * RB_MIXED: FP32 iteration with Dot2 dot products and FP64 residual
 * replacement per system, as rbicgstab_solve's mixed mode: a system whose
 * FP32 iteration stalls, breaks down or overflows is finished in FP64 from
 * its current x; converged when ||b_i - A_i x_i|| <= tol ||b_i||), k_max <=
 * 16 (0: plain BiCGSTAB only).  Errors as for the single-system calls. */
typedef struct rb_batch_ctx* rb_batch;
int rbicgstab_batch_create(rb_batch* h, const rb_opts* opts);
int rbicgstab_batch_destroy(rb_batch h);
/* nsys systems, host arrays: n[i] rows each; row_ptr = the systems' CSR row
 * pointers one after another (n[i] + 1 entries each, each starting at 0);
 * col = their local column indices and val their values, one after another
 * (sum of the systems' nonzeros).  The pattern is copied; the values are the
 * first set_values.  Errors: RB_EINVAL, RB_EBADCSR, RB_ENONFINITE. */
int rbicgstab_batch_set_matrices(rb_batch h, int32_t nsys, const int64_t* n, const int32_t* row_ptr,
                                 const int32_t* col, const double* val);
/* New values on the same patterns (the layout of set_matrices' val). */
int rbicgstab_batch_set_values(rb_batch h, const double* val, int where);
/* k columns for every system: system i's n_i x k column-major block follows
 * system i-1's (sum_i n_i * k doubles).  k = 0 clears.  The setup runs at
 * the next solve. */
int rbicgstab_batch_set_recycle(rb_batch h, int32_t k, const double* U, int where);
/* b, x: sum_i n_i doubles, system after system; x holds x_{-1} on entry and
 * the solutions on return; st: nsys entries (may be NULL), per system
 * (iters summed over refinement restarts, outer = restarts + 1, k_used, the
 * recursive and FP64 true relative residuals; ms_total of the whole batch).
 * Returns RB_OK when every system converged, else the first system's
 * failure code (every system's status is in st); RB_ETIMEOUT when the
 * host's iteration loop runs past every system's max_itn without all of
 * them reporting done (a safeguard: each system stops at its max_itn). */
int rbicgstab_batch_solve(rb_batch h, const double* b, double* x, int where, rb_stats* st);
/* The work list the autotuner chose: slices per tile, CTAs per SM, tiles,
 * and the tuned time of one SpMV + projection pass (ms). */
int rbicgstab_batch_info(rb_batch h, int32_t* tile_slices, int32_t* ctas_per_sm, int32_t* ntiles, double* tune_ms);

/* The dual system A^T lam = g (the dual system of Sec. 2, real arithmetic):
 * Alg. 2 on A^T with the recycle space's roles swapped, right space U~ and
 * left space U, which reuses the products C~ = A^T U~ and C = A U of the
 * setup (Sec. 3).  This is the adjoint solve of a gradient: for
 * L(x(b, A)), lam = A^-T dL/dx gives dL/db = lam and dL/dA_ij = -lam_i x_j.
 * FP64 and with the space held fixed, whatever the handle's precision and
 * recycle mode.  g, lam: n doubles on RB_HOST or RB_DEVICE; lam holds the
 * initial guess on entry and the solution on return; st as for
 * rbicgstab_solve.  Errors as for rbicgstab_solve. */
int rbicgstab_solve_adjoint(rb_handle h, const double* g, double* lam, int where, rb_stats* st);

/* Recycled BiCGstab(l) (Sleijpen and Fokkema, 1993): the breakdown-robust
 * variant of Alg. 2 behind the paper's remark on omega = 0 (Sec. 4) and its
 * outlook (Sec. 7).  The iteration runs on the projected operator
 * (I - C C-hat^T) A of Sec. 3 from the start of eq. (3.5) with the handle's
 * current recycle space held fixed (no update, whatever the recycle mode);
 * each outer step takes l BiCG steps and then minimises the residual over
 * l directions, so the stabilising polynomial no longer has to take
 * BiCGSTAB's degree-1 steps (whose omega collapses on nearly skew
 * operators).  l = 1 is mathematically Alg. 2.  FP64 throughout, whatever
 * the handle's precision.  b, x: n doubles on RB_HOST or RB_DEVICE; x holds
 * x_{-1} on entry and the solution on return.  st (may be NULL): iters =
 * BiCG steps (l per outer step), outer = outer steps, matvecs, relres of the
 * recursive and the true residual.  Converged when ||r|| <= tol ||b|| after
 * an outer step.  Returns RB_OK, RB_ENOTCONV (max_itn BiCG steps),
 * RB_EBREAKDOWN_RHO ((r~_0, r_j) or (r~_0, u_{j+1}) = 0),
 * RB_EBREAKDOWN_OMEGA (rank-deficient residual block or omega = 0),
 * RB_ENONFINITE, RB_EINVAL (l outside 1..8), RB_EDIM, RB_ECUDA. */
int rbicgstab_solve_l(rb_handle h, int32_t ell, const double* b, double* x, int where, rb_stats* st);

/* Gram step of the recycle update (the harmonic-Ritz update after each cycle,
 * Sec. 6.2; the selection rule is the harmonic-Ritz reading of that update):
 * G = Z^T Z and H = Z^T W for the FP32 column blocks of the mixed path,
 * W = [Y, P, S] and Z = [AY, AP, AS] (AP = A P etc.), m = ky + nit + ns
 * columns each.  Every block is on the device, column-major with leading
 * dimension ld (a multiple of 4, >= n, 16-byte aligned columns); Y and AY
 * have ky <= kcap columns, P, AP nit <= scap, S, AS ns <= scap (kcap, scap:
 * the recycle dimension and cycle length, which fix the tile layout).
 * G, H: host arrays of m x m doubles, column-major; G is symmetric.
 * path: RB_GRAM_AUTO uses the tensor cores (tcgen05, TF32 pairs, FP64
 * sums over CTAs) when the layout fits (2 * (r8(kcap) + 2 r8(scap)) <= 224,
 * r8 = round up to 8), else the CUDA-core kernel; RB_GRAM_CUDACORE forces
 * the latter, RB_GRAM_TENSOR the former (RB_EINVAL if it does not fit).
 * This is the kernel the solver runs between cycles; the entry point exists
 * so that it can be checked and timed on its own.  It allocates its own
 * scratch, runs on cuda_stream and synchronises it.  ms_kernel (may be NULL)
 * receives the device time of the Gram kernels alone (CUDA events on
 * cuda_stream around them, scratch allocation excluded).  Errors: RB_EINVAL
 * (arguments, m > 90), RB_ENOMEM, RB_ECUDA, RB_ETIMEOUT (a bounded device
 * wait of the tensor-core kernel expired; outputs undefined). */
#define RB_GRAM_AUTO     0
#define RB_GRAM_CUDACORE 1
#define RB_GRAM_TENSOR   2
int rbicgstab_update_gram(int64_t n, int64_t ld, int32_t ky, int32_t nit, int32_t ns, int32_t kcap,
                          int32_t scap, const float* Y, const float* AY, const float* P, const float* AP,
                          const float* S, const float* AS, double* G, double* H, int32_t path,
                          void* cuda_stream, double* ms_kernel);

/* Layout statistics of the current matrix A on the device (SELL-32, slices of
 * 32 rows): the number of slices and of stencil slices, those whose rows use
 * no more distinct column offsets (col - row) than the slice's longest row
 * and whose gathers stay inside the matrix; the fused SpMV passes form their
 * column indices from per-slice offsets there instead of loading them.
 * Errors: RB_EINVAL (NULL argument), RB_EDIM (no matrix). */
int rbicgstab_sell_stats(rb_handle h, int64_t* nslices, int64_t* stencil_slices);

/* Self-test of the bounded device wait (failure detection without a GPU
 * fault).  The kernels that wait on the copy engine or the tensor cores
 * through mbarriers give up after a time limit instead of hanging, leave
 * normally and report RB_ETIMEOUT.  This call runs that same wait in one
 * block on an mbarrier of one arrival: complete != 0 makes a thread arrive
 * first (returns RB_OK); complete == 0 leaves the barrier incomplete, so the
 * wait gives up after limit_ms (0 < limit_ms <= 1000, converted to SM clock
 * cycles at the rated clock) and the call returns RB_ETIMEOUT with the
 * context usable.  *waited_ms (may be NULL) receives the kernel's duration.
 * Current device, legacy default stream, synchronous.  Errors: RB_EINVAL,
 * RB_ENOMEM, RB_ECUDA. */
int rbicgstab_wait_selftest(int32_t complete, double limit_ms, double* waited_ms);

/* Number of CUDA kernels this library has launched in the process so far
 * (each graph replay adds the kernels its graph holds).  Thread-safe. */
long long rbicgstab_kernel_launches(void);

/* Name of a status code (static string). */
const char* rbicgstab_error_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* RBICGSTAB_H */
