/*
 * emin.h -- C ABI of the GB300 energy-minimisation prolongation library.
 *
 * The library minimises the energy tr(P^T A P) of an AMG prolongation P on a
 * fixed sparsity pattern subject to the near-kernel constraint P B_c = B
 * (Eqs. (trace), (inKern), (Constr) of Janna, Franceschini, Schroder and
 * Olson, "Parallel Energy-Minimization Prolongation for Algebraic
 * Multigrid"), with the restricted Jacobi-preconditioned conjugate gradient
 * of Algorithm 3 after the set-up of Algorithm 2.  Every row of P is free
 * (f = 0 in Eq. (11blk)); the paper's classical form P = [W; I] is the
 * special case in which some rows are fixed.
 *
 * Conventions shared by every call:
 *   - Indices are 32-bit signed ints; sparse matrices are CSR with row
 *     pointers of length nrows+1 starting at 0 and column indices sorted
 *     strictly ascending within each row (no duplicates).
 *   - Floating-point inputs and outputs are IEEE double.  Dense blocks are
 *     row-major.  "Values on P's pattern" means an array of nnz(P) doubles
 *     in CSR order of P.
 *   - A pointer argument is a host pointer unless the call's `on_device` /
 *     `inputs_on_device` flag is 1, in which case it is a device pointer of
 *     the context's device.  The caller keeps ownership of its buffers; the
 *     library keeps no caller pointer after a call returns.
 *   - All device work is ordered on the stream given at creation.  Calls
 *     that return host results (status, scalars, host outputs) synchronise
 *     that stream before returning; emin_iterate synchronises once at its
 *     end.
 *   - Every call returns an emin_status.  Device-detected conditions
 *     (breakdown, invalid input found on the device) are recorded in the
 *     context, reported by the call that detects them and by later calls.
 *     The library never calls exit, abort or __trap.  A context in an error
 *     state can always be destroyed.
 */
#ifndef EMIN_H
#define EMIN_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct emin_ctx emin_ctx; /* opaque, owned by the library */

typedef enum {
    EMIN_OK = 0,
    EMIN_ERR_ARG = -1,       /* invalid argument or unsupported size          */
    EMIN_ERR_PATTERN = -2,   /* CSR row pointers / columns invalid, unsorted, */
                             /* duplicated or out of range                    */
    EMIN_ERR_RANK = -3,      /* m_i < k or Gram matrix of a row not SPD       */
                             /* (strict rank policy)                          */
    EMIN_ERR_DIAG = -4,      /* A(i,i) missing or not positive                */
    EMIN_ERR_BREAKDOWN = -5, /* y^T K y <= 0 or a non-finite scalar in CG     */
    EMIN_ERR_CUDA = -6,      /* a CUDA runtime call failed                    */
    EMIN_ERR_NOMEM = -7,     /* device or pinned host allocation failed       */
    EMIN_ERR_TIMEOUT = -8,   /* reserved: a bounded device wait gave up       */
    EMIN_ERR_STATE = -9      /* call not valid in the context's state         */
} emin_status;

enum { EMIN_FP64 = 0,   /* every step in IEEE double                           */
       EMIN_MIXED = 1   /* A, P and the masked products in float; Gram         */
                        /* factorisation, trace/step reductions and the final  */
                        /* constraint-restoring projection in double           */
};
/* Preconditioners of Section 3.4.  EMIN_JACOBI: M_1, the Jacobi scaling of
 * Pi_B K Pi_B (Theorem 1).  EMIN_SGS: M_2 = Z^T M_SGS^{-1} Z, the projected
 * block symmetric Gauss-Seidel, M_SGS^{-1} = (L + D)^{-T} D (L + D)^{-1} with
 * K = L + D + L^T in the row-wise order of p (per column block of P, rows in
 * increasing order), applied as z = Pi_B M_SGS^{-1} r.  EMIN_SGS builds a
 * plan on the host at create (copies of both patterns; time and memory grow
 * with the products inside the column blocks) and fails with EMIN_ERR_ARG
 * when one column of P has more than 65,535 rows or more than 65,535
 * couplings in one sweep, or when the values of one group of columns with
 * the same rows need more than 96 KB (emin_last_error says which). */
enum { EMIN_JACOBI = 0, EMIN_SGS = 1 };
enum { EMIN_RANK_STRICT = 0, EMIN_RANK_PINV = 1 };

typedef struct {
    int precision;    /* EMIN_FP64 or EMIN_MIXED                               */
    int precond;      /* EMIN_JACOBI or EMIN_SGS                               */
    int rank_policy;  /* EMIN_RANK_STRICT: a rank-deficient row is an error;   */
                      /* EMIN_RANK_PINV: pseudo-inverse of that row's Gram     */
                      /* matrix (the SVD branch of Algorithm 2), counted in    */
                      /* emin_stats                                            */
    int checks;       /* 1: bounds checks in the kernels that gather through  */
                      /* the plan (masked products, SGS sweeps, plan builds): */
                      /* an index outside its array is not dereferenced, and  */
                      /* the call returns EMIN_ERR_PATTERN (sticky); results  */
                      /* are otherwise bit-identical to checks = 0, which     */
                      /* runs unchecked kernels (the default)                 */
    void *stream;     /* cudaStream_t; NULL = legacy default stream            */
} emin_opts;

/* Fill *opts with the defaults: FP64, Jacobi, strict rank, stream NULL. */
void emin_default_opts(emin_opts *opts);

/*
 * Create a context for one minimisation problem and run the set-up
 * (Algorithm 2 and the first line of Algorithm 3).
 *   n, nc, k     rows of P (= order of A), columns of P, near-kernel vectors
 *                (1 <= k <= 8).
 *   A_*          n x n symmetric matrix in CSR (A_val: nnz(A) doubles); every
 *                row must hold a positive diagonal entry.
 *   P_rowptr, P_col  the fixed pattern of P (n x nc CSR); at most 1024 entries
 *                per row.
 *   P0_val       tentative prolongation on P's pattern (nnz(P) doubles); need
 *                not satisfy the constraint: the set-up corrects each row by
 *                the least-norm solution of Eq. (resEq).
 *   B            n x k fine near-kernel block V_f (row i = v_i of Eq. (Constr)).
 *   Bc           nc x k coarse block V_c; row i's local block is B_i = Bc(J_i,:).
 *   opts         options (NULL = defaults).
 *   inputs_on_device  1 if every input pointer is a device pointer.
 * All inputs are copied into library-owned device memory.  The set-up
 * validates the CSR arrays on the device, forms the Gram matrix
 * G_i = B_i^T B_i of every row in double, factorises it (Cholesky; rank
 * tolerance 1e-12 relative to max diag G_i), corrects P0, scales rows by
 * 1/A(i,i) for the Jacobi preconditioner (Theorem 1) and forms the initial
 * residual r = -Pi_B K p0.  On error *out is NULL and nothing is leaked.
 */
int emin_create(emin_ctx **out, int n, int nc, int k,
                const int *A_rowptr, const int *A_col, const double *A_val,
                const int *P_rowptr, const int *P_col, const double *P0_val,
                const double *B, const double *Bc,
                const emin_opts *opts, int inputs_on_device);

/*
 * Replace values without changing the patterns, then restart the
 * minimisation from the (new) P0 as emin_create does.  Any of A_val, B,
 * P0_val may be NULL to keep the stored array.  Device or host per
 * `on_device`.
 */
int emin_set_values(emin_ctx *ctx, const double *A_val, const double *B,
                    const double *P0_val, int on_device);

/* Restart the minimisation from the stored inputs (full set-up again). */
int emin_reset(emin_ctx *ctx);

/*
 * Run up to n_iters iterations of Algorithm 3, resuming the state left by
 * earlier calls.  tol is tau of Eq. (relRed): the iteration k whose energy
 * decrease dE_k = gamma alpha (Eq. (CG_dEa)) satisfies dE_k < tau dE_1 is
 * computed but not applied, and the minimisation is then converged (later
 * calls do nothing); tol = 0 runs exactly n_iters steps unless the projected
 * residual reaches rounding level (gamma <= f <K p0, M^{-1} K p0> with
 * f = (100 eps)^2 of the working precision: 1e-28 in EMIN_FP64, 3.6e-11 in
 * EMIN_MIXED), which also ends the minimisation.  *iters_done (may be NULL) receives the steps
 * applied by this call; *rel_dE_last (may be NULL) the last dE_k / dE_1.
 */
int emin_iterate(emin_ctx *ctx, int n_iters, double tol, int *iters_done,
                 double *rel_dE_last);

/* Energy tr(P^T A P) = <P, mask_P(A P)> of the current P, in double. */
int emin_energy(emin_ctx *ctx, double *E);

/*
 * Current prolongation P = P0 + dW on P's pattern (nnz(P) doubles).  The
 * correction (float in EMIN_MIXED) is promoted to double and every row is
 * then projected back onto its constraint in double (least-norm correction
 * as in Algorithm 2); in EMIN_FP64 this changes P at rounding level only.
 */
int emin_get_p(emin_ctx *ctx, double *P_val_out, int out_on_device);

/*
 * Fixed-pattern product out = [Pi_B] mask_P(A X) (Section 4; Pi_B applied
 * when `project` is 1) for X on P's pattern, computed by the same kernel as
 * the iteration in the context's precision.
 */
int emin_kprod(emin_ctx *ctx, const double *X, double *out, int project, int on_device);

/* out = mask_A(U V^T): for every stored (a, b) of A, sum_c U(a,c) V(b,c),
 * U and V on P's pattern; out has nnz(A) doubles.  Double precision. */
int emin_outer(emin_ctx *ctx, const double *U, const double *V, double *out, int on_device);

/*
 * Energy of a given X on P's pattern and its gradient (Eq. (trace),
 * E = tr(X^T A X) = <X, mask_P(A X)>), in double on the stored (unscaled) A:
 *   *E        = <X, mask_P(A X)>              (host double; may be NULL)
 *   dE_dX     = scale * 2 mask_P(A X)         (nnz(P); may be NULL; A symmetric)
 *   dE_dAval  = scale * mask_A(X X^T)         (nnz(A), per stored entry; may be NULL)
 * scale multiplies both gradients (an upstream derivative of the caller's
 * loss, 1 for the plain gradient).  X and the gradient arrays are device or
 * host per `on_device`.  Independent of the iteration state.
 */
int emin_energy_grad(emin_ctx *ctx, const double *X, double scale, double *E,
                     double *dE_dX, double *dE_dAval, int on_device);

/*
 * Implicit adjoint of the converged minimiser P* (not in the paper; derived
 * from the saddle-point system (sadsys)).  Given dL/dP on P's pattern it
 * solves Pi K Pi u = 1/2 Pi dL/dP by the same restricted PCG (in double,
 * from u = 0, at most max_adj_iters steps, tau = adj_tol) and returns
 *   dL_dAval  nnz(A): -2 mask_A(U P^T), the part of dL/dA through P*;
 *   dL_dB     n x k:  mu_i = G_i^{-1} B_i^T (dL/dP - 2 mask_P(A U))_i.
 * The explicit dependence of L on A is the caller's to add.  The current P
 * is taken as P*; only P (not the CG iterates) is kept from the forward.
 * Either output may be NULL.  *adj_iters (may be NULL) receives the steps.
 */
int emin_backward(emin_ctx *ctx, const double *dL_dP, double *dL_dAval, double *dL_dB,
                  int max_adj_iters, double adj_tol, int on_device, int *adj_iters);

/*
 * Gradient of exactly n_iters steps (not in the paper): the vector-Jacobian
 * product of the map (A values, B) -> P_n, P_n = the set-up's corrected P0
 * (Algorithm 2) followed by n_iters steps of Algorithm 3 with the Jacobi
 * preconditioner in double, for a forward that has not converged (for a
 * converged one it approaches emin_backward).  Given dL/dP (nnz(P)) it
 * returns dL_dAval (nnz(A), one value per stored entry, including the terms
 * through the Jacobi scaling and the initial residual) and dL_dB (n x k,
 * through the correction of P0).  The steps are run again in double from
 * the set-up (the context's own iteration state is not used or changed);
 * the iterates are checkpointed every ceil(sqrt(n_iters)) steps and each
 * segment is recomputed before it is reversed, so memory grows with
 * sqrt(n_iters) vectors on P's pattern.  Needs an EMIN_FP64 context with
 * EMIN_JACOBI (else EMIN_ERR_ARG); A must be symmetric.  Either output may
 * be NULL.  EMIN_ERR_BREAKDOWN if a step has y^T K y <= 0.
 */
int emin_backward_unrolled(emin_ctx *ctx, const double *dL_dP, int n_iters, double *dL_dAval,
                           double *dL_dB, int on_device);

/*
 * Statistics: dE_k of the computed iterations since the last (re)start
 * (up to cap values into dE_hist, may be NULL), their count, the number of
 * rank-deficient rows handled by EMIN_RANK_PINV, and the applied steps.
 */
int emin_stats(emin_ctx *ctx, double *dE_hist, int cap, int *n_hist,
               int *n_rank_deficient, int *n_applied);

/*
 * Instrumentation.  emin_set_timing(ctx, p) with p >= 1 makes every later
 * emin_iterate bracket the masked-product launch of every p-th iteration
 * (iterations 0, p, 2p, ... of the call) with CUDA events on the context's
 * stream (p = 0 switches timing off); emin_timing returns in ms[0] / launches[0] the
 * summed event time and the number of timed launches since timing was
 * enabled (entries 1 and 2 are reserved, 0; either array may be NULL and
 * has 3 entries), and in *total_launches the number of kernels the library
 * has run since the context was created.  Enabling (again) clears the sums.
 * On a non-default stream emin_iterate runs the iteration loop as one CUDA
 * graph (captured on first use for a given iteration count).
 */
int emin_set_timing(emin_ctx *ctx, int enable);
int emin_timing(emin_ctx *ctx, double *ms, long long *launches, long long *total_launches);

/*
 * Allocation-free masked product (the paper has no counterpart; it is a
 * service for callers that must not let a library allocate device memory,
 * e.g. processes whose device memory belongs to another allocator's pool or
 * request paths that cannot afford the device synchronisation of
 * cudaMalloc / cudaFree).
 *   out  = mask_P(A Y)   (nnz(P) doubles, P's pattern, CSR order)
 *   *dot = <Y, out>      (one double)
 * Every pointer is a device pointer of the current device; A is n x n and P
 * is n x nc in CSR as for emin_create (sorted columns).  Work is queued on
 * `stream` (cudaStream_t, NULL = legacy default) and the call returns
 * without waiting.  No device or host memory is allocated: the reduction
 * uses a 128 KiB file-scope device array that every GPU loading the library
 * holds until the process exits.  The first call on a device looks that
 * array's address up (once per device, with that device current); make
 * that first call before any stream capture.  Calls share the array, which
 * keeps the last call's contents (the counters that must start at zero are
 * cleared on every call), so calls that overlap on the GPU race.
 * The address is kept for the life of the process, so calls must not
 * continue after the device's primary context has been reset
 * (cudaDeviceReset).  n > 4,194,304 (= 16,384 blocks of 256 rows), or, with
 * n > 0, a NULL array, returns EMIN_ERR_ARG before anything is queued; n = 0
 * sets *dot = 0.  Row pointers or column indices out of range are skipped
 * and make *dot NaN.
 */
int emin_masked_product_noalloc(int n, int nc, const int *A_rowptr, const int *A_col,
                                const double *A_val, const int *P_rowptr, const int *P_col,
                                const double *Y, double *out, double *dot, void *stream);

/*
 * Measurement aid (the paper has no counterpart): the rate of the fused
 * multiply-add pipe of the current device in double (EMIN_FP64) or float
 * (EMIN_MIXED), from one launch of independent FMA chains that fills every
 * SM, timed with CUDA events on `stream` (cudaStream_t, NULL = legacy
 * default; the call waits for it).  *fma_per_s receives FMAs per second (2
 * flops each), *ms (may be NULL) the timed launch's duration.  It is the
 * ceiling against which the FP64 masked products, bound by FP64 arithmetic
 * on this part, are reported.
 */
int emin_fma_rate(int precision, double *fma_per_s, double *ms, void *stream);

/* Sizes of the context: nnz(A), nnz(P) (either may be NULL). */
int emin_sizes(emin_ctx *ctx, long long *nnz_a, long long *nnz_p);

/* Static description of a status code. */
const char *emin_strerror(int status);

/* The last CUDA failure seen by a library call of this thread (the failing
 * step and CUDA's error name and text), "" if none; valid until the next
 * call of this thread. */
const char *emin_last_error(void);

/* Release every resource of the context (NULL is accepted).  The device
 * memory of a context comes from a stream-ordered pool per device that the
 * library owns and that keeps freed memory for the next context (so that
 * creating and destroying contexts of similar sizes maps no new pages and
 * does not synchronise the device); destroy frees it on the context's
 * stream after waiting for that stream's work. */
void emin_destroy(emin_ctx *ctx);

/* Return the device memory cached in the library's pools (what destroyed
 * contexts released) to the driver; the memory of live contexts stays.
 * EMIN_OK, or EMIN_ERR_CUDA if the driver refused. */
int emin_trim_memory(void);

#ifdef __cplusplus
}
#endif
#endif /* EMIN_H */
