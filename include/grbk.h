/*
 * grbk.h -- C ABI of the GB300 (sm_103a) solver library for the matrix
 * equation A X B = C by the greedy randomized block Kaczmarz family
 * (Wang, Liu, Qu, arXiv 2408.05444).
 *
 *   A in R^{m x p}, B in R^{q x n}, C in R^{m x n}, X in R^{p x q}   (Eq. 1.1)
 *
 * Variants (one row index i_k per iteration, then one block update):
 *   GRBK_GRBK   ME-GRBK,  Algorithm 3 (threshold zeta_k, theta fixed 1/2)
 *   GRBK_RGRBK  ME-RGRBK, Algorithm 4 (threshold xi_k, relaxation theta in (0,1])
 *   GRBK_MWRBK  ME-MWRBK, Algorithm 5 (largest ||R_i||^2 / ||A_i||^2; smallest index on ties)
 *   GRBK_RBK    ME-RBK,   Algorithm 1 (row i with probability ||A_i||^2 / ||A||_F^2)
 *   GRBK_BK     ME-BK,    Algorithm 2 (cyclic, i_k = k mod m)
 * Every variant applies  X += (alpha/||A_i||^2) A_i^T (R_i B^T)  and keeps the
 * residual R = C - A X B by the rank-1 update of Algorithm 3:
 *   R -= (alpha/||A_i||^2) (A A_i^T) ((R_i B^T) B).
 *
 * Conventions for every entry point:
 *   - All matrices are row-major; `ld` is the row stride in elements (>= cols).
 *   - Rows are 0-based.  The random variants draw u_k in [0,1) from
 *     Philox4x64-10 with key (seed, 0) and counter (k, system, 0, 0), first
 *     output word, top 53 bits times 2^-53; i_k is the first admitted row (in
 *     ascending order) whose running sum of ||R_i||^2 exceeds u_k times the
 *     admitted total.
 *   - Errors are reported by the returned grbk_status; no entry point aborts
 *     the process.  A CUDA error leaves the context usable for destroy only.
 *   - Work runs on opts.stream (a cudaStream_t; NULL = legacy default stream)
 *     and every call returns after its work has finished.
 *   - Not thread-safe per context; distinct contexts may be used concurrently.
 */
#ifndef GRBK_H
#define GRBK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GRBK_OK = 0,          /* success (converged, exact, or ran the requested iterations) */
    GRBK_EINVAL = 1,      /* bad argument: shape mismatch, theta outside (0,1], alpha outside (0, 2/||B||_2^2), m == 0, ... */
    GRBK_ENOMEM = 2,      /* device allocation failed */
    GRBK_ECUDA = 3,       /* a CUDA runtime call or kernel failed */
    GRBK_ENOTCONV = 4,    /* maxit reached before the tolerance; X_out still written */
    GRBK_ETIMEOUT = 5,    /* a device-side barrier exceeded its spin budget; X_out not trusted */
    GRBK_ENONFINITE = 6   /* NaN/Inf in the inputs or in the residual */
} grbk_status;

typedef enum { GRBK_GRBK = 0, GRBK_RGRBK = 1, GRBK_MWRBK = 2, GRBK_RBK = 3, GRBK_BK = 4 } grbk_variant;

/* Arithmetic of the residual pass.  F64: everything FP64.  F32: A, B, C, R in
 * FP32; row norms, their sums, the threshold, the pick and X kept in FP64;
 * refresh of R as split-BF16 tensor-core products accumulated in FP32. */
typedef enum { GRBK_F64 = 0, GRBK_F32 = 1 } grbk_precision;

typedef enum { GRBK_DT_F64 = 0, GRBK_DT_F32 = 1 } grbk_dtype;

/* Stopping rule, tested before each iteration.  RELRES: ||R||_F <= tol ||C||_F.
 * RSE: ||X - X_ref||_F <= tol ||X_ref||_F, tested every `check_every`
 * iterations (X is folded in at those points).  NONE: run maxit iterations. */
typedef enum { GRBK_STOP_NONE = 0, GRBK_STOP_RELRES = 1, GRBK_STOP_RSE = 2 } grbk_stop;

/* How the residual is kept.  FULL: R = C - A X B, m x n, as in Algorithm 3.
 * ROWSPACE: every residual row is a combination of the rows of B plus a part
 * that the updates never change (each update of Algorithm 3 subtracts a
 * multiple of R_{i_k} B^T B), so R = Z Bt + Rperp with Bt (r x n) an
 * orthonormal basis of the row space of B (r = rank B) and Z = R Bt^T, m x r.
 * The library keeps Z instead of R: s_i = ||Z_i||^2 + ||Rperp_i||^2 and the
 * iterates are those of the full form up to rounding.  Set-up (pivoted
 * Cholesky of B B^T, Z^0 and the Rperp row norms) costs O(m n q) and the
 * residual shrinks by n / r.  Not part of the paper. */
typedef enum { GRBK_FORM_FULL = 0, GRBK_FORM_ROWSPACE = 1 } grbk_form;

/* A matrix argument.  `ptr` is a host pointer (on_device = 0) or a device
 * pointer (on_device = 1); the library never keeps it after the call returns. */
typedef struct {
    const void* ptr;
    int64_t rows, cols, ld;
    int32_t dtype;      /* grbk_dtype */
    int32_t on_device;
} grbk_mat;

typedef struct {
    int32_t precision;    /* grbk_precision */
    int32_t refresh_T;    /* recompute R = C - A X B every refresh_T iterations; 0 = never */
    double alpha;         /* step; <= 0 selects 1/||B||_2^2 estimated on the device (grbk_create: largest
                             Ritz value of up to 40 Lanczos steps on B B^T; batched solvers: power
                             iteration per system) */
    int32_t stop_kind;    /* grbk_stop */
    int32_t split_terms;  /* F32 refresh: 2 (hi+lo, default) or 3 (hi+mid+lo) BF16 terms; 0 = 2 */
    const grbk_mat* x_ref;/* reference solution for GRBK_STOP_RSE and result.rse; may be NULL */
    int32_t* row_trace;   /* host buffer: selected row of iteration k, k < trace_len; may be NULL */
    double* s_trace;      /* host buffer: ||R^k||_F^2 before iteration k, k < trace_len; may be NULL */
    int64_t trace_len;
    void* stream;         /* cudaStream_t */
    int32_t grid_ctas;    /* persistent-kernel CTAs; 0 = chosen by the library */
    int32_t check_every;  /* iterations per device chunk between host checks; 0 = refresh_T or 256 */
    int32_t use_gram;     /* form A A^T once and read u = (A A^T)_{:,i_k} from it (the practice note after
                             Algorithm 3): 1 on, -1 off (u = A A_{i_k}^T every iteration), 0 on when the
                             m x m matrix takes at most 4 GB and, in FP64, forming it takes at most
                             2 m^2 p = 1e11 flops (FP64 runs on the narrow FP64 pipe: about 80 ms) */
    int32_t form;         /* grbk_form; 0 = FULL */
    double rank_tol;      /* ROWSPACE: pivots of B B^T at most rank_tol * max_i (B B^T)_ii end the
                             basis (they set r); <= 0 selects 1e-12 (F64) or 1e-6 (F32) */
    int32_t band_limit;   /* batched solver: a system whose A and B have nonzeros only within half-bandwidths
                             bA, bB <= band_limit of the diagonal (and 4 bA + 1 < m) takes the banded path,
                             which forms w, u, v from the bands and updates only the rows within 2 bA of
                             i_k (u_i = (A A_{i_k}^T)_i vanishes elsewhere); 0 = 64, -1 = always dense */
    const double* alphas; /* batched and sparse solvers: host array of nsys steps, one per system, each in
                             (0, 2/||B_s||_2^2) (checked against the device estimate of ||B_s||_2^2); it
                             replaces `alpha`.  NULL: `alpha` (when > 0) or 1/||B_s||_2^2 for every system */
    int32_t extended;     /* sparse solver: 1 = least-squares extension for inconsistent systems (Eq. 2.1;
                             see grbk_sparse_create); 0 = the paper's iteration */
    int32_t tune;         /* batched solver: 1 = choose each system's kernel variant by timing the compiled
                             variants on it (grbk_tune_*; choices kept per system shape for the process);
                             0 = the default variant (512 threads, two rows per warp) for every system */
    int32_t deferred;     /* F32 single-system solver: -1 = off, 1 = on, 0 = on in the FULL form only; on
                             only when a chunk (check_every) is at most 64 iterations and each CTA owns at
                             most 512 rows.  During a chunk
                             R stays at its value R^0 from the chunk's start and the current residual is
                             R^0 - sum_j U'_j v_j^T (U'_j = c_j A A_{i_j}^T, v_j = w_j B of iteration j);
                             an iteration reads R^0 once (R^0_i . v), the row norms follow by
                             ||R_i - U'_i v||^2 = s_i - 2 U'_i (R_i . v) + U'_i^2 ||v||^2 (not a form of the
                             paper: its iterates, with the update applied later), the selected row is
                             assembled from R^0 and the kept terms, and after the chunk R is written back
                             with the terms in order (the in-place update's arithmetic) unless the periodic
                             refresh recomputes it */
} grbk_opts;

typedef struct {
    int64_t iters;        /* iterations performed */
    double relres;        /* ||C - A X B||_F / ||C||_F of the kept residual at exit */
    double rse;           /* ||X - X_ref||_F / ||X_ref||_F at exit (NaN without x_ref) */
    double seconds;       /* wall time of the solve call */
    double alpha;         /* step actually used */
    double iter_kernel_ms;        /* device time of the persistent iteration kernel (CUDA events on the stream) */
    int64_t iter_kernel_launches; /* its launches in this call */
    int64_t launches;             /* all kernel launches made by this call */
    int32_t gram;         /* 1 when u came from the precomputed A A^T */
    int32_t x0_rejected;  /* batched solves: 1 when the given X0 had ||C - A X0 B|| >= ||C|| and 0 was used */
    int32_t status;       /* grbk_status of the call */
    int32_t deferred;     /* 1 when the solve used the deferred update (grbk_opts.deferred) */
} grbk_result;

typedef struct grbk_ctx grbk_ctx;
typedef struct grbk_batch grbk_batch;

/* Fill `opts` with defaults (F64, no refresh, alpha = 1/||B||_2^2, STOP_NONE). */
void grbk_default_opts(grbk_opts* opts);

/*
 * grbk_create -- set up one system A X B = C (Eq. 1.1).
 * Copies A (m x p), B (q x n), C (m x n) into library-owned device memory in
 * the precision of opts->precision; the caller may free its buffers at once.
 * Computes ||A_i||^2, ||A||_F^2, ||C||_F^2 and alpha (Section 5 uses
 * alpha = 1/||B||_2^2; Lemma 2.2 and Theorems 4.2, 4.5, 4.8 need 0 < alpha < 2/||B||_2^2).
 * Errors: EINVAL (NULL pointers, shape mismatch, m == 0, explicit alpha not in
 * (0, 2/||B||_2^2), non-finite input -> ENONFINITE), ENOMEM, ECUDA.
 */
grbk_status grbk_create(grbk_ctx** out, const grbk_mat* A, const grbk_mat* B, const grbk_mat* C,
                        const grbk_opts* opts);

/*
 * grbk_solve -- run one of Algorithms 1-5 from X0 (NULL = zero matrix) for at
 * most maxit iterations (Algorithm 3's loop "until convergence").
 * theta: RGRBK relaxation in (0, 1] (Algorithm 4); ignored by other variants.
 * tol: tolerance of opts->stop_kind.  seed: Philox key for RGRBK/GRBK/RBK.
 * X_out: p x q, caller-owned, host or device, FP64 or FP32; written on OK and
 * ENOTCONV.  res: may be NULL.
 * The residual starts as R^0 = C - A X0 B; zero rows of A are never selected
 * (an ME-BK step on such a row changes nothing).  ||R||_F = 0 stops with OK.
 */
grbk_status grbk_solve(grbk_ctx* ctx, int32_t variant, double theta, const grbk_mat* X0,
                       double tol, int64_t maxit, uint64_t seed, grbk_mat* X_out,
                       grbk_result* res);

/*
 * grbk_residual -- R_out = C - A X B for a caller X (p x q), with the same
 * device path the solver uses to refresh its kept residual (FP64 SIMT GEMMs
 * in F64 mode; split-BF16 tcgen05 GEMMs accumulated in FP32 in F32 mode).
 * R_out is m x n, caller-owned, host or device, FP64 or FP32.
 */
grbk_status grbk_residual(grbk_ctx* ctx, const grbk_mat* X, grbk_mat* R_out);

/* Copies of the kept state after a solve: residual R (m x n) and row norms
 * ||R_i||^2 (m doubles, host or device per on_device).  grbk_residual and
 * grbk_get_residual return GRBK_EINVAL for the ROWSPACE form, which keeps no
 * m x n residual; its row norms include the fixed ||Rperp_i||^2. */
grbk_status grbk_get_residual(grbk_ctx* ctx, grbk_mat* R_out);
grbk_status grbk_get_rownorms(grbk_ctx* ctx, double* s_out, int32_t on_device);

/* Device blocks of destroyed contexts are kept (per device and size, at most 64 GB)
 * for the next grbk_create; this returns every kept block to the driver, e.g.
 * before another allocator in the process needs the memory.  Not part of the paper. */
void grbk_trim_cache(void);

/* Problem sizes (m, p, q, n of the caller's system) and the step in use. */
grbk_status grbk_info(const grbk_ctx* ctx, int64_t dims[4], double* alpha);

/* The residual form in use (grbk_form) and the columns of the kept residual:
 * n for FULL, r = rank B for ROWSPACE.  Not part of the paper. */
grbk_status grbk_form_info(const grbk_ctx* ctx, int32_t* form, int64_t* cols);

void grbk_destroy(grbk_ctx* ctx);

/*
 * Batched systems: nsys independent problems A_s X_s B_s = C_s of uneven sizes
 * (the colour-image application of Section 6 solves one per channel), solved
 * together in one persistent launch.  Arrays A, B, C have nsys entries.  The
 * batch runs in FP32 (A, B, C, R) with FP64 row-norm sums, threshold and pick.
 * System s draws its random numbers with counter (k, s, 0, 0).
 * stop_kind: NONE, RELRES (per-system ||R_s||_F <= tol ||C_s||_F) or the
 * discrepancy rule via grbk_batch_solve's `targets`.  opts->row_trace, when
 * set, must hold nsys * trace_len entries: system s writes its first
 * trace_len selected rows at row_trace[s * trace_len + k] (s_trace unused).
 * Every side m, p, q, n of a system is at most 1024 (larger systems belong to
 * grbk_create).  Errors: EINVAL (nsys <= 0, NULL pointers, C_s not m x n, a
 * side outside [1, 1024], a row stride below the column count, a dtype other
 * than F32/F64), ENOMEM, ECUDA.
 */
grbk_status grbk_batch_create(grbk_batch** out, int32_t nsys, const grbk_mat* A, const grbk_mat* B,
                              const grbk_mat* C, const grbk_opts* opts);

/*
 * grbk_batch_solve -- iterate every system until its own stop rule holds or
 * maxit.  X0s: NULL (all zero) or nsys matrices; a given X0 whose residual
 * ||C - A X0 B||_F is not below ||C||_F (or is not finite) is replaced by the
 * zero matrix on the device and reported in results[s].x0_rejected.  targets: NULL, or nsys
 * absolute residual targets ||R_s||_F <= targets[s] (discrepancy principle);
 * when given they replace tol.  X_outs: nsys caller matrices (written).
 * results: NULL or nsys entries.  Returns OK when every system stopped by its
 * rule, ENOTCONV when some reached maxit; EINVAL for a bad variant, theta or
 * maxit, or an X0s / X_outs entry that is not p_s x q_s with row stride >= q_s
 * and dtype F32/F64.
 */
grbk_status grbk_batch_solve(grbk_batch* batch, int32_t variant, double theta, const grbk_mat* X0s,
                             double tol, const double* targets, int64_t maxit, uint64_t seed,
                             grbk_mat* X_outs, grbk_result* results);

/* The path a batched system takes: the half-bandwidths of its A and B when it
 * uses the banded path (opts.band_limit), -1 and -1 for the dense path.  Not
 * part of the paper: a layout choice for banded (e.g. blur) matrices. */
grbk_status grbk_batch_info(const grbk_batch* b, int32_t sys, int32_t* bandA, int32_t* bandB);

void grbk_batch_destroy(grbk_batch* batch);

/*
 * Batch autotuner (not part of the paper; Section 6's application solves many
 * systems of uneven sizes).  The batched kernel is compiled in several
 * variants (threads per CTA, rows of R per warp in the fused update pass) that
 * compute the same iteration and differ only in the summation order of the
 * FP64 totals.  With opts.tune = 1, grbk_batch_create times every variant on
 * one system of each class (sides rounded up to multiples of 64, exact
 * half-bandwidths) not yet in the process-wide cache -- ME-GRBK, 48
 * iterations from R = C, CUDA events -- and keeps the fastest (a variant
 * within 2 % of it that uses fewer threads wins).  Solves then launch one
 * kernel per variant in use, side by side on the batch's own streams.
 *
 * grbk_tune_num_variants / grbk_tune_variant_info: the compiled variants.
 * grbk_tune_choose: the rule applied to one class's timings (ms[v] for each of
 *   the grbk_tune_num_variants() variants; entries <= 0 or non-finite are
 *   ignored); returns the variant, or -1 for a wrong count.
 * grbk_tune_lookup / grbk_tune_store / grbk_tune_clear: the cache (variant -1
 *   when the class is absent).  Thread-safe.
 * grbk_batch_variant: the variant a system of a batch runs and the seconds
 *   the batch's tuning took.
 */
int32_t grbk_tune_num_variants(void);
grbk_status grbk_tune_variant_info(int32_t variant, int32_t* threads, int32_t* rows_per_warp);
int32_t grbk_tune_choose(const double* ms, int32_t nvariants);
grbk_status grbk_tune_lookup(int32_t m, int32_t p, int32_t q, int32_t n, int32_t bandA, int32_t bandB,
                             int32_t* variant);
grbk_status grbk_tune_store(int32_t m, int32_t p, int32_t q, int32_t n, int32_t bandA, int32_t bandB,
                            int32_t variant);
void grbk_tune_clear(void);
grbk_status grbk_batch_variant(const grbk_batch* batch, int32_t sys, int32_t* variant, double* tune_seconds);

/*
 * Sparse A and B: nsys independent systems A_s X_s B_s = C_s with A_s and B_s
 * in compressed sparse rows, R dense, all arithmetic FP64 (the paper's
 * precision).  Section 5 draws A and B from sparse test matrices (the sprandn
 * sets of Tables 3, 5 and 7); Section 6's colour model B = A X A_c^T + E has a
 * blur A of mn x mn with a few dozen nonzeros per row and B = A_c^T (3 x 3),
 * one system per image with the three channels as the columns of X.
 *
 * Per iteration the library touches only what the sparsity allows: w =
 * R_{i_k} B^T over the rows of B, X += c A_{i_k}^T w over the nonzeros of
 * A_{i_k}, v = w B over the columns of B, and R -= c (A A_{i_k}^T) v only on
 * the rows k with (A A^T)_{k,i_k} != 0 (the sparse Gram matrix A A^T is formed
 * once on the device at set-up, the practice note after Algorithm 3).  The
 * threshold, the admitted set and the pick are those of Algorithms 1-5, with
 * the totals kept as per-block summaries of 256 rows.  X^0 = 0 (Section 6
 * starts from the zero matrix).
 *
 * opts->extended = 1 solves inconsistent systems in the least-squares sense
 * (Eq. 2.1, whose target the paper defines but does not solve), as the
 * randomized extended Kaczmarz method of Zouzias and Freris (2013) does for
 * A x = b: an auxiliary Y (m x n, Y^0 = C) is driven to (I - A A^+) C by one
 * column projection per iteration, Y -= A_{:,j} (A_{:,j}^T Y) / ||A_{:,j}||^2
 * with column j drawn with probability ||A_{:,j}||^2 / ||A||_F^2 (Philox
 * counter (k, system, 1, 0)), and the row step of the chosen variant runs on
 * R = C - Y - A X B.  With B of full column rank (B^+ B = I) X^k tends to the
 * least-norm least-squares solution A^+ C B^+.  R^0 = 0, so the extension runs
 * a fixed number of iterations (stop_kind NONE, no targets; otherwise EINVAL).
 */
typedef struct {
    int64_t rows, cols, nnz;
    const int64_t* rowptr;  /* rows + 1 host offsets: rowptr[0] = 0, rowptr[rows] = nnz, non-decreasing */
    const int32_t* colind;  /* nnz host column indices, strictly ascending within each row */
    const double* val;      /* nnz host values (finite) */
} grbk_csr;

typedef struct grbk_sparse grbk_sparse;

/*
 * grbk_sparse_create -- copies A[s] (m x p CSR), B[s] (q x n CSR) and C[s]
 * (m x n dense, host or device, FP32/FP64) for s < nsys into library-owned
 * device memory, forms the CSC of B and A A^T, ||A_i||^2, ||A||_F^2, ||C||_F^2
 * and the step (opts->alphas, opts->alpha, else 1/||B||_2^2 from 200 power
 * iterations on B B^T).  Limits: m <= 262144, q and n <= 1024.
 * opts: stop_kind (NONE or RELRES), row_trace / s_trace (host, nsys * trace_len
 * entries: system s at [s * trace_len + k]), stream, grid_ctas.
 * Errors: EINVAL (NULL, malformed CSR: offsets, column range or order; shapes;
 * limits; inadmissible alpha), ENONFINITE, ENOMEM, ECUDA.
 */
grbk_status grbk_sparse_create(grbk_sparse** out, int32_t nsys, const grbk_csr* A, const grbk_csr* B,
                               const grbk_mat* C, const grbk_opts* opts);

/*
 * grbk_sparse_solve -- every system from X^0 = 0 until its stop rule holds or
 * maxit: RELRES with tol, or targets[s] (absolute ||R_s||_F, the discrepancy
 * principle) when targets is not NULL.  X_outs: NULL or nsys caller matrices
 * p_s x q_s (host or device, FP32/FP64, row stride >= q_s).  results: NULL or
 * nsys entries.  Returns OK, or ENOTCONV when some system with a stop rule
 * reached maxit; EINVAL for a bad variant, theta, tol, target or output.
 */
grbk_status grbk_sparse_solve(grbk_sparse* sp, int32_t variant, double theta, double tol, const double* targets,
                              int64_t maxit, uint64_t seed, grbk_mat* X_outs, grbk_result* results);

/* Entries of the sparse Gram matrix A_s A_s^T and the step of system `sys`. */
grbk_status grbk_sparse_info(const grbk_sparse* sp, int32_t sys, int64_t* gram_nnz, double* alpha);

/* CTAs per system of the last grbk_sparse_solve (1 before any solve): a thread-
 * block cluster of up to 8 CTAs, one per SM, shares each system's row update,
 * X update and admitted scan when the systems leave SMs idle and n >= 8
 * (no counterpart in the paper: a layout choice).  Errors: EINVAL (null). */
grbk_status grbk_sparse_cluster(const grbk_sparse* sp, int32_t* ctas);

/* The kept residual R_s (m x n FP64, row-major) and its row norms ||R_i||^2
 * (m doubles) after a solve, into host buffers (either may be NULL). */
grbk_status grbk_sparse_get_residual(const grbk_sparse* sp, int32_t sys, double* R_out, double* s_out);

void grbk_sparse_destroy(grbk_sparse* sp);

/*
 * grbk_solve_small_noalloc -- one small system A X B = C in FP32 solved with no
 * device or host allocation.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate, e.g. processes whose device memory
 * comes from a fixed pool they do not own (a framework's caching allocator, a
 * service with a hard memory budget), or loops where the cost and device-wide
 * synchronisation of cudaMalloc/cudaFree are not acceptable.
 *
 * It runs the batched kernel on a single system (system index 0 for the
 * Philox counter), so its arithmetic is that of grbk_batch_solve.  All working
 * memory (residual, padded copies of A and B, row norms, recorded update
 * terms, counters) lives in one
 * static device array of GRBK_NOALLOC_SCRATCH_BYTES bytes that every GPU which
 * loads this library holds until the process exits.  Limits: m, p, q, n each
 * at most GRBK_NOALLOC_MAX_SIDE; larger sizes return GRBK_EINVAL.
 *
 * A (m x p), B (q x n), C (m x n): device pointers, FP32, row-major and
 * contiguous (row stride = number of columns), owned by the caller.
 * X_out (p x q): device pointer, FP32, contiguous; zeroed, then overwritten
 * (X^0 = 0).  alpha <= 0 selects 1/||B||_2^2 (200 power iterations on the
 * device); an explicit alpha must lie in (0, 2/||B||_2^2).  tol > 0 stops
 * when ||R||_F <= tol ||C||_F (GRBK_ENOTCONV if maxit comes first); tol <= 0
 * runs exactly maxit iterations.  iters_out and relres_out are host pointers
 * (either may be NULL).  stream is a cudaStream_t; the call returns after the
 * work has finished.
 *
 * The first call on a device looks up the device address of the static array
 * (cudaGetSymbolAddress) and caches it; make that first call before any stream
 * capture.  Every call uses the same array and leaves the previous call's
 * contents in it: the call clears what must start at zero itself.  Calls whose
 * work overlaps on the GPU (other streams, other host threads) race on the
 * array and must be serialised by the caller.
 * Errors: EINVAL (NULL pointer, size outside [1, GRBK_NOALLOC_MAX_SIDE],
 * variant, theta, a non-finite alpha or tol, an alpha outside
 * (0, 2/||B||_2^2)), ENONFINITE (NaN/Inf input or residual), ECUDA.
 */
#define GRBK_NOALLOC_MAX_SIDE 512
#define GRBK_NOALLOC_SCRATCH_BYTES (4u * 1024u * 1024u)
grbk_status grbk_solve_small_noalloc(const float* A, const float* B, const float* C, int32_t m, int32_t p,
                                     int32_t q, int32_t n, int32_t variant, double theta, double alpha,
                                     double tol, int64_t maxit, uint64_t seed, float* X_out,
                                     int64_t* iters_out, double* relres_out, void* stream);

/*
 * Learned warm start for the colour-image application (Section 6 solves one
 * deblurring system per channel): a 3-level convolutional U-Net maps a blurred
 * channel C (h x w, h and w multiples of 4) to an initial iterate
 * X0 = C + f(C).  The solver's own iteration decides the answer (A, B square
 * and full rank: X0 changes the iteration count, not the limit); a caller
 * falls back to X0 = 0 when X0 is non-finite or its residual is larger.
 *
 * Architecture for width w: enc 1->w->w | 2x2 avg pool | w->2w->2w | pool |
 * 2w->4w->4w | nearest 2x up, concat | 6w->2w->2w | up, concat | 3w->w->w |
 * w->1; 3x3 convolutions with zero padding, ReLU except the last.  Parameters
 * form one FP32 array, layer by layer in that order, each W[out][in][3][3]
 * followed by b[out] (grbk_unet_num_params entries); the convolutions use a
 * BF16 copy of the weights and accumulate in FP32.  Training minimises
 * mean((X0 - T)^2) with Adam (beta 0.9 / 0.999, eps 1e-8) on the FP32 copy.
 *
 * Images are NCHW with one channel: n images of h x w FP32, contiguous, device
 * pointers.  All calls run on the stream given at creation and return when the
 * work is done.  Errors: EINVAL (shape, NULL), ENOMEM, ECUDA.
 */
typedef struct grbk_unet grbk_unet;
grbk_status grbk_unet_create(grbk_unet** out, int32_t width, void* stream);
int64_t grbk_unet_num_params(const grbk_unet* net);
/* params: FP32 array of grbk_unet_num_params entries, host (on_device = 0) or device; resets Adam */
grbk_status grbk_unet_set_params(grbk_unet* net, const float* params, int32_t on_device);
grbk_status grbk_unet_get_params(grbk_unet* net, float* params, int32_t on_device);
/* X0 = C + f(C) for n images */
grbk_status grbk_unet_forward(grbk_unet* net, const float* C, int32_t n, int32_t h, int32_t w, float* X0);
/* loss = mean((X0 - T)^2) and its gradient w.r.t. the parameters (grad may be NULL) */
grbk_status grbk_unet_loss_grad(grbk_unet* net, const float* C, const float* T, int32_t n, int32_t h, int32_t w,
                                double* loss, float* grad, int32_t grad_on_device);
/* one Adam step on mean((X0 - T)^2); loss (host, may be NULL) is the loss before the step */
grbk_status grbk_unet_train_step(grbk_unet* net, const float* C, const float* T, int32_t n, int32_t h, int32_t w,
                                 float lr, double* loss);
/* Convolution path (not part of the paper): on = 1 (the default) runs every
 * convolution of the forward pass with 16 to 128 input and output channels on
 * the tensor cores -- an implicit GEMM (tcgen05.mma, TMEM accumulators, TMA
 * loads whose out-of-range coordinates give the zero padding) over a
 * three-term BF16 split of the FP32 activations and the BF16 weights,
 * accumulated in FP32; images at least 128 pixels wide load each kernel row's
 * input pixels once for its three taps.  on = 2: tensor cores with one load
 * per tap (the general tiling, for comparison); on = 0: every convolution on
 * the SIMT kernel.  The backward passes always use the SIMT kernels.  A
 * bounded wait of the tensor-core kernel that expires makes the next forward,
 * loss or training call return GRBK_ETIMEOUT.  EINVAL for other values. */
grbk_status grbk_unet_use_tensor_cores(grbk_unet* net, int32_t on);
void grbk_unet_destroy(grbk_unet* net);

/*
 * grbk_barrier_selftest -- no counterpart in the paper: exercises the bounded
 * grid barrier the iteration kernel uses between its phases.  A small
 * cooperative grid (at most 8 CTAs) meets at one barrier with a spin budget of
 * about 0.1 s.  absent_cta < 0: every CTA arrives, returns GRBK_OK.
 * absent_cta = c >= 0: CTA c leaves without arriving, the others give up when
 * the budget runs out and the call returns GRBK_ETIMEOUT; the CUDA context
 * stays usable.  Nothing faults or hangs in either case.
 */
grbk_status grbk_barrier_selftest(int32_t absent_cta, void* stream);

/*
 * grbk_fp64_probe -- no counterpart in the paper: measures the FP64 fused
 * multiply-add rate of the current device, the roof of the FP64 residual pass
 * (two FMAs per element of R: the rank-1 update and the square of the new
 * value; Algorithm 3's update of R and the row norms of the next iteration).
 * Launches blocks_per_sm x (SM count) blocks of 256 threads, each thread
 * running 8 independent FMA chains for `iters` steps; one untimed launch, then
 * one timed with CUDA events on `stream`.  Outputs (host pointers, may be
 * NULL): FMAs per second and the timed launch's milliseconds.
 * Errors: EINVAL (iters <= 0, blocks_per_sm outside [1, 64]), ENOMEM, ECUDA.
 */
grbk_status grbk_fp64_probe(int64_t iters, int32_t blocks_per_sm, double* dfma_per_s, double* ms, void* stream);

/*
 * grbk_fp64_issue_probe -- no counterpart in the paper: the SM clock cycles one
 * warp spends per FP64 operation when `warps` warps of one CTA run dependent
 * chains of `iters` operations on their first `active_lanes` lanes (op: 0 add,
 * 1 fused multiply-add, 2 multiply, 3 division, 4 double -> float -> double
 * round trip plus an add).  On one SM, cycles per operation with one warp give
 * the issue interval, with many warps the share of the SM's FP64 unit; equal
 * figures for 1 and 32 active lanes mean a warp instruction costs the same
 * whatever its active lanes.  This is why the kernels keep FP64 arithmetic on
 * one lane or on full warps of rows and compare non-negative FP64 values on
 * their bit patterns.  Output: *cycles_per_op (host pointer; the largest of the
 * warps' spans / iters).  Errors: EINVAL (op outside [0, 4], warps outside
 * [1, 32], active_lanes outside [1, 32], iters <= 0, null output), ENOMEM, ECUDA.
 */
grbk_status grbk_fp64_issue_probe(int32_t op, int32_t warps, int32_t active_lanes, int64_t iters,
                                  double* cycles_per_op, void* stream);

/* Human-readable name of a status code (static storage). */
const char* grbk_strerror(int32_t status);

#ifdef __cplusplus
}
#endif

#endif /* GRBK_H */
