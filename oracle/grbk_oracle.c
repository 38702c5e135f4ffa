/*
 * grbk_oracle.c -- plain, slow FP64 CPU reference for the matrix-equation
 * block Kaczmarz family (ME-GRBK and its siblings) for A X B = C.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file.  It shares no code, header
 * or constant with the CUDA library; the two only share the seeded input
 * generators.
 *
 * Everything is row-major FP64 with index-ascending loops.  The build the
 * tests use is single-threaded, with -ffp-contract=off so that x86-64 and
 * aarch64 round identically.  A second build with -fopenmp (used only to time
 * the oracle on every host core) runs the loops marked "omp" below with their
 * rows (or columns) split across threads: every output element is still
 * computed by one thread in the same order, and every sum over rows (S, ||C||)
 * stays a serial ascending loop, so both builds give the same bits.
 *
 * Notation (paper, Section 2 and Algorithms 1-5):
 *   A in R^{m x p}, B in R^{q x n}, C in R^{m x n}, X in R^{p x q};
 *   a_i = ||A_{i,:}||^2, F = ||A||_F^2, R^k = C - A X^k B,
 *   s_i = ||R^k_{i,:}||^2, S = ||R^k||_F^2, c_k = alpha / a_{i_k}.
 *
 * Pins (tests/test_oracle_pins.py): least-norm solution A^+ C B^+ (Eq. 2.2),
 * full-rank closed forms (Section 2), ME-BK limit (Theorem 3.3), invariant
 * (Lemma 3.2, Eq. 3.1), per-step error identity (Eqs. 3.4-3.6), recursive
 * residual = C - A X^k B, MWRBK contraction (Eq. 4.18), non-empty admitted
 * set (Remark 4.1), theta = 1/2 reduction (Remark 4.4), hand-built admitted
 * sets and the pick distribution by chi-square,
 * expected-rate bounds (Eqs. 2.3, 4.2), numpy's Philox known answers.
 * No function here is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Wall time of the iteration loop of the last oracle_solve call (set-up
 * excluded), for timing the oracle; not thread-safe. */
static double g_loop_seconds = 0.0;
double oracle_last_loop_seconds(void) { return g_loop_seconds; }

static double wall_seconds(void)
{
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

/* Threads the "omp" loops run on: 1 in the tests' build. */
int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 counter-based generator, written from Salmon, Moraes, Dror,
 * Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11): ten rounds of
 * two 64x64->128 multiplies with a Weyl-sequence key schedule.              */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2E7470EE14C6C93ULL
#define PHILOX_M1 0xCA5A826395121157ULL
#define PHILOX_W0 0x9E3779B97F4A7C15ULL /* golden ratio */
#define PHILOX_W1 0xBB67AE8584CAA73BULL /* sqrt(3) - 1 */

void oracle_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        unsigned __int128 p0 = (unsigned __int128)PHILOX_M0 * x0;
        unsigned __int128 p1 = (unsigned __int128)PHILOX_M1 * x2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t y0 = hi1 ^ x1 ^ k0;
        uint64_t y2 = hi0 ^ x3 ^ k1;
        x0 = y0; x1 = lo1; x2 = y2; x3 = lo0;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Uniform draw of iteration k of system `sys`: key (seed, 0), counter
 * (k, sys, 0, 0), first output word, top 53 bits scaled to [0, 1). */
double oracle_uniform(uint64_t seed, uint64_t k, uint64_t sys)
{
    uint64_t ctr[4] = {k, sys, 0, 0}, key[2] = {seed, 0}, out[4];
    oracle_philox4x64_10(ctr, key, out);
    return (double)(out[0] >> 11) * 0x1.0p-53;
}

/* The extended method's column draw of iteration k: counter (k, sys, 1, 0). */
double oracle_uniform_column(uint64_t seed, uint64_t k, uint64_t sys)
{
    uint64_t ctr[4] = {k, sys, 1, 0}, key[2] = {seed, 0}, out[4];
    oracle_philox4x64_10(ctr, key, out);
    return (double)(out[0] >> 11) * 0x1.0p-53;
}

/* ------------------------------------------------------------------------ */
/* Dense helpers (plain triple loops, ascending index order).               */
/* ------------------------------------------------------------------------ */

/* R = C - A X B, evaluated as (A X) B.  Definition of the residual used by
 * Algorithms 3-4 initialisation and by Algorithms 1, 2, 5 every step. */
void oracle_residual(int64_t m, int64_t p, int64_t q, int64_t n, const double* A,
                     const double* X, const double* B, const double* C, double* R)
{
    double* AX = (double*)malloc(sizeof(double) * (size_t)(m * q > 0 ? m * q : 1));
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < q; ++j) {
            double acc = 0.0;
            for (int64_t c = 0; c < p; ++c) acc += A[i * p + c] * X[c * q + j];
            AX[i * q + j] = acc;
        }
    for (int64_t i = 0; i < m; ++i)
        for (int64_t l = 0; l < n; ++l) {
            double acc = 0.0;
            for (int64_t j = 0; j < q; ++j) acc += AX[i * q + j] * B[j * n + l];
            R[i * n + l] = C[i * n + l] - acc;
        }
    free(AX);
}

/* a_i = ||A_{i,:}||_2^2 for every row (the sampling weights of Algorithm 1 and
 * the denominators of every update). */
void oracle_row_sqnorms(int64_t m, int64_t p, const double* A, double* a)
{
    for (int64_t i = 0; i < m; ++i) {
        double acc = 0.0;
        for (int64_t c = 0; c < p; ++c) acc += A[i * p + c] * A[i * p + c];
        a[i] = acc;
    }
}

/* ||B||_2^2 = largest eigenvalue of B B^T by power iteration with a Rayleigh
 * quotient; alpha = 1 / ||B||_2^2 is the step the experiments use (Section 5). */
double oracle_spectral_norm_sq(int64_t q, int64_t n, const double* B, int64_t iters)
{
    double* x = (double*)malloc(sizeof(double) * (size_t)q);
    double* t = (double*)malloc(sizeof(double) * (size_t)n);
    double* y = (double*)malloc(sizeof(double) * (size_t)q);
    for (int64_t j = 0; j < q; ++j) x[j] = 1.0 + 0.01 * (double)(j % 7);
    double lam = 0.0;
    for (int64_t it = 0; it < iters; ++it) {
        double nx = 0.0;
        for (int64_t j = 0; j < q; ++j) nx += x[j] * x[j];
        nx = sqrt(nx);
        for (int64_t j = 0; j < q; ++j) x[j] /= nx;
        for (int64_t l = 0; l < n; ++l) { /* t = B^T x */
            double acc = 0.0;
            for (int64_t j = 0; j < q; ++j) acc += B[j * n + l] * x[j];
            t[l] = acc;
        }
        for (int64_t j = 0; j < q; ++j) { /* y = B t */
            double acc = 0.0;
            for (int64_t l = 0; l < n; ++l) acc += B[j * n + l] * t[l];
            y[j] = acc;
        }
        double xy = 0.0;
        for (int64_t j = 0; j < q; ++j) xy += x[j] * y[j];
        lam = xy; /* Rayleigh quotient x^T B B^T x with ||x|| = 1 */
        memcpy(x, y, sizeof(double) * (size_t)q);
    }
    free(x); free(t); free(y);
    return lam;
}

/* ------------------------------------------------------------------------ */
/* The iteration.                                                           */
/* ------------------------------------------------------------------------ */

enum { OR_GRBK = 0, OR_RGRBK = 1, OR_MWRBK = 2, OR_RBK = 3, OR_BK = 4 };
/* How R^{k+1} is obtained:
 *  GRAM     -- Algorithms 3-4 as printed: R -= c (A A^T)_{:,i} (R_i B^T B) with
 *              A A^T and B^T B formed once up front (the paper's practice note).
 *  FACTORED -- the same rank-1 update with the products re-associated:
 *              (A A_i^T) and ((R_i B^T) B); no m x m or n x n Gram matrix.
 *  LITERAL  -- R = C - A X B recomputed from the new X (Algorithms 1, 2, 5). */
enum { OR_MODE_GRAM = 0, OR_MODE_FACTORED = 1, OR_MODE_LITERAL = 2 };
enum { OR_STOP_NONE = 0, OR_STOP_RELRES = 1, OR_STOP_RSE = 2 };
/* status */
enum { OR_RAN_MAXIT = 0, OR_TOL_MET = 1, OR_EXACT = 2, OR_NOT_CONVERGED = 3 };

/*
 * oracle_solve -- run one system for at most `maxit` iterations.
 *
 * dims = {m, p, q, n}.  X holds X^0 on entry and X^k on exit (p x q).
 * variant: OR_GRBK (theta ignored, fixed 1/2), OR_RGRBK (theta in (0,1]),
 * OR_MWRBK, OR_RBK, OR_BK.  alpha is the step (Algorithms 1-5).  Random
 * variants draw u_k = oracle_uniform(seed, k, sys).
 *
 * Per iteration k (Algorithm 3 / 4 / 5 / 1 / 2):
 *   s_i = ||R_i||^2, S = sum_i s_i, r_i = s_i / a_i (rows with a_i = 0 skipped);
 *   GRBK/RGRBK: t = theta r_max + (1 - theta) S / F, clamped to r_max;
 *     J = {i : r_i >= t}; S_J = sum_J s_i; i_k = first i in J (ascending) whose
 *     running sum of s exceeds u S_J (last admitted row if none does);
 *   MWRBK: smallest i attaining r_max;  RBK: same inverse CDF over a_i;
 *   BK: i_k = k mod m (a zero row of A makes that step a no-op);
 *   w = R_{i_k} B^T;  X += c A_{i_k}^T w;  R updated per `mode`.
 * The stop test happens before selection at every k, with the current S and X.
 *
 * Optional traces (NULL to skip), length maxit unless noted:
 *   tr_rows   selected rows                tr_S      S before the step
 *   tr_t      threshold t (NaN if unused)  tr_madm   min_i |r_i - t| / t
 *   tr_mpick  min distance of the pick target to a prefix boundary, relative
 *             (for MWRBK: (r_max - second largest r) / r_max)
 *   tr_err2   ||X^k - Xref||_F^2, length maxit + 1 (needs Xref)
 * R_out (m x n) and s_out (m) receive the final residual and row norms.
 *
 * extended = 1: the inconsistent (least-squares, Eq. 2.1) extension, which the
 * paper defines the target of but does not solve.  As in the randomized
 * extended Kaczmarz method of Zouzias and Freris (SIAM J. Matrix Anal. Appl.,
 * 2013) an auxiliary Y (m x n, Y^0 = C) is driven to (I - A A^+) C by column
 * projections, and the row steps run on the residual R = C - Y - A X B of the
 * consistent system A X B = C - Y:
 *   at the start of iteration k < maxit, j_k = first column (ascending) whose
 *   running sum of ||A_{:,j}||^2 exceeds u'_k ||A||_F^2, u'_k =
 *   oracle_uniform_column(seed, k, sys); z = A_{:,j}^T Y (1 x n), g = z /
 *   ||A_{:,j}||^2; Y -= A_{:,j} g and R += A_{:,j} g (R = C - Y - A X B);
 *   then s_i, S, the stop tests (no stop on S = 0: R^0 = -A X^0 B may vanish
 *   while Y still moves) and the row step of `variant` on R.
 * When B has full column rank (B^+ B = I), X^k tends to A^+ C B^+ + (the part
 * of X^0 in the null space), the least-squares solution of least norm.
 * Y_out (m x n) receives the final Y (extended only).
 * Returns the number of iterations performed; *status gets OR_* status.
 */
int64_t oracle_solve(const int64_t* dims, const double* A, const double* B, const double* C,
                     double* X, int variant, double theta, double alpha, uint64_t seed,
                     uint64_t sys, int64_t maxit, int mode, int stop_kind, double tol,
                     const double* Xref, int64_t* tr_rows, double* tr_S, double* tr_t,
                     double* tr_madm, double* tr_mpick, double* tr_err2, double* R_out,
                     double* s_out, int* status, int extended, double* Y_out)
{
    const int64_t m = dims[0], p = dims[1], q = dims[2], n = dims[3];
    if (variant == OR_GRBK) theta = 0.5;

    double* R = (double*)malloc(sizeof(double) * (size_t)(m * n));
    double* a = (double*)malloc(sizeof(double) * (size_t)m);
    double* s = (double*)malloc(sizeof(double) * (size_t)m);
    double* r = (double*)malloc(sizeof(double) * (size_t)m);
    double* w = (double*)malloc(sizeof(double) * (size_t)q);
    double* g = (double*)malloc(sizeof(double) * (size_t)m);
    double* h = (double*)malloc(sizeof(double) * (size_t)n);
    double* GA = NULL;
    double* GB = NULL;
    double* Y = NULL;       /* extended: Y (m x n) */
    double* cn = NULL;      /* extended: ||A_{:,j}||^2 */
    double* zz = NULL;      /* extended: z / ||A_{:,j}||^2 (1 x n) */
    double Fc = 0.0;        /* extended: sum_j ||A_{:,j}||^2 */

    oracle_row_sqnorms(m, p, A, a);
    double F = 0.0;
    for (int64_t i = 0; i < m; ++i) F += a[i];

    if (mode == OR_MODE_GRAM) {
        /* A A^T (m x m) and B^T B (n x n), formed once. */
        GA = (double*)malloc(sizeof(double) * (size_t)(m * m));
        GB = (double*)malloc(sizeof(double) * (size_t)(n * n));
        for (int64_t i = 0; i < m; ++i)
            for (int64_t j = 0; j < m; ++j) {
                double acc = 0.0;
                for (int64_t c = 0; c < p; ++c) acc += A[i * p + c] * A[j * p + c];
                GA[i * m + j] = acc;
            }
        for (int64_t l1 = 0; l1 < n; ++l1)
            for (int64_t l2 = 0; l2 < n; ++l2) {
                double acc = 0.0;
                for (int64_t j = 0; j < q; ++j) acc += B[j * n + l1] * B[j * n + l2];
                GB[l1 * n + l2] = acc;
            }
    }

    /* R^0 = C - A X^0 B.  For X^0 = 0 every product term is a signed zero and
     * their sums are +0, so R^0 = C bit for bit; copying C skips the O(mpq + mqn)
     * loops, which dominate a few iterations on large systems. */
    int x0_zero = 1;
    for (int64_t i = 0; i < p * q && x0_zero; ++i) x0_zero = (X[i] == 0.0);
    if (x0_zero)
        memcpy(R, C, sizeof(double) * (size_t)(m * n));
    else
        oracle_residual(m, p, q, n, A, X, B, C, R);
    if (extended) {
        /* Y^0 = C, R^0 = C - Y^0 - A X^0 B */
        Y = (double*)malloc(sizeof(double) * (size_t)(m * n));
        cn = (double*)malloc(sizeof(double) * (size_t)p);
        zz = (double*)malloc(sizeof(double) * (size_t)n);
        memcpy(Y, C, sizeof(double) * (size_t)(m * n));
        for (int64_t i = 0; i < m * n; ++i) R[i] -= Y[i];
        for (int64_t j = 0; j < p; ++j) {
            double acc = 0.0;
            for (int64_t i = 0; i < m; ++i) acc += A[i * p + j] * A[i * p + j];
            cn[j] = acc;
            Fc += acc;
        }
    }

    int st =(stop_kind == OR_STOP_NONE) ? OR_RAN_MAXIT : OR_NOT_CONVERGED;
    double normC2 = 0.0;
    for (int64_t i = 0; i < m * n; ++i) normC2 += C[i] * C[i];
    double normXref2 = 0.0;
    if (Xref)
        for (int64_t i = 0; i < p * q; ++i) normXref2 += Xref[i] * Xref[i];

    const double t_loop = wall_seconds();
    int64_t k = 0;
    for (;; ++k) {
        if (extended && k < maxit) {
            /* column step: Y -= A_{:,j} (A_{:,j}^T Y) / ||A_{:,j}||^2, R moves the other way */
            double target = oracle_uniform_column(seed, (uint64_t)k, sys) * Fc, run = 0.0;
            int64_t j = -1, lastj = -1;
            for (int64_t c = 0; c < p; ++c) {
                if (cn[c] <= 0.0) continue;
                run += cn[c];
                lastj = c;
                if (run > target) { j = c; break; }
            }
            if (j < 0) j = lastj;
            for (int64_t l = 0; l < n; ++l) {
                double acc = 0.0;
                for (int64_t i = 0; i < m; ++i) acc += A[i * p + j] * Y[i * n + l];
                zz[l] = acc / cn[j];
            }
            for (int64_t i = 0; i < m; ++i)
                for (int64_t l = 0; l < n; ++l) {
                    Y[i * n + l] -= A[i * p + j] * zz[l];
                    R[i * n + l] += A[i * p + j] * zz[l];
                }
        }
        /* row norms and Frobenius norm of the current residual */
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < m; ++i) {
            double acc = 0.0;
            for (int64_t l = 0; l < n; ++l) acc += R[i * n + l] * R[i * n + l];
            s[i] = acc;
        }
        double S = 0.0;
        for (int64_t i = 0; i < m; ++i) S += s[i];
        double err2 = NAN;
        if (Xref) {
            err2 = 0.0;
            for (int64_t i = 0; i < p * q; ++i) {
                double d = X[i] - Xref[i];
                err2 += d * d;
            }
            if (tr_err2) tr_err2[k] = err2;
        }
        if (S == 0.0 && !extended) { st = OR_EXACT; break; }
        if (stop_kind == OR_STOP_RELRES && sqrt(S) <= tol * sqrt(normC2)) { st = OR_TOL_MET; break; }
        if (stop_kind == OR_STOP_RSE && Xref && sqrt(err2) <= tol * sqrt(normXref2)) { st = OR_TOL_MET; break; }
        if (k >= maxit) break;
        if (tr_S) tr_S[k] = S;

        /* weighted row residuals r_i = s_i / a_i and their maximum */
        double rmax = -INFINITY, r2 = -INFINITY;
        int64_t imax = -1;
        for (int64_t i = 0; i < m; ++i) {
            if (a[i] > 0.0) {
                r[i] = s[i] / a[i];
                if (r[i] > rmax) { r2 = rmax; rmax = r[i]; imax = i; }
                else if (r[i] > r2) r2 = r[i];
            } else {
                r[i] = -INFINITY;
            }
        }

        int64_t ik = -1;
        double t = NAN, madm = INFINITY, mpick = INFINITY;
        if (variant == OR_GRBK || variant == OR_RGRBK) {
            /* threshold: xi_k S = theta r_max + (1 - theta) S / F  (Alg. 3 zeta_k, Alg. 4 xi_k) */
            t = theta * rmax + (1.0 - theta) * (S / F);
            if (t > rmax) t = rmax; /* keeps the maximiser admitted (Remark 4.1) */
            double SJ = 0.0;
            for (int64_t i = 0; i < m; ++i) {
                if (a[i] <= 0.0) continue;
                double d = fabs(r[i] - t) / t;
                if (d < madm) madm = d;
                if (r[i] >= t) SJ += s[i];
            }
            double u = oracle_uniform(seed, (uint64_t)k, sys);
            double target = u * SJ, run = 0.0;
            int64_t last = -1;
            for (int64_t i = 0; i < m; ++i) {
                if (a[i] <= 0.0 || !(r[i] >= t)) continue;
                run += s[i];
                last = i;
                double d = fabs(run - target) / SJ;
                if (d < mpick) mpick = d;
                if (ik < 0 && run > target) ik = i;
            }
            if (ik < 0) ik = last;
        } else if (variant == OR_MWRBK) {
            ik = imax; /* first index attaining the max (strict '>' above) */
            mpick = (r2 == -INFINITY) ? INFINITY : (rmax - r2) / rmax;
        } else if (variant == OR_RBK) {
            double u = oracle_uniform(seed, (uint64_t)k, sys);
            double target = u * F, run = 0.0;
            int64_t last = -1;
            for (int64_t i = 0; i < m; ++i) {
                if (a[i] <= 0.0) continue;
                run += a[i];
                last = i;
                double d = fabs(run - target) / F;
                if (d < mpick) mpick = d;
                if (ik < 0 && run > target) ik = i;
            }
            if (ik < 0) ik = last;
        } else { /* OR_BK */
            ik = k % m;
        }
        if (tr_rows) tr_rows[k] = ik;
        if (tr_t) tr_t[k] = t;
        if (tr_madm) tr_madm[k] = madm;
        if (tr_mpick) tr_mpick[k] = mpick;

        if (a[ik] <= 0.0) continue; /* zero row of A (ME-BK only): no update */
        const double c = alpha / a[ik];

        /* w = R_{i_k} B^T  (1 x q) */
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < q; ++j) {
            double acc = 0.0;
            for (int64_t l = 0; l < n; ++l) acc += R[ik * n + l] * B[j * n + l];
            w[j] = acc;
        }
        /* X^{k+1} = X^k + c A_{i_k}^T w */
#pragma omp parallel for schedule(static)
        for (int64_t row = 0; row < p; ++row)
            for (int64_t j = 0; j < q; ++j) X[row * q + j] += c * A[ik * p + row] * w[j];

        if (mode == OR_MODE_LITERAL) {
            oracle_residual(m, p, q, n, A, X, B, C, R);
            if (extended)
                for (int64_t i = 0; i < m * n; ++i) R[i] -= Y[i];
            continue;
        }
        if (mode == OR_MODE_GRAM) {
            for (int64_t i = 0; i < m; ++i) g[i] = GA[i * m + ik]; /* (A A^T)_{:,i_k} */
            for (int64_t l = 0; l < n; ++l) {                      /* R_{i_k} (B^T B) */
                double acc = 0.0;
                for (int64_t l2 = 0; l2 < n; ++l2) acc += R[ik * n + l2] * GB[l2 * n + l];
                h[l] = acc;
            }
        } else {
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < m; ++i) { /* A A_{i_k}^T */
                double acc = 0.0;
                for (int64_t cc = 0; cc < p; ++cc) acc += A[i * p + cc] * A[ik * p + cc];
                g[i] = acc;
            }
#pragma omp parallel for schedule(static)
            for (int64_t l = 0; l < n; ++l) { /* (R_{i_k} B^T) B */
                double acc = 0.0;
                for (int64_t j = 0; j < q; ++j) acc += w[j] * B[j * n + l];
                h[l] = acc;
            }
        }
        /* R^{k+1} = R^k - c g h  (Algorithm 3, last step) */
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < m; ++i)
            for (int64_t l = 0; l < n; ++l) R[i * n + l] -= c * g[i] * h[l];
    }

    g_loop_seconds = wall_seconds() - t_loop;
    if (R_out) memcpy(R_out, R, sizeof(double) * (size_t)(m * n));
    if (s_out) memcpy(s_out, s, sizeof(double) * (size_t)m);
    if (Y_out && Y) memcpy(Y_out, Y, sizeof(double) * (size_t)(m * n));
    if (status) *status = st;
    free(R); free(a); free(s); free(r); free(w); free(g); free(h);
    free(GA); free(GB); free(Y); free(cn); free(zz);
    return k;
}
