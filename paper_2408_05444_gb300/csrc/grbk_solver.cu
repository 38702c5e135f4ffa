// grbk_solver.cu -- single-system solver: set-up kernels, the persistent
// grid-synchronised iteration kernel and the host driver behind grbk_create /
// grbk_solve / grbk_residual / grbk_destroy.
//
// One iteration k (Algorithms 1-5 with the residual recursion of Algorithm 3):
//   select   S = sum_i s_i, r_max, threshold, admitted set, Philox pick i_k
//   W/U      w = R_{i_k} B^T (q values), u = A A_{i_k}^T (m values)
//   V        v = w B (n values)
//   F        R -= (alpha/a_{i_k}) u v  fused with the new s_i = ||R_i||^2,
//            r_i = s_i / a_i and per-CTA partial sums / maxima
// separated by bounded grid barriers.  X is not touched inside the loop: the
// pairs (i_k, c_k, w_k) are recorded and folded into X once per chunk as a
// small GEMM (the sum of the same rank-1 terms, re-associated).
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "grbk_internal.cuh"

namespace grbk {

static thread_local char g_err[512];

void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line)
{
    snprintf(g_err, sizeof(g_err), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    if (getenv("GRBK_VERBOSE")) fprintf(stderr, "grbk: %s\n", g_err);
}

constexpr int kBlock = 512;        // threads per CTA of the persistent kernel
constexpr int kWarps = kBlock / 32;
constexpr int kUnroll = 8;         // independent vector loads in flight per lane
constexpr int kMaxGrid = 320;      // largest grid of the persistent kernel (pick_row: 32 x 10 partials)
constexpr int kPartsCap = 2048;    // per-CTA (row, chunk) partial slots in shared memory

template <typename T> struct VecOf;
template <> struct VecOf<float> { using V = float4; static constexpr int N = 4; };
template <> struct VecOf<double> { using V = double2; static constexpr int N = 2; };

__device__ __forceinline__ float4 ldcg_v(const float4* p) { return __ldcg(p); }
__device__ __forceinline__ double2 ldcg_v(const double2* p) { return __ldcg(p); }
__device__ __forceinline__ void stcg_v(float4* p, float4 v) { __stcg(p, v); }
__device__ __forceinline__ void stcg_v(double2* p, double2 v) { __stcg(p, v); }
// R is streamed once per iteration: evict-first loads and stores keep it from
// pushing B, u and v out of L2
__device__ __forceinline__ float4 ldcs_v(const float4* p) { return __ldcs(p); }
__device__ __forceinline__ double2 ldcs_v(const double2* p) { return __ldcs(p); }
__device__ __forceinline__ void stcs_v(float4* p, float4 v) { __stcs(p, v); }
__device__ __forceinline__ void stcs_v(double2* p, double2 v) { __stcs(p, v); }

// ----------------------------------------------------------------------------
// kernel parameters
// ----------------------------------------------------------------------------
template <typename T>
struct IterParams {
    int64_t m, p, q, n;
    int64_t lda, ldb, ldr;      // row strides (elements) of A, B and R/C (padded)
    const T* A;
    const T* B;
    T* R;
    const double* a;            // ||A_i||^2
    const double* rbk_prefix;   // running sums of a_i (ME-RBK inverse CDF)
    double2* sr;                // (||R_i||^2, s_i / a_i); r = -inf for zero rows of A
    T* u;                       // A A_{i_k}^T
    T* v;                       // w B, ldr entries (padding stays 0)
    T* w;                       // R_{i_k} B^T
    double4* part;              // per CTA: (sum of s_i, max r_i, its row as bits, unused)
    double* part_SJ;            // per-CTA admitted sums
    int* hist_rows;             // per chunk: i_k
    double* hist_c;             //            alpha / a_{i_k}
    double* hist_w;             //            w (q doubles per iteration)
    int* trace_rows;            // whole solve: i_k (device copy of the host trace)
    double* trace_S;
    long long trace_len;
    GridBarrier* bar;
    DevState* st;
    double F, alpha, theta, stop_S;   // stop when S <= stop_S (RELRES), < 0 disables
    int variant;
    uint64_t seed, sys;
    long long k0;
    int nit;
    int smem_v;                 // v / R_{i_k} staged in shared memory
    int smem_arow;              // A_{i_k} staged in shared memory
    const T* G;                 // A A^T (m x ldg) or null
    int64_t ldg;
    const double* soff;         // fixed row offsets added to s_i (row-space form) or null
    const T* K;                 // row-space form: Lt^T Lt (n x ldk); then v = R_{i_k} K and w is formed per chunk
    int64_t ldk;
    T* hist_z;                  // with K: per chunk the selected rows R_{i_k} (ldr per iteration)
    // deferred update (FP32): during a chunk R stays at its value R^0 from the chunk's start;
    // the current residual is R^0 - sum_j U'_j v_j^T over the chunk's iterations j so far,
    // with U'_j = c_j A A_{i_j}^T and v_j kept below; row norms follow by recurrence, and
    // R is written back (or refreshed) after the chunk
    int defer;
    T* uh;                      // cap x m: U'_j
    T* vh;                      // cap x ldr: v_j
    float2* gp;                 // (cap + 1) x G: per-CTA double-float partials of v_j . v_it
    T* rik;                     // ldr: the current row R_{i_k}, assembled across the CTAs
    int defer_stage;            // the slab's v_j of a whole chunk fit in the dynamic shared memory
};

constexpr int kDeferCap = 64;   // longest chunk the deferred update keeps

// (hi, lo) += (bh, bl) in FP32 arithmetic (two-sum, then renormalised)
__device__ __forceinline__ void df_add(float& hi, float& lo, float bh, float bl)
{
    const float s = __fadd_rn(hi, bh);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
    const float l = __fadd_rn(__fadd_rn(err, lo), bl);
    hi = __fadd_rn(s, l);
    lo = __fsub_rn(l, __fsub_rn(hi, s));
}

// (hi, lo) += a * (bh + bl): the product a bh exactly as p + e (one FMA), a bl rounded
__device__ __forceinline__ void df_fma(float& hi, float& lo, float a, float bh, float bl)
{
    const float p = __fmul_rn(a, bh);
    const float e = __fmaf_rn(a, bh, -p);
    df_add(hi, lo, p, __fmaf_rn(a, bl, e));
}

// balanced contiguous row range of CTA c among G
__device__ __forceinline__ void cta_rows(int64_t m, int c, int G, int64_t& r0, int64_t& r1)
{
    r0 = (m * (int64_t)c) / G;
    r1 = (m * (int64_t)(c + 1)) / G;
}

// ----------------------------------------------------------------------------
// Fused residual pass over rows [r0, r1): R_i -= coef_i v (if UPDATE), then
// s_i = ||R_i||^2 (FP64 sum of per-lane partials; FP32 lanes use Kahan
// compensation), r_i = s_i / a_i, and the CTA's partial sum / argmax.
// ----------------------------------------------------------------------------
// sm_sr (optional): this CTA's (s_i, r_i), rows r0.. in order, kept in shared memory
constexpr int kSrCap = 512;

template <typename T, bool UPDATE>
__device__ __noinline__ void fused_pass(const IterParams<T>& P, double ck, const T* vsrc, int64_t r0, int64_t r1,
                           double* sm_parts, double* sm_red, long long* sm_redi, double2* sm_sr = nullptr)
{
    using V = typename VecOf<T>::V;
    constexpr int VN = VecOf<T>::N;
    constexpr int CHV = 32 * kUnroll * 2;       // vectors per (row, chunk) unit
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nvec_row = P.ldr / VN;
    const int nch = (int)((nvec_row + CHV - 1) / CHV);
    int64_t rows_per_batch = kPartsCap / nch;
    if (rows_per_batch < 1) rows_per_batch = 1;
    if (rows_per_batch > kBlock) rows_per_batch = kBlock;

    double cta_S = 0.0;
    long long cta_key = __double_as_longlong(-INFINITY), cta_bi = LLONG_MAX;

    float2* sm_df = reinterpret_cast<float2*>(sm_parts);   // FP32: (row, chunk) partials as double-float pairs
    for (int64_t b0 = r0; b0 < r1; b0 += rows_per_batch) {
        const int64_t b1 = min(r1, b0 + rows_per_batch);
        const int units = (int)((b1 - b0) * nch);
        for (int unit = warp; unit < units; unit += kWarps) {
            const int rq = unit / nch;
            const int64_t row = b0 + rq;
            const int64_t e0 = (int64_t)(unit - rq * nch) * CHV;
            const int64_t e1 = min(nvec_row, e0 + CHV);
            V* Rrow = reinterpret_cast<V*>(P.R + row * P.ldr);
            const V* vrow = reinterpret_cast<const V*>(vsrc);
            T coef = (T)0;
            if (UPDATE) coef = __ldcg(P.u + row);  // c_k u_row, formed once per row
            double acc_d = 0.0;
            float acc_f = 0.f, comp_f = 0.f;
            for (int64_t base = e0; base < e1; base += 32 * kUnroll) {
                V rv[kUnroll];
#pragma unroll
                for (int uu = 0; uu < kUnroll; ++uu) {
                    const int64_t e = base + uu * 32 + lane;
                    if (e < e1) rv[uu] = ldcs_v(Rrow + e);
                }
#pragma unroll
                for (int uu = 0; uu < kUnroll; ++uu) {
                    const int64_t e = base + uu * 32 + lane;
                    if (e < e1) {
                        V vv;
                        if (UPDATE) vv = P.smem_v ? vrow[e] : ldcg_v(vrow + e);
                        T* x = reinterpret_cast<T*>(&rv[uu]);
                        const T* y = reinterpret_cast<const T*>(&vv);
#pragma unroll
                        for (int c = 0; c < VN; ++c) {
                            if (UPDATE) x[c] = fma(-coef, y[c], x[c]);
                            if constexpr (sizeof(T) == 8) {
                                acc_d = fma((double)x[c], (double)x[c], acc_d);
                            } else {
                                const float yk = fmaf((float)x[c], (float)x[c], -comp_f);
                                const float tk = acc_f + yk;
                                comp_f = (tk - acc_f) - yk;
                                acc_f = tk;
                            }
                        }
                        if (UPDATE) stcs_v(Rrow + e, rv[uu]);
                    }
                }
            }
            if constexpr (sizeof(T) == 8) {
                const double tot = warp_sum(acc_d);
                if (lane == 0) sm_parts[unit] = tot;
            } else {
                float hi = acc_f, lo = -comp_f;  // Kahan state as a double-float
                warp_sum_df(hi, lo);
                if (lane == 0) sm_df[unit] = make_float2(hi, lo);
            }
        }
        __syncthreads();
        // finalise the rows of this batch: one thread per row
        double my_S = 0.0;
        long long my_key = LLONG_MIN, my_bi = LLONG_MAX;
        for (int64_t rr = threadIdx.x; rr < b1 - b0; rr += kBlock) {
            double sv = 0.0;
            if constexpr (sizeof(T) == 8) {
                for (int c = 0; c < nch; ++c) sv += sm_parts[rr * nch + c];
            } else {
                float sh = 0.f, sl = 0.f;
                for (int c = 0; c < nch; ++c) df_add(sh, sl, sm_df[rr * nch + c].x, sm_df[rr * nch + c].y);
                sv = (double)sh + (double)sl;
            }
            const int64_t row = b0 + rr;
            if (P.soff) sv += __ldg(P.soff + row);
            const double ai = __ldg(P.a + row);
            const double ri = (ai > 0.0) ? __ddiv_rn(sv, ai) : -INFINITY;
            __stcg(P.sr + row, make_double2(sv, ri));
            if (sm_sr) sm_sr[row - r0] = make_double2(sv, ri);
            my_S += sv;
            const long long rk = __double_as_longlong(ri);  // r >= 0 or -inf: integer order
            if (rk > my_key) { my_key = rk; my_bi = row; }
        }
        // block reduction in a fixed order, only on the warps that hold rows of the batch
        // (an FP64 warp instruction costs the same with idle lanes), argmax on the integer pipe
        const int nact = (int)min((int64_t)kWarps, (b1 - b0 + 31) / 32);
        if (warp < nact) {
            my_S = warp_sum(my_S);
            warp_argmax_key(my_key, my_bi);
            if (lane == 0) {
                sm_red[warp] = my_S;
                sm_red[kWarps + warp] = __longlong_as_double(my_key);
                sm_redi[warp] = my_bi;
            }
        }
        __syncthreads();
        if (warp == 0) {
            double bs = lane < nact ? sm_red[lane] : 0.0;
            long long bk = lane < nact ? __double_as_longlong(sm_red[kWarps + lane]) : LLONG_MIN;
            long long bi = lane < nact ? sm_redi[lane] : LLONG_MAX;
            bs = warp_sum(bs);
            warp_argmax_key(bk, bi);
            if (lane == 0) {
                cta_S += bs;
                if (bk > cta_key || (bk == cta_key && bi < cta_bi)) { cta_key = bk; cta_bi = bi; }
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double2* pp = reinterpret_cast<double2*>(P.part + blockIdx.x);
        __stcg(pp, make_double2(cta_S, __longlong_as_double(cta_key)));
        __stcg(pp + 1, make_double2(__longlong_as_double(cta_bi), 0.0));
    }
}

// The vector slab [e0, e1) of CTA c: the same split as cols_gemv's.
__device__ __forceinline__ void v_slab(int64_t nvt, int c, int G, int64_t& e0, int64_t& e1)
{
    const int64_t slab = (nvt + G - 1) / G;
    e0 = (int64_t)c * slab;
    e1 = min(nvt, e0 + slab);
}

// Deferred update: this CTA's slab of the current row R_ik = R^0_ik - sum_{j<it} U'_{ik,j} v_j
// into P.rik, the terms in iteration order as the in-place update applies them.
// With P.defer_stage the slab's v_j are first copied into `stage` (the dynamic shared
// memory, idle at this point of the iteration) by all threads, one load each.
template <typename T>
__device__ __noinline__ void defer_row(const IterParams<T>& P, int it, long long ik, int c, int G, float* s_uik,
                                       T* stage)
{
    if constexpr (sizeof(T) == 4) {
        using V = typename VecOf<T>::V;
        constexpr int VN = VecOf<T>::N;
        int64_t e0, e1;
        v_slab(P.ldr / VN, c, G, e0, e1);
        const int64_t ns = e1 - e0;
        const V* R0 = reinterpret_cast<const V*>(P.R + ik * P.ldr);
        for (int j = threadIdx.x; j < it; j += kBlock) s_uik[j] = __ldcg(P.uh + (int64_t)j * P.m + ik);
        if (P.defer_stage) {
            V* st = reinterpret_cast<V*>(stage);
            if (ns > 0)
                for (int64_t t = threadIdx.x; t < (int64_t)it * ns; t += kBlock) {
                    const int64_t j = t / ns;
                    st[t] = ldcg_v(reinterpret_cast<const V*>(P.vh + j * P.ldr) + e0 + (t - j * ns));
                }
            __syncthreads();
            for (int64_t e = threadIdx.x; e < ns; e += kBlock) {
                V x = __ldg(R0 + e0 + e);  // R is not written during a deferred chunk
                float* xf = reinterpret_cast<float*>(&x);
#pragma unroll 8
                for (int j = 0; j < it; ++j) {
                    const float cj = s_uik[j];
                    const V y4 = st[(int64_t)j * ns + e];
                    const float* y = reinterpret_cast<const float*>(&y4);
#pragma unroll
                    for (int cc = 0; cc < VN; ++cc) xf[cc] = __fmaf_rn(-cj, y[cc], xf[cc]);
                }
                stcg_v(reinterpret_cast<V*>(P.rik) + e0 + e, x);
            }
            return;
        }
        __syncthreads();
        for (int64_t e = e0 + threadIdx.x; e < e1; e += kBlock) {
            V x = __ldg(R0 + e);  // R is not written during a deferred chunk
            float* xf = reinterpret_cast<float*>(&x);
            for (int jb = 0; jb < it; jb += 8) {
                V vv[8];
#pragma unroll
                for (int uu = 0; uu < 8; ++uu)
                    if (jb + uu < it) vv[uu] = ldcg_v(reinterpret_cast<const V*>(P.vh + (int64_t)(jb + uu) * P.ldr) + e);
#pragma unroll
                for (int uu = 0; uu < 8; ++uu) {
                    if (jb + uu < it) {
                        const float cj = s_uik[jb + uu];
                        const float* y = reinterpret_cast<const float*>(&vv[uu]);
#pragma unroll
                        for (int cc = 0; cc < VN; ++cc) xf[cc] = __fmaf_rn(-cj, y[cc], xf[cc]);
                    }
                }
            }
            stcg_v(reinterpret_cast<V*>(P.rik) + e, x);
        }
    }
}

// Deferred update: this CTA's partials of v_j . v_it, j <= it, over its slab of v (the
// slab cols_gemv just wrote), one warp per j, exact products summed in double-float.
template <typename T>
__device__ __noinline__ void defer_gram_partial(const IterParams<T>& P, int it, int c, int G)
{
    if constexpr (sizeof(T) == 4) {
        constexpr int VN = VecOf<T>::N;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        int64_t e0, e1;
        v_slab((P.K ? P.ldk : P.ldb) / VN, c, G, e0, e1);
        const int64_t f0 = e0 * VN, f1 = max(f0, e1 * VN);
        const float* vi = P.vh + (int64_t)it * P.ldr;
        for (int j = warp; j <= it; j += kWarps) {
            const float* vj = P.vh + (int64_t)j * P.ldr;
            float hi = 0.f, lo = 0.f;
            for (int64_t f = f0 + lane; f < f1; f += 32) {
                const float a = __ldcg(vj + f), b = __ldcg(vi + f);
                const float pr = __fmul_rn(a, b);
                df_add(hi, lo, pr, __fmaf_rn(a, b, -pr));
            }
            warp_sum_df(hi, lo);
            if (lane == 0) __stcg(P.gp + (int64_t)j * G + c, make_float2(hi, lo));
        }
    }
}

// Deferred update: the Gram column v_j . v_it, j <= it, from the CTA partials in one fixed
// order (every CTA forms the same values).
template <typename T>
__device__ __noinline__ void defer_gram_column(const IterParams<T>& P, int it, int G, float2* s_gf)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = warp; j <= it; j += kWarps) {
        float hi = 0.f, lo = 0.f;
        for (int cc = lane; cc < G; cc += 32) {
            const float2 pg = __ldcg(P.gp + (int64_t)j * G + cc);
            df_add(hi, lo, pg.x, pg.y);
        }
        warp_sum_df(hi, lo);
        if (lane == 0) s_gf[j] = make_float2(hi, lo);
    }
}

// ----------------------------------------------------------------------------
// Deferred form of the residual pass over rows [r0, r1) (R itself is not written):
// d_i = R_i . v_it with R_i the current row, then
//     ||R_i - U'_i v||^2 = s_i - 2 U'_i d_i + U'_i^2 ||v||^2,
// with R_i . v_it = R^0_i . v_it - sum_{j<it} U'_{ij} (v_j . v_it): one read of R^0 per
// iteration instead of a read and a write of R.  R^0_i . v_it is summed from exact FP32
// products in double-float (hi, lo) arithmetic, the correction from the Gram column
// s_gf (double-float) and the CTA's U' rows; s_corr holds the correction in four
// partial sums per row (quarters of the j range), formed before the streaming starts.
// ----------------------------------------------------------------------------
template <typename T>
__device__ __noinline__ void deferred_pass(const IterParams<T>& P, int it, const T* vsrc, const T* ucur,
                                           int64_t r0, int64_t r1, const float2* s_gf, double gkk,
                                           float2* s_corr, double* sm_parts, double* sm_red, long long* sm_redi,
                                           double2* sm_sr)
{
    if constexpr (sizeof(T) == 4) {
        using V = typename VecOf<T>::V;
        constexpr int VN = VecOf<T>::N;
        constexpr int CHV = 32 * kUnroll * 2;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int64_t nvec_row = P.ldr / VN;
        const int nch = (int)((nvec_row + CHV - 1) / CHV);
        int64_t rows_per_batch = kPartsCap / nch;
        if (rows_per_batch < 1) rows_per_batch = 1;
        if (rows_per_batch > kBlock) rows_per_batch = kBlock;
        const int nr = (int)(r1 - r0);

        // the correction sum_{j<it} U'_{ij} g_j, four quarters of j per row, coalesced over rows
        {
            const int qlen = (it + 3) / 4;
            for (int t = threadIdx.x; t < 4 * nr; t += kBlock) {
                const int qq = t / nr, rl = t - qq * nr;
                const int j0 = qq * qlen, j1 = min(it, j0 + qlen);
                float hi = 0.f, lo = 0.f;
                for (int jb = j0; jb < j1; jb += 8) {
                    float uv[8];
#pragma unroll
                    for (int uu = 0; uu < 8; ++uu)
                        uv[uu] = (jb + uu < j1) ? __ldcg(P.uh + (int64_t)(jb + uu) * P.m + r0 + rl) : 0.f;
#pragma unroll
                    for (int uu = 0; uu < 8; ++uu)
                        if (jb + uu < j1) df_fma(hi, lo, uv[uu], s_gf[jb + uu].x, s_gf[jb + uu].y);
                }
                s_corr[qq * kSrCap + rl] = make_float2(hi, lo);
            }
        }

        // (row, chunk) partials as double-float pairs: no FP64 instruction per unit
        float2* sm_df = reinterpret_cast<float2*>(sm_parts);
        double cta_S = 0.0;
        long long cta_key = __double_as_longlong(-INFINITY), cta_bi = LLONG_MAX;
        for (int64_t b0 = r0; b0 < r1; b0 += rows_per_batch) {
            const int64_t b1 = min(r1, b0 + rows_per_batch);
            const int units = (int)((b1 - b0) * nch);
            for (int unit = warp; unit < units; unit += kWarps) {
                const int rq = unit / nch;
                const int64_t row = b0 + rq;
                const int64_t e0 = (int64_t)(unit - rq * nch) * CHV;
                const int64_t e1 = min(nvec_row, e0 + CHV);
                const V* Rrow = reinterpret_cast<const V*>(P.R + row * P.ldr);
                const V* vrow = reinterpret_cast<const V*>(vsrc);
                float acc = 0.f, comp = 0.f, err = 0.f;
                for (int64_t base = e0; base < e1; base += 32 * kUnroll) {
                    V rv[kUnroll];
#pragma unroll
                    for (int uu = 0; uu < kUnroll; ++uu) {
                        const int64_t e = base + uu * 32 + lane;
                        if (e < e1) rv[uu] = ldcs_v(Rrow + e);
                    }
#pragma unroll
                    for (int uu = 0; uu < kUnroll; ++uu) {
                        const int64_t e = base + uu * 32 + lane;
                        if (e < e1) {
                            const V vv = P.smem_v ? vrow[e] : ldcg_v(vrow + e);
                            const float* x = reinterpret_cast<const float*>(&rv[uu]);
                            const float* y = reinterpret_cast<const float*>(&vv);
#pragma unroll
                            for (int cc = 0; cc < VN; ++cc) {
                                const float pr = __fmul_rn(x[cc], y[cc]);
                                err = __fadd_rn(err, __fmaf_rn(x[cc], y[cc], -pr));
                                const float yk = __fsub_rn(pr, comp);
                                const float tk = __fadd_rn(acc, yk);
                                comp = __fsub_rn(__fsub_rn(tk, acc), yk);
                                acc = tk;
                            }
                        }
                    }
                }
                float hi = acc, lo = __fsub_rn(err, comp);
                warp_sum_df(hi, lo);
                if (lane == 0) sm_df[unit] = make_float2(hi, lo);
            }
            __syncthreads();
            double my_S = 0.0;
            long long my_key = LLONG_MIN, my_bi = LLONG_MAX;
            for (int64_t rr = threadIdx.x; rr < b1 - b0; rr += kBlock) {
                float dh = 0.f, dl = 0.f;
                for (int c2 = 0; c2 < nch; ++c2) df_add(dh, dl, sm_df[rr * nch + c2].x, sm_df[rr * nch + c2].y);
                const double dot = (double)dh + (double)dl;
                const int64_t row = b0 + rr;
                const int rl = (int)(row - r0);
                float ch = s_corr[rl].x, cl = s_corr[rl].y;
#pragma unroll
                for (int qq = 1; qq < 4; ++qq) df_add(ch, cl, s_corr[qq * kSrCap + rl].x, s_corr[qq * kSrCap + rl].y);
                const double d = dot - ((double)ch + (double)cl);
                const double coef = (double)__ldcg(ucur + row);
                double sv = sm_sr[rl].x + coef * (coef * gkk - 2.0 * d);
                if (sv < 0.0) sv = 0.0;  // rounding below an exactly vanishing row
                const double ai = __ldg(P.a + row);
                const double ri = (ai > 0.0) ? __ddiv_rn(sv, ai) : -INFINITY;
                __stcg(P.sr + row, make_double2(sv, ri));
                sm_sr[rl] = make_double2(sv, ri);
                my_S += sv;
                const long long rk = __double_as_longlong(ri);
                if (rk > my_key) { my_key = rk; my_bi = row; }
            }
            const int nact = (int)min((int64_t)kWarps, (b1 - b0 + 31) / 32);
            if (warp < nact) {
                my_S = warp_sum(my_S);
                warp_argmax_key(my_key, my_bi);
                if (lane == 0) {
                    sm_red[warp] = my_S;
                    sm_red[kWarps + warp] = __longlong_as_double(my_key);
                    sm_redi[warp] = my_bi;
                }
            }
            __syncthreads();
            if (warp == 0) {
                double bs = lane < nact ? sm_red[lane] : 0.0;
                long long bk = lane < nact ? __double_as_longlong(sm_red[kWarps + lane]) : LLONG_MIN;
                long long bi = lane < nact ? sm_redi[lane] : LLONG_MAX;
                bs = warp_sum(bs);
                warp_argmax_key(bk, bi);
                if (lane == 0) {
                    cta_S += bs;
                    if (bk > cta_key || (bk == cta_key && bi < cta_bi)) { cta_key = bk; cta_bi = bi; }
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            double2* pp = reinterpret_cast<double2*>(P.part + blockIdx.x);
            __stcg(pp, make_double2(cta_S, __longlong_as_double(cta_key)));
            __stcg(pp + 1, make_double2(__longlong_as_double(cta_bi), 0.0));
        }
    }
}

// Row norms of the current R (no update), same partition and partials as the
// persistent kernel.  Launched with the solve's grid size.
template <typename T>
__global__ void __launch_bounds__(kBlock) rownorms_kernel(IterParams<T> P)
{
    __shared__ double sm_parts[kPartsCap];
    __shared__ double sm_red[2 * kWarps];
    __shared__ long long sm_redi[kWarps];
    int64_t r0, r1;
    cta_rows(P.m, blockIdx.x, gridDim.x, r0, r1);
    IterParams<T> Q = P;
    Q.smem_v = 0;
    fused_pass<T, false>(Q, 0.0, nullptr, r0, r1, sm_parts, sm_red, sm_redi);
}

// ----------------------------------------------------------------------------
// dst[row] = X_row . y for rows [r0, r1) of X (row stride ld elements), as
// (row, chunk) units per warp with kUnroll independent vector loads in flight;
// per-unit partial sums are combined in a fixed order.  ymode: 0 = y in shared
// memory, 1 = y written earlier in this kernel (L2 loads), 2 = y read-only.
// dst_hist (optional) receives the FP64 sums.
// ----------------------------------------------------------------------------
template <typename T>
__device__ __noinline__ void rows_dot(const T* X, int64_t ld, int64_t r0, int64_t r1, const T* y, int ymode, T* dst,
                         double* dst_hist, double* sm_parts, double scale = 1.0)
{
    using V = typename VecOf<T>::V;
    constexpr int VN = VecOf<T>::N;
    constexpr int CHV = 32 * kUnroll * 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nvec = ld / VN;
    const int nch = (int)((nvec + CHV - 1) / CHV);
    int64_t rows_per_batch = kPartsCap / nch;
    if (rows_per_batch < 1) rows_per_batch = 1;
    if (rows_per_batch > kBlock) rows_per_batch = kBlock;
    const V* yv = reinterpret_cast<const V*>(y);
    for (int64_t b0 = r0; b0 < r1; b0 += rows_per_batch) {
        const int64_t b1 = min(r1, b0 + rows_per_batch);
        const int64_t units = (b1 - b0) * nch;
        for (int64_t unit = warp; unit < units; unit += kWarps) {
            const int64_t row = b0 + unit / nch;
            const int ch = (int)(unit % nch);
            const int64_t e0 = (int64_t)ch * CHV, e1 = min(nvec, e0 + CHV);
            const V* xrow = reinterpret_cast<const V*>(X + row * ld);
            T acc0 = 0, acc1 = 0;
            for (int64_t base = e0; base < e1; base += 32 * kUnroll) {
                V xs[kUnroll];
#pragma unroll
                for (int uu = 0; uu < kUnroll; ++uu) {
                    const int64_t e = base + uu * 32 + lane;
                    if (e < e1) xs[uu] = __ldg(xrow + e);
                }
#pragma unroll
                for (int uu = 0; uu < kUnroll; ++uu) {
                    const int64_t e = base + uu * 32 + lane;
                    if (e < e1) {
                        const V ys = (ymode == 0) ? yv[e] : (ymode == 1 ? ldcg_v(yv + e) : __ldg(yv + e));
                        const T* a = reinterpret_cast<const T*>(&xs[uu]);
                        const T* b = reinterpret_cast<const T*>(&ys);
#pragma unroll
                        for (int cc = 0; cc < VN; cc += 2) {
                            acc0 = fma(a[cc], b[cc], acc0);
                            acc1 = fma(a[cc + 1], b[cc + 1], acc1);
                        }
                    }
                }
            }
            if constexpr (sizeof(T) == 8) {
                const double tot = warp_sum(acc0 + acc1);
                if (lane == 0) sm_parts[unit] = tot;
            } else {
                const float tot = warp_sum_f(acc0 + acc1);
                if (lane == 0) sm_parts[unit] = (double)tot;
            }
        }
        __syncthreads();
        for (int64_t rr = threadIdx.x; rr < b1 - b0; rr += kBlock) {
            double sum = 0.0;
            for (int c2 = 0; c2 < nch; ++c2) sum += sm_parts[rr * nch + c2];
            __stcg(dst + b0 + rr, (T)(scale * sum));
            if (dst_hist) dst_hist[b0 + rr] = sum;
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------
// v = w B for this CTA's slab of vector columns: each thread owns one vector
// column and a residue class of rows, kUnroll rows in flight; the row classes
// are combined in a fixed order in shared memory.  w is in shared memory.
// ----------------------------------------------------------------------------
template <typename T>
__device__ __noinline__ void cols_gemv(const T* B, int64_t ldb, int64_t q, const T* w, T* v, int c, int G, double* sm_parts)
{
    using V = typename VecOf<T>::V;
    constexpr int VN = VecOf<T>::N;
    const int64_t nvt = ldb / VN;
    const int64_t slab = (nvt + G - 1) / G;
    const int64_t e0 = (int64_t)c * slab, e1 = min(nvt, e0 + slab);
    for (int64_t cb = e0; cb < e1; cb += kBlock) {
        const int ncols = (int)min((int64_t)kBlock, e1 - cb);
        const int RG = kBlock / ncols;
        const int e = threadIdx.x % ncols, rg = threadIdx.x / ncols;
        T acc[VN];
#pragma unroll
        for (int cc = 0; cc < VN; ++cc) acc[cc] = 0;
        if (rg < RG) {
            const V* col = reinterpret_cast<const V*>(B) + cb + e;
            const int64_t ldv = ldb / VN;
            for (int64_t jb = rg; jb < q; jb += (int64_t)RG * kUnroll) {
                V bv[kUnroll];
#pragma unroll
                for (int uu = 0; uu < kUnroll; ++uu) {
                    const int64_t j = jb + (int64_t)uu * RG;
                    if (j < q) bv[uu] = __ldg(col + j * ldv);
                }
#pragma unroll
                for (int uu = 0; uu < kUnroll; ++uu) {
                    const int64_t j = jb + (int64_t)uu * RG;
                    if (j < q) {
                        const T wj = w[j];
                        const T* b = reinterpret_cast<const T*>(&bv[uu]);
#pragma unroll
                        for (int cc = 0; cc < VN; ++cc) acc[cc] = fma(wj, b[cc], acc[cc]);
                    }
                }
            }
        }
        __syncthreads();
        T* red = reinterpret_cast<T*>(sm_parts);
        if (rg < RG) {
#pragma unroll
            for (int cc = 0; cc < VN; ++cc) red[((int64_t)rg * ncols + e) * VN + cc] = acc[cc];
        }
        __syncthreads();
        for (int64_t t = threadIdx.x; t < (int64_t)ncols * VN; t += kBlock) {
            T sum = 0;
            for (int r2 = 0; r2 < RG; ++r2) sum += red[(int64_t)r2 * ncols * VN + t];
            __stcg(v + cb * VN + t, sum);
        }
        __syncthreads();
    }
}

// ME-GRBK / ME-RGRBK pick by warp 0 of every CTA (all CTAs take the same row):
// the CTA partials S_J^c (admitted sums, rows in CTA order) are in P.part_SJ.
template <typename T>
__device__ __noinline__ long long pick_row(const IterParams<T>& P, int G, long long tkey, double u, long long imax)
{
    const int lane = threadIdx.x & 31;
    // The CTA partials S_J^c: lane l owns the run of CTAs [l P, l P + P), P = ceil(G / 32)
    // (G <= 32 kPartRegs).  One scan of the run sums gives S_J and the run where the
    // prefix first exceeds u S_J; a second scan, of that run's partials spread over
    // the lanes, gives the owning CTA c*; a third, of c*'s rows in per-lane runs, the
    // row.  Where rounding leaves u S_J uncovered at a level, its last admitted entry
    // is taken (with base -inf below it).
    constexpr int kPartRegs = 10;
    const unsigned FULL = 0xffffffffu;
    const int PPL = (G + 31) / 32;
    double pv[kPartRegs];
    double lsum = 0.0;
#pragma unroll
    for (int j = 0; j < kPartRegs; ++j) {
        const int cc = lane * PPL + j;
        pv[j] = (j < PPL && cc < G) ? __ldcg(P.part_SJ + cc) : 0.0;
    }
#pragma unroll
    for (int j = 0; j < kPartRegs; ++j)
        if (j < PPL) lsum += pv[j];
    const double inc = warp_inclusive_scan(lsum);
    const double SJ = __shfl_sync(FULL, inc, 31);
    const double target = __dmul_rn(u, SJ);
    const long long gkey = __double_as_longlong(target);
    const unsigned hit = __ballot_sync(FULL, dkey(lsum) > 0 && dkey(inc) > gkey);
    int Lc;
    double excl;
    if (hit) {
        Lc = __ffs(hit) - 1;
        excl = __shfl_sync(FULL, inc - lsum, Lc);
    } else {
        const unsigned nz = __ballot_sync(FULL, dkey(lsum) > 0);
        Lc = nz ? 31 - __clz(nz) : -1;
        excl = -INFINITY;
    }
    int cstar = -1;
    double cexcl = -INFINITY;
    if (Lc >= 0) {
        double mine = 0.0;
#pragma unroll
        for (int j = 0; j < kPartRegs; ++j) {
            const double x = __shfl_sync(FULL, pv[j], Lc);
            if (j == lane) mine = x;
        }
        if (!(lane < PPL && Lc * PPL + lane < G)) mine = 0.0;
        const double inc2 = excl + warp_inclusive_scan(mine);
        const unsigned h2 = __ballot_sync(FULL, dkey(mine) > 0 && dkey(inc2) > gkey);
        if (h2) {
            const int l2 = __ffs(h2) - 1;
            cstar = Lc * PPL + l2;
            cexcl = __shfl_sync(FULL, inc2 - mine, l2);
        } else {
            const unsigned nz2 = __ballot_sync(FULL, dkey(mine) > 0);
            if (nz2) cstar = Lc * PPL + 31 - __clz(nz2);
        }
    }
    long long pick = -1, last = -1;
    if (cstar >= 0) {
        int64_t q0 = 0, q1 = 0;
        cta_rows(P.m, cstar, G, q0, q1);
        double run = cexcl;
        // rounds of up to 32 kRowRegs rows; lane l owns a contiguous run of RPL rows
        constexpr int kRowRegs = 8;
        for (int64_t rb = q0; rb < q1 && pick < 0; rb += 32 * kRowRegs) {
            const int64_t rn = min((int64_t)(32 * kRowRegs), q1 - rb);
            const int RPL = (int)((rn + 31) / 32);
            const int64_t lb = rb + (int64_t)lane * RPL;
            double2 rv[kRowRegs];
#pragma unroll
            for (int j = 0; j < kRowRegs; ++j)
                rv[j] = (j < RPL && lb + j < rb + rn) ? __ldcg(P.sr + lb + j) : make_double2(0.0, -INFINITY);
            double ls = 0.0;
            long long lastl = -1;
#pragma unroll
            for (int j = 0; j < kRowRegs; ++j)
                if (j < RPL && dkey(rv[j].y) >= tkey) { ls += rv[j].x; lastl = lb + j; }
            const double incr = run + warp_inclusive_scan(ls);
            const unsigned am = __ballot_sync(FULL, lastl >= 0);
            if (am) last = __shfl_sync(FULL, lastl, 31 - __clz(am));
            const unsigned hr = __ballot_sync(FULL, dkey(ls) > 0 && dkey(incr) > gkey);
            if (hr) {
                const int Lr = __ffs(hr) - 1;
                const double ex = __shfl_sync(FULL, incr - ls, Lr);
                double ms = 0.0;
                long long mk = LLONG_MIN;
#pragma unroll
                for (int j = 0; j < kRowRegs; ++j) {
                    const double xs = __shfl_sync(FULL, rv[j].x, Lr);
                    const long long xk = __shfl_sync(FULL, dkey(rv[j].y), Lr);
                    if (j == lane) { ms = xs; mk = xk; }
                }
                const bool adm = lane < RPL && mk >= tkey;
                const double inc3 = ex + warp_inclusive_scan(adm ? ms : 0.0);
                const unsigned h3 = __ballot_sync(FULL, adm && dkey(inc3) > gkey);
                const unsigned a3 = __ballot_sync(FULL, adm);
                pick = rb + (int64_t)Lr * RPL + (h3 ? __ffs(h3) - 1 : 31 - __clz(a3));
            }
            run = __shfl_sync(FULL, incr, 31);
        }
    }
    if (pick < 0) pick = last;
    if (pick < 0) pick = imax;  // admitted sum vanished (cannot happen with S > 0)
    return pick;
}

// ----------------------------------------------------------------------------
// the persistent iteration kernel
// ----------------------------------------------------------------------------
// DEFER: the deferred update (FP32 only); the in-place instantiation carries none of its code.
template <typename T, bool DEFER = false>
__global__ void __launch_bounds__(kBlock) iterate_kernel(IterParams<T> P)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ double sm_parts[kPartsCap];
    __shared__ double sm_red[2 * kWarps];
    __shared__ long long sm_redi[kWarps];
    __shared__ int s_ok;
    __shared__ unsigned int s_gen;
    __shared__ double s_S, s_t, s_u, s_ck;
    __shared__ long long s_imax, s_ik;
    __shared__ int s_stop;
    __shared__ double2 sm_sr[kSrCap];          // this CTA's (s_i, r_i) when it owns <= kSrCap rows
    // deferred update: U'_{i_k, j} of the chunk so far, the Gram column v_j . v_it (double-float)
    // and the per-row corrections (four partial sums per row)
    __shared__ float s_uik[kDeferCap];
    __shared__ float2 s_gf[kDeferCap + 1];

    T* sv = reinterpret_cast<T*>(dsm);                               // ldr: R_{i_k}, then v
    T* sa = sv + (P.smem_v ? P.ldr : 0);                              // lda: A_{i_k}
    T* sw = sa + (P.smem_arow ? P.lda : 0);                           // q: w
    // deferred update only: the per-row corrections, four partial sums per row (4 kSrCap pairs)
    float2* s_corr = reinterpret_cast<float2*>(sw + ((P.q + VecOf<T>::N - 1) / VecOf<T>::N) * VecOf<T>::N);

    const int G = gridDim.x, c = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t r0, r1;
    cta_rows(P.m, c, G, r0, r1);
    using V = typename VecOf<T>::V;
    constexpr int VN = VecOf<T>::N;
    const bool own_sm = (r1 - r0) <= kSrCap;
    if (own_sm)
        for (int64_t i = r0 + threadIdx.x; i < r1; i += kBlock) sm_sr[i - r0] = __ldcg(P.sr + i);
    grid_gen_init(P.bar, s_gen);

    for (int it = 0; it <= P.nit; ++it) {
        const long long k = P.k0 + it;
        // ---------------- select: totals from the per-CTA partials ----------
        if (warp == 0) {
            // r >= 0 or -inf, so the largest r is the largest bit pattern read as a signed
            // integer: the argmax stays off the FP64 pipe (ties: smallest row)
            double S = 0.0;
            long long bkey = LLONG_MIN, bi = LLONG_MAX;
            // all of this lane's partials (CTAs lane, lane + 32, ...) are requested
            // before any is used: one L2 round trip per 32 * kSelRegs CTAs
            constexpr int kSelRegs = 5;
            for (int cb = 0; cb < G; cb += 32 * kSelRegs) {
                double2 p0[kSelRegs], p1[kSelRegs];
#pragma unroll
                for (int j = 0; j < kSelRegs; ++j) {
                    const int cc = cb + j * 32 + lane;
                    if (cc < G) {
                        const double2* pp = reinterpret_cast<const double2*>(P.part + cc);
                        p0[j] = __ldcg(pp);
                        p1[j] = __ldcg(pp + 1);
                    }
                }
#pragma unroll
                for (int j = 0; j < kSelRegs; ++j) {
                    const int cc = cb + j * 32 + lane;
                    if (cc < G) {
                        S += p0[j].x;
                        const long long rk = __double_as_longlong(p0[j].y);
                        const long long ii = __double_as_longlong(p1[j].x);
                        if (rk > bkey || (rk == bkey && ii < bi)) { bkey = rk; bi = ii; }
                    }
                }
            }
            // the draw of this iteration, while the partials are in flight
            if (lane == 0) s_u = philox_uniform(P.seed, (uint64_t)k, P.sys);
            S = warp_sum(S);
            warp_argmax_key(bkey, bi);
            if (lane == 0) {
                const double br = __longlong_as_double(bkey);
                s_S = S; s_imax = bi;
                int stop = 0;
                if (!(S > 0.0)) stop = (S == 0.0) ? 2 : 3;      // 3: NaN
                else if (P.stop_S >= 0.0 && S <= P.stop_S) stop = 1;
                else if (it == P.nit) stop = 4;
                s_stop = stop;
                // the threshold, once per CTA (Eq. of Algorithm 4; theta = 1/2: Algorithm 3)
                if (stop == 0 && (P.variant == GRBK_GRBK || P.variant == GRBK_RGRBK)) {
                    const double theta = (P.variant == GRBK_GRBK) ? 0.5 : P.theta;
                    double t = __dadd_rn(__dmul_rn(theta, br), __dmul_rn(1.0 - theta, __ddiv_rn(S, P.F)));
                    if (t > br) t = br;
                    s_t = t;
                }
                if (c == 0) {
                    if (stop == 0 && k < P.trace_len) P.trace_S[k] = S;
                    if (stop != 0) {
                        P.st->k = k;
                        P.st->S = S;
                        if (stop == 1) P.st->flag = FLAG_TOL_MET;
                        if (stop == 2) P.st->flag = FLAG_EXACT;
                        if (stop == 3) atomicCAS(&P.st->status, 0, (int)GRBK_ENONFINITE);
                    }
                }
            }
        }
        __syncthreads();
        if (s_stop) break;

        // ---------------- select: the row -----------------------------------
        long long ik = -1;
        const int var = P.variant;
        if (var == GRBK_GRBK || var == GRBK_RGRBK) {
            // admission r_i >= t and the prefix tests below compare bit patterns: t, r_i
            // and the sums are >= 0 (r_i may be -inf), so the integer order is the numeric one
            const long long tkey = __double_as_longlong(s_t);
            // admitted sum of this CTA's rows
            if (warp == 0) {
                double sj = 0.0;
                for (int64_t i = r0 + lane; i < r1; i += 32) {
                    const double2 v = own_sm ? sm_sr[i - r0] : __ldcg(P.sr + i);
                    if (__double_as_longlong(v.y) >= tkey) sj += v.x;
                }
                sj = warp_sum(sj);
                if (lane == 0) __stcg(P.part_SJ + c, sj);
            }
            if (!grid_sync(P.bar, P.st, 1, s_ok, s_gen)) return;
            if (warp == 0) {
                const long long pick = pick_row(P, G, tkey, s_u, s_imax);
                if (lane == 0) s_ik = pick;
            }
            __syncthreads();
            ik = s_ik;
        } else if (var == GRBK_MWRBK) {
            ik = s_imax;
        } else if (var == GRBK_RBK) {
            if (threadIdx.x == 0) {
                const double u = philox_uniform(P.seed, (uint64_t)k, P.sys);
                const double target = __dmul_rn(u, P.F);
                // first i with prefix[i] > target (prefix is non-decreasing)
                int64_t lo = 0, hi = P.m;  // answer in [lo, hi]
                while (lo < hi) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (__ldg(P.rbk_prefix + mid) > target) hi = mid; else lo = mid + 1;
                }
                if (lo >= P.m) {  // none exceeded: last row with a_i > 0
                    lo = P.m - 1;
                    while (lo > 0 && !(__ldg(P.a + lo) > 0.0)) --lo;
                }
                s_ik = lo;
            }
            __syncthreads();
            ik = s_ik;
        } else {  // GRBK_BK
            ik = k % P.m;
        }

        // per-iteration slots of the deferred update's history
        T* ucur = P.u;
        T* vcur = P.v;
        const T* Rik = P.R + ik * P.ldr;
        if constexpr (DEFER) {
            {
                ucur = P.uh + (int64_t)it * P.m;
                vcur = P.vh + (int64_t)it * P.ldr;
                if (it > 0) {
                    // the current row R_ik = R^0_ik - sum_{j<it} U'_{ik,j} v_j, each CTA its slab
                    // of columns, the terms in iteration order as the in-place update applies them
                    defer_row<T>(P, it, ik, c, G, s_uik, reinterpret_cast<T*>(dsm));
                    if (!grid_sync(P.bar, P.st, 5, s_ok, s_gen)) return;
                    Rik = P.rik;
                }
            }
        }

        // ---------------- W/U: w = R_ik B^T, u = A A_ik^T ---------------------
        const T* Aik = P.A + ik * P.lda;
        if (P.smem_v) {
            for (int64_t e = threadIdx.x; e < P.ldr / VN; e += kBlock)
                reinterpret_cast<V*>(sv)[e] = ldcg_v(reinterpret_cast<const V*>(Rik) + e);
        }
        if (P.smem_arow && !P.G) {
            for (int64_t e = threadIdx.x; e < P.lda / VN; e += kBlock)
                reinterpret_cast<V*>(sa)[e] = __ldg(reinterpret_cast<const V*>(Aik) + e);
        }
        // this thread's first entry of row i_k of A A^T, loaded with the staging
        const int64_t ig = r0 + threadIdx.x;
        T g0 = (T)0;
        if (P.G && ig < r1) g0 = __ldg(P.G + ik * P.ldg + ig);
        // c_k = alpha / a_ik by one thread, after its share of the staging loads is issued
        if (threadIdx.x == 0) {
            const double aik = __ldg(P.a + ik);
            const double ckv = (aik > 0.0) ? __ddiv_rn(P.alpha, aik) : 0.0;
            s_ck = ckv;
            if (c == 0) {
                P.hist_rows[it] = (int)ik;
                P.hist_c[it] = ckv;
                if (k < P.trace_len) P.trace_rows[k] = (int)ik;
            }
        }
        __syncthreads();
        const double ck = s_ck;
        // u holds the row coefficients c_k (A A_ik^T)_i of this CTA's rows, read from
        // row i_k of the precomputed A A^T when there is one
        if (P.G) {
            const T* Gi = P.G + ik * P.ldg;
            if (ig < r1) __stcg(ucur + ig, (T)(ck * (double)g0));
            for (int64_t i = ig + kBlock; i < r1; i += kBlock) __stcg(ucur + i, (T)(ck * (double)__ldg(Gi + i)));
        } else {
            rows_dot<T>(P.A, P.lda, r0, r1, P.smem_arow ? sa : Aik, P.smem_arow ? 0 : 2, ucur, nullptr, sm_parts, ck);
        }
        if (P.K) {
            // row-space form: the update vector is R_ik K (K = Lt^T Lt), one pass over
            // K; the row itself is kept for the X update, w = R_ik Lt^T, formed per chunk
            if (c == 0)
                for (int64_t e = threadIdx.x; e < P.ldr / VN; e += kBlock)
                    reinterpret_cast<V*>(P.hist_z + (int64_t)it * P.ldr)[e] = reinterpret_cast<const V*>(sv)[e];
            cols_gemv<T>(P.K, P.ldk, P.n, sv, vcur, c, G, sm_parts);
        } else {
            // each CTA streams a contiguous block of rows of B for w; B is read last
            // here, so the part of it still in L2 serves the v = w B phase that follows
            int64_t j0, j1;
            cta_rows(P.q, c, G, j0, j1);
            rows_dot<T>(P.B, P.ldb, j0, j1, P.smem_v ? sv : Rik, P.smem_v ? 0 : 1, P.w, P.hist_w + (int64_t)it * P.q,
                        sm_parts);
            if (!grid_sync(P.bar, P.st, 2, s_ok, s_gen)) return;

            // ---------------- V: v = w B (column slab of this CTA) -----------
            for (int64_t j = threadIdx.x; j < P.q; j += kBlock) sw[j] = __ldcg(P.w + j);
            __syncthreads();
            cols_gemv<T>(P.B, P.ldb, P.q, sw, vcur, c, G, sm_parts);
        }
        if constexpr (DEFER) {
            {
                defer_gram_partial<T>(P, it, c, G);
            }
        }
        if (!grid_sync(P.bar, P.st, 3, s_ok, s_gen)) return;

        // ---------------- F: fused rank-1 update + row norms -----------------
        if (P.smem_v) {
            for (int64_t e = threadIdx.x; e < P.ldr / VN; e += kBlock)
                reinterpret_cast<V*>(sv)[e] = ldcg_v(reinterpret_cast<const V*>(vcur) + e);
        }
        if constexpr (DEFER) {
            defer_gram_column<T>(P, it, G, s_gf);
            __syncthreads();
            const double gkk = (double)s_gf[it].x + (double)s_gf[it].y;
            deferred_pass<T>(P, it, P.smem_v ? sv : vcur, ucur, r0, r1, s_gf, gkk, s_corr, sm_parts, sm_red,
                             sm_redi, sm_sr);
        } else {
            if (P.smem_v) __syncthreads();
            fused_pass<T, true>(P, ck, P.smem_v ? sv : vcur, r0, r1, sm_parts, sm_red, sm_redi,
                                own_sm ? sm_sr : nullptr);
        }
        if (!grid_sync(P.bar, P.st, 4, s_ok, s_gen)) return;
    }
}

// ----------------------------------------------------------------------------
// Write-back of a deferred chunk: R <- R - sum_{j<nw} U'_j v_j^T with the terms in
// iteration order, each element by one fused multiply-add per term: the in-place
// update's order and rounding.  Tiles of kWbRows rows x kWbVec vectors of 4 columns;
// the tile's U' and v in shared memory (nw KB); each thread keeps 16 rows of one vector.
// ----------------------------------------------------------------------------
constexpr int kWbRows = 128, kWbVec = 32;

__global__ void __launch_bounds__(256) defer_writeback_kernel(float* R, int64_t ldr, int64_t m, const float* uh,
                                                              const float* vh, int nw)
{
    extern __shared__ __align__(16) float wb_sm[];
    float* su = wb_sm;                                                    // nw x kWbRows
    float4* sv4 = reinterpret_cast<float4*>(wb_sm + (int64_t)nw * kWbRows);  // nw x kWbVec
    const int64_t nvr = ldr / 4;
    const int64_t rt = (int64_t)blockIdx.y * kWbRows, vt = (int64_t)blockIdx.x * kWbVec;
    for (int t = threadIdx.x; t < nw * kWbRows; t += blockDim.x) {
        const int j = t / kWbRows, rr = t - j * kWbRows;
        su[t] = (rt + rr < m) ? __ldg(uh + (int64_t)j * m + rt + rr) : 0.f;
    }
    for (int t = threadIdx.x; t < nw * kWbVec; t += blockDim.x) {
        const int j = t / kWbVec, e = t - j * kWbVec;
        sv4[t] = (vt + e < nvr) ? __ldg(reinterpret_cast<const float4*>(vh + (int64_t)j * ldr) + vt + e)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    const int cv = threadIdx.x % kWbVec, rg = threadIdx.x / kWbVec;
    if (vt + cv >= nvr) return;
    float4* R4 = reinterpret_cast<float4*>(R);
    float4 x[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int64_t row = rt + rg * 16 + r;
        x[r] = (row < m) ? __ldcs(R4 + row * nvr + vt + cv) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int j = 0; j < nw; ++j) {
        const float4 vv = sv4[j * kWbVec + cv];
        const float* uj = su + j * kWbRows + rg * 16;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const float cj = uj[r];
            x[r].x = __fmaf_rn(-cj, vv.x, x[r].x);
            x[r].y = __fmaf_rn(-cj, vv.y, x[r].y);
            x[r].z = __fmaf_rn(-cj, vv.z, x[r].z);
            x[r].w = __fmaf_rn(-cj, vv.w, x[r].w);
        }
    }
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int64_t row = rt + rg * 16 + r;
        if (row < m) __stcs(R4 + row * nvr + vt + cv, x[r]);
    }
}

// ----------------------------------------------------------------------------
// small kernels
// ----------------------------------------------------------------------------

// a_i = ||A_i||^2 (FP64), one warp per row
template <typename T>
__global__ void row_sqnorm_kernel(const T* A, int64_t m, int64_t p, int64_t lda, double* a)
{
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= m) return;
    double acc = 0.0;
    for (int64_t c = lane; c < p; c += 32) {
        const double x = (double)A[row * lda + c];
        acc = fma(x, x, acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) a[row] = acc;
}

// sum of squares (and non-finite count) of a matrix, per-block partials
template <typename T>
__global__ void __launch_bounds__(256) sumsq_kernel(const T* M, int64_t rows, int64_t cols, int64_t ld,
                                                    double* part, int* nonfinite)
{
    // one warp per row (grid-stride); FP32 rows: Kahan-compensated per-lane sums of squares
    // combined in double-float arithmetic, FP64 rows: FP64 sums; a fixed order per launch shape
    __shared__ double red[8];
    using V = typename VecOf<T>::V;
    constexpr int VN = VecOf<T>::N;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * 8 + warp, nw = (int64_t)gridDim.x * 8;
    const bool vec = (ld % VN) == 0;
    double wacc = 0.0;
    int bad = 0;
    for (int64_t i = gw; i < rows; i += nw) {
        const T* row = M + i * ld;
        double acc_d = 0.0;
        float acc_f = 0.f, comp_f = 0.f;
        auto add = [&](T x) {
            if (!isfinite(x)) bad = 1;
            if constexpr (sizeof(T) == 8) {
                acc_d = fma((double)x, (double)x, acc_d);
            } else {
                const float yk = fmaf((float)x, (float)x, -comp_f);
                const float tk = acc_f + yk;
                comp_f = (tk - acc_f) - yk;
                acc_f = tk;
            }
        };
        int64_t c0 = 0;
        if (vec) {
            const int64_t nv = cols / VN;
            const V* rv = reinterpret_cast<const V*>(row);
            for (int64_t e = lane; e < nv; e += 32) {
                const V v = __ldg(rv + e);
                const T* x = reinterpret_cast<const T*>(&v);
#pragma unroll
                for (int c = 0; c < VN; ++c) add(x[c]);
            }
            c0 = nv * VN;
        }
        for (int64_t c = c0 + lane; c < cols; c += 32) add(row[c]);
        double tot;
        if constexpr (sizeof(T) == 8) {
            tot = warp_sum(acc_d);
        } else {
            float hi = acc_f, lo = -comp_f;
            warp_sum_df(hi, lo);
            tot = (double)hi + (double)lo;
        }
        wacc += tot;
    }
    if (lane == 0) red[warp] = wacc;
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(nonfinite, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

// ||X - Xref||^2 and ||Xref||^2 partials (FP64 X, Xref with ldr)
__global__ void rse_kernel(const double* X, int64_t p, int64_t q, const double* Xr, double* part)
{
    __shared__ double red[2][32];
    double e2 = 0.0, r2 = 0.0;
    const int64_t total = p * q;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double d = X[e] - Xr[e];
        e2 = fma(d, d, e2);
        r2 = fma(Xr[e], Xr[e], r2);
    }
    e2 = warp_sum(e2);
    r2 = warp_sum(r2);
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = e2; red[1][threadIdx.x >> 5] = r2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += red[0][w]; b += red[1][w]; }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

// X += sum_t c_t A_{i_t}^T w_t   (fold the chunk's rank-1 terms into X)
template <typename T>
__global__ void x_fold_kernel(double* X, int64_t p, int64_t q, const T* A, int64_t lda,
                              const int* rows, const double* cs, const double* W, int nit)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= p * q) return;
    const int64_t rr = idx / q, j = idx % q;
    double acc = 0.0;
    for (int t = 0; t < nit; ++t) {
        const double ca = cs[t] * (double)__ldg(A + (int64_t)rows[t] * lda + rr);
        acc = fma(ca, W[(int64_t)t * q + j], acc);
    }
    X[idx] += acc;
}

// FP32-mode fold: X (FP64) += sum_t c_t A_{i_t}^T w_t with the sum over the
// chunk's terms formed in FP32 on 64 x 128 tiles of X staged in shared memory
// (sa[t][r] = c_t A[i_t][r0 + r], sw[t][j] = w_t[j0 + j]), 64 terms at a time.
// Row-space form: W[t][j] = Z_t . Lt_j for the chunk's selected rows Z_t (ldz
// apart) and the rows of Lt (q x n, ldl) -- the w = R_{i_k} B^T of each
// iteration, written as FP64 for the X fold.  One warp per (t, j).
template <typename T>
__global__ void chunk_w_kernel(int nit, int64_t q, int64_t n, const T* Z, int64_t ldz, const T* Lt, int64_t ldl,
                               double* W)
{
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= (int64_t)nit * q) return;
    const int64_t t = gw / q, j = gw % q;
    const T* z = Z + t * ldz;
    const T* l = Lt + j * ldl;
    T acc = 0;
    for (int64_t e = lane; e < n; e += 32) acc = fma(__ldg(z + e), __ldg(l + e), acc);
    double tot;
    if constexpr (sizeof(T) == 8) tot = warp_sum(acc);
    else tot = (double)warp_sum_f(acc);
    if (lane == 0) W[t * q + j] = tot;
}

constexpr int kFoldR = 64, kFoldC = 128, kFoldT = 64;

__global__ void __launch_bounds__(512) x_fold_f32_kernel(double* X, int64_t p, int64_t q, const float* A,
                                                         int64_t lda, const int* rows, const double* cs,
                                                         const double* W, int nit)
{
    __shared__ float sa[kFoldT][kFoldR];
    __shared__ float sw[kFoldT][kFoldC];
    const int64_t r0 = (int64_t)blockIdx.y * kFoldR, j0 = (int64_t)blockIdx.x * kFoldC;
    const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;  // rows 2tr, 2tr+1; columns tc + 16b
    float acc[2][8];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
    for (int t0 = 0; t0 < nit; t0 += kFoldT) {
        const int nt = min(kFoldT, nit - t0);
        for (int e = threadIdx.x; e < nt * kFoldR; e += 512) {
            const int t = e / kFoldR, r = e % kFoldR;
            sa[t][r] = (r0 + r < p) ? (float)(cs[t0 + t] * (double)__ldg(A + (int64_t)rows[t0 + t] * lda + r0 + r)) : 0.f;
        }
        for (int e = threadIdx.x; e < nt * kFoldC; e += 512) {
            const int t = e / kFoldC, j = e % kFoldC;
            sw[t][j] = (j0 + j < q) ? (float)W[(int64_t)(t0 + t) * q + j0 + j] : 0.f;
        }
        __syncthreads();
        for (int t = 0; t < nt; ++t) {
            const float a0 = sa[t][2 * tr], a1 = sa[t][2 * tr + 1];
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const float wv = sw[t][tc + 16 * b];
                acc[0][b] = fmaf(a0, wv, acc[0][b]);
                acc[1][b] = fmaf(a1, wv, acc[1][b]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const int64_t rr = r0 + 2 * tr + a;
        if (rr >= p) continue;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int64_t j = j0 + tc + 16 * b;
            if (j < q) X[rr * q + j] += (double)acc[a][b];
        }
    }
}

// power iteration pieces for ||B||_2^2 on the streaming helpers:
// t = B^T x (column slabs, x staged in shared memory) ; y = B t (row blocks)
template <typename T>
__global__ void __launch_bounds__(kBlock) bt_x_kernel(const T* B, int64_t q, int64_t ldb, const T* x, T* t)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ double sm_parts[kPartsCap];
    T* sx = reinterpret_cast<T*>(dsm);
    for (int64_t j = threadIdx.x; j < q; j += kBlock) sx[j] = x[j];
    __syncthreads();
    cols_gemv<T>(B, ldb, q, sx, t, blockIdx.x, gridDim.x, sm_parts);
}

template <typename T>
__global__ void __launch_bounds__(kBlock) b_t_kernel(const T* B, int64_t q, int64_t ldb, const T* t, T* y)
{
    __shared__ double sm_parts[kPartsCap];
    int64_t j0, j1;
    cta_rows(q, blockIdx.x, gridDim.x, j0, j1);
    rows_dot<T>(B, ldb, j0, j1, t, 2, y, nullptr, sm_parts);
}

// x <- y / ||y||, lambda = x.y (one block, FP64 sums)
// One Lanczos step on B B^T (one CTA of 1024 threads): with y = B B^T v_j,
// alpha_j = v_j . y, w = y - alpha_j v_j - beta_j v_{j-1}, beta_{j+1} = ||w||,
// v_{j+1} = w / beta_{j+1}.  v and v_prev are kept in FP64; vt is v_{j+1} in the
// bulk precision for the next product.  A step whose beta would vanish (an
// invariant subspace) ends the recurrence: *nsteps stops growing.
template <typename T>
__global__ void __launch_bounds__(1024) lanczos_step_kernel(double* v, double* vprev, T* vt, const T* y, int64_t q,
                                                            double* alpha, double* beta, int j, int* nsteps)
{
    __shared__ double red[32];
    __shared__ double s_val;
    if (*nsteps != j) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    auto block_sum = [&](double x) {
        x = warp_sum(x);
        if (lane == 0) red[warp] = x;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < 32; ++w) t += red[w];
            s_val = t;
        }
        __syncthreads();
        const double r = s_val;
        __syncthreads();
        return r;
    };
    double a = 0.0;
    for (int64_t i = threadIdx.x; i < q; i += 1024) a = fma(v[i], (double)y[i], a);
    a = block_sum(a);
    const double bj = (j > 0) ? beta[j] : 0.0;
    double b2 = 0.0;
    for (int64_t i = threadIdx.x; i < q; i += 1024) {
        const double w = (double)y[i] - a * v[i] - bj * vprev[i];
        b2 = fma(w, w, b2);
    }
    b2 = block_sum(b2);
    const double b = sqrt(b2);
    if (threadIdx.x == 0) alpha[j] = a;
    if (!(b > 1e-12 * fabs(a))) {
        if (threadIdx.x == 0) *nsteps = -(j + 1);  // finished after this step
        return;
    }
    for (int64_t i = threadIdx.x; i < q; i += 1024) {
        const double w = (double)y[i] - a * v[i] - bj * vprev[i];
        vprev[i] = v[i];
        v[i] = w / b;
        vt[i] = (T)(w / b);
    }
    if (threadIdx.x == 0) {
        beta[j + 1] = b;
        *nsteps = j + 1;
    }
}

__global__ void lanczos_init_kernel(double* v, double* vprev, int64_t q, int* nsteps)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < q) { v[i] = 1.0 / sqrt((double)q); vprev[i] = 0.0; }
    if (i == 0) *nsteps = 0;
}

template <typename T>
__global__ void fill_kernel(T* x, int64_t n, double v)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = (T)v;
}

// dtype conversion / re-pitch, device to device
template <typename Td, typename Ts>
__global__ void convert_kernel(Td* dst, int64_t ldd, const Ts* src, int64_t lds, int64_t rows, int64_t cols)
{
    const int64_t total = rows * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / cols, j = e % cols;
        dst[i * ldd + j] = (Td)src[i * lds + j];
    }
}

cudaError_t convert_matrix(void* dst, int dtd, int64_t ldd, const void* src, int dts, int64_t lds,
                           int64_t rows, int64_t cols, cudaStream_t st)
{
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    const int64_t total = rows * cols;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, 4096);
    if (dtd == GRBK_DT_F64 && dts == GRBK_DT_F64)
        convert_kernel<double, double><<<grid, 256, 0, st>>>((double*)dst, ldd, (const double*)src, lds, rows, cols);
    else if (dtd == GRBK_DT_F64 && dts == GRBK_DT_F32)
        convert_kernel<double, float><<<grid, 256, 0, st>>>((double*)dst, ldd, (const float*)src, lds, rows, cols);
    else if (dtd == GRBK_DT_F32 && dts == GRBK_DT_F64)
        convert_kernel<float, double><<<grid, 256, 0, st>>>((float*)dst, ldd, (const double*)src, lds, rows, cols);
    else
        convert_kernel<float, float><<<grid, 256, 0, st>>>((float*)dst, ldd, (const float*)src, lds, rows, cols);
    return cudaGetLastError();
}

}  // namespace grbk

// ============================================================================
// host side
// ============================================================================
using namespace grbk;

struct grbk_ctx {
    int64_t m, p, q, n, lda, ldb, ldr;
    int prec;        // grbk_precision
    int esz;         // element size of the bulk arrays
    grbk_opts opts;
    cudaStream_t stream;
    int G;           // persistent grid
    int smem_v, smem_arow;
    size_t dyn_smem;
    // device buffers
    void *A, *B, *C, *R, *u, *v, *w;
    double *a, *rbk_prefix, *X;
    double2* sr;
    double4* part;
    double* part_SJ;
    int* hist_rows;
    double *hist_c, *hist_w;
    int chunk_cap;
    GridBarrier* bar;
    DevState* st;
    DevState* st_host;      // pinned
    double* scratch;        // reductions
    double* scratch_host;   // pinned
    // scalars
    double F, alpha, normC2, lambda;
    SplitGemm* sg;
    void* tmp;              // staging for host <-> device conversions
    size_t tmp_bytes;
    void* gram;             // A A^T (m x ldg) when used
    int64_t ldg;
    int form;               // grbk_form
    int64_t n_orig;         // columns of the caller's B and C (n is the kept residual's)
    double* soff;           // row-space form: ||Rperp_i||^2
    void* K;                // row-space form: Lt^T Lt (n x ldr), when the row fits in shared memory
    void* hist_z;           // with K: the selected rows of a chunk (chunk_cap x ldr)
    cudaStream_t side;      // set-up only: the copy of a host C overlapped with the rest
    cudaEvent_t side_done;
    struct {                // set-up only: the Lanczos run for ||B||_2^2 (begun, then read back)
        void *vt, *t, *y;
        double *v, *vprev, *ab;
        int* nst;
        int steps;
    } lz;
    cudaEvent_t ev0, ev1;   // around each persistent-kernel launch
    long long launches;     // kernel launches issued (reset per solve)
    int defer;              // FP32 deferred update (R read once per iteration, written back per chunk)
    int defer_stage;        //   a chunk's v_j over one CTA's slab fit in the dynamic shared memory
    void *uh, *vh, *rik;    //   its U' and v of the chunk, and the assembled row R_{i_k}
    float2* gp;             //   per-CTA partials of the Gram column
};

static grbk_status ensure_tmp(grbk_ctx* c, size_t bytes)
{
    if (c->tmp_bytes >= bytes) return GRBK_OK;
    if (c->tmp) {  // queued copies may still use the old block
        cudaStreamSynchronize(c->stream);
        dev_free(c->tmp);
    }
    c->tmp = nullptr;
    c->tmp_bytes = 0;
    if (dev_alloc(&c->tmp, bytes) != cudaSuccess) return GRBK_ENOMEM;
    c->tmp_bytes = bytes;
    return GRBK_OK;
}

static int dsize(int dt) { return dt == GRBK_DT_F64 ? 8 : 4; }

// Copy a caller matrix (host or device, any dtype, any ld) into a device
// buffer dst (dtype dtd, row stride ldd); padding columns are left untouched.
static grbk_status load_matrix(grbk_ctx* c, const grbk_mat* M, void* dst, int dtd, int64_t ldd)
{
    const int64_t rows = M->rows, cols = M->cols;
    if (rows == 0 || cols == 0) return GRBK_OK;
    const int es = dsize(M->dtype);
    if (M->on_device) {
        GRBK_CK(convert_matrix(dst, dtd, ldd, M->ptr, M->dtype, M->ld, rows, cols, c->stream));
        return GRBK_OK;
    }
    if (M->dtype == dtd) {  // same element type: straight into the padded rows
        GRBK_CK(cudaMemcpy2DAsync(dst, ldd * es, M->ptr, M->ld * es, cols * es, rows, cudaMemcpyHostToDevice,
                                  c->stream));
        return GRBK_OK;
    }
    grbk_status s = ensure_tmp(c, (size_t)rows * cols * es);
    if (s != GRBK_OK) return s;
    GRBK_CK(cudaMemcpy2DAsync(c->tmp, cols * es, M->ptr, M->ld * es, cols * es, rows,
                              cudaMemcpyHostToDevice, c->stream));
    GRBK_CK(convert_matrix(dst, dtd, ldd, c->tmp, M->dtype, cols, rows, cols, c->stream));
    return GRBK_OK;
}

// Write a device matrix (dtype dts, ld lds) into a caller matrix.
static grbk_status store_matrix(grbk_ctx* c, grbk_mat* M, const void* src, int dts, int64_t lds)
{
    const int64_t rows = M->rows, cols = M->cols;
    if (rows == 0 || cols == 0) return GRBK_OK;
    const int es = dsize(M->dtype);
    if (M->on_device) {
        GRBK_CK(convert_matrix((void*)M->ptr, M->dtype, M->ld, src, dts, lds, rows, cols, c->stream));
        return GRBK_OK;
    }
    grbk_status s = ensure_tmp(c, (size_t)rows * cols * es);
    if (s != GRBK_OK) return s;
    GRBK_CK(convert_matrix(c->tmp, M->dtype, cols, src, dts, lds, rows, cols, c->stream));
    GRBK_CK(cudaMemcpy2DAsync((void*)M->ptr, M->ld * es, c->tmp, cols * es, cols * es, rows,
                              cudaMemcpyDeviceToHost, c->stream));
    return GRBK_OK;
}

static bool mat_ok(const grbk_mat* M)
{
    return M && M->ptr && M->rows >= 0 && M->cols >= 0 && M->ld >= M->cols &&
           (M->dtype == GRBK_DT_F64 || M->dtype == GRBK_DT_F32);
}

template <typename T>
static IterParams<T> make_params(grbk_ctx* c)
{
    IterParams<T> P;
    memset(&P, 0, sizeof(P));
    P.m = c->m; P.p = c->p; P.q = c->q; P.n = c->n;
    P.lda = c->lda; P.ldb = c->ldb; P.ldr = c->ldr;
    P.A = (const T*)c->A; P.B = (const T*)c->B; P.R = (T*)c->R;
    P.a = c->a; P.rbk_prefix = c->rbk_prefix; P.sr = c->sr;
    P.u = (T*)c->u; P.v = (T*)c->v; P.w = (T*)c->w;
    P.part = c->part;
    P.part_SJ = c->part_SJ;
    P.hist_rows = c->hist_rows; P.hist_c = c->hist_c; P.hist_w = c->hist_w;
    P.bar = c->bar; P.st = c->st;
    P.F = c->F; P.alpha = c->alpha;
    P.smem_v = c->smem_v; P.smem_arow = c->smem_arow;
    P.G = (const T*)c->gram; P.ldg = c->ldg;
    P.soff = c->soff;
    P.K = (const T*)c->K; P.ldk = c->ldr; P.hist_z = (T*)c->hist_z;
    P.defer = c->defer;
    P.uh = (T*)c->uh; P.vh = (T*)c->vh; P.gp = c->gp; P.rik = (T*)c->rik;
    P.defer_stage = c->defer_stage;
    P.stop_S = -1.0;
    return P;
}

static grbk_status run_rownorms(grbk_ctx* c)
{
    c->launches += 1;
    if (c->prec == GRBK_F64) {
        IterParams<double> P = make_params<double>(c);
        rownorms_kernel<double><<<c->G, kBlock, 0, c->stream>>>(P);
    } else {
        IterParams<float> P = make_params<float>(c);
        rownorms_kernel<float><<<c->G, kBlock, 0, c->stream>>>(P);
    }
    GRBK_CK(cudaGetLastError());
    return GRBK_OK;
}

// R = C - A X B with the context's device X (FP64 master), into dst (ld ldr, bulk precision)
static grbk_status compute_residual(grbk_ctx* c, const double* Xd, void* dst)
{
    const int64_t m = c->m, p = c->p, q = c->q, n = c->n;
    c->launches += (c->prec == GRBK_F64) ? 2 : splitgemm_launches(c->sg);
    if (c->prec == GRBK_F64) {
        // T1 = A X (m x q), then dst = C - T1 B, evaluated in whichever order has fewer flops
        const bool ax_first = (m * p * q + m * q * n) <= (p * q * n + m * p * n);
        if (ax_first) {
            grbk_status s = ensure_tmp(c, (size_t)m * q * 8);
            if (s != GRBK_OK) return s;
            GRBK_CK(gemm_simt<double>(m, q, p, 1.0, (const double*)c->A, c->lda, Xd, q, 0.0, nullptr, 0,
                                      (double*)c->tmp, q, c->stream));
            GRBK_CK(gemm_simt<double>(m, n, q, -1.0, (const double*)c->tmp, q, (const double*)c->B, c->ldb,
                                      1.0, (const double*)c->C, c->ldr, (double*)dst, c->ldr, c->stream));
        } else {
            grbk_status s = ensure_tmp(c, (size_t)p * n * 8);
            if (s != GRBK_OK) return s;
            GRBK_CK(gemm_simt<double>(p, n, q, 1.0, Xd, q, (const double*)c->B, c->ldb, 0.0, nullptr, 0,
                                      (double*)c->tmp, n, c->stream));
            GRBK_CK(gemm_simt<double>(m, n, p, -1.0, (const double*)c->A, c->lda, (const double*)c->tmp, n,
                                      1.0, (const double*)c->C, c->ldr, (double*)dst, c->ldr, c->stream));
        }
        return GRBK_OK;
    }
    grbk_status s = splitgemm_residual(c->sg, Xd, q, (const float*)c->C, (float*)dst, c->ldr, c->stream);
    if (s != GRBK_OK) return s;
    return splitgemm_check(c->sg, c->stream);
}

extern "C" void grbk_default_opts(grbk_opts* o)
{
    memset(o, 0, sizeof(*o));
    o->precision = GRBK_F64;
    o->refresh_T = 0;
    o->alpha = 0.0;
    o->stop_kind = GRBK_STOP_NONE;
    o->split_terms = 2;
}

extern "C" const char* grbk_strerror(int32_t s)
{
    switch (s) {
    case GRBK_OK: return "ok";
    case GRBK_EINVAL: return "invalid argument";
    case GRBK_ENOMEM: return "out of device memory";
    case GRBK_ECUDA: return "CUDA error";
    case GRBK_ENOTCONV: return "not converged within maxit";
    case GRBK_ETIMEOUT: return "device barrier timed out";
    case GRBK_ENONFINITE: return "non-finite value";
    default: return "unknown status";
    }
}

// waits for and releases the set-up's side stream (a copy into c->C may be in flight)
static void end_side(grbk_ctx* c)
{
    if (c->side) {
        cudaStreamSynchronize(c->side);
        cudaStreamDestroy(c->side);
        c->side = nullptr;
    }
    if (c->side_done) {
        cudaEventDestroy(c->side_done);
        c->side_done = nullptr;
    }
}

extern "C" void grbk_destroy(grbk_ctx* c)
{
    if (!c) return;
    end_side(c);
    void* bufs[] = {c->A, c->B, c->C, c->R, c->u, c->v, c->w, c->a, c->rbk_prefix, c->sr, c->X,
                    c->part, c->part_SJ, c->hist_rows, c->hist_c,
                    c->hist_w, c->bar, c->st, c->scratch, c->tmp, c->gram, c->soff, c->K, c->hist_z,
                    c->uh, c->vh, c->rik, c->gp};
    // the blocks go back to the cache: let queued work on the context's stream finish first
    cudaStreamSynchronize(c->stream);
    for (void* b : bufs)
        if (b) dev_free(b);
    void* lzb[] = {c->lz.vt, c->lz.t, c->lz.y, c->lz.v, c->lz.vprev, c->lz.ab, c->lz.nst};
    for (void* b : lzb)
        if (b) dev_free(b);
    if (c->st_host) cudaFreeHost(c->st_host);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->scratch_host) cudaFreeHost(c->scratch_host);
    if (c->sg) splitgemm_destroy(c->sg);
    delete c;
}

#define ALLOC(ptr, bytes)                                                     \
    do {                                                                      \
        if (dev_alloc((void**)&(ptr), (bytes) > 0 ? (bytes) : 16) != cudaSuccess) { \
            grbk_destroy(c);                                                  \
            return GRBK_ENOMEM;                                               \
        }                                                                     \
    } while (0)

#define TRY(expr)                          \
    do {                                   \
        grbk_status s_ = (expr);           \
        if (s_ != GRBK_OK) {               \
            grbk_destroy(c);               \
            return s_;                     \
        }                                  \
    } while (0)

static grbk_status reduce_scratch(grbk_ctx* c, int nparts, int stride, double* out)
{
    GRBK_CK(cudaMemcpyAsync(c->scratch_host, c->scratch, sizeof(double) * nparts * stride,
                            cudaMemcpyDeviceToHost, c->stream));
    GRBK_CK(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < stride; ++k) out[k] = 0.0;
    for (int i = 0; i < nparts; ++i)
        for (int k = 0; k < stride; ++k) out[k] += c->scratch_host[i * stride + k];
    return GRBK_OK;
}

static grbk_status sumsq_nonfinite(grbk_ctx* c, const void* M, int64_t rows, int64_t cols, int64_t ld,
                                   double* ss, int* bad)
{
    int* d_bad = (int*)(c->scratch + 1024);
    GRBK_CK(cudaMemsetAsync(d_bad, 0, sizeof(int), c->stream));
    if (c->prec == GRBK_F64)
        sumsq_kernel<double><<<256, 256, 0, c->stream>>>((const double*)M, rows, cols, ld, c->scratch, d_bad);
    else
        sumsq_kernel<float><<<256, 256, 0, c->stream>>>((const float*)M, rows, cols, ld, c->scratch, d_bad);
    GRBK_CK(cudaGetLastError());
    int hb = 0;
    GRBK_CK(cudaMemcpyAsync(&hb, d_bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    grbk_status s = reduce_scratch(c, 256, 1, ss);
    if (s != GRBK_OK) return s;
    *bad = hb;
    return GRBK_OK;
}

template <typename T>
static grbk_status setup_launch_shape(grbk_ctx* c)
{
    int dev = 0, optin = 0, nsm = 0;
    GRBK_CK(cudaGetDevice(&dev));
    GRBK_CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    GRBK_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const size_t esz = sizeof(T);
    cudaFuncAttributes fa;
    GRBK_CK(cudaFuncGetAttributes(&fa, iterate_kernel<T>));
    const size_t budget = (size_t)optin - fa.sharedSizeBytes - 1024;
    size_t need = (size_t)c->q * esz;
    c->smem_arow = 0;
    c->smem_v = 0;
    if (need + (size_t)c->ldr * esz <= budget) { c->smem_v = 1; need += (size_t)c->ldr * esz; }
    if (need + (size_t)c->lda * esz <= budget) { c->smem_arow = 1; need += (size_t)c->lda * esz; }
    if (need > budget) return GRBK_EINVAL;  // q too large for the w buffer
    // (row, chunk) partial slots: one row's chunks must fit in shared memory
    const int64_t chv = 32 * kUnroll * 2, vn = 16 / (int64_t)esz;
    if ((c->ldr / vn + chv - 1) / chv > kPartsCap) return GRBK_EINVAL;
    c->dyn_smem = need;
    GRBK_CK(cudaFuncSetAttribute(iterate_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need));
    int per_sm = 0;
    GRBK_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, iterate_kernel<T>, kBlock, need));
    if (per_sm < 1) return GRBK_EINVAL;
    int G = nsm * min(per_sm, 1);
    // small systems: fewer CTAs keep the barriers cheap (about 4K elements of R per CTA)
    const int64_t want = std::max<int64_t>(1, (c->m * c->ldr) / 4096);
    if (want < G) G = (int)want;
    if (c->opts.grid_ctas > 0) G = min(c->opts.grid_ctas, nsm * per_sm);
    if (G > c->m) G = (int)std::max<int64_t>(1, c->m);
    G = min(G, kMaxGrid);  // the pick holds up to 32 kPartRegs CTA partials in registers
    c->G = G;
    return GRBK_OK;
}

// lambda = ||B||_2^2: the largest eigenvalue of the tridiagonal matrix of up to
// kLanczosSteps Lanczos steps on B B^T from the normalised ones vector (the
// extreme Ritz value converges first and is not disturbed by the loss of
// orthogonality of plain Lanczos); bisection with Sturm counts on the host.
constexpr int kLanczosSteps = 40;

static double tridiag_max_eig(const std::vector<double>& al, const std::vector<double>& be)
{
    // al[0..k), be[1..k) off-diagonal (be[0] unused)
    const int k = (int)al.size();
    double lo = INFINITY, hi = -INFINITY;
    for (int i = 0; i < k; ++i) {
        const double r = (i > 0 ? fabs(be[i]) : 0.0) + (i + 1 < k ? fabs(be[i + 1]) : 0.0);
        lo = std::min(lo, al[i] - r);
        hi = std::max(hi, al[i] + r);
    }
    auto count_below = [&](double x) {  // eigenvalues < x (Sturm sequence of T - x I)
        int cnt = 0;
        double d = 1.0;
        for (int i = 0; i < k; ++i) {
            const double b2 = (i > 0) ? be[i] * be[i] : 0.0;
            d = (al[i] - x) - (i > 0 ? b2 / d : 0.0);
            if (d == 0.0) d = -1e-300;
            if (d < 0.0) ++cnt;
        }
        return cnt;
    };
    for (int it = 0; it < 200 && hi - lo > 1e-15 * fabs(hi); ++it) {
        const double mid = 0.5 * (lo + hi);
        if (count_below(mid) >= k) hi = mid; else lo = mid;
    }
    return hi;
}

// begin: the Lanczos steps are queued on the context's stream (no host wait)
template <typename T>
static grbk_status lanczos_begin(grbk_ctx* c)
{
    const int64_t q = c->q, ldb = c->ldb;
    cudaStream_t st = c->stream;
    auto& L = c->lz;
    L.steps = (int)std::min<int64_t>(kLanczosSteps, q);
    if (dev_alloc(&L.vt, q * sizeof(T)) != cudaSuccess || dev_alloc(&L.t, ldb * sizeof(T)) != cudaSuccess ||
        dev_alloc(&L.y, q * sizeof(T)) != cudaSuccess || dev_alloc((void**)&L.v, q * 8) != cudaSuccess ||
        dev_alloc((void**)&L.vprev, q * 8) != cudaSuccess ||
        dev_alloc((void**)&L.ab, (size_t)2 * (L.steps + 1) * 8) != cudaSuccess ||
        dev_alloc((void**)&L.nst, sizeof(int)) != cudaSuccess)
        return GRBK_ENOMEM;
    double* alpha = L.ab;
    double* beta = L.ab + L.steps + 1;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const size_t xs = (size_t)q * sizeof(T);
    if (xs > 48 * 1024 &&
        cudaFuncSetAttribute(bt_x_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xs) != cudaSuccess)
        return GRBK_EINVAL;
    const int gcols = (int)std::max<int64_t>(1, std::min<int64_t>(nsm, (ldb / (16 / (int64_t)sizeof(T)) + 31) / 32));
    const int grows = (int)std::max<int64_t>(1, std::min<int64_t>(nsm, q));
    T* vt = (T*)L.vt;
    lanczos_init_kernel<<<(unsigned)((q + 255) / 256), 256, 0, st>>>(L.v, L.vprev, q, L.nst);
    fill_kernel<T><<<(unsigned)((q + 255) / 256), 256, 0, st>>>(vt, q, 1.0 / sqrt((double)q));
    for (int j = 0; j < L.steps; ++j) {
        bt_x_kernel<T><<<gcols, kBlock, xs, st>>>((const T*)c->B, q, ldb, vt, (T*)L.t);
        b_t_kernel<T><<<grows, kBlock, 0, st>>>((const T*)c->B, q, ldb, (const T*)L.t, (T*)L.y);
        lanczos_step_kernel<T><<<1, 1024, 0, st>>>(L.v, L.vprev, vt, (const T*)L.y, q, alpha, beta, j, L.nst);
    }
    c->launches += 3 * L.steps;
    GRBK_CK(cudaGetLastError());
    return GRBK_OK;
}

// end: read the tridiagonal back (waits for the stream), its largest eigenvalue
static grbk_status lanczos_end(grbk_ctx* c, double* lambda_out)
{
    auto& L = c->lz;
    cudaStream_t st = c->stream;
    int hn = 0;
    std::vector<double> hab((size_t)2 * (L.steps + 1), 0.0);
    GRBK_CK(cudaMemcpyAsync(&hn, L.nst, sizeof(int), cudaMemcpyDeviceToHost, st));
    GRBK_CK(cudaMemcpyAsync(hab.data(), L.ab, hab.size() * 8, cudaMemcpyDeviceToHost, st));
    GRBK_CK(cudaStreamSynchronize(st));
    const int k = hn < 0 ? -hn : hn;  // steps whose alpha was computed
    if (k <= 0) {
        *lambda_out = 0.0;
    } else {
        std::vector<double> al(hab.begin(), hab.begin() + k), be(k, 0.0);
        for (int i = 1; i < k; ++i) be[i] = hab[L.steps + 1 + i];
        *lambda_out = tridiag_max_eig(al, be);
    }
    void* b[] = {L.vt, L.t, L.y, L.v, L.vprev, L.ab, L.nst};
    for (void* x : b) dev_free(x);
    memset(&L, 0, sizeof(L));
    return GRBK_OK;
}

// the step from the estimate of ||B||_2^2: 1/lambda, or the caller's alpha when it is admissible
static grbk_status set_step(grbk_ctx* c, double hl)
{
    c->lambda = hl;
    if (!(hl > 0.0)) return GRBK_EINVAL;
    if (c->opts.alpha > 0.0) {
        // Lemma 2.2 / Theorems 4.2-4.6 need 0 < alpha < 2/||B||_2^2 (small slack for the estimate)
        if (!(c->opts.alpha * hl < 2.0 * (1.0 + 1e-9))) return GRBK_EINVAL;
        c->alpha = c->opts.alpha;
    } else {
        c->alpha = 1.0 / hl;
    }
    return GRBK_OK;
}

extern "C" grbk_status grbk_create(grbk_ctx** out, const grbk_mat* A, const grbk_mat* B,
                                   const grbk_mat* C, const grbk_opts* opts)
{
    if (!out) return GRBK_EINVAL;
    *out = nullptr;
    if (!mat_ok(A) || !mat_ok(B) || !mat_ok(C)) return GRBK_EINVAL;
    const int64_t m = A->rows, p = A->cols, q = B->rows, n = B->cols;
    if (m <= 0 || p <= 0 || q <= 0 || n <= 0) return GRBK_EINVAL;
    if (C->rows != m || C->cols != n) return GRBK_EINVAL;
    if (m > 0x7fffffffLL) return GRBK_EINVAL;
    grbk_opts o;
    if (opts) o = *opts; else grbk_default_opts(&o);
    if (o.precision != GRBK_F64 && o.precision != GRBK_F32) return GRBK_EINVAL;
    if (!std::isfinite(o.alpha) || !std::isfinite(o.rank_tol)) return GRBK_EINVAL;
    if (o.split_terms == 0) o.split_terms = 2;
    if (o.split_terms != 2 && o.split_terms != 3) return GRBK_EINVAL;
    if (o.refresh_T < 0) return GRBK_EINVAL;
    if (o.form != GRBK_FORM_FULL && o.form != GRBK_FORM_ROWSPACE) return GRBK_EINVAL;

    grbk_ctx* c = new grbk_ctx;
    memset(c, 0, sizeof(*c));
    c->m = m; c->p = p; c->q = q; c->n = n;
    c->n_orig = n;
    c->form = o.form;
    c->opts = o;
    c->prec = o.precision;
    c->esz = (c->prec == GRBK_F64) ? 8 : 4;
    c->stream = (cudaStream_t)o.stream;
    c->lda = round_up(p, 32);
    c->ldb = round_up(n, 32);
    c->ldr = c->ldb;
    const int dt = (c->prec == GRBK_F64) ? GRBK_DT_F64 : GRBK_DT_F32;
    const size_t es = c->esz;

    ALLOC(c->A, (size_t)m * c->lda * es);
    ALLOC(c->B, (size_t)q * c->ldb * es);
    ALLOC(c->C, (size_t)m * c->ldr * es);
    ALLOC(c->R, (size_t)m * c->ldr * es);
    ALLOC(c->u, (size_t)m * es);
    ALLOC(c->v, (size_t)c->ldr * es);
    ALLOC(c->w, (size_t)q * es);
    ALLOC(c->a, (size_t)m * 8);
    ALLOC(c->rbk_prefix, (size_t)m * 8);
    ALLOC(c->sr, (size_t)m * 16);
    ALLOC(c->X, (size_t)p * q * 8);
    ALLOC(c->bar, sizeof(GridBarrier));
    ALLOC(c->st, sizeof(DevState));
    ALLOC(c->scratch, sizeof(double) * 2048);
    if (cudaMallocHost((void**)&c->st_host, sizeof(DevState)) != cudaSuccess) { grbk_destroy(c); return GRBK_ENOMEM; }
    if (cudaMallocHost((void**)&c->scratch_host, sizeof(double) * 2048) != cudaSuccess) { grbk_destroy(c); return GRBK_ENOMEM; }
    if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess) { grbk_destroy(c); return GRBK_ECUDA; }

    cudaStream_t st = c->stream;
    // a host C of the working type is copied on a side stream while the set-up that
    // needs only A and B runs (the Lanczos steps, the split planes, A A^T); the
    // set-up's read-backs come before that copy starts or after that work
    const bool c_async = c->form == GRBK_FORM_FULL && !C->on_device && C->dtype == dt;
    if (cudaMemsetAsync(c->A, 0, (size_t)m * c->lda * es, st) != cudaSuccess ||
        cudaMemsetAsync(c->B, 0, (size_t)q * c->ldb * es, st) != cudaSuccess ||
        (!c_async && cudaMemsetAsync(c->C, 0, (size_t)m * c->ldr * es, st) != cudaSuccess) ||
        cudaMemsetAsync(c->R, 0, (size_t)m * c->ldr * es, st) != cudaSuccess ||
        cudaMemsetAsync(c->v, 0, (size_t)c->ldr * es, st) != cudaSuccess ||
        cudaMemsetAsync(c->bar, 0, sizeof(GridBarrier), st) != cudaSuccess ||
        cudaMemsetAsync(c->st, 0, sizeof(DevState), st) != cudaSuccess) {
        grbk_destroy(c);
        return GRBK_ECUDA;
    }
    TRY(load_matrix(c, A, c->A, dt, c->lda));
    TRY(load_matrix(c, B, c->B, dt, c->ldb));
    if (!c_async) TRY(load_matrix(c, C, c->C, dt, c->ldr));


    // non-finite check and norms (C's once it has arrived)
    double ssA, ssB, ssC = 0.0;
    int badA, badB, badC = 0;
    TRY(sumsq_nonfinite(c, c->A, m, p, c->lda, &ssA, &badA));
    TRY(sumsq_nonfinite(c, c->B, q, n, c->ldb, &ssB, &badB));
    if (!c_async) TRY(sumsq_nonfinite(c, c->C, m, n, c->ldr, &ssC, &badC));
    if (badA || badB || badC) { grbk_destroy(c); return GRBK_ENONFINITE; }
    c->normC2 = ssC;

    if (c->form == GRBK_FORM_ROWSPACE) {
        // keep Z = R Bt^T (m x r) instead of R: solve the system (A, Lt, Chat) with
        // the fixed row offsets ||Rperp_i||^2 (the derivation is in grbk_rowspace.cu)
        const double tol = o.rank_tol > 0.0 ? o.rank_tol : (c->prec == GRBK_F64 ? 1e-12 : 1e-6);
        RowspaceResult rs;
        memset(&rs, 0, sizeof(rs));
        TRY(rowspace_transform(c->prec == GRBK_F64, m, q, n, c->B, c->ldb, c->C, c->ldr, tol, st, &rs));
        c->soff = rs.rperp;
        const int64_t r = rs.r;
        cudaStreamSynchronize(st);
        dev_free(c->B); c->B = nullptr;
        dev_free(c->C); c->C = nullptr;
        dev_free(c->R); c->R = nullptr;
        dev_free(c->v); c->v = nullptr;
        c->n = r;
        c->ldb = round_up(r, 32);
        c->ldr = c->ldb;
        bool ok = dev_alloc(&c->B, (size_t)q * c->ldb * es) == cudaSuccess &&
                  dev_alloc(&c->C, (size_t)m * c->ldr * es) == cudaSuccess &&
                  dev_alloc(&c->R, (size_t)m * c->ldr * es) == cudaSuccess &&
                  dev_alloc(&c->v, (size_t)c->ldr * es) == cudaSuccess;
        if (ok)
            ok = cudaMemsetAsync(c->B, 0, (size_t)q * c->ldb * es, st) == cudaSuccess &&
                 cudaMemsetAsync(c->C, 0, (size_t)m * c->ldr * es, st) == cudaSuccess &&
                 cudaMemsetAsync(c->R, 0, (size_t)m * c->ldr * es, st) == cudaSuccess &&
                 cudaMemsetAsync(c->v, 0, (size_t)c->ldr * es, st) == cudaSuccess &&
                 convert_matrix(c->B, dt, c->ldb, rs.Lt, dt, r, q, r, st) == cudaSuccess &&
                 convert_matrix(c->C, dt, c->ldr, rs.Chat, dt, r, m, r, st) == cudaSuccess &&
                 cudaStreamSynchronize(st) == cudaSuccess;
        if (ok)
            ok = dev_alloc(&c->K, (size_t)r * c->ldr * es) == cudaSuccess &&
                 cudaMemsetAsync(c->K, 0, (size_t)r * c->ldr * es, st) == cudaSuccess &&
                 convert_matrix(c->K, dt, c->ldr, rs.K, dt, r, r, r, st) == cudaSuccess &&
                 cudaStreamSynchronize(st) == cudaSuccess;
        cudaFree(rs.Lt);
        cudaFree(rs.Chat);
        cudaFree(rs.K);
        if (!ok) { grbk_destroy(c); return GRBK_ENOMEM; }
    }

    // a_i, F and the RBK prefix (sequential, ascending rows)
    {
        const int threads = 256;
        const int64_t blocks = (m * 32 + threads - 1) / threads;
        if (c->prec == GRBK_F64)
            row_sqnorm_kernel<double><<<(unsigned)blocks, threads, 0, st>>>((const double*)c->A, m, p, c->lda, c->a);
        else
            row_sqnorm_kernel<float><<<(unsigned)blocks, threads, 0, st>>>((const float*)c->A, m, p, c->lda, c->a);
        if (cudaGetLastError() != cudaSuccess) { grbk_destroy(c); return GRBK_ECUDA; }
        std::vector<double> ha(m), pref(m);
        if (cudaMemcpyAsync(ha.data(), c->a, m * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) { grbk_destroy(c); return GRBK_ECUDA; }
        double run = 0.0;
        for (int64_t i = 0; i < m; ++i) { run += ha[i]; pref[i] = run; }
        c->F = run;
        if (!(c->F > 0.0)) { grbk_destroy(c); return GRBK_EINVAL; }
        if (cudaMemcpyAsync(c->rbk_prefix, pref.data(), m * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) { grbk_destroy(c); return GRBK_ECUDA; }
    }

    // ||B||_2^2 by Lanczos on B B^T; with a host C in flight its result is read after A A^T,
    // so that no read-back waits behind the copy of C
    TRY(c->prec == GRBK_F64 ? lanczos_begin<double>(c) : lanczos_begin<float>(c));
    if (c_async) {
        if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->side_done, cudaEventDisableTiming) != cudaSuccess ||
            cudaMemsetAsync(c->C, 0, (size_t)m * c->ldr * es, c->side) != cudaSuccess ||
            cudaMemcpy2DAsync(c->C, c->ldr * es, C->ptr, C->ld * es, n * es, m, cudaMemcpyHostToDevice,
                              c->side) != cudaSuccess ||
            cudaEventRecord(c->side_done, c->side) != cudaSuccess) {
            grbk_destroy(c);
            return GRBK_ECUDA;
        }
    } else {
        double hl = 0.0;
        TRY(lanczos_end(c, &hl));
        TRY(set_step(c, hl));
    }

    TRY(c->prec == GRBK_F64 ? setup_launch_shape<double>(c) : setup_launch_shape<float>(c));
    ALLOC(c->part, (size_t)c->G * sizeof(double4));
    ALLOC(c->part_SJ, (size_t)c->G * 8);
    c->chunk_cap = o.check_every > 0 ? o.check_every : (o.refresh_T > 0 ? o.refresh_T : 256);
    if (o.refresh_T > 0 && c->chunk_cap > o.refresh_T) c->chunk_cap = o.refresh_T;
    ALLOC(c->hist_rows, (size_t)c->chunk_cap * 4);
    ALLOC(c->hist_c, (size_t)c->chunk_cap * 8);
    ALLOC(c->hist_w, (size_t)c->chunk_cap * q * 8);
    // the deferred update: FP32, chunks of at most kDeferCap iterations, at most kSrCap rows per CTA; by default
    // only in the full form (in the row-space form the assembly barrier and the Gram column cost about what the
    // halved pass over Z saves)
    c->defer = 0;
    c->defer_stage = 0;
    const bool want_defer = o.deferred > 0 || (o.deferred == 0 && c->form == GRBK_FORM_FULL);
    if (c->prec == GRBK_F32 && want_defer && c->chunk_cap <= kDeferCap && (m + c->G - 1) / c->G <= kSrCap) {
        ALLOC(c->uh, (size_t)c->chunk_cap * m * 4);
        ALLOC(c->vh, (size_t)c->chunk_cap * c->ldr * 4);
        ALLOC(c->gp, (size_t)(c->chunk_cap + 1) * c->G * sizeof(float2));
        ALLOC(c->rik, (size_t)c->ldr * 4);
        if (cudaMemsetAsync(c->vh, 0, (size_t)c->chunk_cap * c->ldr * 4, st) != cudaSuccess ||
            cudaMemsetAsync(c->rik, 0, (size_t)c->ldr * 4, st) != cudaSuccess ||
            cudaFuncSetAttribute(defer_writeback_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kDeferCap * (kWbRows + 4 * kWbVec) * 4) != cudaSuccess) {
            grbk_destroy(c);
            return GRBK_ECUDA;
        }
        const int64_t nvr = c->ldr / 4, slab = (nvr + c->G - 1) / c->G;
        c->defer_stage = (size_t)c->chunk_cap * slab * 16 <= c->dyn_smem;
        // the per-row corrections after the row, A_ik and w buffers in the dynamic shared memory
        int dev = 0, optin = 0;
        cudaFuncAttributes fa;
        const size_t need = (size_t)(c->ldr + (c->smem_arow ? c->lda : 0) + (q + 3) / 4 * 4) * 4 +
                            (size_t)4 * kSrCap * sizeof(float2);
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, iterate_kernel<float, true>) != cudaSuccess) {
            grbk_destroy(c);
            return GRBK_ECUDA;
        }
        if (c->smem_v && need + fa.sharedSizeBytes + 1024 <= (size_t)optin) {
            if (cudaFuncSetAttribute(iterate_kernel<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)need) != cudaSuccess) {
                grbk_destroy(c);
                return GRBK_ECUDA;
            }
            c->dyn_smem = std::max(c->dyn_smem, need);
            c->defer = 1;
        }
    }
    if (c->K) {
        if (c->smem_v) {
            ALLOC(c->hist_z, (size_t)c->chunk_cap * c->ldr * es);
        } else {  // the row does not fit in shared memory: w and v from Lt as in the full form
            dev_free(c->K);
            c->K = nullptr;
        }
    }

    if (c->prec == GRBK_F32)
        TRY(splitgemm_create(&c->sg, m, p, q, c->n, (const float*)c->A, c->lda, (const float*)c->B, c->ldb,
                             o.split_terms, st));
    // A A^T, formed once (the practice note after Algorithm 3)
    c->ldg = round_up(m, 32);
    // automatic choice: at most 4 GB, and in FP64 (SIMT, on the narrow FP64 pipe) at most
    // 1e11 flops of set-up; the FP32 form builds it on the tensor cores in milliseconds
    const double gram_flops = 2.0 * (double)m * (double)m * (double)p;
    const bool want_gram = o.use_gram > 0 || (o.use_gram == 0 && (double)m * c->ldg * es <= 4.0e9 &&
                                              (c->prec == GRBK_F32 || gram_flops <= 1.0e11));
    if (want_gram) {
        ALLOC(c->gram, (size_t)m * c->ldg * es);
        if (c->prec == GRBK_F64) {
            if (gram_simt<double>(m, p, (const double*)c->A, c->lda, (double*)c->gram, c->ldg, st) != cudaSuccess) {
                grbk_destroy(c);
                return GRBK_ECUDA;
            }
        } else {
            TRY(splitgemm_gram(c->sg, (float*)c->gram, c->ldg, st));
            TRY(splitgemm_check(c->sg, st));
        }
    }
    if (c_async) {
        double hl = 0.0;
        TRY(lanczos_end(c, &hl));
        TRY(set_step(c, hl));
        if (cudaStreamWaitEvent(st, c->side_done, 0) != cudaSuccess) { grbk_destroy(c); return GRBK_ECUDA; }
        end_side(c);
        TRY(sumsq_nonfinite(c, c->C, m, n, c->ldr, &ssC, &badC));
        if (badC) { grbk_destroy(c); return GRBK_ENONFINITE; }
        c->normC2 = ssC;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) { grbk_destroy(c); return GRBK_ECUDA; }
    *out = c;
    return GRBK_OK;
}

static grbk_status launch_chunk(grbk_ctx* c, int variant, double theta, uint64_t seed, long long k0,
                                int nit, double stop_S, int* d_trace_rows, double* d_trace_S,
                                long long trace_len)
{
    void* args[1];
    if (c->prec == GRBK_F64) {
        IterParams<double> P = make_params<double>(c);
        P.variant = variant; P.theta = theta; P.seed = seed; P.sys = 0; P.k0 = k0; P.nit = nit;
        P.stop_S = stop_S; P.trace_rows = d_trace_rows; P.trace_S = d_trace_S; P.trace_len = trace_len;
        args[0] = &P;
        GRBK_CK(cudaLaunchCooperativeKernel((const void*)iterate_kernel<double>, dim3(c->G), dim3(kBlock),
                                            args, c->dyn_smem, c->stream));
    } else {
        IterParams<float> P = make_params<float>(c);
        P.variant = variant; P.theta = theta; P.seed = seed; P.sys = 0; P.k0 = k0; P.nit = nit;
        P.stop_S = stop_S; P.trace_rows = d_trace_rows; P.trace_S = d_trace_S; P.trace_len = trace_len;
        args[0] = &P;
        GRBK_CK(cudaLaunchCooperativeKernel(c->defer ? (const void*)iterate_kernel<float, true>
                                                     : (const void*)iterate_kernel<float>, dim3(c->G), dim3(kBlock),
                                            args, c->dyn_smem, c->stream));
    }
    return GRBK_OK;
}

static grbk_status fold_x(grbk_ctx* c, int nit)
{
    if (nit <= 0) return GRBK_OK;
    c->launches += 1;
    if (c->K) {
        // row-space form: w of each iteration from its kept row
        c->launches += 1;
        const int64_t warps = (int64_t)nit * c->q;
        const unsigned blocks = (unsigned)((warps * 32 + 255) / 256);
        if (c->prec == GRBK_F64)
            chunk_w_kernel<double><<<blocks, 256, 0, c->stream>>>(nit, c->q, c->n, (const double*)c->hist_z, c->ldr,
                                                                 (const double*)c->B, c->ldb, c->hist_w);
        else
            chunk_w_kernel<float><<<blocks, 256, 0, c->stream>>>(nit, c->q, c->n, (const float*)c->hist_z, c->ldr,
                                                                (const float*)c->B, c->ldb, c->hist_w);
        GRBK_CK(cudaGetLastError());
    }
    const int64_t tot = c->p * c->q;
    const unsigned blocks = (unsigned)((tot + 255) / 256);
    if (c->prec == GRBK_F64)
        x_fold_kernel<double><<<blocks, 256, 0, c->stream>>>(c->X, c->p, c->q, (const double*)c->A, c->lda,
                                                            c->hist_rows, c->hist_c, c->hist_w, nit);
    else {
        dim3 grid((unsigned)((c->q + kFoldC - 1) / kFoldC), (unsigned)((c->p + kFoldR - 1) / kFoldR));
        x_fold_f32_kernel<<<grid, 512, 0, c->stream>>>(c->X, c->p, c->q, (const float*)c->A, c->lda, c->hist_rows,
                                                       c->hist_c, c->hist_w, nit);
    }
    GRBK_CK(cudaGetLastError());
    return GRBK_OK;
}

// R <- R - sum_j U'_j v_j^T over the nw iterations of a deferred chunk, then the row norms of
// the written-back R (they replace the ones the chunk carried by recurrence)
static grbk_status defer_writeback(grbk_ctx* c, int nw)
{
    if (nw <= 0) return GRBK_OK;
    c->launches += 1;
    const int64_t nvr = c->ldr / 4;
    const dim3 grid((unsigned)((nvr + kWbVec - 1) / kWbVec), (unsigned)((c->m + kWbRows - 1) / kWbRows));
    const size_t smem = (size_t)nw * (kWbRows + 4 * kWbVec) * 4;
    defer_writeback_kernel<<<grid, 256, smem, c->stream>>>((float*)c->R, c->ldr, c->m, (const float*)c->uh,
                                                           (const float*)c->vh, nw);
    GRBK_CK(cudaGetLastError());
    return run_rownorms(c);
}

static grbk_status compute_rse(grbk_ctx* c, const double* Xref_d, double* rse)
{
    c->launches += 1;
    rse_kernel<<<256, 256, 0, c->stream>>>(c->X, c->p, c->q, Xref_d, c->scratch);
    GRBK_CK(cudaGetLastError());
    double out[2];
    grbk_status s = reduce_scratch(c, 256, 2, out);
    if (s != GRBK_OK) return s;
    *rse = out[1] > 0.0 ? sqrt(out[0] / out[1]) : sqrt(out[0]);
    return GRBK_OK;
}

extern "C" grbk_status grbk_solve(grbk_ctx* c, int32_t variant, double theta, const grbk_mat* X0,
                                  double tol, int64_t maxit, uint64_t seed, grbk_mat* X_out,
                                  grbk_result* res)
{
    const auto t_start = std::chrono::steady_clock::now();
    if (!c) return GRBK_EINVAL;
    if (variant < GRBK_GRBK || variant > GRBK_BK) return GRBK_EINVAL;
    if (variant == GRBK_RGRBK && !(theta > 0.0 && theta <= 1.0)) return GRBK_EINVAL;
    if (maxit < 0 || !std::isfinite(tol)) return GRBK_EINVAL;
    if (X0 && (!mat_ok(X0) || X0->rows != c->p || X0->cols != c->q)) return GRBK_EINVAL;
    if (X_out && (!X_out->ptr || X_out->rows != c->p || X_out->cols != c->q || X_out->ld < c->q)) return GRBK_EINVAL;
    const grbk_opts& o = c->opts;
    const grbk_mat* xr = o.x_ref;
    if (xr && (!mat_ok(xr) || xr->rows != c->p || xr->cols != c->q)) return GRBK_EINVAL;
    if (o.stop_kind == GRBK_STOP_RSE && !xr) return GRBK_EINVAL;
    cudaStream_t st = c->stream;

    // X^0 and R^0 = C - A X^0 B
    if (X0) {
        c->launches += 1;
        grbk_status s = load_matrix(c, X0, c->X, GRBK_DT_F64, c->q);
        if (s != GRBK_OK) return s;
        s = compute_residual(c, c->X, c->R);
        if (s != GRBK_OK) return s;
    } else {
        GRBK_CK(cudaMemsetAsync(c->X, 0, (size_t)c->p * c->q * 8, st));
        GRBK_CK(cudaMemcpyAsync(c->R, c->C, (size_t)c->m * c->ldr * c->esz, cudaMemcpyDeviceToDevice, st));
    }
    double* Xref_d = nullptr;
    if (xr) {
        GRBK_CK(cudaMalloc(&Xref_d, (size_t)c->p * c->q * 8));
        grbk_status s = load_matrix(c, xr, Xref_d, GRBK_DT_F64, c->q);
        if (s != GRBK_OK) { cudaFree(Xref_d); return s; }
    }
    const long long trace_len = (o.row_trace || o.s_trace) ? o.trace_len : 0;
    int* d_trace_rows = nullptr;
    double* d_trace_S = nullptr;
    if (trace_len > 0) {
        if (cudaMalloc(&d_trace_rows, trace_len * 4) != cudaSuccess ||
            cudaMalloc(&d_trace_S, trace_len * 8) != cudaSuccess) {
            cudaFree(d_trace_rows); cudaFree(Xref_d);
            return GRBK_ENOMEM;
        }
        cudaMemsetAsync(d_trace_rows, 0xff, trace_len * 4, st);
        cudaMemsetAsync(d_trace_S, 0, trace_len * 8, st);
    }
    grbk_status result = GRBK_OK;
    double stop_S = -1.0;
    if (o.stop_kind == GRBK_STOP_RELRES) stop_S = tol * tol * c->normC2;

    GRBK_CK(cudaMemsetAsync(c->st, 0, sizeof(DevState), st));
    GRBK_CK(cudaMemsetAsync(c->bar, 0, sizeof(GridBarrier), st));
    c->launches = 0;
    double iter_ms = 0.0;
    long long iter_launches = 0;
    result = run_rownorms(c);

    long long k = 0;
    int flag = FLAG_RUNNING;
    double S = NAN, rse = NAN;
    while (result == GRBK_OK) {
        const long long left = maxit - k;
        const int nit = (int)std::min<long long>(left, (long long)c->chunk_cap);
        if (cudaEventRecord(c->ev0, st) != cudaSuccess) { result = GRBK_ECUDA; break; }
        result = launch_chunk(c, variant, theta, seed, k, nit, stop_S, d_trace_rows, d_trace_S, trace_len);
        if (result != GRBK_OK) break;
        c->launches += 1;
        iter_launches += 1;
        if (cudaEventRecord(c->ev1, st) != cudaSuccess) { result = GRBK_ECUDA; break; }
        if (cudaMemcpyAsync(c->st_host, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) { result = GRBK_ECUDA; break; }
        {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, c->ev0, c->ev1) == cudaSuccess) iter_ms += ms;
        }
        const DevState ds = *c->st_host;
        if (ds.status != 0) { result = (grbk_status)ds.status; break; }
        const int done = (int)(ds.k - k);
        result = fold_x(c, done);
        if (result != GRBK_OK) break;
        k = ds.k;
        S = ds.S;
        flag = ds.flag;
        bool stop = flag != FLAG_RUNNING;
        if (!stop && o.stop_kind == GRBK_STOP_RSE) {
            result = compute_rse(c, Xref_d, &rse);
            if (result != GRBK_OK) break;
            if (rse <= tol) { flag = FLAG_TOL_MET; stop = true; }
        }
        if (!stop && k >= maxit) stop = true;
        const bool refresh = !stop && o.refresh_T > 0 && k % o.refresh_T == 0;
        // a deferred chunk leaves R at its start: write it back unless a refresh replaces it
        if (c->defer && !refresh) {
            result = defer_writeback(c, done);
            if (result != GRBK_OK) break;
        }
        if (stop) break;
        if (refresh) {
            result = compute_residual(c, c->X, c->R);
            if (result == GRBK_OK) result = run_rownorms(c);
        }
    }
    if (result == GRBK_OK && xr) result = compute_rse(c, Xref_d, &rse);
    if (result == GRBK_OK && X_out) result = store_matrix(c, X_out, c->X, GRBK_DT_F64, c->q);
    if (trace_len > 0 && result == GRBK_OK) {
        if (o.row_trace) cudaMemcpyAsync(o.row_trace, d_trace_rows, trace_len * 4, cudaMemcpyDeviceToHost, st);
        if (o.s_trace) cudaMemcpyAsync(o.s_trace, d_trace_S, trace_len * 8, cudaMemcpyDeviceToHost, st);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess && result == GRBK_OK) result = GRBK_ECUDA;
    cudaFree(d_trace_rows);
    cudaFree(d_trace_S);
    cudaFree(Xref_d);
    if (result == GRBK_OK && o.stop_kind != GRBK_STOP_NONE && flag == FLAG_RUNNING) result = GRBK_ENOTCONV;
    if (res) {
        res->iters = k;
        res->relres = sqrt(S / c->normC2);
        res->rse = rse;
        res->alpha = c->alpha;
        res->iter_kernel_ms = iter_ms;
        res->iter_kernel_launches = iter_launches;
        res->gram = c->gram != nullptr;
        res->deferred = c->defer;
        res->launches = c->launches;
        res->status = result;
        res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    }
    return result;
}

extern "C" grbk_status grbk_residual(grbk_ctx* c, const grbk_mat* X, grbk_mat* R_out)
{
    if (!c || !mat_ok(X) || X->rows != c->p || X->cols != c->q) return GRBK_EINVAL;
    if (c->form != GRBK_FORM_FULL) return GRBK_EINVAL;
    if (!R_out || !R_out->ptr || R_out->rows != c->m || R_out->cols != c->n || R_out->ld < c->n) return GRBK_EINVAL;
    double* Xd = nullptr;
    void* Rd = nullptr;
    GRBK_CK(cudaMalloc(&Xd, (size_t)c->p * c->q * 8));
    if (cudaMalloc(&Rd, (size_t)c->m * c->ldr * c->esz) != cudaSuccess) { cudaFree(Xd); return GRBK_ENOMEM; }
    grbk_status s = load_matrix(c, X, Xd, GRBK_DT_F64, c->q);
    if (s == GRBK_OK) s = compute_residual(c, Xd, Rd);
    if (s == GRBK_OK) s = store_matrix(c, R_out, Rd, c->prec == GRBK_F64 ? GRBK_DT_F64 : GRBK_DT_F32, c->ldr);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess && s == GRBK_OK) s = GRBK_ECUDA;
    cudaFree(Xd);
    cudaFree(Rd);
    return s;
}

extern "C" grbk_status grbk_get_residual(grbk_ctx* c, grbk_mat* R_out)
{
    if (!c || c->form != GRBK_FORM_FULL) return GRBK_EINVAL;
    if (!R_out || !R_out->ptr || R_out->rows != c->m || R_out->cols != c->n || R_out->ld < c->n) return GRBK_EINVAL;
    grbk_status s = store_matrix(c, R_out, c->R, c->prec == GRBK_F64 ? GRBK_DT_F64 : GRBK_DT_F32, c->ldr);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess && s == GRBK_OK) s = GRBK_ECUDA;
    return s;
}

extern "C" grbk_status grbk_get_rownorms(grbk_ctx* c, double* s_out, int32_t on_device)
{
    if (!c || !s_out) return GRBK_EINVAL;
    // the row norms are the first members of the (s_i, r_i) pairs
    GRBK_CK(cudaMemcpy2DAsync(s_out, 8, c->sr, 16, 8, c->m,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    GRBK_CK(cudaStreamSynchronize(c->stream));
    return GRBK_OK;
}

// One grid barrier of the iteration kernel with a short spin budget; CTA
// `absent` (if >= 0) leaves without arriving, so the others must give up.
__global__ void barrier_selftest_kernel(GridBarrier* bar, DevState* st, int absent, long long budget)
{
    __shared__ int s_ok;
    __shared__ unsigned int s_gen;
    if ((int)blockIdx.x == absent) return;
    grid_gen_init(bar, s_gen);
    grid_sync(bar, st, 9, s_ok, s_gen, budget);
}

extern "C" grbk_status grbk_barrier_selftest(int32_t absent_cta, void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    GRBK_CK(cudaGetDevice(&dev));
    GRBK_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int G = std::max(2, std::min(nsm, 8));
    if (absent_cta >= G) return GRBK_EINVAL;
    GridBarrier* bar = nullptr;
    DevState* ds = nullptr;
    if (cudaMalloc(&bar, sizeof(GridBarrier)) != cudaSuccess) return GRBK_ENOMEM;
    if (cudaMalloc(&ds, sizeof(DevState)) != cudaSuccess) { cudaFree(bar); return GRBK_ENOMEM; }
    grbk_status r = GRBK_OK;
    DevState h;
    memset(&h, 0, sizeof(h));
    int absent = absent_cta;
    long long budget = 200000000LL;  // about 0.1 s at 2 GHz
    void* args[] = {&bar, &ds, &absent, &budget};
    if (cudaMemsetAsync(bar, 0, sizeof(GridBarrier), st) != cudaSuccess ||
        cudaMemsetAsync(ds, 0, sizeof(DevState), st) != cudaSuccess ||
        cudaLaunchCooperativeKernel((const void*)barrier_selftest_kernel, dim3(G), dim3(32), args, 0, st) != cudaSuccess ||
        cudaMemcpyAsync(&h, ds, sizeof(DevState), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        r = GRBK_ECUDA;
    cudaFree(bar);
    cudaFree(ds);
    if (r != GRBK_OK) return r;
    return (grbk_status)h.status;
}

extern "C" grbk_status grbk_form_info(const grbk_ctx* c, int32_t* form, int64_t* cols)
{
    if (!c) return GRBK_EINVAL;
    if (form) *form = c->form;
    if (cols) *cols = c->n;
    return GRBK_OK;
}

extern "C" grbk_status grbk_info(const grbk_ctx* c, int64_t dims[4], double* alpha)
{
    if (!c) return GRBK_EINVAL;
    if (dims) { dims[0] = c->m; dims[1] = c->p; dims[2] = c->q; dims[3] = c->n_orig; }
    if (alpha) *alpha = c->alpha;
    return GRBK_OK;
}
