// grbk_batch.cu -- many independent systems A_s X_s B_s = C_s of uneven sizes
// (one per colour channel of many images, Section 6) in ONE persistent launch.
//
// Each CTA takes systems from a queue ordered by decreasing work (longest
// first) and runs the whole iteration of Algorithms 1-5 for its system with
// CTA-local barriers only: no CTA ever waits on another.  R, A, B, C are FP32;
// the row norms, their sums, the threshold and the pick are FP64; X (FP32) is
// folded from the recorded rank-1 terms every `chunk` iterations.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstddef>
#include <map>
#include <mutex>
#include <vector>

#include "grbk_internal.cuh"

namespace grbk {

constexpr int kBB = 512;            // threads per CTA
constexpr int kBW = kBB / 32;
constexpr int kMaxSide = 1024;      // largest m, p, q, n of one system
constexpr int kDefaultBandLimit = 64;

struct SysDesc {
    int m, p, q, n;
    int lda, ldb, ldr;              // row strides (elements)
    int bandA, bandB;               // banded path: A_ic = 0 for |c - i| > bandA, B_jl = 0 for |l - j| > bandB;
                                    // -1: dense path
    int pad;
    long long offA, offB, offR, offX, offRow, offHist, offHistW;
    double F, alpha, stop_S;        // stop when S <= stop_S (< 0: never)
    double normC2;                  // ||C||_F^2 (the test of a caller's X0)
};

struct BatchParams {
    int nsys;
    const SysDesc* sys;
    const int* order;               // queue order (system ids)
    int* queue;                     // next queue slot
    const float* A;
    const float* B;
    const float* C;                 // may alias R when init_from_x == 0 (the no-allocation entry point keeps
                                    // C's copy in R): then C is read only by the R^0 = C copy, which skips
                                    // the copy when the two are the same array
    float* R;
    float* X;
    const double* a;                // ||A_i||^2 per row
    const double* rbk_prefix;       // running sums of a_i per system
    int* hist_rows;                 // [chunk] per system
    float* hist_c;                  // [chunk] per system
    float* hist_w;                  // [chunk x q] per system
    long long* iters;               // out
    double* S_out;                  // out
    int* flag_out;                  // out: FLAG_*
    int* trace_rows;                // [nsys x trace_len] selected rows, or null
    long long trace_len;
    int* x0_rejected;               // per system: 1 when the caller's X0 was replaced by 0, or null
    int variant;
    double theta;
    uint64_t seed;
    long long maxit;
    int chunk;
    int init_from_x;                // R = C - A X B before iterating (X holds X0)
    int band_smem;                  // dynamic shared memory of the launch, bytes (a banded system whose
                                    // bands fit iterates from a shared-memory copy of them)
};

// block-wide sum in a fixed order; one thread adds the warp partials (FP64 is
// 1/64 of the FP32 rate here, so it is kept off the other threads)
template <int NW = kBW>
__device__ __forceinline__ double block_sum_fixed(double v, double* red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < NW; ++w) t += red[w];
        red[NW] = t;
    }
    __syncthreads();
    const double t = red[NW];
    __syncthreads();
    return t;
}

// X += sum_t c_t A_{i_t}^T w_t over the recorded terms (FP32), as a small GEMM
// over tiles of NT/8 rows x 128 columns of X (each thread two rows and eight
// columns) with the chunk's terms staged in shared memory:
// sa[t][r] = c_t A[i_t][r0 + r], sw[t][j] = w_t[j0 + j].  Every element of X
// sums its terms in the same order t = 0, 1, ... for every CTA size.
constexpr int kFoldCols = 128, kMaxChunk = 64;
template <int NT> struct FoldCfg {
    static constexpr int ROWS = NT / 8;
    static constexpr int SMEM_BYTES = kMaxChunk * (ROWS + kFoldCols) * 4;
};
constexpr int kFoldSmemBytes = FoldCfg<kBB>::SMEM_BYTES;

template <int NT>
__device__ void batch_fold(const BatchParams& P, const SysDesc& d, int nh, float* fsm)
{
    constexpr int kFoldRows = FoldCfg<NT>::ROWS;
    if (nh <= 0) return;
    const float* A = P.A + d.offA;
    const int* hr = P.hist_rows + d.offHist;
    const float* hc = P.hist_c + d.offHist;
    const float* hw = P.hist_w + d.offHistW;
    float* X = P.X + d.offX;
    float* sa = fsm;                          // [nh][kFoldRows]
    float* sw = fsm + kMaxChunk * kFoldRows;  // [nh][kFoldCols]
    const int tr = threadIdx.x / 16, tcol = threadIdx.x % 16;  // rows 2tr, 2tr+1; cols tcol + 16k
    __syncthreads();
    for (int r0 = 0; r0 < d.p; r0 += kFoldRows) {
        for (int e = threadIdx.x; e < nh * kFoldRows; e += NT) {
            const int t = e / kFoldRows, r = e % kFoldRows;
            sa[e] = (r0 + r < d.p) ? hc[t] * A[(long long)hr[t] * d.lda + r0 + r] : 0.f;
        }
        for (int j0 = 0; j0 < d.q; j0 += kFoldCols) {
            for (int e = threadIdx.x; e < nh * kFoldCols; e += NT) {
                const int t = e / kFoldCols, j = e % kFoldCols;
                sw[e] = (j0 + j < d.q) ? hw[(long long)t * d.q + j0 + j] : 0.f;
            }
            __syncthreads();
            float acc[2][8];
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
            for (int t = 0; t < nh; ++t) {
                const float a0 = sa[t * kFoldRows + 2 * tr], a1 = sa[t * kFoldRows + 2 * tr + 1];
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    const float wv = sw[t * kFoldCols + tcol + 16 * b];
                    acc[0][b] = fmaf(a0, wv, acc[0][b]);
                    acc[1][b] = fmaf(a1, wv, acc[1][b]);
                }
            }
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const int rr = r0 + 2 * tr + a;
                if (rr >= d.p) continue;
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    const int j = j0 + tcol + 16 * b;
                    if (j < d.q) X[(long long)rr * d.q + j] += acc[a][b];
                }
            }
            __syncthreads();
        }
    }
}

// dst[r] = X_r . y for rows r < rows (rows of nv float4 vectors, stride ldx
// floats); y in shared memory.  Each warp takes RP rows at a time, so a lane
// has RP independent vector loads in flight per step.
template <int RP, int NW>
__device__ __forceinline__ void batch_rows_dot(const float* X, int ldx, int rows, int nv, const float* y, float* dst)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float4* y4 = reinterpret_cast<const float4*>(y);
    for (int r0 = warp * RP; r0 < rows; r0 += NW * RP) {
        float acc[RP];
#pragma unroll
        for (int k = 0; k < RP; ++k) acc[k] = 0.f;
#pragma unroll 2
        for (int e = lane; e < nv; e += 32) {
            float4 xv[RP];
#pragma unroll
            for (int k = 0; k < RP; ++k)
                if (r0 + k < rows) xv[k] = __ldg(reinterpret_cast<const float4*>(X + (long long)(r0 + k) * ldx) + e);
            const float4 yv = y4[e];
#pragma unroll
            for (int k = 0; k < RP; ++k)
                if (r0 + k < rows)
                    acc[k] = fmaf(xv[k].x, yv.x, fmaf(xv[k].y, yv.y, fmaf(xv[k].z, yv.z, fmaf(xv[k].w, yv.w, acc[k]))));
        }
#pragma unroll
        for (int k = 0; k < RP; ++k) {
            const float t = warp_sum_f(acc[k]);
            if (lane == 0 && r0 + k < rows) dst[r0 + k] = t;
        }
    }
}

// Set-up of one system by one CTA: a_i = ||A_i||^2 (FP64, ascending columns) and
// their running sums, F = ||A||_F^2, ||C||_F^2, lambda ~ ||B||_2^2 from 200 power
// iterations x <- B B^T x / ||.|| (Rayleigh quotient), and a non-finite flag.
// x, t, y: FP64 work vectors of q, n, q entries.  Results valid in thread 0.
struct SetupOut {
    double F, normC2, lambda;
    int bad;
};

__device__ SetupOut system_setup(const float* A, int lda, const float* B, int ldb, const float* C, int ldr, int m,
                                 int p, int q, int n, double* a, double* pref, double* x, double* t, double* y,
                                 double* red, int* s_bad)
{
    if (threadIdx.x == 0) *s_bad = 0;
    __syncthreads();
    int mybad = 0;
    for (int i = threadIdx.x; i < m; i += kBB) {
        double acc = 0.0;
        for (int c = 0; c < p; ++c) {
            const double v = (double)A[(long long)i * lda + c];
            if (!isfinite(v)) mybad = 1;
            acc = __dadd_rn(acc, __dmul_rn(v, v));
        }
        a[i] = acc;
    }
    double c2 = 0.0;
    for (long long e = threadIdx.x; e < (long long)m * n; e += kBB) {
        const double v = (double)C[(e / n) * ldr + e % n];
        if (!isfinite(v)) mybad = 1;
        c2 = fma(v, v, c2);
    }
    for (long long e = threadIdx.x; e < (long long)q * n; e += kBB)
        if (!isfinite(B[(e / n) * ldb + e % n])) mybad = 1;
    if (mybad) atomicOr(s_bad, 1);
    c2 = block_sum_fixed(c2, red);
    SetupOut o;
    o.normC2 = c2;
    o.F = 0.0;
    if (threadIdx.x == 0) {
        double run = 0.0;
        for (int i = 0; i < m; ++i) { run += a[i]; pref[i] = run; }
        o.F = run;
    }
    for (int j = threadIdx.x; j < q; j += kBB) x[j] = 1.0 / sqrt((double)q);
    __syncthreads();
    double lam = 0.0;
    for (int it = 0; it < 200; ++it) {
        for (int l = threadIdx.x; l < n; l += kBB) {
            double acc = 0.0;
            for (int j = 0; j < q; ++j) acc = fma((double)B[(long long)j * ldb + l], x[j], acc);
            t[l] = acc;
        }
        __syncthreads();
        double xy = 0.0, yy = 0.0;
        for (int j = threadIdx.x; j < q; j += kBB) {
            double acc = 0.0;
            for (int l = 0; l < n; ++l) acc = fma((double)B[(long long)j * ldb + l], t[l], acc);
            y[j] = acc;
            xy = fma(x[j], acc, xy);
            yy = fma(acc, acc, yy);
        }
        xy = block_sum_fixed(xy, red);
        yy = block_sum_fixed(yy, red);
        lam = xy;
        const double nrm = sqrt(yy);
        for (int j = threadIdx.x; j < q; j += kBB) x[j] = nrm > 0.0 ? y[j] / nrm : 0.0;
        __syncthreads();
    }
    o.lambda = lam;
    o.bad = *s_bad;
    return o;
}

// largest |c - i| over the nonzero entries M_ic (rows x cols, stride ld), by one CTA
__device__ int half_bandwidth(const float* M, int ld, int rows, int cols, int* s_band)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) *s_band = 0;
    __syncthreads();
    int bw = 0;
    for (int i = warp; i < rows; i += kBW)
        for (int c = lane; c < cols; c += 32)
            if (M[(long long)i * ld + c] != 0.f) bw = max(bw, abs(c - i));
    for (int o = 16; o > 0; o >>= 1) bw = max(bw, __shfl_xor_sync(0xffffffffu, bw, o));
    if (lane == 0) atomicMax(s_band, bw);
    __syncthreads();
    const int r = *s_band;
    __syncthreads();
    return r;
}

// one CTA per system: scalars[s] = {F, ||C||^2, lambda, bad, half-bandwidth of A, of B}
constexpr int kSetupScalars = 6;
__global__ void __launch_bounds__(kBB) batch_setup_kernel(const SysDesc* sys, const float* A, const float* B,
                                                          const float* C, double* a, double* pref, double* scalars)
{
    __shared__ double x[kMaxSide], t[kMaxSide], y[kMaxSide];
    __shared__ double red[2 * kBW];
    __shared__ int bad, band;
    const SysDesc d = sys[blockIdx.x];
    const SetupOut o = system_setup(A + d.offA, d.lda, B + d.offB, d.ldb, C + d.offR, d.ldr, d.m, d.p, d.q, d.n,
                                    a + d.offRow, pref + d.offRow, x, t, y, red, &bad);
    const int bA = half_bandwidth(A + d.offA, d.lda, d.m, d.p, &band);
    const int bB = half_bandwidth(B + d.offB, d.ldb, d.q, d.n, &band);
    if (threadIdx.x == 0) {
        double* sc = scalars + (long long)kSetupScalars * blockIdx.x;
        sc[0] = o.F;
        sc[1] = o.normC2;
        sc[2] = o.lambda;
        sc[3] = (double)o.bad;
        sc[4] = (double)bA;
        sc[5] = (double)bB;
    }
}

// R_i -= coef[i - rb] v for rows [rb, re), fused with the new ||R_i||^2 (Kahan
// FP32 per lane, double-float across lanes); RPW rows per warp at a time, float4
// columns.  v has ldr entries (padding zero).  The norm is left in s_s[i] as a
// (hi, lo) float pair for batch_finalize, which does the FP64 work with full warps.
template <int NW, int RPW>
__device__ __forceinline__ void batch_update_rows(float* R, int ldr, int rb, int re, const float* coef,
                                                  const float* v, double* s_s)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float4* v4 = reinterpret_cast<const float4*>(v);
    const int nv = ldr / 4;
    for (int i0 = rb + RPW * warp; i0 < re; i0 += RPW * NW) {
        float acc[RPW], comp[RPW], cf[RPW];
#pragma unroll
        for (int k2 = 0; k2 < RPW; ++k2) { acc[k2] = 0.f; comp[k2] = 0.f; }
#pragma unroll
        for (int k2 = 0; k2 < RPW; ++k2) cf[k2] = (i0 + k2 < re) ? coef[i0 + k2 - rb] : 0.f;
        for (int e = lane; e < nv; e += 32) {
            float4 rv[RPW];
#pragma unroll
            for (int k2 = 0; k2 < RPW; ++k2)
                if (i0 + k2 < re) rv[k2] = reinterpret_cast<float4*>(R + (long long)(i0 + k2) * ldr)[e];
            const float4 vv = v4[e];
#pragma unroll
            for (int k2 = 0; k2 < RPW; ++k2) {
                if (i0 + k2 >= re) continue;
                float* x = reinterpret_cast<float*>(&rv[k2]);
                const float* y = reinterpret_cast<const float*>(&vv);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    x[c] = fmaf(-cf[k2], y[c], x[c]);
                    const float yk = fmaf(x[c], x[c], -comp[k2]);
                    const float tk = acc[k2] + yk;
                    comp[k2] = (tk - acc[k2]) - yk;
                    acc[k2] = tk;
                }
                reinterpret_cast<float4*>(R + (long long)(i0 + k2) * ldr)[e] = rv[k2];
            }
        }
#pragma unroll
        for (int k2 = 0; k2 < RPW; ++k2) {
            float hi = acc[k2], lo = -comp[k2];
            warp_sum_df(hi, lo);
            if (lane == 0 && i0 + k2 < re) reinterpret_cast<float2*>(s_s)[i0 + k2] = make_float2(hi, lo);
        }
    }
}

// Rows [rb, re) hold their new norms as (hi, lo) float pairs in s_s.  Each warp
// takes a block of 32 rows (lane = row): s_i = hi + lo and r_i = s_i / a_i in
// FP64, then the block's summary: the sum of its s (fixed butterfly order), its
// largest r as an IEEE bit pattern (r >= 0 or -inf, so the integer order is the
// numeric one; ties: smallest row) and that row.  Blocks outside [rb, re) keep
// their summaries.  A warp instruction on the FP64 pipe costs about as much with
// one active lane as with 32, so the FP64 work is spread one row per lane.
template <int NW>
__device__ __forceinline__ void batch_finalize(int m, int rb, int re, const double* a, double* s_s, double* s_r,
                                               double* bsum, long long* bkey, int* barg)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (re <= rb) return;
    const int b0 = rb >> 5, b1 = (re - 1) >> 5;
    for (int b = b0 + warp; b <= b1; b += NW) {
        const int i = (b << 5) + lane;
        double s = 0.0;
        long long key = LLONG_MIN;
        if (i < m) {
            if (i >= rb && i < re) {
                const float2 hl = reinterpret_cast<const float2*>(s_s)[i];
                s = (double)hl.x + (double)hl.y;
                const double ai = __ldg(a + i);
                const double r = ai > 0.0 ? __ddiv_rn(s, ai) : -INFINITY;
                s_s[i] = s;
                s_r[i] = r;
                key = __double_as_longlong(r);
            } else {
                s = s_s[i];
                key = __double_as_longlong(s_r[i]);
            }
        }
        s = warp_sum(s);
        int arg = i;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const long long ok = __shfl_xor_sync(0xffffffffu, key, o);
            const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
            if (ok > key || (ok == key && oa < arg)) { key = ok; arg = oa; }
        }
        if (lane == 0) { bsum[b] = s; bkey[b] = key; barg[b] = arg; }
    }
}

// The banded forms of w_j = R_ik . B_j, (A A_ik^T)_i and v_l = w . B_{:,l} read
// their bands through A(i, c) = A_ic and B(j, l) = B_jl.
struct BandShared {   // the bands of A and B copied to shared memory, diagonal by diagonal
    const float* Ab;  // Ab[(c - i + bA) * m + i] = A_ic
    const float* Bb;  // Bb[(l - j + bB) * q + j] = B_jl
    int m, q, bA, bB;
    __device__ float A(int i, int c) const { return Ab[(c - i + bA) * m + i]; }
    __device__ float B(int j, int l) const { return Bb[(l - j + bB) * q + j]; }
};
struct BandGlobal {   // the bands read from the padded rows in global memory
    const float* Ag;
    const float* Bg;
    int lda, ldb;
    __device__ float A(int i, int c) const { return __ldg(Ag + (long long)i * lda + c); }
    __device__ float B(int j, int l) const { return __ldg(Bg + (long long)j * ldb + l); }
};

// One banded iteration after the pick (R_ik staged in s_vec): w, c_k u on the rows
// within 2 bA of i_k, v, this term's X update (the rows of A_ik's band), then R
// and the norms of the touched rows; each band is summed in ascending index
// order, one thread per output.  Returns with s_s holding (hi, lo) pairs for rows
// [u0, u1] (batch_finalize completes them).
template <int NT, int RPW, class Band>
__device__ __forceinline__ void batch_banded_step(const Band& bd, const SysDesc& d, float* R, float* X, int ik,
                                                  double ck, float* s_vec, float* s_w, float* s_u, double* s_s,
                                                  int& u0, int& u1)
{
    constexpr int NW = NT / 32;
    const int bA = d.bandA, bB = d.bandB;
    // w_j = sum over |l - j| <= bB of R_ik,l B_jl
    for (int j = threadIdx.x; j < d.q; j += NT) {
        const int l0 = max(0, j - bB), l1 = min(d.n - 1, j + bB);
        float acc = 0.f;
        for (int l = l0; l <= l1; ++l) acc = fmaf(s_vec[l], bd.B(j, l), acc);
        s_w[j] = acc;
    }
    // c_k u_i for |i - ik| <= 2 bA: u_i = (A A_ik^T)_i vanishes elsewhere
    u0 = max(0, ik - 2 * bA);
    u1 = min(d.m - 1, ik + 2 * bA);
    for (int i = u0 + threadIdx.x; i <= u1; i += NT) {
        const int c0 = max(0, max(i, ik) - bA), c1 = min(d.p - 1, min(i, ik) + bA);
        float acc = 0.f;
        for (int c = c0; c <= c1; ++c) acc = fmaf(bd.A(i, c), bd.A(ik, c), acc);
        s_u[i - u0] = (float)(ck * (double)acc);
    }
    __syncthreads();
    // v_l = sum over |j - l| <= bB of w_j B_jl (padding columns 0)
    for (int l = threadIdx.x; l < d.ldr; l += NT) {
        float acc = 0.f;
        if (l < d.n) {
            const int j0 = max(0, l - bB), j1 = min(d.q - 1, l + bB);
            for (int j = j0; j <= j1; ++j) acc = fmaf(s_w[j], bd.B(j, l), acc);
        }
        s_vec[l] = acc;
    }
    // X_c += c_k A_ik,c w for the rows c of A_ik's band (this term of the X update,
    // applied at once: A_ik^T w has no other nonzero rows)
    {
        const int xc0 = max(0, ik - bA), xc1 = min(d.p - 1, ik + bA);
        const float ckf = (float)ck;
        for (int j = threadIdx.x; j < d.q; j += NT) {
            const float wj = s_w[j];
            for (int c0 = xc0; c0 <= xc1; c0 += 8) {
                float xv[8];
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    if (c0 + e <= xc1) xv[e] = X[(long long)(c0 + e) * d.q + j];
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    if (c0 + e <= xc1) X[(long long)(c0 + e) * d.q + j] = fmaf(ckf * bd.A(ik, c0 + e), wj, xv[e]);
            }
        }
    }
    __syncthreads();
    batch_update_rows<NW, RPW>(R, d.ldr, u0, u1 + 1, s_u, s_vec, s_s);
}

template <int NT, int RPW>
__global__ void __launch_bounds__(NT, 1) batch_kernel_t(BatchParams P)
{
    constexpr int NW = NT / 32;
    constexpr int NB = kMaxSide / 32;                     // row blocks of 32
    __shared__ double s_s[kMaxSide];                      // ||R_i||^2 (or its (hi, lo) pair while updated)
    __shared__ double s_r[kMaxSide];                      // s_i / a_i
    __shared__ double s_ck[kMaxSide];                     // c_i = alpha / a_i
    __shared__ __align__(16) float s_vec[kMaxSide];       // R_{i_k} row, then v
    __shared__ __align__(16) float s_arow[kMaxSide];      // A_{i_k} (dense path)
    __shared__ __align__(16) float s_w[kMaxSide];         // w
    __shared__ __align__(16) float s_u[kMaxSide];         // c_k u
    extern __shared__ __align__(16) float dyn_smem[];     // dense path: fold tiles; banded path: the bands
    __shared__ double s_bsum[NB], s_bJ[NB];               // per block: sum of s, admitted sum
    __shared__ long long s_bkey[NB];                      // per block: largest r (bit pattern)
    __shared__ int s_barg[NB];                            // per block: its row
    __shared__ double red[2 * 32];
    __shared__ int s_sys, s_first, s_stop, s_ik;
    __shared__ double s_S, s_t, s_uk;
    __shared__ long long s_imax;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const int slot = atomicAdd(P.queue, 1);
            s_sys = (slot < P.nsys) ? P.order[slot] : -1;
        }
        __syncthreads();
        const int sid = s_sys;
        if (sid < 0) return;
        const SysDesc d = P.sys[sid];
        const float* A = P.A + d.offA;
        const float* B = P.B + d.offB;
        const float* C = P.C + d.offR;
        float* R = P.R + d.offR;
        float* X = P.X + d.offX;
        const double* a = P.a + d.offRow;
        const double* pref = P.rbk_prefix + d.offRow;
        int* hrow = P.hist_rows + d.offHist;
        float* hcf = P.hist_c + d.offHist;
        float* hw = P.hist_w + d.offHistW;
        const bool banded = d.bandA >= 0;
        const bool band_sm =
            banded && 4LL * ((2LL * d.bandA + 1) * d.m + (2LL * d.bandB + 1) * d.q) <= (long long)P.band_smem;

        for (int i = threadIdx.x; i < d.m; i += NT) {
            const double ai = a[i];
            s_ck[i] = ai > 0.0 ? __ddiv_rn(d.alpha, ai) : 0.0;
        }
        if (band_sm) {  // the bands of A and B, diagonal by diagonal (zero outside the matrix)
            float* Ab = dyn_smem;
            float* Bb = dyn_smem + (2 * d.bandA + 1) * d.m;
            for (int e = threadIdx.x; e < (2 * d.bandA + 1) * d.m; e += NT) {
                const int i = e % d.m, c = i + e / d.m - d.bandA;
                Ab[e] = (c >= 0 && c < d.p) ? A[(long long)i * d.lda + c] : 0.f;
            }
            for (int e = threadIdx.x; e < (2 * d.bandB + 1) * d.q; e += NT) {
                const int j = e % d.q, l = j + e / d.q - d.bandB;
                Bb[e] = (l >= 0 && l < d.n) ? B[(long long)j * d.ldb + l] : 0.f;
            }
        }

        // R^0 = C - A X^0 B (row by row) or R^0 = C
        if (P.init_from_x) {
            // on the banded path only the bands of A_i and of B's columns contribute
            for (int i = 0; i < d.m; ++i) {
                const int c0 = banded ? max(0, i - d.bandA) : 0, c1 = banded ? min(d.p - 1, i + d.bandA) : d.p - 1;
                for (int j = threadIdx.x; j < d.q; j += NT) {  // t = A_i X
                    float acc = 0.f;
                    for (int c2 = c0; c2 <= c1; ++c2)
                        acc = fmaf(A[(long long)i * d.lda + c2], X[(long long)c2 * d.q + j], acc);
                    s_w[j] = acc;
                }
                __syncthreads();
                for (int l = threadIdx.x; l < d.n; l += NT) {  // R_i = C_i - t B
                    const int j0 = banded ? max(0, l - d.bandB) : 0, j1 = banded ? min(d.q - 1, l + d.bandB) : d.q - 1;
                    float acc = 0.f;
                    for (int j = j0; j <= j1; ++j) acc = fmaf(s_w[j], B[(long long)j * d.ldb + l], acc);
                    R[(long long)i * d.ldr + l] = C[(long long)i * d.ldr + l] - acc;
                }
                __syncthreads();
            }
        } else if (C != R) {
            const float4* C4 = reinterpret_cast<const float4*>(C);
            float4* R4 = reinterpret_cast<float4*>(R);
            for (long long e = threadIdx.x; e < (long long)d.m * d.ldr / 4; e += NT) R4[e] = __ldg(C4 + e);
        }
        __syncthreads();

        // row norms of R^0: warp per row (Kahan FP32 lanes, double-float across lanes),
        // then the FP64 values and the block summaries
        for (int pass = 0; pass < 2; ++pass) {
            for (int i = warp; i < d.m; i += NW) {
                float acc = 0.f, comp = 0.f;
                for (int l = lane; l < d.n; l += 32) {
                    const float x = R[(long long)i * d.ldr + l];
                    const float y = fmaf(x, x, -comp);
                    const float t = acc + y;
                    comp = (t - acc) - y;
                    acc = t;
                }
                float hi = acc, lo = -comp;
                warp_sum_df(hi, lo);
                if (lane == 0) reinterpret_cast<float2*>(s_s)[i] = make_float2(hi, lo);
            }
            __syncthreads();
            batch_finalize<NW>(d.m, 0, d.m, a, s_s, s_r, s_bsum, s_bkey, s_barg);
            __syncthreads();
            if (!P.init_from_x || pass == 1) break;
            // test the caller's X0 against X0 = 0: keep it only if ||C - A X0 B|| < ||C||
            double S0 = 0.0;
            for (int i = threadIdx.x; i < d.m; i += NT) S0 += s_s[i];
            S0 = block_sum_fixed<NW>(S0, red);
            const bool reject = !(S0 < d.normC2);
            if (threadIdx.x == 0 && P.x0_rejected) P.x0_rejected[sid] = reject ? 1 : 0;
            if (!reject) break;
            for (long long e = threadIdx.x; e < (long long)d.p * d.q; e += NT) X[e] = 0.f;
            for (long long e = threadIdx.x; e < (long long)d.m * d.ldr; e += NT) R[e] = C[e];
            __syncthreads();
        }

        const int nb = (d.m + 31) >> 5;
        const int var = P.variant;
        long long k = 0;
        int nh = 0, flag = FLAG_RUNNING;
        for (;;) {
            // ---- totals from the block summaries (one warp), threshold, draw and stop test
            if (warp == 0) {
                double S = lane < nb ? s_bsum[lane] : 0.0;
                long long key = lane < nb ? s_bkey[lane] : LLONG_MIN;
                int arg = lane < nb ? s_barg[lane] : INT_MAX;
                S = warp_sum(S);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const long long ok = __shfl_xor_sync(0xffffffffu, key, o);
                    const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
                    if (ok > key || (ok == key && oa < arg)) { key = ok; arg = oa; }
                }
                if (lane == 0) {
                    // S >= 0 (or NaN), stop_S >= 0 or -1: the tests compare bit patterns, off the
                    // FP64 pipe (a NaN S has a pattern above +inf's and is caught by !(S > 0))
                    const double rmax = __longlong_as_double(key);
                    const long long Sk = __double_as_longlong(S);
                    s_S = S;
                    s_imax = arg;
                    int stop = 0;
                    if (!(Sk > 0 && Sk < 0x7ff0000000000001LL)) stop = 2;
                    else if (__double_as_longlong(d.stop_S) >= 0 && Sk <= __double_as_longlong(d.stop_S)) stop = 1;
                    else if (k >= P.maxit) stop = 4;
                    s_stop = stop;
                    if (!stop && (var == GRBK_GRBK || var == GRBK_RGRBK)) {
                        const double theta = (var == GRBK_GRBK) ? 0.5 : P.theta;
                        double t = __dadd_rn(__dmul_rn(theta, rmax), __dmul_rn(1.0 - theta, __ddiv_rn(S, d.F)));
                        if (__double_as_longlong(t) > key) t = rmax;
                        s_t = t;
                    }
                }
            } else if (warp == 1 && lane == 0 && var != GRBK_MWRBK && var != GRBK_BK) {
                // the draw of this iteration, beside the totals
                s_uk = philox_uniform(P.seed, (uint64_t)k, (uint64_t)sid);
            }
            __syncthreads();
            if (s_stop) {
                if (s_stop == 1) flag = FLAG_TOL_MET;
                if (s_stop == 2) flag = FLAG_EXACT;
                break;
            }
            // ---- select i_k
            int ik;
            if (var == GRBK_GRBK || var == GRBK_RGRBK) {
                // the admitted (r_i >= t, compared as bit patterns) sum of every block that
                // has an admitted row; then one warp finds the block and the row where the
                // prefix of the admitted s_i first exceeds u S_J
                const long long tkey = __double_as_longlong(s_t);
                for (int b = warp; b < nb; b += NW) {
                    double v = 0.0;
                    if (s_bkey[b] >= tkey) {
                        const int i = (b << 5) + lane;
                        if (i < d.m && __double_as_longlong(s_r[i]) >= tkey) v = s_s[i];
                        v = warp_sum(v);
                    }
                    if (lane == 0) s_bJ[b] = v;
                }
                __syncthreads();
                if (warp == 0) {
                    const double bv = lane < nb ? s_bJ[lane] : 0.0;
                    const double inc = warp_inclusive_scan(bv);
                    const double SJ = __shfl_sync(0xffffffffu, inc, 31);
                    const double target = __dmul_rn(s_uk, SJ);
                    const long long gk = __double_as_longlong(target);
                    const unsigned hit =
                        __ballot_sync(0xffffffffu, __double_as_longlong(bv) > 0 && __double_as_longlong(inc) > gk);
                    int cb;
                    double base;
                    if (hit) {
                        cb = __ffs(hit) - 1;
                        base = __shfl_sync(0xffffffffu, inc - bv, cb);
                    } else {  // rounding left u S_J uncovered: the last admitted row
                        const unsigned nz = __ballot_sync(0xffffffffu, __double_as_longlong(bv) > 0);
                        cb = nz ? 31 - __clz(nz) : -1;
                        base = -INFINITY;
                    }
                    int pick = -1;
                    if (cb >= 0) {
                        const int i = (cb << 5) + lane;
                        const bool adm = i < d.m && __double_as_longlong(s_r[i]) >= tkey;
                        const double inc2 = base + warp_inclusive_scan(adm ? s_s[i] : 0.0);
                        const unsigned h2 = __ballot_sync(0xffffffffu, adm && __double_as_longlong(inc2) > gk);
                        const unsigned am = __ballot_sync(0xffffffffu, adm);
                        if (h2) pick = (cb << 5) + __ffs(h2) - 1;
                        else if (am) pick = (cb << 5) + 31 - __clz(am);
                    }
                    if (pick < 0) pick = (int)s_imax;
                    if (lane == 0) s_ik = pick;
                }
                __syncthreads();
                ik = s_ik;
            } else if (var == GRBK_MWRBK) {
                ik = (int)s_imax;
            } else if (var == GRBK_RBK) {
                if (threadIdx.x == 0) {
                    const double target = __dmul_rn(s_uk, d.F);
                    int lo = 0, hi = d.m;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (pref[mid] > target) hi = mid; else lo = mid + 1;
                    }
                    if (lo >= d.m) {
                        lo = d.m - 1;
                        while (lo > 0 && !(a[lo] > 0.0)) --lo;
                    }
                    s_first = lo;
                }
                __syncthreads();
                ik = s_first;
            } else {
                ik = (int)(k % d.m);
            }
            const double ck = s_ck[ik];
            if (threadIdx.x == 0 && k < P.trace_len) P.trace_rows[(long long)sid * P.trace_len + k] = ik;

            int rb = 0, re = d.m;
            if (banded) {
                // ---- banded A and B: u_i = (A A_ik^T)_i vanishes for |i - ik| > 2 bandA, so the
                // update touches those rows only; w and v use the band of B
                {
                    const float4* Rr = reinterpret_cast<const float4*>(R + (long long)ik * d.ldr);
                    for (int e = threadIdx.x; e < d.ldr / 4; e += NT) reinterpret_cast<float4*>(s_vec)[e] = Rr[e];
                }
                __syncthreads();
                int u0, u1;
                if (band_sm) {
                    const BandShared bd{dyn_smem, dyn_smem + (2 * d.bandA + 1) * d.m, d.m, d.q, d.bandA, d.bandB};
                    batch_banded_step<NT, RPW>(bd, d, R, X, ik, ck, s_vec, s_w, s_u, s_s, u0, u1);
                } else {
                    const BandGlobal bd{A, B, d.lda, d.ldb};
                    batch_banded_step<NT, RPW>(bd, d, R, X, ik, ck, s_vec, s_w, s_u, s_s, u0, u1);
                }
                rb = u0;
                re = u1 + 1;
            } else {
                // ---- w = R_ik B^T, u = A A_ik^T (rows of B and A streamed as float4, 4 rows per warp)
                {
                    const float4* Rr = reinterpret_cast<const float4*>(R + (long long)ik * d.ldr);
                    const float4* Ar = reinterpret_cast<const float4*>(A + (long long)ik * d.lda);
                    for (int e = threadIdx.x; e < d.ldr / 4; e += NT) reinterpret_cast<float4*>(s_vec)[e] = Rr[e];
                    for (int e = threadIdx.x; e < d.lda / 4; e += NT) reinterpret_cast<float4*>(s_arow)[e] = __ldg(Ar + e);
                }
                __syncthreads();
                batch_rows_dot<4, NW>(B, d.ldb, d.q, d.ldb / 4, s_vec, s_w);
                batch_rows_dot<4, NW>(A, d.lda, d.m, d.lda / 4, s_arow, s_u);
                __syncthreads();
                for (int i = threadIdx.x; i < d.m; i += NT) s_u[i] = (float)(ck * (double)s_u[i]);  // coefficient c_k u_i
                // ---- record the term, v = w B (vector columns, row classes reduced in shared memory)
                if (threadIdx.x == 0) { hrow[nh] = ik; hcf[nh] = (float)ck; }
                for (int j = threadIdx.x; j < d.q; j += NT) hw[(long long)nh * d.q + j] = s_w[j];
                {
                    const int nv4 = d.ldb / 4;
                    float4* red4 = reinterpret_cast<float4*>(dyn_smem);  // [RG][cols] float4
                    for (int cb = 0; cb < nv4; cb += NT) {
                        const int ncols = min(NT, nv4 - cb);
                        const int RG = NT / ncols;
                        const int e = threadIdx.x % ncols, rg = threadIdx.x / ncols;
                        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (rg < RG) {
                            const float4* col = reinterpret_cast<const float4*>(B) + cb + e;
                            const int ldv = d.ldb / 4;
    #pragma unroll 8
                            for (int j = rg; j < d.q; j += RG) {
                                const float4 bv = __ldg(col + (long long)j * ldv);
                                const float wj = s_w[j];
                                acc.x = fmaf(wj, bv.x, acc.x);
                                acc.y = fmaf(wj, bv.y, acc.y);
                                acc.z = fmaf(wj, bv.z, acc.z);
                                acc.w = fmaf(wj, bv.w, acc.w);
                            }
                            red4[rg * ncols + e] = acc;
                        }
                        __syncthreads();
                        for (int t = threadIdx.x; t < ncols; t += NT) {
                            float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
                            for (int r2 = 0; r2 < RG; ++r2) {
                                const float4 v = red4[r2 * ncols + t];
                                sum.x += v.x; sum.y += v.y; sum.z += v.z; sum.w += v.w;
                            }
                            reinterpret_cast<float4*>(s_vec)[cb + t] = sum;
                        }
                        __syncthreads();
                    }
                }
                // ---- R -= c u v fused with the new row norms
                batch_update_rows<NW, RPW>(R, d.ldr, 0, d.m, s_u, s_vec, s_s);
                ++nh;
            }
            __syncthreads();
            batch_finalize<NW>(d.m, rb, re, a, s_s, s_r, s_bsum, s_bkey, s_barg);
            ++k;
            if (nh == P.chunk) {
                batch_fold<NT>(P, d, nh, dyn_smem);
                nh = 0;
            }
            __syncthreads();
        }
        batch_fold<NT>(P, d, nh, dyn_smem);
        if (threadIdx.x == 0) {
            P.iters[sid] = k;
            P.S_out[sid] = s_S;
            P.flag_out[sid] = flag;
        }
    }
}

// ---------------------------------------------------------------------------
// Batch autotuner: the compiled variants of the batched kernel (threads per
// CTA, rows per warp of the fused update pass).  All variants compute the same
// iteration; they differ in how the work of one system is spread over the CTA
// (and so in how many CTAs fit on an SM) and only in the summation order of
// the FP64 totals.  A system's variant is chosen by timing every variant on it
// and kept per system shape for the rest of the process.
// ---------------------------------------------------------------------------
struct BatchVariant {
    int threads, rpw;
    void (*kern)(BatchParams);
    int smem;
};
static const BatchVariant kVariants[] = {
    {256, 1, batch_kernel_t<256, 1>, FoldCfg<256>::SMEM_BYTES},
    {256, 2, batch_kernel_t<256, 2>, FoldCfg<256>::SMEM_BYTES},
    {256, 4, batch_kernel_t<256, 4>, FoldCfg<256>::SMEM_BYTES},
    {512, 1, batch_kernel_t<512, 1>, FoldCfg<512>::SMEM_BYTES},
    {512, 2, batch_kernel_t<512, 2>, FoldCfg<512>::SMEM_BYTES},
    {512, 4, batch_kernel_t<512, 4>, FoldCfg<512>::SMEM_BYTES},
};
constexpr int kNumVariants = (int)(sizeof(kVariants) / sizeof(kVariants[0]));
constexpr int kDefaultVariant = 4;   // 512 threads, two rows per warp
constexpr int kTuneIters = 48;       // iterations of one timed trial

}  // namespace grbk

// ============================================================================
// host side
// ============================================================================
using namespace grbk;

struct grbk_batch {
    int nsys;
    grbk_opts opts;
    cudaStream_t stream;
    std::vector<SysDesc> hsys;
    std::vector<int> order;
    std::vector<double> normC2;
    SysDesc* dsys;
    int* dorder;
    int* dqueue;
    float *A, *B, *C, *R, *X;
    double *a, *pref;
    int* hist_rows;
    float *hist_c, *hist_w;
    long long* iters;
    double* S;
    int* flags;
    int* trace;
    int* rejected;
    int chunk;
    long long totA, totB, totR, totX, totRow, totHist, totHistW;
    std::vector<int> variant;        // kernel variant of each system
    int goff[grbk::kNumVariants] = {}, gcnt[grbk::kNumVariants] = {};   // systems of each variant in dorder
    int* dids = nullptr;             // system ids 0 .. nsys-1 (one-system tuning launches)
    cudaStream_t side[grbk::kNumVariants] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[grbk::kNumVariants] = {};
    double tune_seconds = 0.0;
};

static void* dmalloc(size_t bytes)
{
    void* p = nullptr;
    if (cudaMalloc(&p, bytes > 0 ? bytes : 16) != cudaSuccess) return nullptr;
    return p;
}

// ---- autotuner bookkeeping (host only) -------------------------------------
// A system's class: its sides rounded up to multiples of 64 and its exact
// half-bandwidths (-1 on the dense path).
struct TuneKey {
    int m, p, q, n, bandA, bandB;
    bool operator<(const TuneKey& o) const
    {
        const int a[6] = {m, p, q, n, bandA, bandB}, b[6] = {o.m, o.p, o.q, o.n, o.bandA, o.bandB};
        return std::lexicographical_compare(a, a + 6, b, b + 6);
    }
};
static std::map<TuneKey, int> g_tune_cache;
static std::mutex g_tune_mu;

static TuneKey tune_key(int m, int p, int q, int n, int bandA, int bandB)
{
    auto r64 = [](int x) { return (x + 63) / 64 * 64; };
    return TuneKey{r64(m), r64(p), r64(q), r64(n), bandA, bandB};
}

// The fastest variant; a variant within 2 % of the fastest that uses fewer
// threads wins (more CTAs fit on an SM, which helps the other systems).
static int tune_choose(const double* ms, int nv)
{
    int best = -1;
    for (int v = 0; v < nv; ++v)
        if (ms[v] > 0.0 && std::isfinite(ms[v]) && (best < 0 || ms[v] < ms[best])) best = v;
    if (best < 0) return kDefaultVariant;
    int pick = best;
    for (int v = 0; v < nv; ++v)
        if (ms[v] > 0.0 && std::isfinite(ms[v]) && ms[v] <= 1.02 * ms[best] &&
            kVariants[v].threads < kVariants[pick].threads)
            pick = v;
    return pick;
}

extern "C" int32_t grbk_tune_num_variants(void) { return kNumVariants; }

extern "C" grbk_status grbk_tune_variant_info(int32_t v, int32_t* threads, int32_t* rows_per_warp)
{
    if (v < 0 || v >= kNumVariants) return GRBK_EINVAL;
    if (threads) *threads = kVariants[v].threads;
    if (rows_per_warp) *rows_per_warp = kVariants[v].rpw;
    return GRBK_OK;
}

extern "C" int32_t grbk_tune_choose(const double* ms, int32_t nv)
{
    if (!ms || nv != kNumVariants) return -1;
    return tune_choose(ms, nv);
}

extern "C" grbk_status grbk_tune_lookup(int32_t m, int32_t p, int32_t q, int32_t n, int32_t bandA, int32_t bandB,
                                        int32_t* variant)
{
    if (!variant) return GRBK_EINVAL;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    const auto it = g_tune_cache.find(tune_key(m, p, q, n, bandA, bandB));
    *variant = it == g_tune_cache.end() ? -1 : it->second;
    return GRBK_OK;
}

extern "C" grbk_status grbk_tune_store(int32_t m, int32_t p, int32_t q, int32_t n, int32_t bandA, int32_t bandB,
                                       int32_t variant)
{
    if (variant < 0 || variant >= kNumVariants) return GRBK_EINVAL;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[tune_key(m, p, q, n, bandA, bandB)] = variant;
    return GRBK_OK;
}

extern "C" void grbk_tune_clear(void)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache.clear();
}

extern "C" void grbk_batch_destroy(grbk_batch* b)
{
    if (!b) return;
    void* bufs[] = {b->dsys, b->dorder, b->dqueue, b->A, b->B, b->C, b->R, b->X, b->a, b->pref,
                    b->hist_rows, b->hist_c, b->hist_w, b->iters, b->S, b->flags, b->trace, b->rejected, b->dids};
    for (void* p : bufs)
        if (p) cudaFree(p);
    for (int v = 0; v < kNumVariants; ++v) {
        if (b->side[v]) cudaStreamDestroy(b->side[v]);
        if (b->ev_join[v]) cudaEventDestroy(b->ev_join[v]);
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    delete b;
}

// Caller matrices -> padded FP32 device rows, for many systems in one call.  An FP32
// host matrix is copied straight into its rows; an FP64 host matrix goes through one
// staging block (largest of them, reused in stream order, released after one wait).
struct BatchLoader {
    cudaStream_t st;
    void* tmp = nullptr;
    size_t tmp_bytes = 0;
    grbk_status load(const grbk_mat* M, float* dst, int64_t ldd)
    {
        const int64_t rows = M->rows, cols = M->cols;
        if (M->on_device) {
            GRBK_CK(convert_matrix(dst, GRBK_DT_F32, ldd, M->ptr, M->dtype, M->ld, rows, cols, st));
            return GRBK_OK;
        }
        if (M->dtype == GRBK_DT_F32) {
            GRBK_CK(cudaMemcpy2DAsync(dst, ldd * 4, M->ptr, M->ld * 4, cols * 4, rows, cudaMemcpyHostToDevice, st));
            return GRBK_OK;
        }
        const size_t need = (size_t)rows * cols * 8;
        if (need > tmp_bytes) {
            if (tmp) { cudaStreamSynchronize(st); dev_free(tmp); tmp = nullptr; tmp_bytes = 0; }
            if (dev_alloc(&tmp, need) != cudaSuccess) return GRBK_ENOMEM;
            tmp_bytes = need;
        }
        GRBK_CK(cudaMemcpy2DAsync(tmp, cols * 8, M->ptr, M->ld * 8, cols * 8, rows, cudaMemcpyHostToDevice, st));
        GRBK_CK(convert_matrix(dst, GRBK_DT_F32, ldd, tmp, M->dtype, cols, rows, cols, st));
        return GRBK_OK;
    }
    grbk_status finish()
    {
        const cudaError_t e = cudaStreamSynchronize(st);
        if (tmp) dev_free(tmp);
        tmp = nullptr;
        tmp_bytes = 0;
        return e == cudaSuccess ? GRBK_OK : GRBK_ECUDA;
    }
    ~BatchLoader() { finish(); }
};

static bool dtype_ok(int32_t dt) { return dt == GRBK_DT_F64 || dt == GRBK_DT_F32; }

// an X^0 or X output descriptor the copies can follow: p x q, row stride >= q, FP32 or FP64
static bool x_desc_ok(const grbk_mat& M, int p, int q)
{
    return M.ptr && M.rows == p && M.cols == q && M.ld >= q && dtype_ok(M.dtype);
}

// The kernel parameters of a launch over the systems order[0 .. n) (queue counter at queue).
static BatchParams batch_params(grbk_batch* b, const int* order, int n, int* queue)
{
    BatchParams P;
    memset(&P, 0, sizeof(P));
    P.nsys = n; P.sys = b->dsys; P.order = order; P.queue = queue;
    P.A = b->A; P.B = b->B; P.C = b->C; P.R = b->R; P.X = b->X; P.a = b->a; P.rbk_prefix = b->pref;
    P.hist_rows = b->hist_rows; P.hist_c = b->hist_c; P.hist_w = b->hist_w;
    P.iters = b->iters; P.S_out = b->S; P.flag_out = b->flags;
    P.chunk = b->chunk;
    P.x0_rejected = b->rejected;
    return P;
}

// Shared-memory bytes of a banded system's band copies (0 on the dense path, and
// when they exceed kBandSmemCap: such a system reads its bands from global memory).
constexpr int kBandSmemCap = 150 * 1024;
static int band_smem_bytes(const SysDesc& d)
{
    if (d.bandA < 0) return 0;
    const long long bytes = 4LL * ((2LL * d.bandA + 1) * d.m + (2LL * d.bandB + 1) * d.q);
    return bytes <= kBandSmemCap ? (int)bytes : 0;
}

// One launch of variant v over nsys_launch systems; band_bytes: the largest band
// copy among them (the dynamic shared memory is the larger of it and the dense
// path's fold tiles).
static grbk_status launch_variant(int v, BatchParams P, int nsys_launch, int grid_cap, int band_bytes,
                                  cudaStream_t st)
{
    const BatchVariant& V = kVariants[v];
    int dev = 0, nsm = 0, per_sm = 0;
    const int smem = std::max(V.smem, band_bytes);
    P.band_smem = smem;
    GRBK_CK(cudaGetDevice(&dev));
    GRBK_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    GRBK_CK(cudaFuncSetAttribute(V.kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    GRBK_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, V.kern, V.threads, smem));
    int grid = nsm * (per_sm > 0 ? per_sm : 1);
    if (grid_cap > 0) grid = std::min(grid, grid_cap);
    grid = std::min(grid, nsys_launch);
    V.kern<<<grid, V.threads, smem, st>>>(P);
    GRBK_CK(cudaGetLastError());
    return GRBK_OK;
}

// Time every variant on one system of each class not yet in the cache (ME-GRBK,
// kTuneIters iterations from R = C, one untimed and one timed launch each) and
// keep the choice.  The systems' R and X are left as the trials leave them;
// every solve starts them afresh.
static grbk_status batch_autotune(grbk_batch* b)
{
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t st = b->stream;
    std::vector<int> ids(b->nsys);
    for (int s = 0; s < b->nsys; ++s) ids[s] = s;
    b->dids = (int*)dmalloc(4 * b->nsys);
    if (!b->dids) return GRBK_ENOMEM;
    GRBK_CK(cudaMemcpyAsync(b->dids, ids.data(), 4 * b->nsys, cudaMemcpyHostToDevice, st));
    GRBK_CK(cudaMemcpyAsync(b->dsys, b->hsys.data(), sizeof(SysDesc) * b->nsys, cudaMemcpyHostToDevice, st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    GRBK_CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return GRBK_ECUDA; }
    grbk_status res = GRBK_OK;
    for (int s : b->order) {
        const SysDesc& d = b->hsys[s];
        int32_t v = -1;
        grbk_tune_lookup(d.m, d.p, d.q, d.n, d.bandA, d.bandB, &v);
        if (v >= 0) { b->variant[s] = v; continue; }
        double ms[kNumVariants];
        BatchParams P = batch_params(b, b->dids + s, 1, b->dqueue);
        P.variant = GRBK_GRBK; P.theta = 0.5; P.seed = 1; P.maxit = kTuneIters;
        for (int vv = 0; vv < kNumVariants && res == GRBK_OK; ++vv) {
            float el = 0.f;
            for (int rep = 0; rep < 2 && res == GRBK_OK; ++rep) {
                if (cudaMemsetAsync(b->dqueue, 0, 4, st) != cudaSuccess) { res = GRBK_ECUDA; break; }
                if (rep == 1 && cudaEventRecord(e0, st) != cudaSuccess) { res = GRBK_ECUDA; break; }
                res = launch_variant(vv, P, 1, 1, band_smem_bytes(d), st);
                if (res == GRBK_OK && rep == 1 && cudaEventRecord(e1, st) != cudaSuccess) res = GRBK_ECUDA;
            }
            if (res == GRBK_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&el, e0, e1) != cudaSuccess))
                res = GRBK_ECUDA;
            ms[vv] = el;
        }
        if (res != GRBK_OK) break;
        v = tune_choose(ms, kNumVariants);
        grbk_tune_store(d.m, d.p, d.q, d.n, d.bandA, d.bandB, v);
        b->variant[s] = v;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tune_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return res;
}

extern "C" grbk_status grbk_batch_create(grbk_batch** out, int32_t nsys, const grbk_mat* A, const grbk_mat* B,
                                         const grbk_mat* C, const grbk_opts* opts)
{
    if (!out || nsys <= 0 || !A || !B || !C) return GRBK_EINVAL;
    *out = nullptr;
    grbk_opts o;
    if (opts) o = *opts; else grbk_default_opts(&o);
    if (!std::isfinite(o.alpha)) return GRBK_EINVAL;
    for (int s = 0; s < nsys; ++s) {
        const int64_t m = A[s].rows, p = A[s].cols, q = B[s].rows, n = B[s].cols;
        if (o.alphas && !(std::isfinite(o.alphas[s]) && o.alphas[s] > 0.0)) return GRBK_EINVAL;
        if (!A[s].ptr || !B[s].ptr || !C[s].ptr) return GRBK_EINVAL;
        if (m <= 0 || p <= 0 || q <= 0 || n <= 0 || C[s].rows != m || C[s].cols != n) return GRBK_EINVAL;
        if (m > kMaxSide || p > kMaxSide || q > kMaxSide || n > kMaxSide) return GRBK_EINVAL;
        if (A[s].ld < p || B[s].ld < n || C[s].ld < n) return GRBK_EINVAL;
        if (!dtype_ok(A[s].dtype) || !dtype_ok(B[s].dtype) || !dtype_ok(C[s].dtype)) return GRBK_EINVAL;
    }
    grbk_batch* b = new grbk_batch();
    b->nsys = nsys;
    b->opts = o;
    b->stream = (cudaStream_t)o.stream;
    b->chunk = o.check_every > 0 ? std::min(o.check_every, kMaxChunk) : kMaxChunk;
    b->hsys.resize(nsys);
    long long oA = 0, oB = 0, oR = 0, oX = 0, oRow = 0, oH = 0, oHW = 0;
    for (int s = 0; s < nsys; ++s) {
        SysDesc& d = b->hsys[s];
        memset(&d, 0, sizeof(d));
        d.m = (int)A[s].rows; d.p = (int)A[s].cols; d.q = (int)B[s].rows; d.n = (int)B[s].cols;
        d.lda = (int)round_up(d.p, 4); d.ldb = (int)round_up(d.n, 4); d.ldr = d.ldb;
        d.offA = oA; d.offB = oB; d.offR = oR; d.offX = oX; d.offRow = oRow; d.offHist = oH; d.offHistW = oHW;
        oA += (long long)d.m * d.lda; oB += (long long)d.q * d.ldb; oR += (long long)d.m * d.ldr;
        oX += (long long)d.p * d.q; oRow += d.m; oH += b->chunk; oHW += (long long)b->chunk * d.q;
    }
    b->totA = oA; b->totB = oB; b->totR = oR; b->totX = oX; b->totRow = oRow; b->totHist = oH; b->totHistW = oHW;
    b->A = (float*)dmalloc(oA * 4); b->B = (float*)dmalloc(oB * 4); b->C = (float*)dmalloc(oR * 4);
    b->R = (float*)dmalloc(oR * 4); b->X = (float*)dmalloc(oX * 4);
    b->a = (double*)dmalloc(oRow * 8); b->pref = (double*)dmalloc(oRow * 8);
    b->hist_rows = (int*)dmalloc(oH * 4); b->hist_c = (float*)dmalloc(oH * 4); b->hist_w = (float*)dmalloc(oHW * 4);
    b->dsys = (SysDesc*)dmalloc(sizeof(SysDesc) * nsys); b->dorder = (int*)dmalloc(4 * nsys);
    b->dqueue = (int*)dmalloc(4 * kNumVariants); b->iters = (long long*)dmalloc(8 * nsys); b->S = (double*)dmalloc(8 * nsys);
    b->flags = (int*)dmalloc(4 * nsys);
    b->rejected = (int*)dmalloc(4 * nsys);
    if (!b->rejected || !b->A || !b->B || !b->C || !b->R || !b->X || !b->a || !b->pref || !b->hist_rows || !b->hist_c ||
        !b->hist_w || !b->dsys || !b->dorder || !b->dqueue || !b->iters || !b->S || !b->flags) {
        grbk_batch_destroy(b);
        return GRBK_ENOMEM;
    }
    cudaStream_t st = b->stream;
    cudaMemsetAsync(b->A, 0, oA * 4, st);
    cudaMemsetAsync(b->B, 0, oB * 4, st);
    cudaMemsetAsync(b->C, 0, oR * 4, st);
    b->normC2.resize(nsys);
    {
        BatchLoader ld{st};
        for (int s = 0; s < nsys; ++s) {
            SysDesc& d = b->hsys[s];
            grbk_status e;
            if ((e = ld.load(&A[s], b->A + d.offA, d.lda)) != GRBK_OK ||
                (e = ld.load(&B[s], b->B + d.offB, d.ldb)) != GRBK_OK ||
                (e = ld.load(&C[s], b->C + d.offR, d.ldr)) != GRBK_OK) {
                ld.finish();
                grbk_batch_destroy(b);
                return e;
            }
        }
        const grbk_status e = ld.finish();
        if (e != GRBK_OK) { grbk_batch_destroy(b); return e; }
    }
    // per-system set-up on the device (one CTA per system)
    {
        std::vector<double> sc(kSetupScalars * (size_t)nsys);
        double* dsc = (double*)dmalloc(sizeof(double) * kSetupScalars * nsys);
        if (!dsc) { grbk_batch_destroy(b); return GRBK_ENOMEM; }
        cudaError_t e = cudaMemcpyAsync(b->dsys, b->hsys.data(), sizeof(SysDesc) * nsys, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) {
            batch_setup_kernel<<<nsys, kBB, 0, st>>>(b->dsys, b->A, b->B, b->C, b->a, b->pref, dsc);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sc.data(), dsc, sizeof(double) * kSetupScalars * nsys, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFree(dsc);
        if (e != cudaSuccess) { grbk_batch_destroy(b); return GRBK_ECUDA; }
        for (int s = 0; s < nsys; ++s) {
            SysDesc& d = b->hsys[s];
            const double* scs = sc.data() + (size_t)kSetupScalars * s;
            const double F = scs[0], c2s = scs[1], lam = scs[2];
            if (scs[3] != 0.0) { grbk_batch_destroy(b); return GRBK_ENONFINITE; }
            // banded path when both half-bandwidths are within the limit and the rows an update
            // touches (within 2 bandA of i_k) are a small part of R
            const int limit = o.band_limit == 0 ? kDefaultBandLimit : o.band_limit;
            const int bA = (int)scs[4], bB = (int)scs[5];
            const bool banded = limit > 0 && bA <= limit && bB <= limit && 4 * (long long)bA + 1 < d.m;
            d.bandA = banded ? bA : -1;
            d.bandB = banded ? bB : -1;
            if (!(F > 0.0) || !(lam > 0.0)) { grbk_batch_destroy(b); return GRBK_EINVAL; }
            d.F = F;
            b->normC2[s] = c2s;
            d.normC2 = c2s;
            const double a_in = o.alphas ? o.alphas[s] : o.alpha;
            if (o.alphas || a_in > 0.0) {
                // Lemma 2.2 / Theorems 4.2-4.8 need 0 < alpha < 2/||B||_2^2 (small slack for the estimate)
                if (!(a_in > 0.0 && a_in * lam < 2.0 * (1.0 + 1e-9))) { grbk_batch_destroy(b); return GRBK_EINVAL; }
                d.alpha = a_in;
            } else {
                d.alpha = 1.0 / lam;
            }
            d.stop_S = -1.0;
        }
    }
    // longest-processing-time order: largest R first
    b->order.resize(nsys);
    for (int s = 0; s < nsys; ++s) b->order[s] = s;
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
        return (long long)b->hsys[x].m * b->hsys[x].n > (long long)b->hsys[y].m * b->hsys[y].n;
    });
    // kernel variant of every system: the default, or the autotuner's choice
    b->variant.assign(nsys, kDefaultVariant);
    if (o.tune) {
        const grbk_status e = batch_autotune(b);
        if (e != GRBK_OK) { grbk_batch_destroy(b); return e; }
    }
    // queue order: systems grouped by variant, longest first within a group
    std::vector<int> grouped;
    for (int v = 0; v < kNumVariants; ++v) {
        b->goff[v] = (int)grouped.size();
        for (int s : b->order)
            if (b->variant[s] == v) grouped.push_back(s);
        b->gcnt[v] = (int)grouped.size() - b->goff[v];
    }
    b->order = grouped;
    if (cudaMemcpyAsync(b->dorder, b->order.data(), 4 * nsys, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        grbk_batch_destroy(b);
        return GRBK_ECUDA;
    }
    *out = b;
    return GRBK_OK;
}

extern "C" grbk_status grbk_batch_variant(const grbk_batch* b, int32_t sys, int32_t* variant, double* tune_seconds)
{
    if (!b || sys < 0 || sys >= b->nsys) return GRBK_EINVAL;
    if (variant) *variant = b->variant[sys];
    if (tune_seconds) *tune_seconds = b->tune_seconds;
    return GRBK_OK;
}

extern "C" grbk_status grbk_batch_info(const grbk_batch* b, int32_t sys, int32_t* bandA, int32_t* bandB)
{
    if (!b || sys < 0 || sys >= b->nsys) return GRBK_EINVAL;
    if (bandA) *bandA = b->hsys[sys].bandA;
    if (bandB) *bandB = b->hsys[sys].bandB;
    return GRBK_OK;
}

extern "C" grbk_status grbk_batch_solve(grbk_batch* b, int32_t variant, double theta, const grbk_mat* X0s,
                                        double tol, const double* targets, int64_t maxit, uint64_t seed,
                                        grbk_mat* X_outs, grbk_result* results)
{
    const auto t0 = std::chrono::steady_clock::now();
    if (!b) return GRBK_EINVAL;
    if (variant < GRBK_GRBK || variant > GRBK_BK) return GRBK_EINVAL;
    if (variant == GRBK_RGRBK && !(theta > 0.0 && theta <= 1.0)) return GRBK_EINVAL;
    if (maxit < 0 || !std::isfinite(tol)) return GRBK_EINVAL;
    cudaStream_t st = b->stream;
    for (int s = 0; s < b->nsys; ++s) {
        SysDesc& d = b->hsys[s];
        if (X0s && !x_desc_ok(X0s[s], d.p, d.q)) return GRBK_EINVAL;
        if (X_outs && !x_desc_ok(X_outs[s], d.p, d.q)) return GRBK_EINVAL;
        if (targets && !(std::isfinite(targets[s]) && targets[s] >= 0.0)) return GRBK_EINVAL;
        if (targets) d.stop_S = targets[s] * targets[s];
        else if (b->opts.stop_kind == GRBK_STOP_RELRES) d.stop_S = tol * tol * b->normC2[s];
        else d.stop_S = -1.0;
    }
    GRBK_CK(cudaMemcpyAsync(b->dsys, b->hsys.data(), sizeof(SysDesc) * b->nsys, cudaMemcpyHostToDevice, st));
    if (X0s) {
        BatchLoader ld{st};
        for (int s = 0; s < b->nsys; ++s) {
            const SysDesc& d = b->hsys[s];
            const grbk_status e = ld.load(&X0s[s], b->X + d.offX, d.q);
            if (e != GRBK_OK) return e;
        }
        const grbk_status e = ld.finish();
        if (e != GRBK_OK) return e;
    } else {
        GRBK_CK(cudaMemsetAsync(b->X, 0, b->totX * 4, st));
    }
    GRBK_CK(cudaMemsetAsync(b->dqueue, 0, 4 * kNumVariants, st));
    GRBK_CK(cudaMemsetAsync(b->rejected, 0, 4 * b->nsys, st));
    BatchParams P;
    memset(&P, 0, sizeof(P));
    P.nsys = b->nsys; P.sys = b->dsys; P.order = b->dorder; P.queue = b->dqueue;
    P.A = b->A; P.B = b->B; P.C = b->C; P.R = b->R; P.X = b->X; P.a = b->a; P.rbk_prefix = b->pref;
    P.hist_rows = b->hist_rows; P.hist_c = b->hist_c; P.hist_w = b->hist_w;
    P.iters = b->iters; P.S_out = b->S; P.flag_out = b->flags;
    P.variant = variant; P.theta = theta; P.seed = seed; P.maxit = maxit; P.chunk = b->chunk;
    const long long tlen = b->opts.row_trace ? b->opts.trace_len : 0;
    if (tlen > 0) {
        if (b->trace) cudaFree(b->trace);
        b->trace = (int*)dmalloc((size_t)tlen * b->nsys * 4);
        if (!b->trace) return GRBK_ENOMEM;
        GRBK_CK(cudaMemsetAsync(b->trace, 0xff, (size_t)tlen * b->nsys * 4, st));
        P.trace_rows = b->trace;
        P.trace_len = tlen;
    }
    P.init_from_x = X0s != nullptr;
    P.x0_rejected = b->rejected;
    // one launch per kernel variant in use, each over its own systems; with more
    // than one, the launches run side by side on the batch's side streams
    int ngroups = 0;
    for (int v = 0; v < kNumVariants; ++v) ngroups += b->gcnt[v] > 0;
    if (ngroups > 1 && !b->ev_fork) {
        GRBK_CK(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
        for (int v = 0; v < kNumVariants; ++v) {
            GRBK_CK(cudaStreamCreateWithFlags(&b->side[v], cudaStreamNonBlocking));
            GRBK_CK(cudaEventCreateWithFlags(&b->ev_join[v], cudaEventDisableTiming));
        }
    }
    if (ngroups > 1) GRBK_CK(cudaEventRecord(b->ev_fork, st));
    for (int v = 0; v < kNumVariants; ++v) {
        if (!b->gcnt[v]) continue;
        BatchParams Pv = P;
        Pv.nsys = b->gcnt[v];
        Pv.order = b->dorder + b->goff[v];
        Pv.queue = b->dqueue + v;
        cudaStream_t sv = st;
        if (ngroups > 1) {
            sv = b->side[v];
            GRBK_CK(cudaStreamWaitEvent(sv, b->ev_fork, 0));
        }
        int bbytes = 0;
        for (int g2 = 0; g2 < b->gcnt[v]; ++g2)
            bbytes = std::max(bbytes, band_smem_bytes(b->hsys[b->order[b->goff[v] + g2]]));
        const grbk_status e = launch_variant(v, Pv, b->gcnt[v], b->opts.grid_ctas, bbytes, sv);
        if (e != GRBK_OK) return e;
        if (ngroups > 1) {
            GRBK_CK(cudaEventRecord(b->ev_join[v], sv));
            GRBK_CK(cudaStreamWaitEvent(st, b->ev_join[v], 0));
        }
    }
    std::vector<long long> it(b->nsys);
    std::vector<double> S(b->nsys);
    std::vector<int> fl(b->nsys), rej(b->nsys);
    GRBK_CK(cudaMemcpyAsync(it.data(), b->iters, 8 * b->nsys, cudaMemcpyDeviceToHost, st));
    GRBK_CK(cudaMemcpyAsync(S.data(), b->S, 8 * b->nsys, cudaMemcpyDeviceToHost, st));
    GRBK_CK(cudaMemcpyAsync(fl.data(), b->flags, 4 * b->nsys, cudaMemcpyDeviceToHost, st));
    GRBK_CK(cudaMemcpyAsync(rej.data(), b->rejected, 4 * b->nsys, cudaMemcpyDeviceToHost, st));
    if (tlen > 0)
        GRBK_CK(cudaMemcpyAsync(b->opts.row_trace, b->trace, (size_t)tlen * b->nsys * 4, cudaMemcpyDeviceToHost, st));
    if (X_outs) {
        // host outputs go through one staging block: every system converted into it at its own
        // offset, each copied out, one wait at the end
        size_t stage_bytes = 0;
        for (int s = 0; s < b->nsys; ++s)
            if (!X_outs[s].on_device)
                stage_bytes += (size_t)b->hsys[s].p * b->hsys[s].q * (X_outs[s].dtype == GRBK_DT_F64 ? 8 : 4);
        char* stage = nullptr;
        if (stage_bytes && dev_alloc((void**)&stage, stage_bytes) != cudaSuccess) return GRBK_ENOMEM;
        size_t off = 0;
        cudaError_t e = cudaSuccess;
        for (int s = 0; s < b->nsys && e == cudaSuccess; ++s) {
            const SysDesc& d = b->hsys[s];
            grbk_mat& M = X_outs[s];
            const int es = M.dtype == GRBK_DT_F64 ? 8 : 4;
            if (M.on_device) {
                e = convert_matrix((void*)M.ptr, M.dtype, M.ld, b->X + d.offX, GRBK_DT_F32, d.q, d.p, d.q, st);
            } else {
                e = convert_matrix(stage + off, M.dtype, d.q, b->X + d.offX, GRBK_DT_F32, d.q, d.p, d.q, st);
                if (e == cudaSuccess)
                    e = cudaMemcpy2DAsync((void*)M.ptr, M.ld * es, stage + off, d.q * es, d.q * es, d.p,
                                          cudaMemcpyDeviceToHost, st);
                off += (size_t)d.p * d.q * es;
            }
        }
        const cudaError_t e2 = cudaStreamSynchronize(st);
        if (stage) dev_free(stage);
        if (e != cudaSuccess || e2 != cudaSuccess) return GRBK_ECUDA;
    }
    GRBK_CK(cudaStreamSynchronize(st));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    grbk_status overall = GRBK_OK;
    for (int s = 0; s < b->nsys; ++s) {
        const bool stopped_by_rule = fl[s] != FLAG_RUNNING;
        grbk_status ss = GRBK_OK;
        if (b->hsys[s].stop_S >= 0.0 && !stopped_by_rule) ss = GRBK_ENOTCONV;
        if (!std::isfinite(S[s])) ss = GRBK_ENONFINITE;
        if (ss != GRBK_OK && overall == GRBK_OK) overall = ss;
        if (results) {
            results[s].iters = it[s];
            results[s].relres = b->normC2[s] > 0 ? sqrt(S[s] / b->normC2[s]) : 0.0;
            results[s].rse = NAN;
            results[s].seconds = secs;
            results[s].alpha = b->hsys[s].alpha;
            results[s].x0_rejected = rej[s];
            results[s].status = ss;
        }
    }
    return overall;
}

// ============================================================================
// grbk_solve_small_noalloc: one small FP32 system, no allocation at all.
//
// Some callers cannot allocate device memory: processes whose device memory
// is handed out by a fixed pool they do not own (a framework's caching
// allocator or a service's memory budget), or latency-critical loops where a
// cudaMalloc / cudaFree (and the device-wide synchronisation cudaFree implies)
// is not acceptable.  For them this entry point runs the batch kernel above on one
// system with every working buffer (residual, row norms, recorded terms,
// queue, outputs) taken from the file-scope array below.  The array lives as
// long as the library is loaded on a device; every call shares it.
// ============================================================================
namespace grbk {

constexpr int kNoAllocSide = GRBK_NOALLOC_MAX_SIDE;
constexpr int kNoAllocChunk = 64;

struct NoAllocScratch {
    SysDesc desc;
    int order;
    int queue;
    long long iters;
    double S;
    int flag;
    int status;
    double normC2;
    double lambda;
    int hist_rows[kNoAllocChunk];
    float hist_c[kNoAllocChunk];
    double a[kNoAllocSide];
    double pref[kNoAllocSide];
    double px[kNoAllocSide];
    double pt[kNoAllocSide];
    double py[kNoAllocSide];
    float hist_w[kNoAllocChunk * kNoAllocSide];
    // the batched kernel reads these with 16-byte vector loads: keep them 16-byte aligned
    __align__(16) float R[kNoAllocSide * kNoAllocSide];   // rows padded to a multiple of 4
    __align__(16) float A[kNoAllocSide * kNoAllocSide];   // padded copy of the caller's A
    __align__(16) float B[kNoAllocSide * kNoAllocSide];   // padded copy of the caller's B
};
static_assert(sizeof(NoAllocScratch) <= GRBK_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the stated size");
static_assert(offsetof(NoAllocScratch, R) % 16 == 0 && offsetof(NoAllocScratch, A) % 16 == 0 &&
                  offsetof(NoAllocScratch, B) % 16 == 0,
              "vector-loaded arrays must be 16-byte aligned");

// The working memory of grbk_solve_small_noalloc.  In host code this name is a
// host-side stand-in, not a device address: host code only ever passes the
// address obtained from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GRBK_NOALLOC_SCRATCH_BYTES];

// Set-up for one system in one CTA: ||A_i||^2 and their running sums, ||A||_F^2,
// ||C||_F^2, ||B||_2^2 by 200 power iterations on B B^T, the step, the stop
// level, a non-finite scan.  On an error the queue is filled so that the batch
// kernel finds no work.
// caller's contiguous A, B, C -> the array's rows padded to a multiple of 4 (zeros in the padding)
__global__ void noalloc_copy_kernel(NoAllocScratch* S, const float* A, const float* B, const float* C, int m, int p,
                                    int q, int n)
{
    const int lda = (p + 3) & ~3, ldb = (n + 3) & ~3;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)m * lda;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / lda), c = (int)(e % lda);
        S->A[e] = c < p ? A[(long long)i * p + c] : 0.f;
    }
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)q * ldb;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / ldb), c = (int)(e % ldb);
        S->B[e] = c < n ? B[(long long)i * n + c] : 0.f;
    }
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)m * ldb;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / ldb), c = (int)(e % ldb);
        S->R[e] = c < n ? C[(long long)i * n + c] : 0.f;
    }
}

__global__ void __launch_bounds__(kBB) noalloc_setup_kernel(NoAllocScratch* S, const float* A, const float* B,
                                                            const float* C, int m, int p, int q, int n,
                                                            double alpha_in, double tol)
{
    __shared__ double red[2 * kBW];
    __shared__ int bad;
    const SetupOut o = system_setup(A, p, B, n, C, n, m, p, q, n, S->a, S->pref, S->px, S->pt, S->py, red, &bad);
    if (threadIdx.x == 0) {
        int status = 0;
        const double lam = o.lambda;
        if (o.bad) status = GRBK_ENONFINITE;
        else if (!(o.F > 0.0) || !(lam > 0.0)) status = GRBK_EINVAL;
        else if (alpha_in > 0.0 && !(alpha_in * lam < 2.0 * (1.0 + 1e-9))) status = GRBK_EINVAL;
        SysDesc& d = S->desc;
        d.m = m; d.p = p; d.q = q; d.n = n;
        d.lda = (p + 3) & ~3; d.ldb = (n + 3) & ~3; d.ldr = d.ldb;
        d.bandA = -1; d.bandB = -1;
        d.pad = 0;
        d.offA = 0; d.offB = 0; d.offR = 0; d.offX = 0; d.offRow = 0; d.offHist = 0; d.offHistW = 0;
        d.F = o.F;
        d.alpha = alpha_in > 0.0 ? alpha_in : 1.0 / lam;
        d.stop_S = tol > 0.0 ? tol * tol * o.normC2 : -1.0;
        d.normC2 = o.normC2;
        S->normC2 = o.normC2;
        S->lambda = lam;
        S->status = status;
        S->order = 0;
        S->iters = 0;
        S->S = 0.0;
        S->flag = FLAG_RUNNING;
        S->queue = status ? 1 : 0;   // an error leaves the batch kernel without work
    }
}

// Device address of the scratch array, looked up once per device.
static void* g_noalloc_ptr[64];
static std::mutex g_noalloc_mu;

static grbk_status noalloc_scratch_address(void** out)
{
    int dev = 0;
    GRBK_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return GRBK_EINVAL;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* ptr = nullptr;
        GRBK_CK(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
        GRBK_CK(cudaFuncSetAttribute(batch_kernel_t<kBB, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFoldSmemBytes));
        g_noalloc_ptr[dev] = ptr;
    }
    *out = g_noalloc_ptr[dev];
    return GRBK_OK;
}

}  // namespace grbk

extern "C" grbk_status grbk_solve_small_noalloc(const float* A, const float* B, const float* C, int32_t m, int32_t p,
                                                int32_t q, int32_t n, int32_t variant, double theta, double alpha,
                                                double tol, int64_t maxit, uint64_t seed, float* X_out,
                                                int64_t* iters_out, double* relres_out, void* stream)
{
    if (!A || !B || !C || !X_out) return GRBK_EINVAL;
    if (m <= 0 || p <= 0 || q <= 0 || n <= 0) return GRBK_EINVAL;
    if (m > GRBK_NOALLOC_MAX_SIDE || p > GRBK_NOALLOC_MAX_SIDE || q > GRBK_NOALLOC_MAX_SIDE ||
        n > GRBK_NOALLOC_MAX_SIDE)
        return GRBK_EINVAL;
    if (variant < GRBK_GRBK || variant > GRBK_BK) return GRBK_EINVAL;
    if (variant == GRBK_RGRBK && !(theta > 0.0 && theta <= 1.0)) return GRBK_EINVAL;
    if (maxit < 0 || !std::isfinite(alpha) || !std::isfinite(tol)) return GRBK_EINVAL;
    void* base = nullptr;
    grbk_status s = noalloc_scratch_address(&base);
    if (s != GRBK_OK) return s;
    NoAllocScratch* S = reinterpret_cast<NoAllocScratch*>(base);
    cudaStream_t st = (cudaStream_t)stream;
    GRBK_CK(cudaMemsetAsync(X_out, 0, sizeof(float) * (size_t)p * q, st));
    noalloc_copy_kernel<<<64, 256, 0, st>>>(S, A, B, C, m, p, q, n);
    noalloc_setup_kernel<<<1, kBB, 0, st>>>(S, A, B, C, m, p, q, n, alpha, tol);
    GRBK_CK(cudaGetLastError());
    BatchParams P;
    memset(&P, 0, sizeof(P));
    P.nsys = 1;
    P.sys = &S->desc;
    P.order = &S->order;
    P.queue = &S->queue;
    // R starts as the padded copy of C: C aliases R, which the kernel allows when init_from_x == 0
    P.A = S->A; P.B = S->B; P.C = S->R;
    P.R = S->R;
    P.X = X_out;
    P.a = S->a;
    P.rbk_prefix = S->pref;
    P.hist_rows = S->hist_rows;
    P.hist_c = S->hist_c;
    P.hist_w = S->hist_w;
    P.iters = &S->iters;
    P.S_out = &S->S;
    P.flag_out = &S->flag;
    P.variant = variant;
    P.theta = theta;
    P.seed = seed;
    P.maxit = maxit;
    P.chunk = kNoAllocChunk;
    P.init_from_x = 0;
    batch_kernel_t<kBB, 2><<<1, kBB, kFoldSmemBytes, st>>>(P);
    GRBK_CK(cudaGetLastError());
    struct {
        long long iters;
        double S;
        int flag;
        int status;
        double normC2;
    } h;
    GRBK_CK(cudaMemcpyAsync(&h.iters, &S->iters, sizeof(long long), cudaMemcpyDeviceToHost, st));
    GRBK_CK(cudaMemcpyAsync(&h.S, &S->S, sizeof(double), cudaMemcpyDeviceToHost, st));
    GRBK_CK(cudaMemcpyAsync(&h.flag, &S->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    GRBK_CK(cudaMemcpyAsync(&h.status, &S->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    GRBK_CK(cudaMemcpyAsync(&h.normC2, &S->normC2, sizeof(double), cudaMemcpyDeviceToHost, st));
    GRBK_CK(cudaStreamSynchronize(st));
    if (h.status != 0) return (grbk_status)h.status;
    if (iters_out) *iters_out = h.iters;
    if (relres_out) *relres_out = h.normC2 > 0.0 ? sqrt(h.S / h.normC2) : 0.0;
    if (!std::isfinite(h.S)) return GRBK_ENONFINITE;
    if (tol > 0.0 && h.flag == FLAG_RUNNING) return GRBK_ENOTCONV;
    return GRBK_OK;
}
