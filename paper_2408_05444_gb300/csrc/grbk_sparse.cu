// grbk_sparse.cu -- systems A X B = C with sparse A and B (CSR), R dense, in
// FP64: the sparse test sets of Section 5 (sprandn matrices, Tables 3, 5, 7)
// and the colour-image model of Section 6, B = A X A_c^T, where A (mn x mn) is
// the within-channel blur with a few dozen nonzeros per row and B = A_c^T is
// 3 x 3.
//
// One CTA runs one system at a time (systems taken from a longest-first
// queue); CTAs never wait on each other.  Per iteration (Algorithms 1-5):
//   * the totals S = sum_i s_i and r_max = max_i s_i / a_i come from per-block
//     summaries of 256 rows (sum of s, largest r and its row), kept up to date
//     by recomputing only the blocks whose rows changed;
//   * ME-GRBK/ME-RGRBK admit the rows with r_i >= t; only blocks whose largest
//     r reaches t are scanned for S_J and for the pick;
//   * w = R_{i_k} B^T over the rows of B (CSR), X += c A_{i_k}^T w over the
//     nonzeros of A_{i_k} only, v = w B over the columns of B (CSC);
//   * R -= c (A A_{i_k}^T) v touches only the rows k with (A A^T)_{k,i_k} != 0,
//     read from the precomputed sparse Gram matrix A A^T (the practice note
//     after Algorithm 3), and their s_k, r_k are recomputed;
//   * the least-squares extension (Eq. 2.1) first projects column j of A out of
//     an auxiliary Y, Y -= A_{:,j} (A_{:,j}^T Y) / ||A_{:,j}||^2, over the
//     nonzeros of that column (CSC of A), and moves R = C - Y - A X B with it.
// Every product and sum of w, v, u, the X and R updates, a_i and s_i is taken
// in the oracle's order with explicitly rounded operations (no fused
// multiply-add), so R, X and s follow the FP64 oracle bit for bit while the
// selected rows agree; only S and S_J are summed in another (fixed) order.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <vector>

#include <cooperative_groups.h>

#include "grbk_internal.cuh"

namespace cg = cooperative_groups;

namespace grbk {

constexpr int kSpT = 256;                 // threads per CTA
constexpr int kSpW = kSpT / 32;
constexpr int kSpBlk = 256;               // rows per summary block
constexpr int kSpRowsPerLane = kSpBlk / 32;
constexpr int kSpMaxBlocks = 1024;        // m <= 262144
constexpr int kSpMaxSide = 1024;          // q, n <= 1024 (R_{i_k}, w, v in shared memory)
constexpr int kSpMaxRowNnz = 256;         // nonzeros of one row of A staged in shared memory (more: read from L2)
constexpr long long kSpSqCap = 23552;     // doubles of dynamic shared memory for the row update's squares (184 KB)

struct SpDesc {
    int m, p, q, n;
    int nb;                    // summary blocks = ceil(m / kSpBlk)
    int pad;
    long long aRow, aNz;       // A: rowptr base (m + 1 entries), entry base
    long long bRow, bNz;       // B: CSR rowptr base (q + 1), entry base
    long long bCol;            // B: CSC colptr base (n + 1); CSC entries share bNz
    long long gRow, gNz;       // A A^T: rowptr base (m + 1), entry base
    long long aCol;            // A: CSC colptr base (p + 1); CSC entries share aNz
    long long offR, offX, offRow, offBlk, offCol;
    double F, alpha, stop_S, normC2;
    double Fc;                 // sum of the column norms ||A_{:,j}||^2 (extended method)
};

struct SpParams {
    int nsys;
    const SpDesc* sys;
    const int* order;
    int* queue;
    const long long* a_rowptr; const int* a_col; const double* a_val;
    const long long* b_rowptr; const int* b_col; const double* b_val;     // CSR of B
    const long long* bc_colptr; const int* bc_row; const double* bc_val;  // CSC of B
    const long long* g_rowptr; const int* g_col; const double* g_val;     // A A^T (CSR)
    const long long* ac_colptr; const int* ac_row; const double* ac_val;  // CSC of A
    const double* cn;          // ||A_{:,j}||^2
    const double* cpref;       // running sums of the nonzero column norms
    double* Y;                 // extended method: Y (m x n)
    int extended;
    const double* C;
    double* R;
    double* X;
    const double* a;           // ||A_i||^2
    const double* pref;        // running sums of a_i (ME-RBK)
    double* s;                 // ||R_i||^2
    double* r;                 // s_i / a_i (-inf for a zero row of A)
    long long* iters;
    double* S_out;
    int* flag_out;
    int* trace_rows;           // [nsys x trace_len] or null
    double* trace_S;           // [nsys x trace_len] or null
    long long trace_len;
    int variant;
    double theta;
    uint64_t seed;
    long long maxit;
    long long sq_cap;          // doubles of dynamic shared memory for the row update's squares
};

// ---------------------------------------------------------------------------
// set-up kernels
// ---------------------------------------------------------------------------

// exclusive scan of cnt[0..len) into out[0..len] (out[len] = total), one CTA,
// chunks of kSpT in order
__global__ void __launch_bounds__(kSpT) sp_scan_kernel(const long long* cnt, long long len, long long* out)
{
    __shared__ long long tot[kSpW + 1];
    __shared__ long long base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (long long c0 = 0; c0 < len; c0 += kSpT) {
        const long long i = c0 + threadIdx.x;
        const long long v = i < len ? cnt[i] : 0;
        long long inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) tot[warp] = inc;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long run = 0;
            for (int w = 0; w < kSpW; ++w) { const long long t = tot[w]; tot[w] = run; run += t; }
            tot[kSpW] = run;
        }
        __syncthreads();
        if (i < len) out[i] = base + tot[warp] + inc - v;
        __syncthreads();
        if (threadIdx.x == 0) base += tot[kSpW];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[len] = base;
}

// per-column entry counts of a CSR matrix (rows x cols)
// largest entry of cnt[0..len) into *out (atomic maximum; *out zeroed before)
__global__ void sp_rowmax_kernel(const long long* cnt, long long len, unsigned long long* out)
{
    unsigned long long mx = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
        mx = max(mx, (unsigned long long)cnt[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, mx);
}

__global__ void sp_colcount_kernel(const int* col, long long nnz, long long* cnt)
{
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (long long)gridDim.x * blockDim.x)
        atomicAdd((unsigned long long*)&cnt[col[e]], 1ull);
}

// scatter the CSR entries into CSC slots (order within a column fixed later)
__global__ void sp_csc_fill_kernel(const long long* rowptr, const int* col, const double* val, int rows,
                                   const long long* colptr, long long* fill, int* crow, double* cval)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x)
        for (long long e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            const int c = col[e];
            const long long pos = colptr[c] + (long long)atomicAdd((unsigned long long*)&fill[c], 1ull);
            crow[pos] = i;
            cval[pos] = val[e];
        }
}

// sort every column's entries by row (insertion sort; columns are short)
__global__ void sp_csc_sort_kernel(const long long* colptr, int cols, int* crow, double* cval)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x) {
        const long long b = colptr[c], e = colptr[c + 1];
        for (long long i = b + 1; i < e; ++i) {
            const int kr = crow[i];
            const double kv = cval[i];
            long long j = i - 1;
            while (j >= b && crow[j] > kr) { crow[j + 1] = crow[j]; cval[j + 1] = cval[j]; --j; }
            crow[j + 1] = kr;
            cval[j + 1] = kv;
        }
    }
}

// Merge of two sorted sparse rows: the first common column and the dot product
// over all common columns, summed in ascending column order with rounded
// products (as a dense dot in ascending order, whose other terms are zeros).
__device__ __forceinline__ int sp_merge_dot(const int* ca, const double* va, long long na, const int* cb,
                                            const double* vb, long long nb, double* dot)
{
    long long i = 0, j = 0;
    int first = -1;
    double acc = 0.0;
    while (i < na && j < nb) {
        const int x = ca[i], y = cb[j];
        if (x == y) {
            if (first < 0) first = x;
            acc = __dadd_rn(acc, __dmul_rn(va[i], vb[j]));
            ++i; ++j;
        } else if (x < y) {
            ++i;
        } else {
            ++j;
        }
    }
    *dot = acc;
    return first;
}

// Sparse Gram matrix G = A A^T, one warp per row i.  The candidates k are the
// rows of every column c of A_i (from the CSC of A); k is taken at the column
// c that is the first column A_i and A_k share, so each neighbour appears
// once.  fill == null: count the entries of each row; otherwise write them at
// g_rowptr[i] in (column of A_i, row of the column) order.
__global__ void __launch_bounds__(kSpT) sp_gram_kernel(const long long* rowptr, const int* col, const double* val,
                                                       int m, const long long* colptr, const int* crow,
                                                       long long* count, const long long* g_rowptr, int* g_col,
                                                       double* g_val, int fill)
{
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x / 32);
    for (int i = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); i < m; i += warps) {
        const long long ib = rowptr[i], ie = rowptr[i + 1];
        long long pos = fill ? g_rowptr[i] : 0;
        long long cnt = 0;
        for (long long e = ib; e < ie; ++e) {
            const int c = col[e];
            const long long cb = colptr[c], ce = colptr[c + 1];
            for (long long t0 = cb; t0 < ce; t0 += 32) {
                const long long t = t0 + lane;
                bool take = false;
                double dot = 0.0;
                int k = 0;
                if (t < ce) {
                    k = crow[t];
                    const int first = sp_merge_dot(col + ib, val + ib, ie - ib, col + rowptr[k], val + rowptr[k],
                                                   rowptr[k + 1] - rowptr[k], &dot);
                    take = (first == c);
                }
                const unsigned mask = __ballot_sync(0xffffffffu, take);
                if (fill && take) {
                    const long long at = pos + __popc(mask & ((1u << lane) - 1u));
                    g_col[at] = k;
                    g_val[at] = dot;
                }
                pos += __popc(mask);
                cnt += __popc(mask);
            }
        }
        if (!fill && lane == 0) count[i] = cnt;
    }
}

// One CTA per system: a_i = sum_c A_ic^2 (ascending, rounded products), their
// running sums and F, ||C||_F^2, ||B||_2^2 by 200 power iterations on B B^T
// (Rayleigh quotient; B^T x over the CSC, B t over the CSR), a non-finite flag.
constexpr int kSpSetupScalars = 5;  // F, ||C||^2, lambda, bad, sum of the column norms
__global__ void __launch_bounds__(kSpT) sp_setup_kernel(SpParams P, double* a_out, double* pref_out,
                                                        double* cn_out, double* cpref_out, double* scalars)
{
    __shared__ double x[kSpMaxSide], t[kSpMaxSide], y[kSpMaxSide];
    __shared__ double red[kSpW + 1], red2[kSpW];
    __shared__ int bad;
    const SpDesc d = P.sys[blockIdx.x];
    const long long* rp = P.a_rowptr + d.aRow;
    const int* ac = P.a_col + d.aNz;
    const double* av = P.a_val + d.aNz;
    double* a = a_out + d.offRow;
    double* pref = pref_out + d.offRow;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    int mybad = 0;
    for (int i = threadIdx.x; i < d.m; i += kSpT) {
        double acc = 0.0;
        for (long long e = rp[i]; e < rp[i + 1]; ++e) {
            const double v = av[e];
            if (!isfinite(v)) mybad = 1;
            acc = __dadd_rn(acc, __dmul_rn(v, v));
        }
        a[i] = acc;
    }
    const double* C = P.C + d.offR;
    double c2 = 0.0;
    for (long long e = threadIdx.x; e < (long long)d.m * d.n; e += kSpT) {
        const double v = C[e];
        if (!isfinite(v)) mybad = 1;
        c2 = fma(v, v, c2);
    }
    const long long* brp = P.b_rowptr + d.bRow;
    const int* bcl = P.b_col + d.bNz;
    const double* bv = P.b_val + d.bNz;
    const long long* ccp = P.bc_colptr + d.bCol;
    const int* crw = P.bc_row + d.bNz;
    const double* cvl = P.bc_val + d.bNz;
    for (long long e = threadIdx.x; e < brp[d.q]; e += kSpT)
        if (!isfinite(bv[e])) mybad = 1;
    if (mybad) atomicOr(&bad, 1);
    c2 = warp_sum(c2);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tt = 0.0;
        for (int w = 0; w < kSpW; ++w) tt += red[w];
        red[kSpW] = tt;
        double run = 0.0;
        for (int i = 0; i < d.m; ++i) {
            if (a[i] > 0.0) run = __dadd_rn(run, a[i]);
            pref[i] = run;
        }
        scalars[kSpSetupScalars * blockIdx.x + 0] = run;
        scalars[kSpSetupScalars * blockIdx.x + 1] = tt;
    }
    // ||A_{:,j}||^2 over the CSC of A (ascending rows) and their running sums
    {
        const long long* acp = P.ac_colptr + d.aCol;
        const double* acv = P.ac_val + d.aNz;
        double* cn = cn_out + d.offCol;
        for (int j = threadIdx.x; j < d.p; j += kSpT) {
            double acc = 0.0;
            for (long long e = acp[j]; e < acp[j + 1]; ++e) acc = __dadd_rn(acc, __dmul_rn(acv[e], acv[e]));
            cn[j] = acc;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double run = 0.0;
            for (int j = 0; j < d.p; ++j) {
                if (cn[j] > 0.0) run = __dadd_rn(run, cn[j]);
                cpref_out[d.offCol + j] = run;
            }
            scalars[kSpSetupScalars * blockIdx.x + 4] = run;
        }
    }
    for (int j = threadIdx.x; j < d.q; j += kSpT) x[j] = 1.0 / sqrt((double)d.q);
    __syncthreads();
    double lam = 0.0;
    for (int it = 0; it < 200; ++it) {
        for (int l = threadIdx.x; l < d.n; l += kSpT) {      // t = B^T x
            double acc = 0.0;
            for (long long e = ccp[l]; e < ccp[l + 1]; ++e) acc = fma(cvl[e], x[crw[e]], acc);
            t[l] = acc;
        }
        __syncthreads();
        double xy = 0.0, yy = 0.0;
        for (int j = threadIdx.x; j < d.q; j += kSpT) {      // y = B t
            double acc = 0.0;
            for (long long e = brp[j]; e < brp[j + 1]; ++e) acc = fma(bv[e], t[bcl[e]], acc);
            y[j] = acc;
            xy = fma(x[j], acc, xy);
            yy = fma(acc, acc, yy);
        }
        xy = warp_sum(xy);
        yy = warp_sum(yy);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5] = xy; red2[threadIdx.x >> 5] = yy; }
        __syncthreads();
        double sxy = 0.0, syy = 0.0;
        for (int w = 0; w < kSpW; ++w) { sxy += red[w]; syy += red2[w]; }
        lam = sxy;
        const double nrm = sqrt(syy);
        __syncthreads();
        for (int j = threadIdx.x; j < d.q; j += kSpT) x[j] = nrm > 0.0 ? y[j] / nrm : 0.0;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        scalars[kSpSetupScalars * blockIdx.x + 2] = lam;
        scalars[kSpSetupScalars * blockIdx.x + 3] = (double)bad;
    }
}

// ---------------------------------------------------------------------------
// the iteration
// ---------------------------------------------------------------------------

// floor(s 2^(62 - E)) for 0 <= s <= S < 2^E, where ebS is S's biased exponent
// (E = ebS - 1022): s = mant 2^(e - 1075) scaled by 2^(1084 - ebS), a shift of
// e - ebS + 9 <= 9 places, so the result and any sum of results stay below 2^62.
__device__ __forceinline__ unsigned long long sp_fix(double s, int ebS)
{
    const long long b = __double_as_longlong(s);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e == 0) return 0ull;   // zero (a subnormal is below every admitted row's share)
    const unsigned long long mant = (unsigned long long)(b & 0xfffffffffffffLL) | (1ull << 52);
    const int sh = e - ebS + 9;
    if (sh >= 0) return mant << sh;
    return sh > -64 ? (mant >> (-sh)) : 0ull;
}

// summary of block b: sum of s over its rows (lane partials in row order, then
// a fixed tree), largest r key and the smallest row attaining it; one warp.
// The summaries live in the shared memory of the CTA that runs the system.
// Cluster form (CL) or one CTA per system: loads of rows other CTAs of the cluster
// write go through L2 (ld.global.cg) and the CTA barriers are cluster barriers; the
// one-CTA form keeps cached loads and block barriers.
template <bool CL>
__device__ __forceinline__ double ldx(const double* p)
{
    if constexpr (CL) return __ldcg(p);
    else return *p;
}
template <bool CL>
__device__ __forceinline__ void csync(cg::cluster_group& cl)
{
    if constexpr (CL) cl.sync();
    else __syncthreads();
}
template <bool CL, class T>
__device__ __forceinline__ T rank_read(cg::cluster_group& cl, T* p, int rank)
{
    if constexpr (CL) return *cl.map_shared_rank(p, rank);
    else return *p;
}

template <bool CL>
__device__ __forceinline__ void sp_block_summary(const SpParams& P, const SpDesc& d, int b, double* bsum,
                                                 long long* bkey, int* barg)
{
    const int lane = threadIdx.x & 31;
    const double* s = P.s + d.offRow;
    const double* r = P.r + d.offRow;
    const int r0 = b * kSpBlk + lane * kSpRowsPerLane;
    double sum = 0.0;
    long long key = LLONG_MIN;
    int arg = INT_MAX;
#pragma unroll
    for (int k = 0; k < kSpRowsPerLane; ++k) {
        const int i = r0 + k;
        if (i < d.m) {
            sum += ldx<CL>(s + i);
            const long long kk = __double_as_longlong(ldx<CL>(r + i));
            if (kk > key) { key = kk; arg = i; }
        }
    }
    sum = warp_sum(sum);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long ok = __shfl_xor_sync(0xffffffffu, key, o);
        const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
        if (ok > key || (ok == key && oa < arg)) { key = ok; arg = oa; }
    }
    if (lane == 0) {
        bsum[b] = sum;
        bkey[b] = key;
        barg[b] = arg;
    }
}

// R^0 = C, s_i, r_i and every block summary of one system (one CTA per system)
__global__ void __launch_bounds__(kSpT) sp_init_kernel(SpParams P)
{
    const SpDesc d = P.sys[blockIdx.x];
    const double* C = P.C + d.offR;
    double* R = P.R + d.offR;
    if (P.extended) {   // Y^0 = C, R^0 = C - Y^0 (X^0 = 0)
        double* Y = P.Y + d.offR;
        for (long long e = threadIdx.x; e < (long long)d.m * d.n; e += kSpT) {
            Y[e] = C[e];
            R[e] = __dsub_rn(C[e], C[e]);
        }
    } else {
        for (long long e = threadIdx.x; e < (long long)d.m * d.n; e += kSpT) R[e] = C[e];
    }
    double* X = P.X + d.offX;
    for (long long e = threadIdx.x; e < (long long)d.p * d.q; e += kSpT) X[e] = 0.0;
    __syncthreads();
    const double* a = P.a + d.offRow;
    for (int i = threadIdx.x; i < d.m; i += kSpT) {
        double acc = 0.0;
        for (int l = 0; l < d.n; ++l) {
            const double v = R[(long long)i * d.n + l];
            acc = __dadd_rn(acc, __dmul_rn(v, v));
        }
        P.s[d.offRow + i] = acc;
        P.r[d.offRow + i] = a[i] > 0.0 ? __ddiv_rn(acc, a[i]) : -INFINITY;
    }
}

template <bool CL>
__global__ void __launch_bounds__(kSpT, 2) sp_solve_kernel(SpParams P)
{
    extern __shared__ double sp_sq[];        // squares of the updated rows (row update) / the select's block sums
    __shared__ double s_row[kSpMaxSide];      // R_{i_k}, then v
    __shared__ double s_w[kSpMaxSide];        // w; the extended method's z / ||A_{:,j}||^2
    __shared__ double s_bsum[kSpMaxBlocks];   // per block of 256 rows: sum of s,
    __shared__ long long s_bkey[kSpMaxBlocks];//   its largest r (IEEE bits)
    __shared__ int s_barg[kSpMaxBlocks];      //   and the smallest row attaining it
    __shared__ int s_anz_c[kSpMaxRowNnz];     // nonzeros of A_{i_k}
    __shared__ double s_anz_v[kSpMaxRowNnz];
    __shared__ unsigned s_dirty[kSpMaxBlocks / 32];
    __shared__ double red[kSpW + 1];
    __shared__ double s_wbase[kSpW];          // exclusive bases of the warps' admitted sums
    __shared__ int s_sys, s_stop, s_pick, s_last_adm, s_col;
    __shared__ double s_S, s_t, s_u, s_ck;
    __shared__ int s_imax;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // A cluster of CS CTAs (one per SM) runs one system: every CTA forms the totals, the
    // pick, R_{i_k}, w and v itself; CTA `crank` scans the blocks b = crank mod CS, updates
    // the X rows of A_{i_k}'s nonzeros e = crank mod CS and the rows of Gram row i_k at
    // positions t = crank mod CS.  Rows written by one CTA and read by another go through
    // L2 (ld.global.cg) after a cluster barrier.  CS = 1 is the plain one-CTA solver.
    cg::cluster_group cl = cg::this_cluster();
    const int crank = (int)cl.block_rank(), CS = (int)cl.num_blocks();
    for (;;) {
        csync<CL>(cl);
        if (crank == 0 && threadIdx.x == 0) {
            const int slot = atomicAdd(P.queue, 1);
            s_sys = slot < P.nsys ? P.order[slot] : -1;
        }
        csync<CL>(cl);
        const int sid = rank_read<CL>(cl, &s_sys, 0);
        if (sid < 0) {
            csync<CL>(cl);   // no CTA leaves while another may still read its shared memory
            return;
        }
        const SpDesc d = P.sys[sid];
        double* R = P.R + d.offR;
        double* X = P.X + d.offX;
        const double* a = P.a + d.offRow;
        double* s = P.s + d.offRow;
        double* r = P.r + d.offRow;
        const long long* arp = P.a_rowptr + d.aRow;
        const int* acol = P.a_col + d.aNz;
        const double* aval = P.a_val + d.aNz;
        const long long* brp = P.b_rowptr + d.bRow;
        const int* bcol = P.b_col + d.bNz;
        const double* bval = P.b_val + d.bNz;
        const long long* ccp = P.bc_colptr + d.bCol;
        const int* crow = P.bc_row + d.bNz;
        const double* cval = P.bc_val + d.bNz;
        const long long* grp = P.g_rowptr + d.gRow;
        const int* gcol = P.g_col + d.gNz;
        const double* gval = P.g_val + d.gNz;
        for (int b = threadIdx.x; b < kSpMaxBlocks / 32; b += kSpT) s_dirty[b] = 0u;
        for (int b = warp; b < d.nb; b += kSpW) sp_block_summary<CL>(P, d, b, s_bsum, s_bkey, s_barg);
        __syncthreads();

        long long k = 0;
        int flag = FLAG_RUNNING;
        for (;;) {
            // ---- extended method: project column j of A out of Y; R = C - Y - A X B follows
            if (P.extended && k < P.maxit) {
                if (threadIdx.x == 0) {
                    const double* cpref = P.cpref + d.offCol;
                    const double* cn = P.cn + d.offCol;
                    const double target = __dmul_rn(philox_uniform(P.seed, (uint64_t)k, (uint64_t)sid, 1), d.Fc);
                    int lo = 0, hi = d.p;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (cpref[mid] > target) hi = mid; else lo = mid + 1;
                    }
                    if (lo >= d.p) {
                        lo = d.p - 1;
                        while (lo > 0 && !(cn[lo] > 0.0)) --lo;
                    }
                    s_col = lo;
                }
                __syncthreads();
                const int j = s_col;
                const long long cb = P.ac_colptr[d.aCol + j], ce = P.ac_colptr[d.aCol + j + 1];
                const int* crw = P.ac_row + d.aNz;
                const double* cvl = P.ac_val + d.aNz;
                double* Y = P.Y + d.offR;
                const double cnj = P.cn[d.offCol + j];
                for (int l = threadIdx.x; l < d.n; l += kSpT) {
                    double acc = 0.0;
                    for (long long e = cb; e < ce; ++e)
                        acc = __dadd_rn(acc, __dmul_rn(cvl[e], ldx<CL>(Y + (long long)crw[e] * d.n + l)));
                    s_w[l] = __ddiv_rn(acc, cnj);
                }
                csync<CL>(cl);   // every CTA has z before any CTA updates Y
                for (long long e = cb + (long long)crank * kSpT + threadIdx.x; e < ce; e += (long long)CS * kSpT) {
                    const int i = crw[e];
                    const double av = cvl[e];
                    double* Yi = Y + (long long)i * d.n;
                    double* Ri = R + (long long)i * d.n;
                    double acc = 0.0;
                    for (int l = 0; l < d.n; ++l) {
                        const double gl = __dmul_rn(av, s_w[l]);
                        Yi[l] = __dsub_rn(ldx<CL>(Yi + l), gl);
                        const double v = __dadd_rn(ldx<CL>(Ri + l), gl);
                        Ri[l] = v;
                        acc = __dadd_rn(acc, __dmul_rn(v, v));
                    }
                    s[i] = acc;
                    r[i] = a[i] > 0.0 ? __ddiv_rn(acc, a[i]) : -INFINITY;
                }
                for (long long e = cb + threadIdx.x; e < ce; e += kSpT) {   // every CTA marks every row
                    const int b = crw[e] / kSpBlk;
                    atomicOr(&s_dirty[b >> 5], 1u << (b & 31));
                }
                csync<CL>(cl);
                {
                    const int nw = (d.nb + 31) / 32;
                    for (int wi = 0; wi < nw; ++wi) {
                        unsigned bits = s_dirty[wi];
                        int idx = 0;
                        while (bits) {
                            const int bit = __ffs(bits) - 1;
                            bits &= bits - 1;
                            if (idx % kSpW == warp) sp_block_summary<CL>(P, d, wi * 32 + bit, s_bsum, s_bkey, s_barg);
                            ++idx;
                        }
                    }
                }
                __syncthreads();
                for (int b = threadIdx.x; b < (d.nb + 31) / 32; b += kSpT) s_dirty[b] = 0u;
            }
            // ---- totals from the block summaries (one warp, fixed order), threshold and stop test;
            // the draw on a second warp beside it
            const int var = P.variant;
            if (warp == 0) {
                double Sv = 0.0;
                long long key = LLONG_MIN;
                int arg = INT_MAX;
                for (int b = lane; b < d.nb; b += 32) {
                    Sv += s_bsum[b];
                    const long long kk = s_bkey[b];
                    const int aa = s_barg[b];
                    if (kk > key || (kk == key && aa < arg)) { key = kk; arg = aa; }
                }
                Sv = warp_sum(Sv);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const long long ok = __shfl_xor_sync(0xffffffffu, key, o);
                    const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
                    if (ok > key || (ok == key && oa < arg)) { key = ok; arg = oa; }
                }
                if (lane == 0) {
                    const double S = Sv;
                    const double rmax = __longlong_as_double(key);
                    s_S = S;
                    s_imax = arg;
                    int stop = 0;
                    if (!(S > 0.0) && !P.extended) stop = 2;   // the extension's R^0 = 0 while Y moves
                    else if (d.stop_S >= 0.0 && S <= d.stop_S) stop = 1;
                    else if (k >= P.maxit) stop = 4;
                    s_stop = stop;
                    if (!stop && k < P.trace_len && crank == 0) {
                        if (P.trace_S) P.trace_S[(long long)sid * P.trace_len + k] = S;
                    }
                    s_pick = INT_MAX;
                    s_last_adm = -1;
                    if (!stop && (var == GRBK_GRBK || var == GRBK_RGRBK)) {
                        const double theta = (var == GRBK_GRBK) ? 0.5 : P.theta;
                        double t = __dadd_rn(__dmul_rn(theta, rmax), __dmul_rn(1.0 - theta, __ddiv_rn(S, d.F)));
                        if (t > rmax) t = rmax;
                        s_t = t;
                    }
                }
            } else if (warp == 1 && lane == 0 && (var == GRBK_GRBK || var == GRBK_RGRBK || var == GRBK_RBK)) {
                s_u = philox_uniform(P.seed, (uint64_t)k, (uint64_t)sid);
            }
            __syncthreads();
            if (s_stop) {
                if (s_stop == 1) flag = FLAG_TOL_MET;
                if (s_stop == 2) flag = FLAG_EXACT;
                break;
            }

            // ---- select i_k
            if (var == GRBK_GRBK || var == GRBK_RGRBK) {
                // Admission compares bit patterns (r_i and t are >= 0 or -inf).  The admitted sums
                // are exact 64-bit fixed-point sums on the integer pipe (sp_fix: s_i truncated to
                // a multiple of 2^(E-62), S < 2^E), so their order does not matter; they differ
                // from the oracle's sequential FP64 sums only by that sum's own rounding.
                const long long tkey = __double_as_longlong(s_t);
                const int ebS = (int)((__double_as_longlong(s_S) >> 52) & 0x7ff);
                // Warps take the 256-row summary blocks round robin; a block whose largest r is
                // below t counts 0 without loads, the others are read in 8 chunks of 32 rows (lane =
                // row: coalesced loads, all 16 in flight), each lane adds its rows' fixed-point
                // shares and one warp reduction gives the block's admitted sum (bs[b], shared
                // memory).  Warp 0 then scans the block sums for the block where the prefix first
                // exceeds floor(u S_J) and scans that block's rows for the row.
                unsigned long long* bs = reinterpret_cast<unsigned long long*>(sp_sq);
                int lastadm = -1;
                for (int bb = crank + CS * warp; bb < d.nb; bb += CS * kSpW) {
                    unsigned long long f = 0;
                    if (s_bkey[bb] >= tkey) {
                        double rv[8], sv[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const int i = bb * kSpBlk + 32 * u + lane;
                            rv[u] = (i < d.m) ? ldx<CL>(r + i) : -INFINITY;
                            sv[u] = (i < d.m) ? ldx<CL>(s + i) : 0.0;
                        }
#pragma unroll
                        for (int u = 0; u < 8; ++u)
                            if (__double_as_longlong(rv[u]) >= tkey) {
                                f += sp_fix(sv[u], ebS);
                                lastadm = max(lastadm, bb * kSpBlk + 32 * u + lane);
                            }
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
                    }
                    if (lane == 0) bs[bb] = f;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) lastadm = max(lastadm, __shfl_xor_sync(0xffffffffu, lastadm, o));
                if (lane == 0 && lastadm >= 0) atomicMax(&s_last_adm, lastadm);   // this CTA's last admitted row
                csync<CL>(cl);   // every CTA's block sums are in its shared memory
                if (warp == 0) {
                    // lanes take runs of `per` block sums; one scan gives S_J and the crossing run
                    const int per = (d.nb + 31) / 32;
                    unsigned long long ls = 0;
                    for (int j = 0; j < per; ++j) {
                        const int bb = lane * per + j;
                        if (bb < d.nb) ls += rank_read<CL>(cl, bs + bb, bb % CS);
                    }
                    unsigned long long inc = ls;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const unsigned long long t2 = __shfl_up_sync(0xffffffffu, inc, o);
                        if (lane >= o) inc += t2;
                    }
                    const unsigned long long SJ = __shfl_sync(0xffffffffu, inc, 31);
                    // floor(u S_J) in the same fixed point: u = U 2^-53 exactly (the draw's 53 bits)
                    const unsigned long long U = (unsigned long long)__dmul_rn(s_u, 9007199254740992.0);
                    const unsigned long long target = __umul64hi(U << 11, SJ);
                    const unsigned hl = __ballot_sync(0xffffffffu, ls > 0 && inc > target);
                    int pick = -1;
                    if (hl) {
                        const int L = __ffs(hl) - 1;
                        unsigned long long run = __shfl_sync(0xffffffffu, inc - ls, L);
                        int bstar = -1;
                        for (int j = 0; j < per && bstar < 0; ++j) {   // lane L's blocks, every lane follows
                            const int bb = L * per + j;
                            if (bb >= d.nb) break;
                            const unsigned long long v = rank_read<CL>(cl, bs + bb, bb % CS);
                            if (v > 0 && run + v > target) bstar = bb;
                            else run += v;
                        }
                        if (bstar >= 0) {
                            double rv[8], sv[8];
#pragma unroll
                            for (int u = 0; u < 8; ++u) {
                                const int i = bstar * kSpBlk + 32 * u + lane;
                                rv[u] = (i < d.m) ? ldx<CL>(r + i) : -INFINITY;
                                sv[u] = (i < d.m) ? ldx<CL>(s + i) : 0.0;
                            }
#pragma unroll
                            for (int u = 0; u < 8; ++u) {
                                if (pick >= 0) break;
                                const bool adm = __double_as_longlong(rv[u]) >= tkey;
                                unsigned long long ic = adm ? sp_fix(sv[u], ebS) : 0ull;
#pragma unroll
                                for (int o = 1; o < 32; o <<= 1) {
                                    const unsigned long long t2 = __shfl_up_sync(0xffffffffu, ic, o);
                                    if (lane >= o) ic += t2;
                                }
                                const unsigned h2 = __ballot_sync(0xffffffffu, adm && run + ic > target);
                                if (h2) pick = bstar * kSpBlk + 32 * u + __ffs(h2) - 1;
                                run += __shfl_sync(0xffffffffu, ic, 31);
                            }
                        }
                    }
                    if (pick < 0) {   // no admitted mass (every s_i below 2^(E-62)): the last admitted row
                        int gl = lane < CS ? rank_read<CL>(cl, &s_last_adm, lane) : -1;
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) gl = max(gl, __shfl_xor_sync(0xffffffffu, gl, o));
                        pick = gl >= 0 ? gl : s_imax;
                    }
                    if (lane == 0) s_pick = pick;
                }
                __syncthreads();
            } else if (var == GRBK_MWRBK) {
                if (threadIdx.x == 0) s_pick = s_imax;
            } else if (var == GRBK_RBK) {
                if (threadIdx.x == 0) {
                    const double* pref = P.pref + d.offRow;
                    const double target = __dmul_rn(s_u, d.F);
                    int lo = 0, hi = d.m;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (pref[mid] > target) hi = mid; else lo = mid + 1;
                    }
                    if (lo >= d.m) {
                        lo = d.m - 1;
                        while (lo > 0 && !(a[lo] > 0.0)) --lo;
                    }
                    s_pick = lo;
                }
            } else {
                if (threadIdx.x == 0) s_pick = (int)(k % d.m);
            }
            __syncthreads();
            const int ik = s_pick;
            if (crank == 0 && threadIdx.x == 0 && k < P.trace_len && P.trace_rows)
                P.trace_rows[(long long)sid * P.trace_len + k] = ik;
            const double aik = a[ik];
            if (!(__double_as_longlong(aik) > 0)) {   // zero row of A (ME-BK only): the step changes nothing
                ++k;
                continue;
            }

            // ---- R_{i_k} and A_{i_k} to shared memory
            const long long ab = arp[ik], ae = arp[ik + 1];
            const int anz = (int)min(ae - ab, (long long)kSpMaxRowNnz);
            for (int l = threadIdx.x; l < d.n; l += kSpT) s_row[l] = ldx<CL>(R + (long long)ik * d.n + l);
            if (threadIdx.x == 0) s_ck = __ddiv_rn(d.alpha, aik);   // c_k, once
            __syncthreads();
            const double ck = s_ck;
            // A_{i_k}'s nonzeros, scaled by c_k once (c_k a_c: the X update's coefficients)
            for (int e = threadIdx.x; e < anz; e += kSpT) {
                s_anz_c[e] = acol[ab + e];
                s_anz_v[e] = __dmul_rn(ck, aval[ab + e]);
            }
            __syncthreads();
            // ---- w = R_{i_k} B^T over the rows of B, in ascending column order
            for (int j = threadIdx.x; j < d.q; j += kSpT) {
                double acc = 0.0;
                for (long long e = brp[j]; e < brp[j + 1]; ++e)
                    acc = __dadd_rn(acc, __dmul_rn(s_row[bcol[e]], bval[e]));
                s_w[j] = acc;
            }
            csync<CL>(cl);   // every CTA has R_{i_k} (and is done with the block sums) before rows change
            // ---- X += (c A_{i_k}^T) w over the nonzeros of A_{i_k}; v = w B over the columns of B
            {
                const int anz_all = (int)(ae - ab);
                if (d.q >= 32) {
                    // one warp per nonzero c of A_{i_k}: row c of X, lanes over its columns, 8
                    // columns per lane loaded together before their updates
                    for (int e = crank + CS * warp; e < anz_all; e += CS * kSpW) {
                        const int c = e < kSpMaxRowNnz ? s_anz_c[e] : acol[ab + e];
                        const double cav = e < kSpMaxRowNnz ? s_anz_v[e] : __dmul_rn(ck, aval[ab + e]);
                        double* Xc = X + (long long)c * d.q;
                        for (int j0 = lane; j0 < d.q; j0 += 256) {
                            double xv[8];
#pragma unroll
                            for (int u = 0; u < 8; ++u)
                                if (j0 + 32 * u < d.q) xv[u] = ldx<CL>(Xc + j0 + 32 * u);
#pragma unroll
                            for (int u = 0; u < 8; ++u) {
                                const int j = j0 + 32 * u;
                                if (j < d.q) Xc[j] = __fma_rn(cav, s_w[j], xv[u]);
                            }
                        }
                    }
                } else {
                    // few columns (the colour model's q = 3): one thread per element
                    const long long nx = (long long)anz_all * d.q;
                    for (long long t2 = (long long)crank * kSpT + threadIdx.x; t2 < nx; t2 += (long long)CS * kSpT) {
                        const int e = (int)(t2 / d.q), j = (int)(t2 % d.q);
                        const int c = e < kSpMaxRowNnz ? s_anz_c[e] : acol[ab + e];
                        const double cav = e < kSpMaxRowNnz ? s_anz_v[e] : __dmul_rn(ck, aval[ab + e]);
                        double* xp = X + (long long)c * d.q + j;
                        *xp = __fma_rn(cav, s_w[j], ldx<CL>(xp));
                    }
                }
            }
            for (int l = threadIdx.x; l < d.n; l += kSpT) {
                double acc = 0.0;
                for (long long e = ccp[l]; e < ccp[l + 1]; ++e) acc = __dadd_rn(acc, __dmul_rn(s_w[crow[e]], cval[e]));
                s_row[l] = acc;   // v_l (R_{i_k} is no longer needed)
            }
            __syncthreads();
            // ---- R_k -= (c g_k) v for the rows k sharing a column with A_{i_k}; new s_k, r_k.
            // w, v, R and the row norms are formed with the oracle's rounded operations in its
            // order (one thread per row, ascending columns): rows whose r are equal in exact
            // arithmetic (a row of A with one nonzero makes several) then tie exactly as in the
            // oracle, which keeps ME-MWRBK's argmax and the threshold tests identical.
            const long long gb = grp[ik], ge = grp[ik + 1];
            const int nrow = (int)(ge - gb);
            if (d.n >= 8 && (long long)nrow * d.n <= P.sq_cap) {
                // the same operations in two phases: (1) every element, one warp per row and
                // lanes over columns: v = R - (c g) v_l and its square, rounded as above; (2) one
                // thread per row adds its squares in ascending column order.  Phase 1 keeps the
                // FP64 unit busy with full warps; phase 2 is the oracle's chain of additions.
                for (int t = crank + CS * warp; t < nrow; t += CS * kSpW) {
                    const int kr = gcol[gb + t];
                    const double cg = __dmul_rn(ck, gval[gb + t]);
                    double* Rk = R + (long long)kr * d.n;
                    double* q = sp_sq + (long long)(t / CS) * d.n;
                    // 8 columns per lane at a time: their loads are issued before the first store
                    for (int l0 = lane; l0 < d.n; l0 += 256) {
                        double rv[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u)
                            if (l0 + 32 * u < d.n) rv[u] = ldx<CL>(Rk + l0 + 32 * u);
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const int l = l0 + 32 * u;
                            if (l < d.n) {
                                const double v = __dsub_rn(rv[u], __dmul_rn(cg, s_row[l]));
                                Rk[l] = v;
                                q[l] = __dmul_rn(v, v);
                            }
                        }
                    }
                }
                __syncthreads();
                for (int t = crank + CS * threadIdx.x; t < nrow; t += CS * kSpT) {
                    const int kr = gcol[gb + t];
                    const double* q = sp_sq + (long long)(t / CS) * d.n;
                    double acc = 0.0;
                    for (int l = 0; l < d.n; ++l) acc = __dadd_rn(acc, q[l]);
                    s[kr] = acc;
                    r[kr] = a[kr] > 0.0 ? __ddiv_rn(acc, a[kr]) : -INFINITY;
                }
            } else {
                for (long long e = gb + crank + (long long)CS * threadIdx.x; e < ge; e += (long long)CS * kSpT) {
                    const int kr = gcol[e];
                    const double cg = __dmul_rn(ck, gval[e]);
                    double* Rk = R + (long long)kr * d.n;
                    double acc = 0.0;
                    for (int l = 0; l < d.n; ++l) {
                        const double v = __dsub_rn(ldx<CL>(Rk + l), __dmul_rn(cg, s_row[l]));
                        Rk[l] = v;
                        acc = __dadd_rn(acc, __dmul_rn(v, v));
                    }
                    s[kr] = acc;
                    r[kr] = a[kr] > 0.0 ? __ddiv_rn(acc, a[kr]) : -INFINITY;
                }
            }
            for (long long e = gb + threadIdx.x; e < ge; e += kSpT) {   // every CTA marks every updated row
                const int b = gcol[e] / kSpBlk;
                atomicOr(&s_dirty[b >> 5], 1u << (b & 31));
            }
            csync<CL>(cl);   // every CTA's rows, s and r written before the summaries are refreshed
            // ---- refresh the summaries of the blocks that changed
            {
                const int nw = (d.nb + 31) / 32;
                for (int wi = 0; wi < nw; ++wi) {
                    unsigned bits = s_dirty[wi];
                    int idx = 0;
                    while (bits) {
                        const int bit = __ffs(bits) - 1;
                        bits &= bits - 1;
                        if (idx % kSpW == warp) sp_block_summary<CL>(P, d, wi * 32 + bit, s_bsum, s_bkey, s_barg);
                        ++idx;
                    }
                }
            }
            __syncthreads();
            for (int b = threadIdx.x; b < (d.nb + 31) / 32; b += kSpT) s_dirty[b] = 0u;
            ++k;
        }
        if (crank == 0 && threadIdx.x == 0) {
            P.iters[sid] = k;
            P.S_out[sid] = s_S;
            P.flag_out[sid] = flag;
        }
    }
}

}  // namespace grbk

// ============================================================================
// host side
// ============================================================================
using namespace grbk;

struct grbk_sparse {
    int nsys;
    grbk_opts opts;
    cudaStream_t stream;
    std::vector<SpDesc> hsys;
    std::vector<int> order;
    std::vector<long long> gnnz;
    std::vector<long long> growmax;    // largest row of A A^T per system
    int last_cluster = 1;               // CTAs per system of the last solve
    SpDesc* dsys = nullptr;
    int* dorder = nullptr;
    int* dqueue = nullptr;
    long long *a_rowptr = nullptr, *b_rowptr = nullptr, *bc_colptr = nullptr, *g_rowptr = nullptr;
    int *a_col = nullptr, *b_col = nullptr, *bc_row = nullptr, *g_col = nullptr;
    double *a_val = nullptr, *b_val = nullptr, *bc_val = nullptr, *g_val = nullptr;
    long long* ac_colptr = nullptr;
    int* ac_row = nullptr;
    double *ac_val = nullptr, *cn = nullptr, *cpref = nullptr, *Y = nullptr;
    double *C = nullptr, *R = nullptr, *X = nullptr, *a = nullptr, *pref = nullptr, *s = nullptr, *r = nullptr;
    long long* iters = nullptr;
    double* S = nullptr;
    int* flags = nullptr;
    int* trace = nullptr;
    double* traceS = nullptr;
    long long totR = 0, totX = 0;
};

extern "C" void grbk_sparse_destroy(grbk_sparse* b)
{
    if (!b) return;
    void* bufs[] = {b->dsys, b->dorder, b->dqueue, b->a_rowptr, b->b_rowptr, b->bc_colptr, b->g_rowptr,
                    b->a_col, b->b_col, b->bc_row, b->g_col, b->a_val, b->b_val, b->bc_val, b->g_val, b->C,
                    b->R, b->X, b->a, b->pref, b->s, b->r, b->iters, b->S,
                    b->flags, b->trace, b->traceS, b->ac_colptr, b->ac_row, b->ac_val, b->cn, b->cpref, b->Y};
    for (void* p : bufs)
        if (p) cudaFree(p);
    delete b;
}

template <typename T>
static bool sp_alloc(T** p, size_t count)
{
    return cudaMalloc((void**)p, sizeof(T) * (count > 0 ? count : 1)) == cudaSuccess;
}

// the structure of a caller CSR matrix: offsets from 0 to nnz, columns in range and strictly ascending per row
static bool csr_ok(const grbk_csr& M, int64_t max_rows, int64_t max_cols)
{
    if (M.rows <= 0 || M.cols <= 0 || M.rows > max_rows || M.cols > max_cols || M.nnz < 0) return false;
    if (!M.rowptr || (M.nnz > 0 && (!M.colind || !M.val))) return false;
    if (M.rowptr[0] != 0 || M.rowptr[M.rows] != M.nnz) return false;
    for (int64_t i = 0; i < M.rows; ++i) {
        if (M.rowptr[i + 1] < M.rowptr[i]) return false;
        for (int64_t e = M.rowptr[i]; e < M.rowptr[i + 1]; ++e) {
            const int32_t c = M.colind[e];
            if (c < 0 || c >= M.cols) return false;
            if (e > M.rowptr[i] && c <= M.colind[e - 1]) return false;
        }
    }
    return true;
}

extern "C" grbk_status grbk_sparse_create(grbk_sparse** out, int32_t nsys, const grbk_csr* A, const grbk_csr* B,
                                          const grbk_mat* C, const grbk_opts* opts)
{
    if (!out || nsys <= 0 || !A || !B || !C) return GRBK_EINVAL;
    *out = nullptr;
    grbk_opts o;
    if (opts) o = *opts; else grbk_default_opts(&o);
    if (!std::isfinite(o.alpha)) return GRBK_EINVAL;
    for (int s = 0; s < nsys; ++s) {
        if (!csr_ok(A[s], (int64_t)kSpMaxBlocks * kSpBlk, INT_MAX) || !csr_ok(B[s], kSpMaxSide, kSpMaxSide))
            return GRBK_EINVAL;
        if (!C[s].ptr || C[s].rows != A[s].rows || C[s].cols != B[s].cols || C[s].ld < C[s].cols) return GRBK_EINVAL;
        if (C[s].dtype != GRBK_DT_F64 && C[s].dtype != GRBK_DT_F32) return GRBK_EINVAL;
        if (o.alphas && !(std::isfinite(o.alphas[s]) && o.alphas[s] > 0.0)) return GRBK_EINVAL;
    }
    grbk_sparse* b = new grbk_sparse();
    b->nsys = nsys;
    b->opts = o;
    b->stream = (cudaStream_t)o.stream;
    b->hsys.resize(nsys);
    long long oAR = 0, oAN = 0, oBR = 0, oBN = 0, oBC = 0, oGR = 0, oR = 0, oX = 0, oRow = 0, oBlk = 0, oAC = 0;
    long long oCol = 0;
    for (int s = 0; s < nsys; ++s) {
        SpDesc& d = b->hsys[s];
        memset(&d, 0, sizeof(d));
        d.m = (int)A[s].rows; d.p = (int)A[s].cols; d.q = (int)B[s].rows; d.n = (int)B[s].cols;
        d.nb = (d.m + kSpBlk - 1) / kSpBlk;
        d.aRow = oAR; d.aNz = oAN; d.bRow = oBR; d.bNz = oBN; d.bCol = oBC; d.gRow = oGR;
        d.offR = oR; d.offX = oX; d.offRow = oRow; d.offBlk = oBlk; d.aCol = oAC; d.offCol = oCol;
        oAC += d.p + 1; oCol += d.p;
        oAR += d.m + 1; oAN += A[s].nnz; oBR += d.q + 1; oBN += B[s].nnz; oBC += d.n + 1; oGR += d.m + 1;
        oR += (long long)d.m * d.n; oX += (long long)d.p * d.q; oRow += d.m; oBlk += d.nb;
    }
    b->totR = oR;
    b->totX = oX;
    bool ok = sp_alloc(&b->a_rowptr, oAR) && sp_alloc(&b->a_col, oAN) && sp_alloc(&b->a_val, oAN) &&
              sp_alloc(&b->b_rowptr, oBR) && sp_alloc(&b->b_col, oBN) && sp_alloc(&b->b_val, oBN) &&
              sp_alloc(&b->bc_colptr, oBC) && sp_alloc(&b->bc_row, oBN) && sp_alloc(&b->bc_val, oBN) &&
              sp_alloc(&b->g_rowptr, oGR) && sp_alloc(&b->C, oR) && sp_alloc(&b->R, oR) && sp_alloc(&b->X, oX) &&
              sp_alloc(&b->a, oRow) && sp_alloc(&b->pref, oRow) && sp_alloc(&b->s, oRow) && sp_alloc(&b->r, oRow) &&
              sp_alloc(&b->ac_colptr, oAC) && sp_alloc(&b->ac_row, oAN) && sp_alloc(&b->ac_val, oAN) &&
              sp_alloc(&b->cn, oCol) && sp_alloc(&b->cpref, oCol) && (!o.extended || sp_alloc(&b->Y, oR)) &&
              sp_alloc(&b->dsys, nsys) && sp_alloc(&b->dorder, nsys) && sp_alloc(&b->dqueue, 1) &&
              sp_alloc(&b->iters, nsys) && sp_alloc(&b->S, nsys) && sp_alloc(&b->flags, nsys);
    if (!ok) { grbk_sparse_destroy(b); return GRBK_ENOMEM; }
    cudaStream_t st = b->stream;
    // caller arrays -> device; C converted to FP64
    std::vector<long long> rp;
    std::vector<long long*> scratch;
    long long* cnt = nullptr;
    long long* fill = nullptr;
    long long maxdim = 1;
    for (int s = 0; s < nsys; ++s) maxdim = std::max<long long>({maxdim, (long long)A[s].cols + 1, (long long)A[s].rows + 1,
                                                               (long long)B[s].cols + 1});
    grbk_status err = GRBK_OK;
    auto fail = [&](grbk_status e) {
        cudaStreamSynchronize(st);
        cudaFree(cnt);
        cudaFree(fill);
        grbk_sparse_destroy(b);
        return e;
    };
    if (!sp_alloc(&cnt, maxdim) || !sp_alloc(&fill, maxdim)) return fail(GRBK_ENOMEM);
    for (int s = 0; s < nsys && err == GRBK_OK; ++s) {
        const SpDesc& d = b->hsys[s];
        if (cudaMemcpyAsync(b->a_rowptr + d.aRow, A[s].rowptr, 8 * (d.m + 1), cudaMemcpyHostToDevice, st) ||
            cudaMemcpyAsync(b->a_col + d.aNz, A[s].colind, 4 * A[s].nnz, cudaMemcpyHostToDevice, st) ||
            cudaMemcpyAsync(b->a_val + d.aNz, A[s].val, 8 * A[s].nnz, cudaMemcpyHostToDevice, st) ||
            cudaMemcpyAsync(b->b_rowptr + d.bRow, B[s].rowptr, 8 * (d.q + 1), cudaMemcpyHostToDevice, st) ||
            cudaMemcpyAsync(b->b_col + d.bNz, B[s].colind, 4 * B[s].nnz, cudaMemcpyHostToDevice, st) ||
            cudaMemcpyAsync(b->b_val + d.bNz, B[s].val, 8 * B[s].nnz, cudaMemcpyHostToDevice, st))
            err = GRBK_ECUDA;
        if (err != GRBK_OK) break;
        // C: host matrices of either type go through a device staging copy of their own type
        const grbk_mat& M = C[s];
        if (M.on_device) {
            if (convert_matrix(b->C + d.offR, GRBK_DT_F64, d.n, M.ptr, M.dtype, M.ld, d.m, d.n, st)) err = GRBK_ECUDA;
        } else if (M.dtype == GRBK_DT_F64) {
            if (cudaMemcpy2DAsync(b->C + d.offR, 8 * d.n, M.ptr, 8 * M.ld, 8 * d.n, d.m, cudaMemcpyHostToDevice, st))
                err = GRBK_ECUDA;
        } else {
            float* tmp = nullptr;
            if (!sp_alloc(&tmp, (size_t)d.m * d.n)) { err = GRBK_ENOMEM; break; }
            if (cudaMemcpy2DAsync(tmp, 4 * d.n, M.ptr, 4 * M.ld, 4 * d.n, d.m, cudaMemcpyHostToDevice, st) ||
                convert_matrix(b->C + d.offR, GRBK_DT_F64, d.n, tmp, GRBK_DT_F32, d.n, d.m, d.n, st))
                err = GRBK_ECUDA;
            cudaStreamSynchronize(st);
            cudaFree(tmp);
        }
    }
    if (err != GRBK_OK) return fail(err);
    // CSC of B (for v = w B) and of A (for the Gram matrix), then A A^T: count, scan, fill
    b->gnnz.assign(nsys, 0);
    b->growmax.assign(nsys, 0);
    for (int s = 0; s < nsys; ++s) {
        const SpDesc& d = b->hsys[s];
        const int grid = 64;
        // B^T
        cudaMemsetAsync(cnt, 0, 8 * (d.n + 1), st);
        cudaMemsetAsync(fill, 0, 8 * (d.n + 1), st);
        sp_colcount_kernel<<<grid, 256, 0, st>>>(b->b_col + d.bNz, B[s].nnz, cnt);
        sp_scan_kernel<<<1, kSpT, 0, st>>>(cnt, d.n, b->bc_colptr + d.bCol);
        sp_csc_fill_kernel<<<grid, 256, 0, st>>>(b->b_rowptr + d.bRow, b->b_col + d.bNz, b->b_val + d.bNz, d.q,
                                                  b->bc_colptr + d.bCol, fill, b->bc_row + d.bNz, b->bc_val + d.bNz);
        sp_csc_sort_kernel<<<grid, 256, 0, st>>>(b->bc_colptr + d.bCol, d.n, b->bc_row + d.bNz, b->bc_val + d.bNz);
        // A^T (kept: the Gram matrix below and the extended method's column steps read it)
        long long* a_colptr = b->ac_colptr + d.aCol;
        int* a_crow = b->ac_row + d.aNz;
        double* a_cval = b->ac_val + d.aNz;
        cudaMemsetAsync(cnt, 0, 8 * (d.p + 1), st);
        cudaMemsetAsync(fill, 0, 8 * (d.p + 1), st);
        sp_colcount_kernel<<<grid, 256, 0, st>>>(b->a_col + d.aNz, A[s].nnz, cnt);
        sp_scan_kernel<<<1, kSpT, 0, st>>>(cnt, d.p, a_colptr);
        sp_csc_fill_kernel<<<grid, 256, 0, st>>>(b->a_rowptr + d.aRow, b->a_col + d.aNz, b->a_val + d.aNz, d.m,
                                                  a_colptr, fill, a_crow, a_cval);
        sp_csc_sort_kernel<<<grid, 256, 0, st>>>(a_colptr, d.p, a_crow, a_cval);
        // A A^T: entries per row, their offsets
        const int gb = std::max(1, std::min(1024, (d.m + kSpW - 1) / kSpW));
        sp_gram_kernel<<<gb, kSpT, 0, st>>>(b->a_rowptr + d.aRow, b->a_col + d.aNz, b->a_val + d.aNz, d.m,
                                            a_colptr, a_crow, cnt, nullptr, nullptr, nullptr, 0);
        sp_scan_kernel<<<1, kSpT, 0, st>>>(cnt, d.m, b->g_rowptr + d.gRow);
        // the largest row, in the scan's last slot's neighbour (fill is free until the next system)
        unsigned long long* dmax = reinterpret_cast<unsigned long long*>(fill);
        cudaMemsetAsync(dmax, 0, 8, st);
        sp_rowmax_kernel<<<std::max(1, std::min(256, (d.m + 255) / 256)), 256, 0, st>>>(cnt, d.m, dmax);
        if (cudaGetLastError() != cudaSuccess) return fail(GRBK_ECUDA);
        long long gn = 0;
        unsigned long long gmax = 0;
        if (cudaMemcpyAsync(&gn, b->g_rowptr + d.gRow + d.m, 8, cudaMemcpyDeviceToHost, st) ||
            cudaMemcpyAsync(&gmax, dmax, 8, cudaMemcpyDeviceToHost, st) || cudaStreamSynchronize(st))
            return fail(GRBK_ECUDA);
        b->gnnz[s] = gn;
        b->growmax[s] = (long long)gmax;
    }
    long long oGN = 0;
    for (int s = 0; s < nsys; ++s) { b->hsys[s].gNz = oGN; oGN += b->gnnz[s]; }
    if (!sp_alloc(&b->g_col, oGN) || !sp_alloc(&b->g_val, oGN)) return fail(GRBK_ENOMEM);
    for (int s = 0; s < nsys; ++s) {
        const SpDesc& d = b->hsys[s];
        const int gb = std::max(1, std::min(1024, (d.m + kSpW - 1) / kSpW));
        sp_gram_kernel<<<gb, kSpT, 0, st>>>(b->a_rowptr + d.aRow, b->a_col + d.aNz, b->a_val + d.aNz, d.m,
                                            b->ac_colptr + d.aCol, b->ac_row + d.aNz, nullptr, b->g_rowptr + d.gRow,
                                            b->g_col + d.gNz, b->g_val + d.gNz, 1);
    }
    if (cudaGetLastError() != cudaSuccess) return fail(GRBK_ECUDA);
    // per-system scalars
    SpParams P;
    memset(&P, 0, sizeof(P));
    P.nsys = nsys; P.sys = b->dsys;
    P.a_rowptr = b->a_rowptr; P.a_col = b->a_col; P.a_val = b->a_val;
    P.b_rowptr = b->b_rowptr; P.b_col = b->b_col; P.b_val = b->b_val;
    P.bc_colptr = b->bc_colptr; P.bc_row = b->bc_row; P.bc_val = b->bc_val;
    P.ac_colptr = b->ac_colptr; P.ac_row = b->ac_row; P.ac_val = b->ac_val;
    P.C = b->C;
    std::vector<double> sc(kSpSetupScalars * (size_t)nsys);
    double* dsc = nullptr;
    if (!sp_alloc(&dsc, sc.size())) return fail(GRBK_ENOMEM);
    cudaError_t e = cudaMemcpyAsync(b->dsys, b->hsys.data(), sizeof(SpDesc) * nsys, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        sp_setup_kernel<<<nsys, kSpT, 0, st>>>(P, b->a, b->pref, b->cn, b->cpref, dsc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(sc.data(), dsc, 8 * sc.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(dsc);
    if (e != cudaSuccess) return fail(GRBK_ECUDA);
    for (int s = 0; s < nsys; ++s) {
        SpDesc& d = b->hsys[s];
        const double* x = sc.data() + (size_t)kSpSetupScalars * s;
        if (x[3] != 0.0) return fail(GRBK_ENONFINITE);
        const double F = x[0], lam = x[2];
        if (!(F > 0.0) || !(lam > 0.0)) return fail(GRBK_EINVAL);
        d.F = F;
        d.normC2 = x[1];
        d.Fc = x[4];
        const double a_in = o.alphas ? o.alphas[s] : o.alpha;
        if (o.alphas || a_in > 0.0) {
            // Lemma 2.2 / Theorems 4.2-4.8 need 0 < alpha < 2/||B||_2^2
            if (!(a_in > 0.0 && a_in * lam < 2.0 * (1.0 + 1e-9))) return fail(GRBK_EINVAL);
            d.alpha = a_in;
        } else {
            d.alpha = 1.0 / lam;
        }
        d.stop_S = -1.0;
    }
    // longest first: rows of R times the entries of an average Gram row
    b->order.resize(nsys);
    for (int s = 0; s < nsys; ++s) b->order[s] = s;
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
        return (long long)b->hsys[x].m * b->hsys[x].n > (long long)b->hsys[y].m * b->hsys[y].n;
    });
    if (cudaMemcpyAsync(b->dorder, b->order.data(), 4 * nsys, cudaMemcpyHostToDevice, st) ||
        cudaStreamSynchronize(st))
        return fail(GRBK_ECUDA);
    cudaFree(cnt);
    cudaFree(fill);
    *out = b;
    return GRBK_OK;
}

extern "C" grbk_status grbk_sparse_cluster(const grbk_sparse* b, int32_t* ctas)
{
    if (!b || !ctas) return GRBK_EINVAL;
    *ctas = b->last_cluster;
    return GRBK_OK;
}

extern "C" grbk_status grbk_sparse_info(const grbk_sparse* b, int32_t sys, int64_t* gram_nnz, double* alpha)
{
    if (!b || sys < 0 || sys >= b->nsys) return GRBK_EINVAL;
    if (gram_nnz) *gram_nnz = b->gnnz[sys];
    if (alpha) *alpha = b->hsys[sys].alpha;
    return GRBK_OK;
}

extern "C" grbk_status grbk_sparse_solve(grbk_sparse* b, int32_t variant, double theta, double tol,
                                         const double* targets, int64_t maxit, uint64_t seed, grbk_mat* X_outs,
                                         grbk_result* results)
{
    const auto t0 = std::chrono::steady_clock::now();
    if (!b) return GRBK_EINVAL;
    if (variant < GRBK_GRBK || variant > GRBK_BK) return GRBK_EINVAL;
    if (variant == GRBK_RGRBK && !(theta > 0.0 && theta <= 1.0)) return GRBK_EINVAL;
    if (maxit < 0 || !std::isfinite(tol)) return GRBK_EINVAL;
    // the extension's residual starts at zero: it runs a fixed number of iterations
    if (b->opts.extended && (targets || b->opts.stop_kind != GRBK_STOP_NONE)) return GRBK_EINVAL;
    cudaStream_t st = b->stream;
    for (int s = 0; s < b->nsys; ++s) {
        SpDesc& d = b->hsys[s];
        if (X_outs) {
            const grbk_mat& M = X_outs[s];
            if (!M.ptr || M.rows != d.p || M.cols != d.q || M.ld < d.q) return GRBK_EINVAL;
            if (M.dtype != GRBK_DT_F64 && M.dtype != GRBK_DT_F32) return GRBK_EINVAL;
        }
        if (targets && !(std::isfinite(targets[s]) && targets[s] >= 0.0)) return GRBK_EINVAL;
        if (targets) d.stop_S = targets[s] * targets[s];
        else if (b->opts.stop_kind == GRBK_STOP_RELRES) d.stop_S = tol * tol * d.normC2;
        else d.stop_S = -1.0;
    }
    GRBK_CK(cudaMemcpyAsync(b->dsys, b->hsys.data(), sizeof(SpDesc) * b->nsys, cudaMemcpyHostToDevice, st));
    GRBK_CK(cudaMemsetAsync(b->dqueue, 0, 4, st));
    SpParams P;
    memset(&P, 0, sizeof(P));
    P.nsys = b->nsys; P.sys = b->dsys; P.order = b->dorder; P.queue = b->dqueue;
    P.a_rowptr = b->a_rowptr; P.a_col = b->a_col; P.a_val = b->a_val;
    P.b_rowptr = b->b_rowptr; P.b_col = b->b_col; P.b_val = b->b_val;
    P.bc_colptr = b->bc_colptr; P.bc_row = b->bc_row; P.bc_val = b->bc_val;
    P.g_rowptr = b->g_rowptr; P.g_col = b->g_col; P.g_val = b->g_val;
    P.ac_colptr = b->ac_colptr; P.ac_row = b->ac_row; P.ac_val = b->ac_val;
    P.cn = b->cn; P.cpref = b->cpref; P.Y = b->Y; P.extended = b->opts.extended ? 1 : 0;
    P.C = b->C; P.R = b->R; P.X = b->X; P.a = b->a; P.pref = b->pref; P.s = b->s; P.r = b->r;
    P.iters = b->iters; P.S_out = b->S; P.flag_out = b->flags;
    P.variant = variant; P.theta = theta; P.seed = seed; P.maxit = maxit;
    const long long tlen = (b->opts.row_trace || b->opts.s_trace) ? b->opts.trace_len : 0;
    if (tlen > 0) {
        cudaFree(b->trace);
        cudaFree(b->traceS);
        b->trace = nullptr;
        b->traceS = nullptr;
        if (!sp_alloc(&b->trace, (size_t)tlen * b->nsys) || !sp_alloc(&b->traceS, (size_t)tlen * b->nsys))
            return GRBK_ENOMEM;
        GRBK_CK(cudaMemsetAsync(b->trace, 0xff, 4 * (size_t)tlen * b->nsys, st));
        GRBK_CK(cudaMemsetAsync(b->traceS, 0, 8 * (size_t)tlen * b->nsys, st));
        P.trace_rows = b->trace;
        P.trace_S = b->traceS;
        P.trace_len = tlen;
    }
    sp_init_kernel<<<b->nsys, kSpT, 0, st>>>(P);
    GRBK_CK(cudaGetLastError());
    int dev = 0, nsm = 0;
    GRBK_CK(cudaGetDevice(&dev));
    GRBK_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    int grid = std::min(b->nsys, nsm * 4);
    if (b->opts.grid_ctas > 0) grid = std::min(grid, (int)b->opts.grid_ctas);
    // shared memory for the row update's squares: the largest (row of A A^T) x n, at most
    // kSpSqCap; an iteration whose row does not fit takes the one-thread-per-row update
    long long sq = 0;
    for (int s = 0; s < b->nsys; ++s) {
        if (b->hsys[s].n >= 8) sq = std::max(sq, std::min(kSpSqCap, b->growmax[s] * b->hsys[s].n));
        // the select's block sums (one 8-byte word per 256-row block) share the same memory
        sq = std::max(sq, (long long)b->hsys[s].nb);
    }
    P.sq_cap = sq;
    // a cluster of CS CTAs per system when the systems leave SMs idle (CS * systems <= SMs) and
    // the row update is heavy (n >= 8: its element work splits over the cluster; with few
    // columns, as in the colour model, three cluster barriers per iteration cost more than the
    // split saves); with clusters every CTA asks for at least 120 KB of shared memory, so that
    // no two CTAs of a cluster share an SM (and its FP64 unit)
    int nmax = 0;
    for (int s = 0; s < b->nsys; ++s) nmax = std::max(nmax, b->hsys[s].n);
    int CS = 1;
    for (int c = 8; c >= 2; c >>= 1)
        if ((long long)b->nsys * c <= nsm && b->opts.grid_ctas <= 0 && nmax >= 8) { CS = c; break; }
    size_t smem = (size_t)sq * 8;
    if (CS > 1) smem = std::max(smem, (size_t)120 * 1024);
    GRBK_CK(cudaFuncSetAttribute(sp_solve_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    GRBK_CK(cudaFuncSetAttribute(sp_solve_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    cfg.blockDim = dim3(kSpT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    for (;;) {
        attr[0].val.clusterDim.x = CS;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)(CS == 1 ? grid : std::min(b->nsys, nsm / CS) * CS));
        int nclus = 0;
        if (CS == 1 || (cudaOccupancyMaxActiveClusters(&nclus, (const void*)sp_solve_kernel<true>, &cfg) == cudaSuccess &&
                        nclus >= 1)) {
            if (CS > 1) cfg.gridDim = dim3((unsigned)(std::min(std::min(b->nsys, nsm / CS), nclus) * CS));
            break;
        }
        cudaGetLastError();
        CS >>= 1;   // that cluster size does not fit: a smaller one
        if (CS == 1) {
            smem = (size_t)sq * 8;
            cfg.dynamicSmemBytes = smem;
        }
    }
    b->last_cluster = CS;
    if (CS > 1) {
        GRBK_CK(cudaLaunchKernelEx(&cfg, sp_solve_kernel<true>, P));
    } else {
        sp_solve_kernel<false><<<cfg.gridDim, kSpT, cfg.dynamicSmemBytes, st>>>(P);
    }
    GRBK_CK(cudaGetLastError());
    std::vector<long long> it(b->nsys);
    std::vector<double> S(b->nsys);
    std::vector<int> fl(b->nsys);
    GRBK_CK(cudaMemcpyAsync(it.data(), b->iters, 8 * b->nsys, cudaMemcpyDeviceToHost, st));
    GRBK_CK(cudaMemcpyAsync(S.data(), b->S, 8 * b->nsys, cudaMemcpyDeviceToHost, st));
    GRBK_CK(cudaMemcpyAsync(fl.data(), b->flags, 4 * b->nsys, cudaMemcpyDeviceToHost, st));
    if (tlen > 0) {
        if (b->opts.row_trace)
            GRBK_CK(cudaMemcpyAsync(b->opts.row_trace, b->trace, 4 * (size_t)tlen * b->nsys, cudaMemcpyDeviceToHost, st));
        if (b->opts.s_trace)
            GRBK_CK(cudaMemcpyAsync(b->opts.s_trace, b->traceS, 8 * (size_t)tlen * b->nsys, cudaMemcpyDeviceToHost, st));
    }
    if (X_outs) {
        for (int s = 0; s < b->nsys; ++s) {
            const SpDesc& d = b->hsys[s];
            grbk_mat& M = X_outs[s];
            if (M.on_device) {
                GRBK_CK(convert_matrix((void*)M.ptr, M.dtype, M.ld, b->X + d.offX, GRBK_DT_F64, d.q, d.p, d.q, st));
            } else if (M.dtype == GRBK_DT_F64) {
                GRBK_CK(cudaMemcpy2DAsync((void*)M.ptr, 8 * M.ld, b->X + d.offX, 8 * d.q, 8 * d.q, d.p,
                                          cudaMemcpyDeviceToHost, st));
            } else {
                float* tmp = nullptr;
                if (!sp_alloc(&tmp, (size_t)d.p * d.q)) return GRBK_ENOMEM;
                cudaError_t e = convert_matrix(tmp, GRBK_DT_F32, d.q, b->X + d.offX, GRBK_DT_F64, d.q, d.p, d.q, st);
                if (e == cudaSuccess)
                    e = cudaMemcpy2DAsync((void*)M.ptr, 4 * M.ld, tmp, 4 * d.q, 4 * d.q, d.p, cudaMemcpyDeviceToHost, st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                cudaFree(tmp);
                if (e != cudaSuccess) return GRBK_ECUDA;
            }
        }
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
            results[s].relres = b->hsys[s].normC2 > 0 ? sqrt(S[s] / b->hsys[s].normC2) : 0.0;
            results[s].rse = NAN;
            results[s].seconds = secs;
            results[s].alpha = b->hsys[s].alpha;
            results[s].x0_rejected = 0;
            results[s].gram = 1;
            results[s].launches = 2;
            results[s].status = ss;
        }
    }
    return overall;
}

// R and the row norms of system `sys` after a solve (host FP64 buffers)
extern "C" grbk_status grbk_sparse_get_residual(const grbk_sparse* b, int32_t sys, double* R_out, double* s_out)
{
    if (!b || sys < 0 || sys >= b->nsys) return GRBK_EINVAL;
    const SpDesc& d = b->hsys[sys];
    if (R_out) GRBK_CK(cudaMemcpyAsync(R_out, b->R + d.offR, 8 * (size_t)d.m * d.n, cudaMemcpyDeviceToHost, b->stream));
    if (s_out) GRBK_CK(cudaMemcpyAsync(s_out, b->s + d.offRow, 8 * (size_t)d.m, cudaMemcpyDeviceToHost, b->stream));
    GRBK_CK(cudaStreamSynchronize(b->stream));
    return GRBK_OK;
}
