// grbk_rowspace.cu -- set-up of the row-space form of the residual.
//
// Every residual row of the method lies in the row space of B plus a part that
// the iteration never changes: R^k = C - A X^k B, and each update subtracts
// c_k u (w B), a combination of the rows of B (Algorithm 3's update of R).
// With an orthonormal basis Bt (r x n, Bt Bt^T = I, r = rank B) of that row
// space and B = Lt Bt (Lt is q x r), write R^k = Z^k Bt + Rperp with
// Z^k = R^k Bt^T (m x r) and Rperp = C - C Bt^T Bt.  Then
//   ||R_i||^2 = ||Z_i||^2 + ||Rperp_i||^2       (s_i of Algorithm 3),
//   w = R_{i_k} B^T = Z_{i_k} Lt^T              (the X update is unchanged),
//   R_{i_k} B^T B = (w Lt) Bt                   (the R update becomes Z -= c u (w Lt)),
// so the method on (A, B, C) performs the same iterations as the method on the
// smaller system (A, Lt, Chat = C Bt^T) with the fixed row offsets
// ||Rperp_i||^2 added to its row norms.  The residual shrinks from m x n to
// m x r.  The refresh becomes Z = Chat - (A X) Lt, since B Bt^T = Lt.
//
// The basis comes from a pivoted Cholesky factorisation of G = B B^T:
// G = P L L^T P^T with L (q x r) lower trapezoidal, L1 = L[0:r, 0:r]; the r
// pivot rows B1 of B are independent and Bt = L1^{-1} B1, Lt = P L.  The
// factorisation stops at the first pivot below tol * max_i G_ii, which sets r.
//
// Set-up products (64 x 64 SIMT tiles; FP64 throughout in the FP64 form; FP32
// inputs with Kahan-compensated accumulation of 16-term tile sums in the FP32
// form): G = B B^T (FP64 output), Y = C B^T, Chat = Y M^T with
// M[t][perm[s]] = L1^{-1}[t][s], Bt = M B, Rperp = C - Chat Bt (formed
// explicitly, then its row norms in FP64, so that no difference of large
// squared norms is taken), and K = Lt^T Lt (r x r): the update vector of the
// kept residual, (w Lt) with w = Z_{i_k} Lt^T, equals Z_{i_k} K, so an
// iteration can form it from the selected row alone.
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>
#include <algorithm>

#include "grbk_internal.cuh"

namespace grbk {

namespace {

// Cout (Tout, ldc) = alpha * A(M x K) * op(B) + beta * Cin, op(B) = B (K x N) or,
// with BT, B given as N x K.  Tile sums of 16 products in Tin precision; for
// Tin = float they are added into a Kahan-compensated FP32 accumulator.
template <typename Tin, typename Tout, bool BT>
__global__ void __launch_bounds__(256) setup_gemm_kernel(int64_t M, int64_t N, int64_t K, double alpha,
                                                         const Tin* __restrict__ A, int64_t lda,
                                                         const Tin* __restrict__ B, int64_t ldb, double beta,
                                                         const Tin* __restrict__ Cin, int64_t ldcin,
                                                         Tout* __restrict__ Cout, int64_t ldc)
{
    constexpr int BM = 64, BN = 64, BK = 16;
    constexpr bool kComp = sizeof(Tin) == 4;
    __shared__ Tin As[BK][BM + 1];
    __shared__ Tin Bs[BK][BN + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int64_t row0 = (int64_t)blockIdx.y * BM, col0 = (int64_t)blockIdx.x * BN;
    Tin acc[4][4], cmp[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = cmp[i][j] = (Tin)0;
    for (int64_t k0 = 0; k0 < K; k0 += BK) {
        for (int e = threadIdx.x; e < BM * BK; e += 256) {
            const int r = e / BK, kk = e % BK;
            const int64_t gr = row0 + r, gk = k0 + kk;
            As[kk][r] = (gr < M && gk < K) ? A[gr * lda + gk] : (Tin)0;
        }
        for (int e = threadIdx.x; e < BK * BN; e += 256) {
            int kk, cc;
            if (BT) { cc = e / BK; kk = e % BK; } else { kk = e / BN; cc = e % BN; }
            const int64_t gk = k0 + kk, gc = col0 + cc;
            Bs[kk][cc] = (gk < K && gc < N) ? (BT ? B[gc * ldb + gk] : B[gk * ldb + gc]) : (Tin)0;
        }
        __syncthreads();
        Tin part[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) part[i][j] = (Tin)0;
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            Tin a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) part[i][j] = fma(a[i], b[j], part[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (kComp) {
                    const Tin y = part[i][j] - cmp[i][j];
                    const Tin t = acc[i][j] + y;
                    cmp[i][j] = (t - acc[i][j]) - y;
                    acc[i][j] = t;
                } else {
                    acc[i][j] += part[i][j];
                }
            }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t gr = row0 + ty + 16 * i;
        if (gr >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t gc = col0 + tx + 16 * j;
            if (gc >= N) continue;
            double val = alpha * ((double)acc[i][j] - (double)cmp[i][j]);
            if (Cin) val += beta * (double)Cin[gr * ldcin + gc];
            Cout[gr * ldc + gc] = (Tout)val;
        }
    }
}

template <typename Tin, typename Tout, bool BT>
cudaError_t setup_gemm(int64_t M, int64_t N, int64_t K, double alpha, const Tin* A, int64_t lda, const Tin* B,
                       int64_t ldb, double beta, const Tin* Cin, int64_t ldcin, Tout* Cout, int64_t ldc,
                       cudaStream_t st)
{
    if (M <= 0 || N <= 0) return cudaSuccess;
    dim3 grid((unsigned)((N + 63) / 64), (unsigned)((M + 63) / 64));
    setup_gemm_kernel<Tin, Tout, BT><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, Cin, ldcin, Cout,
                                                          ldc);
    return cudaGetLastError();
}

struct PcholState {
    int rank;   // -1 while running; else the number of accepted pivots
    int piv;    // position of the pivot of the current step
};

__global__ void pchol_init_kernel(int64_t q, const double* G, int64_t ldg, double* d, int* perm, PcholState* s)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < q) {
        d[i] = G[i * ldg + i];
        perm[i] = (int)i;
    }
    if (i == 0) { s->rank = -1; s->piv = 0; }
}

// Step j, part 1 (one CTA): the pivot is the largest remaining diagonal entry
// d[perm[t]], t >= j (ties: smallest t).  Stops when it is <= tol_abs.
// Otherwise swaps positions j and t in perm and in the computed columns of L,
// and sets L[j][j] = sqrt(pivot).
constexpr int kPivThreads = 1024;
__global__ void __launch_bounds__(kPivThreads) pchol_pivot_kernel(int64_t j, int64_t q, double* L, int64_t ldl,
                                                                  int* perm, const double* d, double tol_abs,
                                                                  PcholState* s)
{
    __shared__ double sv[kPivThreads / 32];
    __shared__ long long si[kPivThreads / 32];
    __shared__ long long s_t;
    if (ld_volatile_int(&s->rank) >= 0) return;
    double best = -INFINITY;
    long long bi = 0x7fffffffffffffffLL;
    for (int64_t t = j + threadIdx.x; t < q; t += kPivThreads) {
        const double v = d[perm[t]];
        if (v > best) { best = v; bi = t; }
    }
    warp_argmax(best, bi);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { sv[warp] = best; si[warp] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = -INFINITY;
        long long t = 0x7fffffffffffffffLL;
        for (int w = 0; w < kPivThreads / 32; ++w)
            if (sv[w] > b || (sv[w] == b && si[w] < t)) { b = sv[w]; t = si[w]; }
        if (!(b > tol_abs)) {
            s->rank = (int)j;
            t = -1;
        } else {
            const int pj = perm[j];
            perm[j] = perm[t];
            perm[t] = pj;
            L[j * ldl + j] = sqrt(b);
            s->piv = (int)t;
        }
        s_t = t;
    }
    __syncthreads();
    const long long t = s_t;
    if (t < 0 || t == j) return;
    for (int64_t c = threadIdx.x; c < j; c += kPivThreads) {
        const double a = L[j * ldl + c];
        L[j * ldl + c] = L[t * ldl + c];
        L[t * ldl + c] = a;
    }
}

// Step j, part 2: column j below the diagonal, one warp per row t > j:
// L[t][j] = (G[perm t][perm j] - L[t][0:j] . L[j][0:j]) / L[j][j], and the
// remaining diagonal d[perm t] -= L[t][j]^2.
__global__ void __launch_bounds__(256) pchol_column_kernel(int64_t j, int64_t q, const double* G, int64_t ldg,
                                                           double* L, int64_t ldl, const int* perm, double* d,
                                                           const PcholState* s)
{
    if (ld_volatile_int(&s->rank) >= 0) return;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const double ljj = L[j * ldl + j];
    const int pj = perm[j];
    for (int64_t t = j + 1 + gw; t < q; t += nw) {
        double acc = 0.0;
        for (int64_t c = lane; c < j; c += 32) acc = fma(L[t * ldl + c], L[j * ldl + c], acc);
        acc = warp_sum(acc);
        if (lane == 0) {
            const int pt = perm[t];
            const double l = (G[(int64_t)pt * ldg + pj] - acc) / ljj;
            L[t * ldl + j] = l;
            d[pt] -= l * l;
        }
    }
}

// LinvT[j][i] = (L1^{-1})[i][j]: forward substitution for column j of the
// inverse, one warp per column (row j of LinvT, written in order).
__global__ void __launch_bounds__(256) tri_inv_kernel(int64_t r, const double* L, int64_t ldl, double* LinvT)
{
    const int lane = threadIdx.x & 31;
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= r) return;
    double* x = LinvT + j * r;
    for (int64_t i = lane; i < j; i += 32) x[i] = 0.0;
    if (lane == 0) __stcg(x + j, 1.0 / L[j * ldl + j]);
    __syncwarp();
    for (int64_t i = j + 1; i < r; ++i) {
        double acc = 0.0;
        for (int64_t c = j + lane; c < i; c += 32) acc = fma(L[i * ldl + c], __ldcg(x + c), acc);
        acc = warp_sum(acc);
        if (lane == 0) __stcg(x + i, -acc / L[i * ldl + i]);
        __syncwarp();
    }
}

// M (r x q, T): M[t][perm[s]] = LinvT[s][t] for s < r, 0 in the other columns.
// Lt (q x r, T): Lt[perm[j]][t] = L[j][t] for t <= j, else 0; LtT (r x q) its transpose.
template <typename T>
__global__ void build_factors_kernel(int64_t q, int64_t r, const double* L, int64_t ldl, const double* LinvT,
                                     const int* perm, T* M, T* Lt, T* LtT)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= q * r) return;
    const int64_t a = e / r, b = e % r;  // a in [0, q), b in [0, r)
    // Lt row perm[a], column b
    const T l = (T)((b <= a) ? L[a * ldl + b] : 0.0);
    Lt[(int64_t)perm[a] * r + b] = l;
    LtT[b * q + perm[a]] = l;
    // M row b, column perm[a]
    M[b * q + perm[a]] = (T)((a < r) ? LinvT[a * r + b] : 0.0);
}

// rperp[i] = ||Rp_i||^2 (FP64), one warp per row
template <typename T>
__global__ void row_norms_kernel(int64_t m, int64_t n, const T* X, int64_t ld, double* out)
{
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= m) return;
    double acc = 0.0;
    for (int64_t c = lane; c < n; c += 32) {
        const double x = (double)X[row * ld + c];
        acc = fma(x, x, acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) out[row] = acc;
}

struct Bufs {
    void* p[10] = {};
    int n = 0;
    cudaError_t alloc(void** ptr, size_t bytes)
    {
        cudaError_t e = cudaMalloc(ptr, bytes > 0 ? bytes : 16);
        if (e == cudaSuccess) p[n++] = *ptr;
        return e;
    }
    ~Bufs()
    {
        for (int i = 0; i < n; ++i) cudaFree(p[i]);
    }
};

#define RS_CK(call)                                                \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) {                                   \
            set_last_cuda_error(e_, #call, __FILE__, __LINE__);    \
            return e_ == cudaErrorMemoryAllocation ? GRBK_ENOMEM : GRBK_ECUDA; \
        }                                                          \
    } while (0)

template <typename T>
grbk_status transform(int64_t m, int64_t q, int64_t n, const T* B, int64_t ldb, const T* C, int64_t ldc,
                      double tol_rel, cudaStream_t st, RowspaceResult* out)
{
    Bufs tmp;
    double *G = nullptr, *L = nullptr, *d = nullptr, *LinvT = nullptr;
    int* perm = nullptr;
    PcholState* ps = nullptr;
    RS_CK(tmp.alloc((void**)&G, (size_t)q * q * 8));
    RS_CK(tmp.alloc((void**)&L, (size_t)q * q * 8));
    RS_CK(tmp.alloc((void**)&d, (size_t)q * 8));
    RS_CK(tmp.alloc((void**)&perm, (size_t)q * 4));
    RS_CK(tmp.alloc((void**)&ps, sizeof(PcholState)));
    RS_CK(cudaMemsetAsync(L, 0, (size_t)q * q * 8, st));

    // G = B B^T (FP64)
    RS_CK((setup_gemm<T, double, true>(q, q, n, 1.0, B, ldb, B, ldb, 0.0, nullptr, 0, G, q, st)));
    pchol_init_kernel<<<(unsigned)((q + 255) / 256), 256, 0, st>>>(q, G, q, d, perm, ps);
    RS_CK(cudaGetLastError());
    double gmax = 0.0;
    {
        // tolerance relative to the largest diagonal entry of G
        double* hd = nullptr;
        RS_CK(cudaMallocHost((void**)&hd, (size_t)q * 8));
        cudaError_t e = cudaMemcpyAsync(hd, d, (size_t)q * 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess)
            for (int64_t i = 0; i < q; ++i) gmax = fmax(gmax, hd[i]);
        cudaFreeHost(hd);
        RS_CK(e);
    }
    if (!(gmax > 0.0) || !isfinite(gmax)) return GRBK_EINVAL;
    const double tol_abs = tol_rel * gmax;
    for (int64_t j = 0; j < q; ++j) {
        pchol_pivot_kernel<<<1, kPivThreads, 0, st>>>(j, q, L, q, perm, d, tol_abs, ps);
        const int64_t rows = q - j - 1;
        if (rows > 0) {
            const unsigned blocks = (unsigned)std::min<int64_t>((rows + 7) / 8, 1024);
            pchol_column_kernel<<<blocks, 256, 0, st>>>(j, q, G, q, L, q, perm, d, ps);
        }
    }
    RS_CK(cudaGetLastError());
    PcholState hs;
    RS_CK(cudaMemcpyAsync(&hs, ps, sizeof(hs), cudaMemcpyDeviceToHost, st));
    RS_CK(cudaStreamSynchronize(st));
    const int64_t r = (hs.rank < 0) ? q : hs.rank;
    if (r <= 0) return GRBK_EINVAL;

    RS_CK(tmp.alloc((void**)&LinvT, (size_t)r * r * 8));
    tri_inv_kernel<<<(unsigned)((r * 32 + 255) / 256), 256, 0, st>>>(r, L, q, LinvT);
    RS_CK(cudaGetLastError());

    T *M = nullptr, *Lt = nullptr, *LtT = nullptr, *Y = nullptr, *Bt = nullptr, *Chat = nullptr, *Rp = nullptr;
    T* K = nullptr;
    double* rperp = nullptr;
    RS_CK(tmp.alloc((void**)&M, (size_t)r * q * sizeof(T)));
    RS_CK(tmp.alloc((void**)&LtT, (size_t)r * q * sizeof(T)));
    RS_CK(tmp.alloc((void**)&Y, (size_t)m * q * sizeof(T)));
    RS_CK(tmp.alloc((void**)&Bt, (size_t)r * n * sizeof(T)));
    RS_CK(tmp.alloc((void**)&Rp, (size_t)m * n * sizeof(T)));
    // results (owned by the caller on success)
    RS_CK(cudaMalloc((void**)&Lt, (size_t)q * r * sizeof(T)));
    if (cudaMalloc((void**)&Chat, (size_t)m * r * sizeof(T)) != cudaSuccess) { cudaFree(Lt); return GRBK_ENOMEM; }
    if (cudaMalloc((void**)&rperp, (size_t)m * 8) != cudaSuccess) { cudaFree(Lt); cudaFree(Chat); return GRBK_ENOMEM; }
    if (cudaMalloc((void**)&K, (size_t)r * r * sizeof(T)) != cudaSuccess) {
        cudaFree(Lt); cudaFree(Chat); cudaFree(rperp);
        return GRBK_ENOMEM;
    }
    auto fail = [&](cudaError_t e, const char* what) {
        set_last_cuda_error(e, what, __FILE__, __LINE__);
        cudaFree(Lt); cudaFree(Chat); cudaFree(rperp); cudaFree(K);
        return GRBK_ECUDA;
    };
    cudaError_t e;
    build_factors_kernel<T><<<(unsigned)((q * r + 255) / 256), 256, 0, st>>>(q, r, L, q, LinvT, perm, M, Lt, LtT);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "build_factors_kernel");
    // K = Lt^T Lt (r x r): R_{i_k} B^T B = Z_{i_k} K Bt, so v in the basis is Z_{i_k} K
    if ((e = setup_gemm<T, T, true>(r, r, q, 1.0, LtT, q, LtT, q, 0.0, nullptr, 0, K, r, st)) != cudaSuccess)
        return fail(e, "K = Lt^T Lt");
    // Y = C B^T (m x q); Chat = Y M^T (m x r); Bt = M B (r x n); Rp = C - Chat Bt
    if ((e = setup_gemm<T, T, true>(m, q, n, 1.0, C, ldc, B, ldb, 0.0, nullptr, 0, Y, q, st)) != cudaSuccess)
        return fail(e, "Y = C B^T");
    if ((e = setup_gemm<T, T, true>(m, r, q, 1.0, Y, q, M, q, 0.0, nullptr, 0, Chat, r, st)) != cudaSuccess)
        return fail(e, "Chat = Y M^T");
    if ((e = setup_gemm<T, T, false>(r, n, q, 1.0, M, q, B, ldb, 0.0, nullptr, 0, Bt, n, st)) != cudaSuccess)
        return fail(e, "Bt = M B");
    if ((e = setup_gemm<T, T, false>(m, n, r, -1.0, Chat, r, Bt, n, 1.0, C, ldc, Rp, n, st)) != cudaSuccess)
        return fail(e, "Rp = C - Chat Bt");
    row_norms_kernel<T><<<(unsigned)((m * 32 + 255) / 256), 256, 0, st>>>(m, n, Rp, n, rperp);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "row_norms_kernel");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(e, "rowspace set-up");
    out->r = r;
    out->Lt = Lt;
    out->Chat = Chat;
    out->rperp = rperp;
    out->K = K;
    out->launches = 4 + 2 * q + 7;
    return GRBK_OK;
}

}  // namespace

grbk_status rowspace_transform(bool fp64, int64_t m, int64_t q, int64_t n, const void* B, int64_t ldb,
                               const void* C, int64_t ldc, double tol_rel, cudaStream_t st, RowspaceResult* out)
{
    if (fp64)
        return transform<double>(m, q, n, (const double*)B, ldb, (const double*)C, ldc, tol_rel, st, out);
    return transform<float>(m, q, n, (const float*)B, ldb, (const float*)C, ldc, tol_rel, st, out);
}

}  // namespace grbk
