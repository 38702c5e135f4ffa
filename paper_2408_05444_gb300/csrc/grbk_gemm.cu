// grbk_gemm.cu -- dense products for the residual refresh R = C - A X B
// (Algorithm 3 initialisation, repeated every refresh period): a tiled SIMT
// GEMM used in FP64 mode, and the FP32-mode refresh engine.
#include <cuda_runtime.h>
#include <stdint.h>

#include "grbk_internal.cuh"

namespace grbk {

// Cout = beta * Cin + alpha * A(MxK) * B(KxN); 64x64 tiles, 16x16 threads, 4x4 per thread.
template <typename T>
__global__ void __launch_bounds__(256) gemm_simt_kernel(int64_t M, int64_t N, int64_t K, double alpha,
                                                        const T* __restrict__ A, int64_t lda,
                                                        const T* __restrict__ B, int64_t ldb, double beta,
                                                        const T* __restrict__ Cin, int64_t ldcin,
                                                        T* __restrict__ Cout, int64_t ldc)
{
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int64_t row0 = (int64_t)blockIdx.y * BM, col0 = (int64_t)blockIdx.x * BN;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = (T)0;
    for (int64_t k0 = 0; k0 < K; k0 += BK) {
        for (int e = threadIdx.x; e < BM * BK; e += 256) {
            const int r = e / BK, kk = e % BK;
            const int64_t gr = row0 + r, gk = k0 + kk;
            As[kk][r] = (gr < M && gk < K) ? A[gr * lda + gk] : (T)0;
        }
        for (int e = threadIdx.x; e < BK * BN; e += 256) {
            const int kk = e / BN, cc = e % BN;
            const int64_t gk = k0 + kk, gc = col0 + cc;
            Bs[kk][cc] = (gk < K && gc < N) ? B[gk * ldb + gc] : (T)0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
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
            double val = alpha * (double)acc[i][j];
            if (Cin) val += beta * (double)Cin[gr * ldcin + gc];
            Cout[gr * ldc + gc] = (T)val;
        }
    }
}

template <typename T>
cudaError_t gemm_simt(int64_t M, int64_t N, int64_t K, double alpha, const T* A, int64_t lda, const T* B,
                      int64_t ldb, double beta, const T* Cin, int64_t ldcin, T* Cout, int64_t ldc,
                      cudaStream_t st)
{
    if (M <= 0 || N <= 0) return cudaSuccess;
    dim3 grid((unsigned)((N + 63) / 64), (unsigned)((M + 63) / 64));
    gemm_simt_kernel<T><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, Cin, ldcin, Cout, ldc);
    return cudaGetLastError();
}

template cudaError_t gemm_simt<double>(int64_t, int64_t, int64_t, double, const double*, int64_t,
                                       const double*, int64_t, double, const double*, int64_t, double*,
                                       int64_t, cudaStream_t);
template cudaError_t gemm_simt<float>(int64_t, int64_t, int64_t, double, const float*, int64_t,
                                      const float*, int64_t, double, const float*, int64_t, float*,
                                      int64_t, cudaStream_t);

// ----------------------------------------------------------------------------
// FP32-mode refresh engine
// ----------------------------------------------------------------------------
struct SplitGemm {
    int64_t m, p, q, n, lda, ldb;
    const float* A;
    const float* B;
    int terms;
    float* Xf;   // p x q
    float* T1;   // m x q
};

__global__ void x_to_f32_kernel(const double* X, int64_t total, float* Xf)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < total) Xf[i] = (float)X[i];
}

grbk_status splitgemm_create(SplitGemm** out, int64_t m, int64_t p, int64_t q, int64_t n, const float* A,
                             int64_t lda, const float* B, int64_t ldb, int terms, cudaStream_t st)
{
    (void)st;
    SplitGemm* g = new SplitGemm();
    g->m = m; g->p = p; g->q = q; g->n = n; g->lda = lda; g->ldb = ldb;
    g->A = A; g->B = B; g->terms = terms;
    g->Xf = nullptr; g->T1 = nullptr;
    if (cudaMalloc(&g->Xf, (size_t)p * q * 4) != cudaSuccess || cudaMalloc(&g->T1, (size_t)m * q * 4) != cudaSuccess) {
        splitgemm_destroy(g);
        return GRBK_ENOMEM;
    }
    *out = g;
    return GRBK_OK;
}

grbk_status splitgemm_residual(SplitGemm* g, const double* X, int64_t ldx, const float* C, float* R,
                               int64_t ldr, cudaStream_t st)
{
    (void)ldx;
    const int64_t tot = g->p * g->q;
    x_to_f32_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(X, tot, g->Xf);
    GRBK_CK(cudaGetLastError());
    GRBK_CK(gemm_simt<float>(g->m, g->q, g->p, 1.0, g->A, g->lda, g->Xf, g->q, 0.0, nullptr, 0, g->T1, g->q, st));
    GRBK_CK(gemm_simt<float>(g->m, g->n, g->q, -1.0, g->T1, g->q, g->B, g->ldb, 1.0, C, ldr, R, ldr, st));
    return GRBK_OK;
}

int splitgemm_launches(const SplitGemm*) { return 3; }

void splitgemm_destroy(SplitGemm* g)
{
    if (!g) return;
    if (g->Xf) cudaFree(g->Xf);
    if (g->T1) cudaFree(g->T1);
    delete g;
}

}  // namespace grbk
