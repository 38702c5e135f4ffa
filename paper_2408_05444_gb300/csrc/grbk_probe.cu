// grbk_probe.cu -- throughput probe of the FP64 pipe.
//
// The FP64 form of the residual pass does two fused multiply-adds per element
// of R (the rank-1 update and the square of the new value).  Whether it is
// bound by HBM or by the FP64 pipe depends on the part's FP64 rate, which this
// probe measures: every thread runs kChains independent DFMA chains for
// `iters` steps, enough blocks to fill every SM, timed with CUDA events on the
// caller's stream.
#include <cuda_runtime.h>
#include <stdint.h>

#include "grbk_internal.cuh"

namespace grbk {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

// x <- x * a + b keeps |x| bounded (a < 1), so no chain overflows or
// underflows; the sum of the chains is stored so the compiler keeps them.
__global__ void __launch_bounds__(kProbeThreads) dfma_probe_kernel(long long iters, double a, double b, double* out)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * (double)(threadIdx.x + c);
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[(long long)blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

}  // namespace grbk

using namespace grbk;

extern "C" grbk_status grbk_fp64_probe(int64_t iters, int32_t blocks_per_sm, double* dfma_per_s, double* ms_out,
                                       void* stream)
{
    if (iters <= 0 || blocks_per_sm <= 0 || blocks_per_sm > 64) return GRBK_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    GRBK_CK(cudaGetDevice(&dev));
    GRBK_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int grid = nsm * blocks_per_sm;
    double* out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * (size_t)grid * kProbeThreads) != cudaSuccess) return GRBK_ENOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    grbk_status r = GRBK_OK;
    float ms = 0.f;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) r = GRBK_ECUDA;
    if (r == GRBK_OK) {
        // one untimed launch brings the clocks up, the second is timed
        dfma_probe_kernel<<<grid, kProbeThreads, 0, st>>>(iters, 0.999999, 1e-6, out);
        cudaEventRecord(e0, st);
        dfma_probe_kernel<<<grid, kProbeThreads, 0, st>>>(iters, 0.999999, 1e-6, out);
        cudaEventRecord(e1, st);
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            r = GRBK_ECUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (r != GRBK_OK) return r;
    const double n_fma = (double)grid * kProbeThreads * (double)iters * kChains;
    if (dfma_per_s) *dfma_per_s = ms > 0.f ? n_fma / (ms * 1e-3) : 0.0;
    if (ms_out) *ms_out = ms;
    return GRBK_OK;
}
