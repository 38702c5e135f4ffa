// grbk_probe.cu -- throughput and issue-cost probes of the FP64 pipe.
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

// Issue cost of one FP64 operation on one SM: one CTA of `warps` warps; in each
// warp the first `active` lanes run a dependent chain of `iters` operations
// (op 0 add, 1 fused multiply-add, 2 multiply, 3 division, 4 a double -> float
// -> double round trip plus an add); the others wait at the end.  Each warp
// records its clock64 span; the chains keep their values finite.
__global__ void fp64_issue_kernel(int op, int active, long long iters, double* out, long long* cyc)
{
    const int lane = threadIdx.x & 31;
    double x = 1.0 + 1e-3 * threadIdx.x;
    const double y = 1e-300 * (threadIdx.x + 1);
    float f = 1.0f;
    __syncthreads();
    const long long t0 = clock64();
    if (lane < active) {
        for (long long i = 0; i < iters; ++i) {
            if (op == 0) x = __dadd_rn(x, y);
            else if (op == 1) x = __fma_rn(x, 0.5, y);
            else if (op == 2) x = __dmul_rn(x, 1.0000001);
            else if (op == 3) x = __ddiv_rn(1.0, x);
            else { f = (float)x; x = (double)f + y; }
        }
    }
    const long long t1 = clock64();
    out[threadIdx.x] = x + (double)f;
    if (lane == 0) cyc[threadIdx.x >> 5] = t1 - t0;
}

}  // namespace grbk

using namespace grbk;

extern "C" grbk_status grbk_fp64_issue_probe(int32_t op, int32_t warps, int32_t active_lanes, int64_t iters,
                                             double* cycles_per_op, void* stream)
{
    if (op < 0 || op > 4 || warps < 1 || warps > 32 || active_lanes < 1 || active_lanes > 32 || iters <= 0 ||
        !cycles_per_op)
        return GRBK_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    double* out = nullptr;
    long long* cyc = nullptr;
    if (cudaMalloc(&out, sizeof(double) * 32 * (size_t)warps) != cudaSuccess) return GRBK_ENOMEM;
    if (cudaMalloc(&cyc, sizeof(long long) * (size_t)warps) != cudaSuccess) { cudaFree(out); return GRBK_ENOMEM; }
    grbk_status r = GRBK_OK;
    long long h[32] = {0};
    // one untimed launch, then the measured one
    fp64_issue_kernel<<<1, 32 * warps, 0, st>>>(op, active_lanes, iters, out, cyc);
    fp64_issue_kernel<<<1, 32 * warps, 0, st>>>(op, active_lanes, iters, out, cyc);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(h, cyc, sizeof(long long) * (size_t)warps, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        r = GRBK_ECUDA;
    cudaFree(out);
    cudaFree(cyc);
    if (r != GRBK_OK) return r;
    long long mx = 0;
    for (int w = 0; w < warps; ++w) mx = h[w] > mx ? h[w] : mx;
    *cycles_per_op = (double)mx / (double)iters;
    return GRBK_OK;
}

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
