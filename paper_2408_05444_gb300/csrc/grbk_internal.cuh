// grbk_internal.cuh -- internal declarations shared by the library's translation
// units: device helpers (bounded grid barrier, Philox4x64-10, warp reductions),
// the context layout and the internal launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#include "grbk.h"

namespace grbk {

// ----------------------------------------------------------------------------
// error plumbing
// ----------------------------------------------------------------------------
#define GRBK_CK(call)                                              \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) {                                   \
            grbk::set_last_cuda_error(e_, #call, __FILE__, __LINE__); \
            return GRBK_ECUDA;                                     \
        }                                                          \
    } while (0)

void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);

inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// Device blocks for contexts (grbk_alloc.cu): freed blocks are kept per device and
// rounded size for the next request instead of returning to the driver.  A block
// may be freed only when no queued work still uses it.
cudaError_t dev_alloc(void** p, size_t bytes);
void dev_free(void* p);

// ----------------------------------------------------------------------------
// device-side status (one per context / batch)
// ----------------------------------------------------------------------------
enum : int { FLAG_RUNNING = 0, FLAG_TOL_MET = 1, FLAG_EXACT = 2 };

struct DevState {
    int status;          // grbk_status raised on the device (0 = none)
    int flag;            // FLAG_*
    long long k;         // iteration index reached by the last chunk
    double S;            // ||R||_F^2 at iteration k
    int timeout_site;    // which barrier gave up (diagnostics)
    int pad;
};

struct GridBarrier {
    unsigned int count;
    unsigned int gen;
};

// Spin budget of one barrier wait, in SM clock cycles (about 2 s at 2 GHz).
// A legitimate wait lasts at most one phase of one iteration.
constexpr long long kBarrierBudget = 4000000000LL;

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned int* p, unsigned int v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile_int(const int* p) { return *(volatile const int*)p; }

// Grid-wide barrier for a co-resident (cooperative) grid.  bar->count counts
// arrivals and bar->gen completed barriers since both were zeroed, so after g
// barriers count = g x grid.  Each CTA keeps its own copy of gen in s_gen (read
// once at kernel start by grid_gen_init, when no barrier of the launch can have
// completed: that needs this CTA's arrival), so an arrival is one atomic add;
// the CTA whose add brings count to (g + 1) x grid completes the barrier by
// releasing gen = g + 1, and the others wait for that (unsigned arithmetic wraps
// consistently).  Every wait is bounded: on expiry the CTA records
// GRBK_ETIMEOUT and the barrier returns false, as it does when it sees, while
// waiting, that any CTA has recorded an error; callers then leave the kernel.
// s_ok and s_gen must be __shared__.
__device__ __forceinline__ void grid_gen_init(const GridBarrier* bar, unsigned int& s_gen)
{
    if (threadIdx.x == 0) s_gen = ld_acquire_u32(&bar->gen);
    __syncthreads();
}

__device__ __forceinline__ bool grid_sync(GridBarrier* bar, DevState* st, int site, int& s_ok, unsigned int& s_gen,
                                          long long budget = kBarrierBudget)
{
    __syncthreads();
    if (gridDim.x == 1) {  // a single CTA: the block barrier is the grid barrier
        if (threadIdx.x == 0) s_ok = (ld_volatile_int(&st->status) == 0);
        __syncthreads();
        return s_ok != 0;
    }
    if (threadIdx.x == 0) {
        // The block barrier orders the CTA's writes before thread 0's release
        // fence; the arrival is a relaxed atomic after it.  The completing CTA
        // fences again (acquire) before its release store; the waiters acquire.
        const unsigned int nb = gridDim.x;
        const unsigned int g = s_gen;
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        const unsigned int arrived = atomicAdd(&bar->count, 1u);
        int ok = 1;
        if (arrived == g * nb + (nb - 1u)) {
            asm volatile("fence.acq_rel.gpu;" ::: "memory");
            st_release_u32(&bar->gen, g + 1u);
        } else {
            const long long t0 = clock64();
            for (;;) {
                const int sv = ld_volatile_int(&st->status);  // issued before the acquire load
                if (ld_acquire_u32(&bar->gen) != g) break;
                if (sv != 0) { ok = 0; break; }
                if (clock64() - t0 > budget) {
                    if (atomicCAS(&st->status, 0, (int)GRBK_ETIMEOUT) == 0) st->timeout_site = site;
                    ok = 0;
                    break;
                }
                __nanosleep(32);  // polling without a pause slows the CTAs still working
            }
        }
        s_gen = g + 1u;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ----------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): key (seed, 0), counter
// (k, sys, stream, 0); u = top 53 bits of the first output word times 2^-53.
// Stream 0 draws the row picks, stream 1 the extended method's columns.
// ----------------------------------------------------------------------------
__device__ __forceinline__ double philox_uniform(uint64_t seed, uint64_t k, uint64_t sys, uint64_t stream = 0)
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t x0 = k, x1 = sys, x2 = stream, x3 = 0, k0 = seed, k1 = 0;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t hi0 = __umul64hi(M0, x0), lo0 = M0 * x0;
        const uint64_t hi1 = __umul64hi(M1, x2), lo1 = M1 * x2;
        const uint64_t y0 = hi1 ^ x1 ^ k0;
        const uint64_t y2 = hi0 ^ x3 ^ k1;
        x0 = y0;
        x1 = lo1;
        x2 = y2;
        x3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    return (double)(x0 >> 11) * 0x1.0p-53;
}

// ----------------------------------------------------------------------------
// warp helpers
// ----------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Double-float (hi + lo) sum across the warp, in FP32 arithmetic only: each
// step adds two (hi, lo) pairs with Knuth's two-sum and renormalises.  Keeps
// about 44 bits without touching the FP64 pipe (1/64 of the FP32 rate here).
__device__ __forceinline__ void warp_sum_df(float& hi, float& lo)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float bh = __shfl_xor_sync(0xffffffffu, hi, o);
        const float bl = __shfl_xor_sync(0xffffffffu, lo, o);
        const float s = __fadd_rn(hi, bh);
        const float bb = __fsub_rn(s, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
        const float l = __fadd_rn(__fadd_rn(err, lo), bl);
        hi = __fadd_rn(s, l);
        lo = __fsub_rn(l, __fsub_rn(hi, s));
    }
}

// argmax of (val, idx) pairs; ties go to the smaller index.
__device__ __forceinline__ void warp_argmax(double& v, long long& i)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const long long oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (ov > v || (ov == v && oi < i)) {
            v = ov;
            i = oi;
        }
    }
}

// argmax of signed integer keys across the warp (ties: smallest index); every lane
// ends with the result
__device__ __forceinline__ void warp_argmax_key(long long& key, long long& i)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long ok = __shfl_xor_sync(0xffffffffu, key, o);
        const long long oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (ok > key || (ok == key && oi < i)) {
            key = ok;
            i = oi;
        }
    }
}

// The bit pattern of a double read as a signed integer: for values >= +0 and -inf
// the integer order is the numeric order, so comparisons of row norms, ratios and
// their sums can run on the integer pipe instead of the (slow) FP64 pipe.
__device__ __forceinline__ long long dkey(double v) { return __double_as_longlong(v); }

// inclusive scan across the warp (fixed order)
__device__ __forceinline__ double warp_inclusive_scan(double v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// ----------------------------------------------------------------------------
// internal launchers implemented in other translation units
// ----------------------------------------------------------------------------

// Cout = beta * Cin + alpha * A * B (row-major; M x K times K x N), SIMT.
template <typename T>
cudaError_t gemm_simt(int64_t M, int64_t N, int64_t K, double alpha, const T* A, int64_t lda,
                      const T* B, int64_t ldb, double beta, const T* Cin, int64_t ldcin, T* Cout,
                      int64_t ldc, cudaStream_t st);

// G = A A^T (M x M, row stride ldg) for A (M x K, row stride lda), SIMT.
template <typename T>
cudaError_t gram_simt(int64_t M, int64_t K, const T* A, int64_t lda, T* G, int64_t ldg, cudaStream_t st);

// dst(rows x cols, ldd) of type Td <- src(rows x cols, lds) of type Ts, device to device.
cudaError_t convert_matrix(void* dst, int dtd, int64_t ldd, const void* src, int dts, int64_t lds,
                           int64_t rows, int64_t cols, cudaStream_t st);

// Split-BF16 tensor-core refresh engine (tcgen05 + TMA), FP32 mode.
struct SplitGemm;
grbk_status splitgemm_create(SplitGemm** out, int64_t m, int64_t p, int64_t q, int64_t n,
                             const float* A, int64_t lda, const float* B, int64_t ldb, int terms,
                             cudaStream_t st);
// R = C - A X B with X (p x q FP64 row-major, ldx); C and R are m x n (ld ldr).
grbk_status splitgemm_residual(SplitGemm* g, const double* X, int64_t ldx, const float* C,
                               float* R, int64_t ldr, cudaStream_t st);
void splitgemm_destroy(SplitGemm* g);
// G = A A^T (m x m, row stride ldg) with the split-BF16 tensor-core GEMM
grbk_status splitgemm_gram(SplitGemm* g, float* G, int64_t ldg, cudaStream_t st);
// reads the device error flag of the tensor-core kernels (GRBK_ETIMEOUT if a wait expired)
grbk_status splitgemm_check(SplitGemm* g, cudaStream_t st);
// kernel launches made by one splitgemm_residual call
int splitgemm_launches(const SplitGemm* g);

// 3x3 convolution, zero padding 1, on the tensor cores (grbk_gemm.cu): input planes
// xs = [3 terms][nimg][H][W][Cp] BF16 (NHWC, Cp a multiple of 64, a three-term split of
// the FP32 activations), weights wtc = [Npad][9 taps][Cp] BF16 (Npad a multiple of 16,
// at most 128); out[n][out_c0 + o][y][x] (NCHW FP32, out_ctot channels) = bias[o] +
// sum over taps and channels, then ReLU when relu != 0, for o < Cout.  err: device
// flag set when a bounded wait expires.  halo: images at least 128 pixels wide
// take the variant that loads each kernel row's 130 input pixels once for its
// three taps.
grbk_status tc_conv3x3(const void* xs, int nimg, int H, int W, int Cp, const void* wtc, int Npad, int Cout,
                       const float* bias, int relu, float* out, int out_ctot, int out_c0, int* err, cudaStream_t st,
                       bool halo);
// whether an H x W image fits the tensor-core convolution's 128-pixel tile (its rows
// of a power-of-two width up to 128 stack no higher than H)
bool tc_conv_fits(int H, int W);

// Row-space form set-up (grbk_rowspace.cu): from B (q x n, ldb) and C (m x n,
// ldc) in the working precision, the rank r of B, Lt (q x r, compact, with
// Lt Lt^T = B B^T), Chat = C Bt^T (m x r, compact), K = Lt^T Lt (r x r) and
// the FP64 row offsets ||Rperp_i||^2 (m).  The four arrays are cudaMalloc'ed
// for the caller.
struct RowspaceResult {
    int64_t r;
    void* Lt;
    void* Chat;
    double* rperp;
    void* K;        // Lt^T Lt (r x r, compact)
    long long launches;
};
grbk_status rowspace_transform(bool fp64, int64_t m, int64_t q, int64_t n, const void* B, int64_t ldb,
                               const void* C, int64_t ldc, double tol_rel, cudaStream_t st, RowspaceResult* out);

}  // namespace grbk
