// grbk_gemm.cu -- dense products for the residual refresh R = C - A X B
// (Algorithm 3 initialisation, repeated every refresh period): a tiled SIMT
// GEMM used in FP64 mode, and the FP32-mode refresh engine.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>
#include <algorithm>

#include "grbk_internal.cuh"

namespace grbk {

// Cout = beta * Cin + alpha * A(MxK) * B(KxN); 64x64 tiles, 16x16 threads, 4x4 per thread.
// BT: B is given as its transpose (N x K, row stride ldb), e.g. A A^T with B = A.
template <typename T, bool BT>
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
            Bs[kk][cc] = (gk < K && gc < N) ? (BT ? B[gc * ldb + gk] : B[gk * ldb + gc]) : (T)0;
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
    gemm_simt_kernel<T, false><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, Cin, ldcin, Cout, ldc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t gram_simt(int64_t M, int64_t K, const T* A, int64_t lda, T* G, int64_t ldg, cudaStream_t st)
{
    if (M <= 0) return cudaSuccess;
    dim3 grid((unsigned)((M + 63) / 64), (unsigned)((M + 63) / 64));
    gemm_simt_kernel<T, true><<<grid, 256, 0, st>>>(M, M, K, 1.0, A, lda, A, lda, 0.0, nullptr, 0, G, ldg);
    return cudaGetLastError();
}
template cudaError_t gram_simt<double>(int64_t, int64_t, const double*, int64_t, double*, int64_t, cudaStream_t);
template cudaError_t gram_simt<float>(int64_t, int64_t, const float*, int64_t, float*, int64_t, cudaStream_t);

template cudaError_t gemm_simt<double>(int64_t, int64_t, int64_t, double, const double*, int64_t,
                                       const double*, int64_t, double, const double*, int64_t, double*,
                                       int64_t, cudaStream_t);
template cudaError_t gemm_simt<float>(int64_t, int64_t, int64_t, double, const float*, int64_t,
                                      const float*, int64_t, double, const float*, int64_t, float*,
                                      int64_t, cudaStream_t);

// ----------------------------------------------------------------------------
// FP32-mode refresh engine: R = C - (A X) B with split-BF16 operands on the
// 5th-generation tensor cores (tcgen05.mma, accumulators in TMEM, operands
// staged by TMA with 128-byte swizzle).
//
// Each FP32 (or FP64) operand x is split into BF16 terms x = x0 + x1 (+ x2)
// with x0 = bf16(x), x1 = bf16(x - x0), x2 = bf16(x - x0 - x1); a product is
// the sum of the cross terms whose orders add up to at most terms-1
// (2 terms: x0 y0 + x0 y1 + x1 y0; 3 terms adds x0 y2 + x2 y0 + x1 y1),
// accumulated in FP32.  The terms are stored as [term][rows][Kpad] planes
// (K contiguous, zero padded to a multiple of 64) so that one 3-D tensor map
// serves every term; the kernel walks (term pair, K block) in one
// accumulation chain.
// ----------------------------------------------------------------------------
namespace tc {

// Tile: BM x BN(TERMS) outputs, K blocks of BK.  A pipeline stage holds every
// split term of one K block of both operands, and the MMA issuer runs all term
// pairs from that stage, so each operand tile crosses L2 once per K block.
// 2 terms: BN = 256, stage = 2 x (16 + 32) KB; 3 terms: BN = 128, stage =
// 3 x (16 + 16) KB.  Two stages (192 KB).
constexpr int BM = 128, BK = 64, STAGES = 2;
constexpr int A_TILE = BM * BK * 2;            // 16 KB per term
template <int TERMS> struct Cfg {
    static constexpr int BN = TERMS == 2 ? 256 : 128;
    static constexpr int B_TILE = BN * BK * 2;
    static constexpr int STAGE_BYTES = TERMS * (A_TILE + B_TILE);
    static constexpr int NPAIRS = TERMS == 2 ? 3 : 6;
};
constexpr int SMEM_BYTES = STAGES * 98304 + 1024 + 256;
static_assert(Cfg<2>::STAGE_BYTES == 98304 && Cfg<3>::STAGE_BYTES == 98304, "stage size");
constexpr int BN_MAX = 256;                    // plane rows are padded to this
constexpr long long kWaitBudget = 2000000000LL;  // cycles (about 1 s)

enum { EPI_SPLIT = 0, EPI_RESID = 1, EPI_STORE = 2 };

struct Args {
    int M, N, K;                 // K: padded inner size (multiple of BK)
    int mode;
    int out_terms;               // EPI_SPLIT: terms written
    int out_rows;                // EPI_SPLIT: rows per output plane (>= M)
    __nv_bfloat16* out_split;    // [out_terms][out_rows][out_ld]
    int64_t out_ld;
    const float* cin;            // EPI_RESID: out = cin - D
    float* out;
    int64_t ld;
    int* err;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// bounded wait for the phase with the given parity; false on expiry
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > kWaitBudget) return false;
    }
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;               // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;     // stride byte offset
    d |= (uint64_t)1 << 46;               // descriptor version
    d |= (uint64_t)2 << 61;               // 128-byte swizzle
    return d;
}

// instruction descriptor, kind::f16: BF16 x BF16 -> FP32, both K-major, BM x N
__host__ __device__ constexpr uint32_t idesc_for(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// term pairs, smallest cross terms first so the FP32 accumulator adds them before the large ones:
// 2 terms: x0 y1, x1 y0, x0 y0;  3 terms: x1 y1, x2 y0, x0 y2, x1 y0, x0 y1, x0 y0
__device__ __forceinline__ void pair_terms(int terms, int p, int& ta, int& tb)
{
    const int a2[3] = {0, 1, 0}, b2[3] = {1, 0, 0};
    const int a3[6] = {1, 2, 0, 1, 0, 0}, b3[6] = {1, 0, 2, 0, 1, 0};
    ta = terms == 2 ? a2[p] : a3[p];
    tb = terms == 2 ? b2[p] : b3[p];
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void split_f(float x, int terms, __nv_bfloat16* t)
{
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    t[0] = h;
    const float r1 = x - __bfloat162float(h);
    const __nv_bfloat16 l = __float2bfloat16_rn(r1);
    t[1] = l;
    if (terms > 2) t[2] = __float2bfloat16_rn(r1 - __bfloat162float(l));
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// D[M x N] = sum over term pairs of A_ta[M x K] * B_tb[N x K]^T, persistent:
// each CTA walks output tiles blockIdx.x, blockIdx.x + gridDim.x, ... (tile
// index = m_block * n_blocks + n_block).  Two TMEM accumulators let the
// epilogue of one tile run while the MMAs of the next are issued.
// 256 threads: warp 0 = TMA producer, warp 1 = MMA issuer, warp 2 = TMEM owner,
// warps 4-7 = epilogue.  Barriers: full/empty per smem stage, acc_full/acc_empty
// per accumulator (acc_empty counts the 4 epilogue warps), done (all MMAs).
template <int TERMS>
__global__ void __launch_bounds__(256, 1) gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                                                      const __grid_constant__ CUtensorMap tmB, Args g)
{
    constexpr int BN = Cfg<TERMS>::BN, B_TILE = Cfg<TERMS>::B_TILE, STAGE_BYTES = Cfg<TERMS>::STAGE_BYTES;
    constexpr int TMEM_COLS = 2 * BN;
    constexpr uint32_t IDESC = idesc_for(BN);
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    // stage s: [A term 0 .. TERMS-1][B term 0 .. TERMS-1]
    auto sA = [&](int s, int t) { return smem + s * STAGE_BYTES + t * A_TILE; };
    auto sB = [&](int s, int t) { return smem + s * STAGE_BYTES + TERMS * A_TILE + t * B_TILE; };
    uint64_t* bars = (uint64_t*)(smem + STAGES * STAGE_BYTES);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES);
    const uint32_t accf0 = smem_u32(bars + 2 * STAGES), acce0 = smem_u32(bars + 2 * STAGES + 2);
    const uint32_t done = smem_u32(bars + 2 * STAGES + 4);
    uint32_t* tmem_slot = (uint32_t*)(bars + 2 * STAGES + 5);
    __shared__ int s_abort;

    // a CTA that finds the error flag already set (an earlier CTA's wait
    // expired) leaves at once, before touching barriers or TMEM
    if (*(volatile int*)g.err != 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nkb = g.K / BK;
    const int n_blocks = (g.N + BN - 1) / BN, m_blocks = (g.M + BM - 1) / BM;
    const int ntiles = n_blocks * m_blocks;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(accf0 + 8 * a, 1);
            mbar_init(acce0 + 8 * a, 4);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *(volatile uint32_t*)tmem_slot;

    if (warp == 0 && lane == 0) {
        int issued = 0;
        bool stop = false;
        for (int tile = blockIdx.x; tile < ntiles && !stop; tile += gridDim.x) {
            const int m0 = (tile / n_blocks) * BM, n0 = (tile % n_blocks) * BN;
            for (int kb = 0; kb < nkb; ++kb) {
                const int it = issued;
                const int s = it % STAGES;
                const uint32_t ph = (uint32_t)((it / STAGES) & 1);
                if (!mbar_wait(empty0 + 8 * s, ph ^ 1u)) { s_abort = 1; stop = true; break; }
                if (*(volatile int*)&s_abort) { stop = true; break; }
                mbar_expect_tx(full0 + 8 * s, STAGE_BYTES);
#pragma unroll
                for (int t = 0; t < TERMS; ++t) {
                    tma_load_3d(smem_u32(sA(s, t)), &tmA, kb * BK, m0, t, full0 + 8 * s);
                    tma_load_3d(smem_u32(sB(s, t)), &tmB, kb * BK, n0, t, full0 + 8 * s);
                }
                ++issued;
            }
        }
        // wait (bounded) for this CTA's copies still in flight before anyone leaves
        for (int it = (issued > STAGES ? issued - STAGES : 0); it < issued; ++it)
            mbar_wait(full0 + 8 * (it % STAGES), (uint32_t)((it / STAGES) & 1));
    } else if (warp == 1 && lane == 0) {
        int it = 0, lt = 0;
        bool stop = false;
        for (int tile = blockIdx.x; tile < ntiles && !stop; tile += gridDim.x, ++lt) {
            const int acc = lt & 1;
            // the epilogue has drained this accumulator (first two tiles pass at once)
            if (!mbar_wait(acce0 + 8 * acc, (uint32_t)(((lt >> 1) & 1) ^ 1))) { s_abort = 1; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t dacc = tmem + (uint32_t)(acc * BN);
            for (int kb = 0; kb < nkb; ++kb, ++it) {
                const int s = it % STAGES;
                const uint32_t ph = (uint32_t)((it / STAGES) & 1);
                if (!mbar_wait(full0 + 8 * s, ph)) { s_abort = 1; stop = true; break; }
                if (*(volatile int*)&s_abort) { stop = true; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int p = 0; p < Cfg<TERMS>::NPAIRS; ++p) {
                    int ta, tb;
                    pair_terms(TERMS, p, ta, tb);
                    const uint32_t a0 = smem_u32(sA(s, ta)), b0 = smem_u32(sB(s, tb));
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk)
                        mma_bf16(dacc, sdesc(a0 + kk * 32), sdesc(b0 + kk * 32), IDESC,
                                 (kb > 0 || p > 0 || kk > 0) ? 1u : 0u);
                }
                mma_commit(empty0 + 8 * s);
            }
            if (!stop) mma_commit(accf0 + 8 * acc);  // this tile's accumulator is complete
        }
        mma_commit(done);  // arrives once every MMA issued above has completed
    } else if (warp >= 4) {
        const int e = warp - 4;
        int lt = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++lt) {
            const int acc = lt & 1;
            const bool ok = mbar_wait(accf0 + 8 * acc, (uint32_t)((lt >> 1) & 1));
            if (!ok || *(volatile int*)&s_abort) { s_abort = 1; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int m0 = (tile / n_blocks) * BM, n0 = (tile % n_blocks) * BN;
            const int row = m0 + e * 32 + lane;
            for (int cb = 0; cb < BN; cb += 32) {
                uint32_t r[32];
                tmem_ld32(tmem + (uint32_t)(acc * BN) + ((uint32_t)(e * 32) << 16) + (uint32_t)cb, r);
                if (row >= g.M || n0 + cb >= g.N) continue;
                const int col0 = n0 + cb;
                const bool full = col0 + 32 <= g.N;
                if (g.mode == EPI_RESID || g.mode == EPI_STORE) {
                    const bool resid = g.mode == EPI_RESID;
                    const float* ci = resid ? g.cin + (int64_t)row * g.ld + col0 : nullptr;
                    float* oi = g.out + (int64_t)row * g.ld + col0;
                    if (full) {
#pragma unroll
                        for (int j = 0; j < 32; j += 4) {
                            float4 ov;
                            if (resid) {
                                const float4 cv = __ldg(reinterpret_cast<const float4*>(ci + j));
                                ov.x = cv.x - __uint_as_float(r[j]);
                                ov.y = cv.y - __uint_as_float(r[j + 1]);
                                ov.z = cv.z - __uint_as_float(r[j + 2]);
                                ov.w = cv.w - __uint_as_float(r[j + 3]);
                            } else {
                                ov = make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                                                 __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]));
                            }
                            *reinterpret_cast<float4*>(oi + j) = ov;
                        }
                    } else {
                        for (int j = 0; j < 32 && col0 + j < g.N; ++j)
                            oi[j] = resid ? ci[j] - __uint_as_float(r[j]) : __uint_as_float(r[j]);
                    }
                } else if (full) {
                    // this lane's 32 columns of each term plane are 64 contiguous bytes
                    // (the split planes have as many terms as the operands: out_terms == TERMS)
#pragma unroll
                    for (int tt = 0; tt < TERMS; ++tt) {
                        uint4* dst = reinterpret_cast<uint4*>(g.out_split + ((int64_t)tt * g.out_rows + row) * g.out_ld +
                                                              col0);
#pragma unroll
                        for (int q4 = 0; q4 < 4; ++q4) {
                            uint32_t w4[4];
#pragma unroll
                            for (int h = 0; h < 4; ++h) {
                                __nv_bfloat16 t0[3], t1[3];
                                split_f(__uint_as_float(r[q4 * 8 + 2 * h]), TERMS, t0);
                                split_f(__uint_as_float(r[q4 * 8 + 2 * h + 1]), TERMS, t1);
                                w4[h] = (uint32_t)__bfloat16_as_ushort(t0[tt]) |
                                        ((uint32_t)__bfloat16_as_ushort(t1[tt]) << 16);
                            }
                            dst[q4] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
                        }
                    }
                } else {
                    for (int j = 0; j < 32 && col0 + j < g.N; ++j) {
                        __nv_bfloat16 t[3];
                        split_f(__uint_as_float(r[j]), g.out_terms, t);
                        for (int tt = 0; tt < g.out_terms; ++tt)
                            g.out_split[((int64_t)tt * g.out_rows + row) * g.out_ld + col0 + j] = t[tt];
                    }
                }
            }
            // hand the accumulator back to the MMA issuer
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(acce0 + 8 * acc);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0 && *(volatile int*)&s_abort) atomicExch(g.err, 1);
    if (warp == 2) {
        // every MMA this CTA issued has completed before the columns are freed
        mbar_wait(done, 0);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// planes [terms][rows][Kpad] of the split of src rows (src[r][k], k < K); K..Kpad-1 left as zeros
template <typename S>
__global__ void split_rows_kernel(const S* src, int64_t ld, int64_t rows, int64_t K, int64_t Kpad, int terms,
                                  int64_t plane_rows, __nv_bfloat16* dst)
{
    const int64_t total = rows * K;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / K, k = e % K;
        const double x = (double)src[r * ld + k];
        const __nv_bfloat16 h = __double2bfloat16(x);
        const double r1 = x - (double)__bfloat162float(h);
        const __nv_bfloat16 l = __double2bfloat16(r1);
        dst[r * Kpad + k] = h;
        dst[(plane_rows + r) * Kpad + k] = l;
        if (terms > 2) dst[(2 * plane_rows + r) * Kpad + k] = __double2bfloat16(r1 - (double)__bfloat162float(l));
    }
}

// planes [terms][N][Kpad] of the split of src^T (src is K x N, row stride ld)
template <typename S>
__global__ void split_transpose_kernel(const S* src, int64_t ld, int64_t K, int64_t N, int64_t Kpad, int terms,
                                       int64_t plane_rows, __nv_bfloat16* dst)
{
    __shared__ double tile[32][33];
    const int64_t k0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int64_t k = k0 + dy, j = j0 + threadIdx.x;
        tile[dy][threadIdx.x] = (k < K && j < N) ? (double)src[k * ld + j] : 0.0;
    }
    __syncthreads();
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int64_t j = j0 + dy, k = k0 + threadIdx.x;
        if (j < N && k < K) {
            const double x = tile[threadIdx.x][dy];
            const __nv_bfloat16 h = __double2bfloat16(x);
            const double r1 = x - (double)__bfloat162float(h);
            const __nv_bfloat16 l = __double2bfloat16(r1);
            dst[j * Kpad + k] = h;
            dst[(plane_rows + j) * Kpad + k] = l;
            if (terms > 2) dst[(2 * plane_rows + j) * Kpad + k] = __double2bfloat16(r1 - (double)__bfloat162float(l));
        }
    }
}


// ----------------------------------------------------------------------------
// 3x3 convolution with zero padding 1 as an implicit GEMM on the tensor cores
// (the warm-start network's convolutions).  Activations are NHWC BF16 planes
// [term][image][H][W][Cp] holding a three-term split of the FP32 values
// (x = x0 + x1 + x2, about 24 significant bits in all); weights are one BF16
// term (they are BF16 already), laid out [Npad][tap][Cp].  An output tile is
// 128 pixels (boxh rows of boxw columns) by Npad output channels, accumulated
// in TMEM over K = 9 taps x Cp channels: for tap (dy, dx) the A operand is the
// input tile shifted by (dy, dx), loaded by a 4-D TMA whose out-of-range
// coordinates fill zeros -- the zero padding costs nothing.  Persistent CTAs,
// two smem stages, two TMEM accumulators so the epilogue (bias, ReLU, NCHW
// FP32 store) of one tile overlaps the MMAs of the next.
// ----------------------------------------------------------------------------
constexpr int CONV_TERMS = 3;
constexpr int CONV_STAGES = 2;
constexpr int CONV_A_BYTES = CONV_TERMS * A_TILE;                 // 48 KB
constexpr int CONV_STAGE_BYTES = CONV_A_BYTES + 128 * BK * 2;       // + B for up to 128 channels
constexpr int CONV_SMEM_BYTES = CONV_STAGES * CONV_STAGE_BYTES + 1024 + 256;

struct ConvArgs {
    int nimg, H, W, Cp, Npad, Cout;
    int boxw, boxh, tiles_x, tiles_y;
    int tmem_cols;                   // two accumulators, the second at column tmem_cols / 2
    const float* bias;
    int relu;
    float* out;
    int out_ctot, out_c0;
    int* err;
};

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

__global__ void __launch_bounds__(256, 1) conv_tc_kernel(const __grid_constant__ CUtensorMap tmX,
                                                         const __grid_constant__ CUtensorMap tmW, ConvArgs g)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    auto sA = [&](int s, int t) { return smem + s * CONV_STAGE_BYTES + t * A_TILE; };
    auto sB = [&](int s) { return smem + s * CONV_STAGE_BYTES + CONV_A_BYTES; };
    uint64_t* bars = (uint64_t*)(smem + CONV_STAGES * CONV_STAGE_BYTES);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + CONV_STAGES);
    const uint32_t accf0 = smem_u32(bars + 2 * CONV_STAGES), acce0 = smem_u32(bars + 2 * CONV_STAGES + 2);
    const uint32_t done = smem_u32(bars + 2 * CONV_STAGES + 4);
    uint32_t* tmem_slot = (uint32_t*)(bars + 2 * CONV_STAGES + 5);
    __shared__ int s_abort;

    if (*(volatile int*)g.err != 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nkc = g.Cp / BK;
    const int nkb = 9 * nkc;
    const int ntiles = g.nimg * g.tiles_y * g.tiles_x;
    const uint32_t idesc = idesc_for(g.Npad);
    const uint32_t stage_tx = (uint32_t)(CONV_A_BYTES + g.Npad * BK * 2);

    if (threadIdx.x == 0) {
        for (int s = 0; s < CONV_STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(accf0 + 8 * a, 1);
            mbar_init(acce0 + 8 * a, 4);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(g.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *(volatile uint32_t*)tmem_slot;

    auto tile_origin = [&](int tile, int& n, int& y0, int& x0) {
        const int per = g.tiles_y * g.tiles_x;
        n = tile / per;
        const int r = tile % per;
        y0 = (r / g.tiles_x) * g.boxh;
        x0 = (r % g.tiles_x) * g.boxw;
    };

    if (warp == 0 && lane == 0) {
        int issued = 0;
        bool stop = false;
        for (int tile = blockIdx.x; tile < ntiles && !stop; tile += gridDim.x) {
            int n, y0, x0;
            tile_origin(tile, n, y0, x0);
            for (int kb = 0; kb < nkb; ++kb) {
                const int tap = kb / nkc, kc = kb % nkc;
                const int dy = tap / 3 - 1, dx = tap % 3 - 1;
                const int s = issued % CONV_STAGES;
                const uint32_t ph = (uint32_t)((issued / CONV_STAGES) & 1);
                if (!mbar_wait(empty0 + 8 * s, ph ^ 1u)) { s_abort = 1; stop = true; break; }
                if (*(volatile int*)&s_abort) { stop = true; break; }
                mbar_expect_tx(full0 + 8 * s, stage_tx);
#pragma unroll
                for (int t = 0; t < CONV_TERMS; ++t)
                    tma_load_4d(smem_u32(sA(s, t)), &tmX, kc * BK, x0 + dx, y0 + dy, t * g.nimg + n, full0 + 8 * s);
                tma_load_2d(smem_u32(sB(s)), &tmW, tap * g.Cp + kc * BK, 0, full0 + 8 * s);
                ++issued;
            }
        }
        for (int it = (issued > CONV_STAGES ? issued - CONV_STAGES : 0); it < issued; ++it)
            mbar_wait(full0 + 8 * (it % CONV_STAGES), (uint32_t)((it / CONV_STAGES) & 1));
    } else if (warp == 1 && lane == 0) {
        int it = 0, lt = 0;
        bool stop = false;
        for (int tile = blockIdx.x; tile < ntiles && !stop; tile += gridDim.x, ++lt) {
            const int acc = lt & 1;
            if (!mbar_wait(acce0 + 8 * acc, (uint32_t)(((lt >> 1) & 1) ^ 1))) { s_abort = 1; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t dacc = tmem + (uint32_t)(acc * (g.tmem_cols / 2));
            for (int kb = 0; kb < nkb; ++kb, ++it) {
                const int s = it % CONV_STAGES;
                const uint32_t ph = (uint32_t)((it / CONV_STAGES) & 1);
                if (!mbar_wait(full0 + 8 * s, ph)) { s_abort = 1; stop = true; break; }
                if (*(volatile int*)&s_abort) { stop = true; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t b0 = smem_u32(sB(s));
                // the smallest terms first, so the FP32 accumulator adds them before the large one
#pragma unroll
                for (int t = CONV_TERMS - 1; t >= 0; --t) {
                    const uint32_t a0 = smem_u32(sA(s, t));
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk)
                        mma_bf16(dacc, sdesc(a0 + kk * 32), sdesc(b0 + kk * 32), idesc,
                                 (kb > 0 || t < CONV_TERMS - 1 || kk > 0) ? 1u : 0u);
                }
                mma_commit(empty0 + 8 * s);
            }
            if (!stop) mma_commit(accf0 + 8 * acc);
        }
        mma_commit(done);
    } else if (warp >= 4) {
        const int e = warp - 4;
        int lt = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++lt) {
            const int acc = lt & 1;
            const bool ok = mbar_wait(accf0 + 8 * acc, (uint32_t)((lt >> 1) & 1));
            if (!ok || *(volatile int*)&s_abort) { s_abort = 1; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            int n, y0, x0;
            tile_origin(tile, n, y0, x0);
            const int r = e * 32 + lane;
            const int y = y0 + r / g.boxw, x = x0 + r % g.boxw;
            const bool valid = y < g.H && x < g.W;
            float* obase = g.out + (((int64_t)n * g.out_ctot + g.out_c0) * g.H + y) * g.W + x;
            const int64_t cstride = (int64_t)g.H * g.W;
            for (int cb = 0; cb < g.Npad; cb += 32) {
                uint32_t v[32];
                tmem_ld32(tmem + (uint32_t)(acc * (g.tmem_cols / 2)) + ((uint32_t)(e * 32) << 16) + (uint32_t)cb, v);
                if (!valid) continue;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int o = cb + j;
                    if (o >= g.Cout) break;
                    float val = __uint_as_float(v[j]) + (g.bias ? g.bias[o] : 0.f);
                    if (g.relu) val = fmaxf(val, 0.f);
                    obase[(int64_t)o * cstride] = val;
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(acce0 + 8 * acc);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0 && *(volatile int*)&s_abort) atomicExch(g.err, 1);
    if (warp == 2) {
        mbar_wait(done, 0);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(g.tmem_cols) : "memory");
    }
}

// Variant for images at least 128 pixels wide: a tile is 128 pixels of one
// image row, and for each kernel row dy one TMA brings the 130 input pixels
// the three taps (dy, -1..1) need (one halo pixel on each side, zeros past the
// image).  The three A operands are that smem tile read from rows 0, 1 and 2:
// start addresses one 128-byte row apart.  The TMA writes the 128-byte swizzle
// as a function of the shared-memory address (the tile starts on a 1024-byte
// boundary), and the MMA unswizzles by address in the same way, so a shifted
// start needs no other change.  Each input pixel crosses L2 three times per
// term instead of nine.
constexpr int HALO_ROWS = 130;
constexpr int HALO_TERM_BYTES = 17 * 1024;                          // 130 rows of 128 B, 1024-aligned
constexpr int HALO_A_BYTES = CONV_TERMS * HALO_TERM_BYTES;          // 51 KB
constexpr int HALO_STAGE_BYTES = HALO_A_BYTES + 3 * 128 * BK * 2;   // + three taps of B, up to 128 channels
constexpr int HALO_SMEM_BYTES = CONV_STAGES * HALO_STAGE_BYTES + 1024 + 256;

__global__ void __launch_bounds__(256, 1) conv_tc_halo_kernel(const __grid_constant__ CUtensorMap tmX,
                                                              const __grid_constant__ CUtensorMap tmW, ConvArgs g)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    auto sA = [&](int s, int t) { return smem + s * HALO_STAGE_BYTES + t * HALO_TERM_BYTES; };
    auto sB = [&](int s, int j) { return smem + s * HALO_STAGE_BYTES + HALO_A_BYTES + j * (g.Npad * BK * 2); };
    uint64_t* bars = (uint64_t*)(smem + CONV_STAGES * HALO_STAGE_BYTES);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + CONV_STAGES);
    const uint32_t accf0 = smem_u32(bars + 2 * CONV_STAGES), acce0 = smem_u32(bars + 2 * CONV_STAGES + 2);
    const uint32_t done = smem_u32(bars + 2 * CONV_STAGES + 4);
    uint32_t* tmem_slot = (uint32_t*)(bars + 2 * CONV_STAGES + 5);
    __shared__ int s_abort;

    if (*(volatile int*)g.err != 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nkc = g.Cp / BK;
    const int nkb = 3 * nkc;                      // (dy, channel chunk)
    const int ntiles = g.nimg * g.H * g.tiles_x;  // one tile = 128 pixels of one row
    const uint32_t idesc = idesc_for(g.Npad);
    const uint32_t stage_tx = (uint32_t)(CONV_TERMS * HALO_ROWS * 128 + 3 * g.Npad * BK * 2);

    if (threadIdx.x == 0) {
        for (int s = 0; s < CONV_STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(accf0 + 8 * a, 1);
            mbar_init(acce0 + 8 * a, 4);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(g.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *(volatile uint32_t*)tmem_slot;

    auto tile_origin = [&](int tile, int& n, int& y0, int& x0) {
        const int per = g.H * g.tiles_x;
        n = tile / per;
        const int r = tile % per;
        y0 = r / g.tiles_x;
        x0 = (r % g.tiles_x) * 128;
    };

    if (warp == 0 && lane == 0) {
        int issued = 0;
        bool stop = false;
        for (int tile = blockIdx.x; tile < ntiles && !stop; tile += gridDim.x) {
            int n, y0, x0;
            tile_origin(tile, n, y0, x0);
            for (int kb = 0; kb < nkb; ++kb) {
                const int dyi = kb / nkc, kc = kb % nkc;    // dy = dyi - 1
                const int s = issued % CONV_STAGES;
                const uint32_t ph = (uint32_t)((issued / CONV_STAGES) & 1);
                if (!mbar_wait(empty0 + 8 * s, ph ^ 1u)) { s_abort = 1; stop = true; break; }
                if (*(volatile int*)&s_abort) { stop = true; break; }
                mbar_expect_tx(full0 + 8 * s, stage_tx);
#pragma unroll
                for (int t = 0; t < CONV_TERMS; ++t)
                    tma_load_4d(smem_u32(sA(s, t)), &tmX, kc * BK, x0 - 1, y0 + dyi - 1, t * g.nimg + n, full0 + 8 * s);
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    tma_load_2d(smem_u32(sB(s, j)), &tmW, (dyi * 3 + j) * g.Cp + kc * BK, 0, full0 + 8 * s);
                ++issued;
            }
        }
        for (int it = (issued > CONV_STAGES ? issued - CONV_STAGES : 0); it < issued; ++it)
            mbar_wait(full0 + 8 * (it % CONV_STAGES), (uint32_t)((it / CONV_STAGES) & 1));
    } else if (warp == 1 && lane == 0) {
        int it = 0, lt = 0;
        bool stop = false;
        for (int tile = blockIdx.x; tile < ntiles && !stop; tile += gridDim.x, ++lt) {
            const int acc = lt & 1;
            if (!mbar_wait(acce0 + 8 * acc, (uint32_t)(((lt >> 1) & 1) ^ 1))) { s_abort = 1; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t dacc = tmem + (uint32_t)(acc * (g.tmem_cols / 2));
            for (int kb = 0; kb < nkb; ++kb, ++it) {
                const int s = it % CONV_STAGES;
                const uint32_t ph = (uint32_t)((it / CONV_STAGES) & 1);
                if (!mbar_wait(full0 + 8 * s, ph)) { s_abort = 1; stop = true; break; }
                if (*(volatile int*)&s_abort) { stop = true; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 3; ++j) {           // dx = j - 1: A rows j .. j + 127
                    const uint32_t b0 = smem_u32(sB(s, j));
#pragma unroll
                    for (int t = CONV_TERMS - 1; t >= 0; --t) {
                        const uint32_t a0 = smem_u32(sA(s, t)) + (uint32_t)(j * 128);
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk)
                            mma_bf16(dacc, sdesc(a0 + kk * 32), sdesc(b0 + kk * 32), idesc,
                                     (kb > 0 || j > 0 || t < CONV_TERMS - 1 || kk > 0) ? 1u : 0u);
                    }
                }
                mma_commit(empty0 + 8 * s);
            }
            if (!stop) mma_commit(accf0 + 8 * acc);
        }
        mma_commit(done);
    } else if (warp >= 4) {
        const int e = warp - 4;
        int lt = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++lt) {
            const int acc = lt & 1;
            const bool ok = mbar_wait(accf0 + 8 * acc, (uint32_t)((lt >> 1) & 1));
            if (!ok || *(volatile int*)&s_abort) { s_abort = 1; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            int n, y0, x0;
            tile_origin(tile, n, y0, x0);
            const int x = x0 + e * 32 + lane;
            const bool valid = x < g.W;
            float* obase = g.out + (((int64_t)n * g.out_ctot + g.out_c0) * g.H + y0) * g.W + x;
            const int64_t cstride = (int64_t)g.H * g.W;
            for (int cb = 0; cb < g.Npad; cb += 32) {
                uint32_t v[32];
                tmem_ld32(tmem + (uint32_t)(acc * (g.tmem_cols / 2)) + ((uint32_t)(e * 32) << 16) + (uint32_t)cb, v);
                if (!valid) continue;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int o = cb + j;
                    if (o >= g.Cout) break;
                    float val = __uint_as_float(v[j]) + (g.bias ? g.bias[o] : 0.f);
                    if (g.relu) val = fmaxf(val, 0.f);
                    obase[(int64_t)o * cstride] = val;
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(acce0 + 8 * acc);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0 && *(volatile int*)&s_abort) atomicExch(g.err, 1);
    if (warp == 2) {
        mbar_wait(done, 0);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(g.tmem_cols) : "memory");
    }
}

}  // namespace tc

struct SplitGemm {
    int64_t m, p, q, n, lda, ldb;
    int terms;
    int64_t Kp, Kq;                 // p and q padded to multiples of 64
    int64_t mr, nr, qr;             // m padded to BM, n and q padded to BN (plane rows)
    __nv_bfloat16* As;              // [terms][mr][Kp]
    __nv_bfloat16* BTs;             // [terms][nr][Kq]
    __nv_bfloat16* XTs;             // [terms][qr][Kp]
    __nv_bfloat16* T1s;             // [terms][mr][Kq]
    CUtensorMap tmA, tmXT, tmT1, tmBT;
    CUtensorMap tmAn;               // A's planes as the N-side operand (for A A^T)
    int* err;
    int nsm;                        // persistent grid size
};

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 3-D map over [terms][rows][Kpad] BF16 planes, box 64 x box_rows x 1, 128-byte swizzle
static bool make_map(CUtensorMap* map, void* base, int64_t Kpad, int64_t rows, int terms, int box_rows)
{
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)Kpad, (cuuint64_t)rows, (cuuint64_t)terms};
    cuuint64_t strides[2] = {(cuuint64_t)(Kpad * 2), (cuuint64_t)(rows * Kpad * 2)};
    cuuint32_t box[3] = {(cuuint32_t)tc::BK, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

grbk_status splitgemm_create(SplitGemm** out, int64_t m, int64_t p, int64_t q, int64_t n, const float* A,
                             int64_t lda, const float* B, int64_t ldb, int terms, cudaStream_t st)
{
    SplitGemm* g = new SplitGemm();
    memset(g, 0, sizeof(*g));
    g->m = m; g->p = p; g->q = q; g->n = n; g->lda = lda; g->ldb = ldb; g->terms = terms;
    g->Kp = round_up(p, tc::BK);
    g->Kq = round_up(q, tc::BK);
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g->nsm, cudaDevAttrMultiProcessorCount, dev);
        if (g->nsm < 1) g->nsm = 1;
    }
    g->mr = round_up(m, tc::BN_MAX);   // A's planes also serve as the N-side operand of A A^T
    g->nr = round_up(n, tc::BN_MAX);
    g->qr = round_up(q, tc::BN_MAX);
    const size_t szA = (size_t)terms * g->mr * g->Kp * 2, szB = (size_t)terms * g->nr * g->Kq * 2;
    const size_t szX = (size_t)terms * g->qr * g->Kp * 2, szT = (size_t)terms * g->mr * g->Kq * 2;
    if (dev_alloc((void**)&g->As, szA) != cudaSuccess || dev_alloc((void**)&g->BTs, szB) != cudaSuccess ||
        dev_alloc((void**)&g->XTs, szX) != cudaSuccess || dev_alloc((void**)&g->T1s, szT) != cudaSuccess ||
        dev_alloc((void**)&g->err, sizeof(int)) != cudaSuccess) {
        splitgemm_destroy(g);
        return GRBK_ENOMEM;
    }
    if (cudaMemsetAsync(g->As, 0, szA, st) != cudaSuccess || cudaMemsetAsync(g->BTs, 0, szB, st) != cudaSuccess ||
        cudaMemsetAsync(g->XTs, 0, szX, st) != cudaSuccess || cudaMemsetAsync(g->T1s, 0, szT, st) != cudaSuccess ||
        cudaMemsetAsync(g->err, 0, sizeof(int), st) != cudaSuccess) {
        splitgemm_destroy(g);
        return GRBK_ECUDA;
    }
    tc::split_rows_kernel<float><<<2048, 256, 0, st>>>(A, lda, m, p, g->Kp, terms, g->mr, g->As);
    dim3 tb(32, 8), grd((unsigned)((n + 31) / 32), (unsigned)((q + 31) / 32));
    tc::split_transpose_kernel<float><<<grd, tb, 0, st>>>(B, ldb, q, n, g->Kq, terms, g->nr, g->BTs);
    if (cudaGetLastError() != cudaSuccess) { splitgemm_destroy(g); return GRBK_ECUDA; }
    const int bn = terms == 2 ? tc::Cfg<2>::BN : tc::Cfg<3>::BN;
    if (!make_map(&g->tmA, g->As, g->Kp, g->mr, terms, tc::BM) ||
        !make_map(&g->tmXT, g->XTs, g->Kp, g->qr, terms, bn) ||
        !make_map(&g->tmT1, g->T1s, g->Kq, g->mr, terms, tc::BM) ||
        !make_map(&g->tmBT, g->BTs, g->Kq, g->nr, terms, bn) ||
        !make_map(&g->tmAn, g->As, g->Kp, g->mr, terms, bn)) {
        splitgemm_destroy(g);
        return GRBK_ECUDA;
    }
    if (cudaFuncSetAttribute(tc::gemm_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES) !=
            cudaSuccess ||
        cudaFuncSetAttribute(tc::gemm_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES) !=
            cudaSuccess) {
        splitgemm_destroy(g);
        return GRBK_ECUDA;
    }
    *out = g;
    return GRBK_OK;
}

grbk_status splitgemm_residual(SplitGemm* g, const double* X, int64_t ldx, const float* C, float* R, int64_t ldr,
                               cudaStream_t st)
{
    // X^T terms: [terms][q][Kp] from X (p x q, FP64)
    dim3 tb(32, 8), grd((unsigned)((g->q + 31) / 32), (unsigned)((g->p + 31) / 32));
    tc::split_transpose_kernel<double><<<grd, tb, 0, st>>>(X, ldx, g->p, g->q, g->Kp, g->terms, g->qr, g->XTs);
    GRBK_CK(cudaGetLastError());
    // T1 = A X  (M = m, N = q, K = p); epilogue writes the split terms of T1
    tc::Args a1;
    memset(&a1, 0, sizeof(a1));
    a1.M = (int)g->m; a1.N = (int)g->q; a1.K = (int)g->Kp;
    a1.mode = tc::EPI_SPLIT; a1.out_terms = g->terms; a1.out_rows = (int)g->mr; a1.out_split = g->T1s;
    a1.out_ld = g->Kq; a1.err = g->err;
    // R = C - T1 B  (M = m, N = n, K = q)
    tc::Args a2;
    memset(&a2, 0, sizeof(a2));
    a2.M = (int)g->m; a2.N = (int)g->n; a2.K = (int)g->Kq;
    a2.mode = tc::EPI_RESID; a2.cin = C; a2.out = R; a2.ld = ldr; a2.err = g->err;
    const int bn = g->terms == 2 ? tc::Cfg<2>::BN : tc::Cfg<3>::BN;
    const int64_t t1 = ((g->q + bn - 1) / bn) * ((g->m + tc::BM - 1) / tc::BM);
    const int64_t t2 = ((g->n + bn - 1) / bn) * ((g->m + tc::BM - 1) / tc::BM);
    dim3 g1((unsigned)std::min<int64_t>(t1, g->nsm)), g2((unsigned)std::min<int64_t>(t2, g->nsm));
    if (g->terms == 2) {
        tc::gemm_kernel<2><<<g1, 256, tc::SMEM_BYTES, st>>>(g->tmA, g->tmXT, a1);
        GRBK_CK(cudaGetLastError());
        tc::gemm_kernel<2><<<g2, 256, tc::SMEM_BYTES, st>>>(g->tmT1, g->tmBT, a2);
    } else {
        tc::gemm_kernel<3><<<g1, 256, tc::SMEM_BYTES, st>>>(g->tmA, g->tmXT, a1);
        GRBK_CK(cudaGetLastError());
        tc::gemm_kernel<3><<<g2, 256, tc::SMEM_BYTES, st>>>(g->tmT1, g->tmBT, a2);
    }
    GRBK_CK(cudaGetLastError());
    return GRBK_OK;
}

grbk_status splitgemm_gram(SplitGemm* g, float* G, int64_t ldg, cudaStream_t st)
{
    tc::Args a;
    memset(&a, 0, sizeof(a));
    a.M = (int)g->m; a.N = (int)g->m; a.K = (int)g->Kp;
    a.mode = tc::EPI_STORE; a.out = G; a.ld = ldg; a.err = g->err;
    const int bn = g->terms == 2 ? tc::Cfg<2>::BN : tc::Cfg<3>::BN;
    const int64_t tiles = ((g->m + bn - 1) / bn) * ((g->m + tc::BM - 1) / tc::BM);
    dim3 grid((unsigned)std::min<int64_t>(tiles, g->nsm));
    if (g->terms == 2) tc::gemm_kernel<2><<<grid, 256, tc::SMEM_BYTES, st>>>(g->tmA, g->tmAn, a);
    else tc::gemm_kernel<3><<<grid, 256, tc::SMEM_BYTES, st>>>(g->tmA, g->tmAn, a);
    GRBK_CK(cudaGetLastError());
    return GRBK_OK;
}

grbk_status splitgemm_check(SplitGemm* g, cudaStream_t st)
{
    int h = 0;
    GRBK_CK(cudaMemcpyAsync(&h, g->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    GRBK_CK(cudaStreamSynchronize(st));
    return h ? GRBK_ETIMEOUT : GRBK_OK;
}

int splitgemm_launches(const SplitGemm*) { return 3; }

// pixel tile of the tensor-core convolution: 128 pixels, boxw a power of two up
// to 128 and no wider than the image, boxh = 128 / boxw rows
static int conv_boxw(int W)
{
    int boxw = 128;
    while (boxw > W && boxw > 1) boxw >>= 1;
    return boxw;
}

bool tc_conv_fits(int H, int W) { return W >= 1 && 128 / conv_boxw(W) <= H; }

grbk_status tc_conv3x3(const void* xs, int nimg, int H, int W, int Cp, const void* wtc, int Npad, int Cout,
                       const float* bias, int relu, float* out, int out_ctot, int out_c0, int* err, cudaStream_t st,
                       bool halo)
{
    if (Cp % tc::BK != 0 || Npad % 16 != 0 || Npad < 16 || Npad > 128 || Cout > Npad) return GRBK_EINVAL;
    if (!tc_conv_fits(H, W)) return GRBK_EINVAL;
    auto enc = tensor_map_encoder();
    if (!enc) return GRBK_ECUDA;
    const int boxw = conv_boxw(W);
    const int boxh = 128 / boxw;
    halo = halo && boxw == 128;   // the row variant needs images at least 128 pixels wide
    CUtensorMap tmX, tmW;
    {
        cuuint64_t dims[4] = {(cuuint64_t)Cp, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)(tc::CONV_TERMS * nimg)};
        cuuint64_t strides[3] = {(cuuint64_t)Cp * 2, (cuuint64_t)W * Cp * 2, (cuuint64_t)H * W * Cp * 2};
        cuuint32_t box[4] = {(cuuint32_t)tc::BK, halo ? (cuuint32_t)tc::HALO_ROWS : (cuuint32_t)boxw,
                             halo ? 1u : (cuuint32_t)boxh, 1};
        cuuint32_t estr[4] = {1, 1, 1, 1};
        if (enc(&tmX, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)xs, dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return GRBK_ECUDA;
    }
    {
        cuuint64_t dims[2] = {(cuuint64_t)(9 * Cp), (cuuint64_t)Npad};
        cuuint64_t strides[1] = {(cuuint64_t)9 * Cp * 2};
        cuuint32_t box[2] = {(cuuint32_t)tc::BK, (cuuint32_t)Npad};
        cuuint32_t estr[2] = {1, 1};
        if (enc(&tmW, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)wtc, dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return GRBK_ECUDA;
    }
    tc::ConvArgs a;
    memset(&a, 0, sizeof(a));
    a.nimg = nimg; a.H = H; a.W = W; a.Cp = Cp; a.Npad = Npad; a.Cout = Cout;
    a.boxw = boxw; a.boxh = boxh;
    a.tiles_x = (W + boxw - 1) / boxw;
    a.tiles_y = (H + boxh - 1) / boxh;
    int cols = 64;
    while (cols < 2 * ((Npad + 31) / 32 * 32)) cols <<= 1;   // two accumulators, each a power-of-two slot
    a.tmem_cols = cols;
    a.bias = bias; a.relu = relu; a.out = out; a.out_ctot = out_ctot; a.out_c0 = out_c0; a.err = err;
    int dev = 0, nsm = 0;
    GRBK_CK(cudaGetDevice(&dev));
    GRBK_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if (halo) {
        GRBK_CK(cudaFuncSetAttribute(tc::conv_tc_halo_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     tc::HALO_SMEM_BYTES));
        const int64_t ntiles = (int64_t)nimg * H * a.tiles_x;
        dim3 grid((unsigned)std::min<int64_t>(ntiles, nsm));
        tc::conv_tc_halo_kernel<<<grid, 256, tc::HALO_SMEM_BYTES, st>>>(tmX, tmW, a);
    } else {
        GRBK_CK(cudaFuncSetAttribute(tc::conv_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     tc::CONV_SMEM_BYTES));
        const int64_t ntiles = (int64_t)nimg * a.tiles_y * a.tiles_x;
        dim3 grid((unsigned)std::min<int64_t>(ntiles, nsm));
        tc::conv_tc_kernel<<<grid, 256, tc::CONV_SMEM_BYTES, st>>>(tmX, tmW, a);
    }
    GRBK_CK(cudaGetLastError());
    return GRBK_OK;
}

void splitgemm_destroy(SplitGemm* g)
{
    if (!g) return;
    void* bufs[] = {g->As, g->BTs, g->XTs, g->T1s, g->err};
    for (void* b : bufs)
        if (b) dev_free(b);
    delete g;
}

}  // namespace grbk
