// grbk_unet.cu -- learned warm start for the colour-image application
// (Section 6): a 3-level convolutional U-Net maps a blurred channel C to an
// initial iterate X0 = C + f(C) for the block Kaczmarz solve.  Hand-written
// kernels for the forward pass, both backward passes, pooling, upsampling,
// the L2 loss and Adam; BF16 weights (rounded from an FP32 master copy), FP32
// activations and accumulation.
//
// Architecture (w = width): enc1 1->w->w | pool | enc2 w->2w->2w | pool |
// bottleneck 2w->4w->4w | up, concat enc2 | dec2 6w->2w->2w | up, concat enc1 |
// dec1 3w->w->w | out w->1.  Every conv is 3x3, zero padding 1, ReLU except
// the last.  Pooling is 2x2 average, upsampling nearest; concatenations are
// free: the skip tensors are written straight into the decoder input buffers.
// Parameters are one flat FP32 array, layer by layer in the order above, each
// layer W[out][in][3][3] then b[out].
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>
#include <math.h>
#include <algorithm>
#include <vector>

#include "grbk_internal.cuh"

namespace grbk {
namespace unet {

constexpr int TILE = 16;       // output tile side (weight-gradient kernel; width of the convolution's tile)
constexpr int PIX = 4;         // convolution: output pixels per thread, stacked vertically
constexpr int TILE_H = TILE * PIX;  // convolution: output tile height
constexpr int CO_T = 16;       // output channels per CTA
constexpr int CI_T = 8;        // input channels staged per step

// A channel range of an NCHW buffer with `ctot` channels.
struct View {
    float* p;
    int ctot;
    int c0;
};

__device__ __forceinline__ float* at(const View& v, int n, int c, int H, int W)
{
    return v.p + ((size_t)n * v.ctot + v.c0 + c) * H * W;
}

// out[n][o] = sum_i sum_k w(o, i, k) in[n][i](y + ky - 1, x + kx - 1) (+ b[o], ReLU)
//   FLIP = false: w(o, i, k) = W[o][i][k]         (forward)
//   FLIP = true : w(o, i, k) = W[i][o][8 - k]     (gradient w.r.t. the input)
// mask (optional): the input is multiplied by (mask > 0) (ReLU derivative).
template <bool FLIP, int COT>
__global__ void __launch_bounds__(256) conv3x3_kernel(View in, int Cin, View mask, View out, int Cout,
                                                      const __nv_bfloat16* __restrict__ Wt, const float* __restrict__ b,
                                                      int H, int W, int relu, int accumulate)
{
    // output tile TILE wide and TILE_H tall, COT output channels; thread (lx, ly) computes
    // PIX pixels of one column, so every weight read from shared memory feeds PIX
    // multiply-adds.
    __shared__ float s_in[CI_T][TILE_H + 2][TILE + 2];
    __shared__ float s_w[COT][CI_T][9];
    const int tiles_x = (W + TILE - 1) / TILE;
    const int tx0 = (blockIdx.x % tiles_x) * TILE, ty0 = (blockIdx.x / tiles_x) * TILE_H;
    const int o0 = blockIdx.y * COT, n = blockIdx.z;
    const int lx = threadIdx.x % TILE, ly = threadIdx.x / TILE;
    const int x = tx0 + lx, y0 = ty0 + ly * PIX;
    float acc[COT][PIX];
#pragma unroll
    for (int o = 0; o < COT; ++o)
#pragma unroll
        for (int p = 0; p < PIX; ++p) acc[o][p] = 0.f;
    for (int i0 = 0; i0 < Cin; i0 += CI_T) {
        // stage CI_T input channels with a 1-pixel halo (zeros past Cin)
        for (int e = threadIdx.x; e < CI_T * (TILE_H + 2) * (TILE + 2); e += 256) {
            const int ci = e / ((TILE_H + 2) * (TILE + 2));
            const int r = e % ((TILE_H + 2) * (TILE + 2));
            const int hy = r / (TILE + 2), hx = r % (TILE + 2);
            const int gy = ty0 + hy - 1, gx = tx0 + hx - 1;
            float v = 0.f;
            if (i0 + ci < Cin && gy >= 0 && gy < H && gx >= 0 && gx < W) {
                v = at(in, n, i0 + ci, H, W)[gy * W + gx];
                if (mask.p && !(at(mask, n, i0 + ci, H, W)[gy * W + gx] > 0.f)) v = 0.f;
            }
            s_in[ci][hy][hx] = v;
        }
        for (int e = threadIdx.x; e < COT * CI_T * 9; e += 256) {
            const int o = e / (CI_T * 9), r = e % (CI_T * 9), ci = r / 9, k = r % 9;
            float wv = 0.f;
            if (o0 + o < Cout && i0 + ci < Cin) {
                const size_t idx = FLIP ? (((size_t)(i0 + ci) * Cout + (o0 + o)) * 9 + (8 - k))
                                        : (((size_t)(o0 + o) * Cin + (i0 + ci)) * 9 + k);
                wv = __bfloat162float(Wt[idx]);
            }
            s_w[o][ci][k] = wv;
        }
        __syncthreads();
#pragma unroll 2
        for (int ci = 0; ci < CI_T; ++ci) {
            float nb[PIX + 2][3];
#pragma unroll
            for (int r = 0; r < PIX + 2; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) nb[r][c] = s_in[ci][ly * PIX + r][lx + c];
#pragma unroll
            for (int o = 0; o < COT; ++o) {
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    const float wv = s_w[o][ci][k];
#pragma unroll
                    for (int p = 0; p < PIX; ++p) acc[o][p] = fmaf(wv, nb[p + k / 3][k % 3], acc[o][p]);
                }
            }
        }
        __syncthreads();
    }
    if (x >= W) return;
#pragma unroll
    for (int p = 0; p < PIX; ++p) {
        const int y = y0 + p;
        if (y >= H) break;
#pragma unroll
        for (int o = 0; o < COT; ++o) {
            if (o0 + o >= Cout) break;
            float v = acc[o][p] + (b ? b[o0 + o] : 0.f);
            if (relu) v = fmaxf(v, 0.f);
            float* dst = at(out, n, o0 + o, H, W) + y * W + x;
            if (accumulate) *dst += v; else *dst = v;
        }
    }
}

// partial dW[o][i][k] and db[o] over a slice of the (image, tile) space:
// part[s][o][i][k] = sum over the slice of g[n][o](p) in[n][i](p + k - 1),
// g = dY (masked by mask > 0 when given).  Grid: (Cout / CO_T, Cin / CI_T, S).
__global__ void __launch_bounds__(256) conv3x3_wgrad_kernel(View in, int Cin, View dy, View mask, int Cout, int N, int H,
                                                            int W, float* __restrict__ part, float* __restrict__ bpart)
{
    __shared__ float s_in[CI_T][TILE + 2][TILE + 2];
    __shared__ float s_g[CO_T][TILE * TILE];
    const int o0 = blockIdx.x * CO_T, i0 = blockIdx.y * CI_T, S = gridDim.z, sl = blockIdx.z;
    const int tiles_x = (W + TILE - 1) / TILE, tiles_y = (H + TILE - 1) / TILE;
    const int ntile = N * tiles_x * tiles_y;
    // thread -> (o, i) pair and half of the tile's pixels
    const int pair = threadIdx.x % (CO_T * CI_T), half = threadIdx.x / (CO_T * CI_T);
    const int po = pair / CI_T, pi = pair % CI_T;
    float acc[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] = 0.f;
    float bacc = 0.f;
    for (int t = sl; t < ntile; t += S) {
        const int n = t / (tiles_x * tiles_y), r = t % (tiles_x * tiles_y);
        const int tx0 = (r % tiles_x) * TILE, ty0 = (r / tiles_x) * TILE;
        __syncthreads();
        for (int e = threadIdx.x; e < CI_T * (TILE + 2) * (TILE + 2); e += 256) {
            const int ci = e / ((TILE + 2) * (TILE + 2));
            const int rr = e % ((TILE + 2) * (TILE + 2));
            const int hy = rr / (TILE + 2), hx = rr % (TILE + 2);
            const int gy = ty0 + hy - 1, gx = tx0 + hx - 1;
            float v = 0.f;
            if (i0 + ci < Cin && gy >= 0 && gy < H && gx >= 0 && gx < W) v = at(in, n, i0 + ci, H, W)[gy * W + gx];
            s_in[ci][hy][hx] = v;
        }
        for (int e = threadIdx.x; e < CO_T * TILE * TILE; e += 256) {
            const int o = e / (TILE * TILE), px = e % (TILE * TILE);
            const int gy = ty0 + px / TILE, gx = tx0 + px % TILE;
            float v = 0.f;
            if (o0 + o < Cout && gy < H && gx < W) {
                v = at(dy, n, o0 + o, H, W)[gy * W + gx];
                if (mask.p && !(at(mask, n, o0 + o, H, W)[gy * W + gx] > 0.f)) v = 0.f;
            }
            s_g[o][px] = v;
        }
        __syncthreads();
        for (int px = half; px < TILE * TILE; px += 2) {
            const float gv = s_g[po][px];
            const int ly = px / TILE, lx = px % TILE;
#pragma unroll
            for (int k = 0; k < 9; ++k) acc[k] = fmaf(gv, s_in[pi][ly + k / 3][lx + k % 3], acc[k]);
            if (pi == 0) bacc += gv;
        }
    }
    // combine the two pixel halves in shared memory, then write this slice's partials
    __syncthreads();
    float* red = &s_g[0][0];  // CO_T * CI_T * 10 floats needed (<= CO_T * TILE * TILE)
    if (half == 1) {
#pragma unroll
        for (int k = 0; k < 9; ++k) red[pair * 10 + k] = acc[k];
        red[pair * 10 + 9] = bacc;
    }
    __syncthreads();
    if (half == 0) {
#pragma unroll
        for (int k = 0; k < 9; ++k) acc[k] += red[pair * 10 + k];
        bacc += red[pair * 10 + 9];
        const int o = o0 + po, i = i0 + pi;
        if (o < Cout && i < Cin) {
#pragma unroll
            for (int k = 0; k < 9; ++k) part[(((size_t)sl * Cout + o) * Cin + i) * 9 + k] = acc[k];
        }
        if (pi == 0 && o < Cout && blockIdx.y == 0) bpart[(size_t)sl * Cout + o] = bacc;
    }
}

// g[j] = sum_s part[s][j] (fixed order); optional second array for the bias
__global__ void reduce_slices_kernel(const float* part, int S, int64_t len, float* g)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= len) return;
    float acc = 0.f;
    for (int s = 0; s < S; ++s) acc += part[(int64_t)s * len + j];
    g[j] = acc;
}

// 2x2 average pooling and its adjoint.  Grid: (tiles of the plane, channel, image); 32-bit
// offsets within a plane (H W < 2^31) keep the index arithmetic off 64-bit division.
__global__ void pool_fwd_kernel(View in, View out, int C, int N, int H, int W)
{
    const int Ho = H / 2, Wo = W / 2;
    const int c = blockIdx.y, n = blockIdx.z;
    const float* s = at(in, n, c, H, W);
    float* d = at(out, n, c, Ho, Wo);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Ho * Wo; e += gridDim.x * blockDim.x) {
        const int y = e / Wo, x = e - y * Wo;
        d[e] = 0.25f * (s[(2 * y) * W + 2 * x] + s[(2 * y) * W + 2 * x + 1] + s[(2 * y + 1) * W + 2 * x] +
                        s[(2 * y + 1) * W + 2 * x + 1]);
    }
}

__global__ void pool_bwd_kernel(View gout, View gin, int C, int N, int H, int W, int accumulate)
{
    const int c = blockIdx.y, n = blockIdx.z;
    const float* g = at(gout, n, c, H / 2, W / 2);
    float* d = at(gin, n, c, H, W);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < H * W; e += gridDim.x * blockDim.x) {
        const int y = e / W, x = e - y * W;
        const float v = 0.25f * g[(y / 2) * (W / 2) + x / 2];
        if (accumulate) d[e] += v; else d[e] = v;
    }
}

// nearest 2x upsampling (H, W are the low-resolution sizes) and its adjoint
__global__ void up_fwd_kernel(View in, View out, int C, int N, int H, int W)
{
    const int Ho = 2 * H, Wo = 2 * W;
    const int c = blockIdx.y, n = blockIdx.z;
    const float* s = at(in, n, c, H, W);
    float* d = at(out, n, c, Ho, Wo);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Ho * Wo; e += gridDim.x * blockDim.x) {
        const int y = e / Wo, x = e - y * Wo;
        d[e] = s[(y / 2) * W + x / 2];
    }
}

__global__ void up_bwd_kernel(View gout, View gin, int C, int N, int H, int W)
{
    const int Wo = 2 * W;
    const int c = blockIdx.y, n = blockIdx.z;
    const float* g = at(gout, n, c, 2 * H, Wo);
    float* d = at(gin, n, c, H, W);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < H * W; e += gridDim.x * blockDim.x) {
        const int y = e / W, x = e - y * W;
        d[e] = g[(2 * y) * Wo + 2 * x] + g[(2 * y) * Wo + 2 * x + 1] + g[(2 * y + 1) * Wo + 2 * x] +
               g[(2 * y + 1) * Wo + 2 * x + 1];
    }
}

// X0 = C + y ; with a target: loss partials of (X0 - T)^2 and dy = 2 (X0 - T) / count
__global__ void residual_out_kernel(const float* C, const float* y, float* X0, int64_t total)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        X0[e] = C[e] + y[e];
}

__global__ void loss_kernel(const float* C, const float* y, const float* T, float* dy, int64_t total, double* part)
{
    __shared__ double red[32];
    double acc = 0.0;
    const float scale = 2.0f / (float)total;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const float d = C[e] + y[e] - T[e];
        acc += (double)d * (double)d;
        dy[e] = scale * d;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

// Adam (Kingma & Ba) on the FP32 master weights, then the BF16 copy used by the convolutions
__global__ void adam_kernel(float* w, __nv_bfloat16* wb, const float* g, float* m1, float* m2, int64_t len, float lr,
                            float b1, float b2, float eps, float c1, float c2)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= len) return;
    const float gj = g[j];
    const float a = b1 * m1[j] + (1.f - b1) * gj;
    const float v = b2 * m2[j] + (1.f - b2) * gj * gj;
    m1[j] = a;
    m2[j] = v;
    const float wn = w[j] - lr * (a / c1) / (sqrtf(v / c2) + eps);
    w[j] = wn;
    wb[j] = __float2bfloat16_rn(wn);
}

__global__ void to_bf16_kernel(const float* w, __nv_bfloat16* wb, int64_t len)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < len) wb[j] = __float2bfloat16_rn(w[j]);
}

// Input of a tensor-core convolution: channels [0, Cin) of an NCHW FP32 view as
// three BF16 planes [term][n][y][x][Cp] (NHWC, channels padded with zeros to Cp)
// with x = x0 + x1 + x2, x0 = bf16(x), x1 = bf16(x - x0), x2 = bf16(x - x0 - x1).
// A CTA transposes 64 consecutive pixels of one image through shared memory:
// reads of a channel run along the pixels, writes of a pixel run along its
// channels, both coalesced.
constexpr int PACK_PIX = 64;
// mask (optional): the input is multiplied by (mask > 0) (the ReLU derivative, for the
// gradient with respect to a layer's input).
__global__ void __launch_bounds__(256) pack_nhwc3_kernel(View in, int Cin, View mask, int N, int H, int W, int Cp,
                                                         __nv_bfloat16* dst)
{
    __shared__ float tile[128][PACK_PIX + 1];          // Cp <= 128
    const int64_t hw = (int64_t)H * W;
    const int64_t blocks_per_img = (hw + PACK_PIX - 1) / PACK_PIX;
    const int64_t plane = (int64_t)N * hw * Cp;
    for (int64_t blk = blockIdx.x; blk < (int64_t)N * blocks_per_img; blk += gridDim.x) {
        const int n = (int)(blk / blocks_per_img);
        const int64_t p0 = (blk % blocks_per_img) * PACK_PIX;
        __syncthreads();
        for (int e = threadIdx.x; e < Cp * PACK_PIX; e += blockDim.x) {
            const int c = e / PACK_PIX, j = e % PACK_PIX;
            float x = 0.f;
            if (c < Cin && p0 + j < hw) {
                x = at(in, n, c, H, W)[p0 + j];
                if (mask.p && !(at(mask, n, c, H, W)[p0 + j] > 0.f)) x = 0.f;
            }
            tile[c][j] = x;
        }
        __syncthreads();
        const int groups = Cp / 8;
        for (int e = threadIdx.x; e < PACK_PIX * groups; e += blockDim.x) {
            const int j = e / groups, cg = e % groups;
            if (p0 + j >= hw) continue;
            __align__(16) __nv_bfloat16 t0[8], t1[8], t2[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float x = tile[cg * 8 + k][j];
                const __nv_bfloat16 h = __float2bfloat16_rn(x);
                const float r1 = x - __bfloat162float(h);
                const __nv_bfloat16 l = __float2bfloat16_rn(r1);
                t0[k] = h;
                t1[k] = l;
                t2[k] = __float2bfloat16_rn(r1 - __bfloat162float(l));
            }
            const int64_t off = ((int64_t)n * hw + p0 + j) * Cp + cg * 8;
            *reinterpret_cast<uint4*>(dst + off) = *reinterpret_cast<const uint4*>(t0);
            *reinterpret_cast<uint4*>(dst + plane + off) = *reinterpret_cast<const uint4*>(t1);
            *reinterpret_cast<uint4*>(dst + 2 * plane + off) = *reinterpret_cast<const uint4*>(t2);
        }
    }
}

// Weights of a tensor-core convolution with Cin input and Cout output channels:
// wt[o][tap][c] = W[o][c][tap] (BF16 copy; flip = 0), or, for the gradient with
// respect to the input of a layer whose weights are W[c][o][tap] (Cout of this
// convolution = the layer's inputs), wt[o][tap][c] = W[c][o][8 - tap] (flip = 1).
// Zero for o >= Cout or c >= Cin.
__global__ void pack_wtc_kernel(const __nv_bfloat16* wb, int Cin, int Cout, int Cp, int Npad, int flip,
                                __nv_bfloat16* wt)
{
    const int64_t total = (int64_t)Npad * 9 * Cp;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % Cp), tap = (int)((e / Cp) % 9), o = (int)(e / (9 * (int64_t)Cp));
        __nv_bfloat16 v = __float2bfloat16_rn(0.f);
        if (o < Cout && c < Cin)
            v = flip ? wb[((int64_t)c * Cout + o) * 9 + (8 - tap)] : wb[((int64_t)o * Cin + c) * 9 + tap];
        wt[e] = v;
    }
}

}  // namespace unet
}  // namespace grbk

// ============================================================================
// host side
// ============================================================================
using namespace grbk;
using namespace grbk::unet;

namespace {

enum { ENC1A, ENC1B, ENC2A, ENC2B, BOTA, BOTB, DEC2A, DEC2B, DEC1A, DEC1B, OUTL, NLAYERS };

struct LayerDef {
    int cin, cout, relu;
    int64_t woff, boff;
};

// activation / gradient buffers of one sub-batch (NCHW FP32)
struct Acts {
    float *a1, *D1, *p1, *a2, *D2, *p2, *a3, *a3b, *d2a, *d2b, *d1a, *d1b, *y;
};

}  // namespace

struct grbk_unet {
    int w;
    LayerDef L[NLAYERS];
    int64_t nparams;
    float* params;            // FP32 master
    __nv_bfloat16* wb;        // BF16 copy used by the convolutions
    float* grad;
    float *m1, *m2;           // Adam moments
    long long step;
    float* arena;             // activations + gradients
    size_t arena_floats;
    float* wpart;             // weight-gradient slices
    size_t wpart_floats;
    double* lpart;            // loss partials
    double* lpart_host;
    cudaStream_t stream;
    int cap_n, cap_h, cap_w;  // arena capacity
    int use_tc;               // tensor-core convolutions where the layer allows (default on)
    __nv_bfloat16* xs;        // tensor-core input planes (largest layer)
    size_t xs_elems;
    __nv_bfloat16* wtc;       // tensor-core weight layouts, per layer at wtc_off (forward) and
    int64_t wtc_off[16];      // wtcb_off (gradient with respect to the layer's input)
    int64_t wtcb_off[16];
    int* tc_err;              // device flag: a bounded wait of the tensor-core kernel expired
};

static void unet_layers(grbk_unet* u)
{
    const int w = u->w;
    const int io[NLAYERS][3] = {{1, w, 1},         {w, w, 1},         {w, 2 * w, 1},     {2 * w, 2 * w, 1},
                                {2 * w, 4 * w, 1}, {4 * w, 4 * w, 1}, {6 * w, 2 * w, 1}, {2 * w, 2 * w, 1},
                                {3 * w, w, 1},     {w, w, 1},         {w, 1, 0}};
    int64_t off = 0;
    for (int l = 0; l < NLAYERS; ++l) {
        u->L[l].cin = io[l][0];
        u->L[l].cout = io[l][1];
        u->L[l].relu = io[l][2];
        u->L[l].woff = off;
        off += (int64_t)io[l][0] * io[l][1] * 9;
        u->L[l].boff = off;
        off += io[l][1];
    }
    u->nparams = off;
}

// floats per image of every activation (or gradient) buffer for an H x W input
static size_t acts_floats(int w, int H, int W)
{
    const size_t l1 = (size_t)H * W, l2 = l1 / 4, l3 = l1 / 16;
    return l1 * (w + 3 * w + w + w + 1) + l2 * (w + 2 * w + 6 * w + 2 * w + 2 * w) + l3 * (2 * w + 4 * w + 4 * w);
}

static Acts carve(float*& p, int w, int N, int H, int W)
{
    const size_t l1 = (size_t)N * H * W, l2 = l1 / 4, l3 = l1 / 16;
    Acts a;
    a.a1 = p; p += l1 * w;
    a.D1 = p; p += l1 * 3 * w;
    a.d1a = p; p += l1 * w;
    a.d1b = p; p += l1 * w;
    a.y = p; p += l1;
    a.p1 = p; p += l2 * w;
    a.a2 = p; p += l2 * 2 * w;
    a.D2 = p; p += l2 * 6 * w;
    a.d2a = p; p += l2 * 2 * w;
    a.d2b = p; p += l2 * 2 * w;
    a.p2 = p; p += l3 * 2 * w;
    a.a3 = p; p += l3 * 4 * w;
    a.a3b = p; p += l3 * 4 * w;
    return a;
}

static View V(float* p, int ctot, int c0 = 0) { return View{p, ctot, c0}; }
static const View kNone = {nullptr, 0, 0};

static unsigned blocks_for(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 65535); }

// grid of the per-plane kernels (pooling, upsampling): tiles of a plane of `plane` pixels x C x N
static dim3 plane_grid(int64_t plane, int C, int N)
{
    return dim3((unsigned)std::min<int64_t>((plane + 255) / 256, 4096), (unsigned)C, (unsigned)N);
}

// The tensor-core path takes layers with 16 to 128 input and output channels (the
// first and last layers, with one channel, stay on the SIMT kernel).
static bool tc_layer(const grbk_unet* u, int l)
{
    return u->use_tc && u->L[l].cin >= 16 && u->L[l].cin <= 128 && u->L[l].cout >= 16 && u->L[l].cout <= 128;
}
// the gradient with respect to a layer's input is a 3x3 convolution of the output
// gradient (cout channels in, cin out), so the same channel limits apply
static bool tc_bwd_layer(const grbk_unet* u, int l) { return l != ENC1A && tc_layer(u, l); }
static int tc_cp(int cin) { return (cin + 63) / 64 * 64; }
static int tc_npad(int cout) { return (cout + 15) / 16 * 16; }

// resolution level (1, 2, 3) of each layer's input
static int layer_level(int l)
{
    switch (l) {
    case ENC2A: case ENC2B: case DEC2A: case DEC2B: return 2;
    case BOTA: case BOTB: return 3;
    default: return 1;
    }
}

static grbk_status tc_prepare(grbk_unet* u, int N, int H, int W)
{
    size_t need = 0;
    for (int l = 0; l < NLAYERS; ++l) {
        if (!tc_layer(u, l)) continue;
        const int sh = layer_level(l) - 1;
        need = std::max(need, (size_t)3 * N * (H >> sh) * (W >> sh) * tc_cp(u->L[l].cin));
        if (tc_bwd_layer(u, l)) need = std::max(need, (size_t)3 * N * (H >> sh) * (W >> sh) * tc_cp(u->L[l].cout));
    }
    if (need > u->xs_elems) {
        if (u->xs) cudaFree(u->xs);
        u->xs = nullptr;
        u->xs_elems = 0;
        if (cudaMalloc(&u->xs, need * 2) != cudaSuccess) return GRBK_ENOMEM;
        u->xs_elems = need;
    }
    if (!u->wtc) {
        int64_t off = 0;
        for (int l = 0; l < NLAYERS; ++l) {
            u->wtc_off[l] = off;
            if (tc_layer(u, l)) off += (int64_t)tc_npad(u->L[l].cout) * 9 * tc_cp(u->L[l].cin);
            u->wtcb_off[l] = off;
            if (tc_bwd_layer(u, l)) off += (int64_t)tc_npad(u->L[l].cin) * 9 * tc_cp(u->L[l].cout);
        }
        if (cudaMalloc(&u->wtc, std::max<int64_t>(off, 1) * 2) != cudaSuccess) return GRBK_ENOMEM;
        if (cudaMalloc(&u->tc_err, sizeof(int)) != cudaSuccess) return GRBK_ENOMEM;
        if (cudaMemsetAsync(u->tc_err, 0, sizeof(int), u->stream) != cudaSuccess) return GRBK_ECUDA;
    }
    return GRBK_OK;
}

static cudaError_t conv(grbk_unet* u, int l, View in, View out, int N, int H, int W)
{
    const LayerDef& d = u->L[l];
    if (tc_layer(u, l) && tc_conv_fits(H, W)) {
        const int Cp = tc_cp(d.cin), Np = tc_npad(d.cout);
        const int64_t npix = (int64_t)N * H * W;
        const int64_t pblocks = (int64_t)N * (((int64_t)H * W + PACK_PIX - 1) / PACK_PIX);
        pack_nhwc3_kernel<<<(unsigned)std::min<int64_t>(pblocks, 65535), 256, 0, u->stream>>>(in, d.cin, kNone, N, H, W,
                                                                                              Cp, u->xs);
        pack_wtc_kernel<<<blocks_for((int64_t)Np * 9 * Cp), 256, 0, u->stream>>>(u->wb + d.woff, d.cin, d.cout, Cp, Np, 0,
                                                                                u->wtc + u->wtc_off[l]);
        const grbk_status s = tc_conv3x3(u->xs, N, H, W, Cp, u->wtc + u->wtc_off[l], Np, d.cout, u->params + d.boff,
                                         d.relu, out.p, out.ctot, out.c0, u->tc_err, u->stream, u->use_tc == 1);
        if (s != GRBK_OK) return cudaErrorUnknown;
        return cudaGetLastError();
    }
    const int tiles = ((W + TILE - 1) / TILE) * ((H + TILE_H - 1) / TILE_H);
    if (d.cout == 1) {  // the output layer: one channel per CTA instead of CO_T mostly empty ones
        dim3 grid((unsigned)tiles, 1u, (unsigned)N);
        conv3x3_kernel<false, 1><<<grid, 256, 0, u->stream>>>(in, d.cin, kNone, out, d.cout, u->wb + d.woff,
                                                              u->params + d.boff, H, W, d.relu, 0);
    } else {
        dim3 grid((unsigned)tiles, (unsigned)((d.cout + CO_T - 1) / CO_T), (unsigned)N);
        conv3x3_kernel<false, CO_T><<<grid, 256, 0, u->stream>>>(in, d.cin, kNone, out, d.cout, u->wb + d.woff,
                                                                 u->params + d.boff, H, W, d.relu, 0);
    }
    return cudaGetLastError();
}

// backward of layer l: gout = dL/d(output), outv = the layer's output (ReLU mask), in = its input.
// Writes dW, db into u->grad and (if gin.p) dL/d(input) into gin (accumulating when asked).
static cudaError_t conv_bwd(grbk_unet* u, int l, View in, View outv, View gout, View gin, int accumulate, int N, int H,
                            int W)
{
    const LayerDef& d = u->L[l];
    const View mask = d.relu ? outv : kNone;
    const int tiles = ((W + TILE - 1) / TILE) * ((H + TILE - 1) / TILE);
    const int S = std::max(1, std::min(N * tiles, 128));
    dim3 gw((unsigned)((d.cout + CO_T - 1) / CO_T), (unsigned)((d.cin + CI_T - 1) / CI_T), (unsigned)S);
    float* bpart = u->wpart + (size_t)S * d.cout * d.cin * 9;
    conv3x3_wgrad_kernel<<<gw, 256, 0, u->stream>>>(in, d.cin, gout, mask, d.cout, N, H, W, u->wpart, bpart);
    const int64_t wl = (int64_t)d.cout * d.cin * 9;
    reduce_slices_kernel<<<blocks_for(wl), 256, 0, u->stream>>>(u->wpart, S, wl, u->grad + d.woff);
    reduce_slices_kernel<<<blocks_for(d.cout), 256, 0, u->stream>>>(bpart, S, d.cout, u->grad + d.boff);
    if (gin.p && !accumulate && tc_bwd_layer(u, l) && tc_conv_fits(H, W) && u->xs) {
        // dL/d(input) on the tensor cores: the output gradient (masked by the ReLU
        // derivative) convolved with the flipped, channel-transposed weights
        const int Cp = tc_cp(d.cout), Np = tc_npad(d.cin);
        const int64_t pblocks = (int64_t)N * (((int64_t)H * W + PACK_PIX - 1) / PACK_PIX);
        pack_nhwc3_kernel<<<(unsigned)std::min<int64_t>(pblocks, 65535), 256, 0, u->stream>>>(gout, d.cout, mask, N, H, W,
                                                                                              Cp, u->xs);
        pack_wtc_kernel<<<blocks_for((int64_t)Np * 9 * Cp), 256, 0, u->stream>>>(u->wb + d.woff, d.cout, d.cin, Cp, Np, 1,
                                                                                u->wtc + u->wtcb_off[l]);
        const grbk_status s = tc_conv3x3(u->xs, N, H, W, Cp, u->wtc + u->wtcb_off[l], Np, d.cin, nullptr, 0, gin.p,
                                         gin.ctot, gin.c0, u->tc_err, u->stream, u->use_tc == 1);
        if (s != GRBK_OK) return cudaErrorUnknown;
    } else if (gin.p) {
        const int ctiles = ((W + TILE - 1) / TILE) * ((H + TILE_H - 1) / TILE_H);
        dim3 grid((unsigned)ctiles, (unsigned)((d.cin + CO_T - 1) / CO_T), (unsigned)N);
        conv3x3_kernel<true, CO_T><<<grid, 256, 0, u->stream>>>(gout, d.cout, mask, gin, d.cin, u->wb + d.woff, nullptr, H, W,
                                                          0, accumulate);
    }
    return cudaGetLastError();
}

static grbk_status ensure_arena(grbk_unet* u, int N, int H, int W, bool train)
{
    const size_t need = acts_floats(u->w, H, W) * (size_t)N * (train ? 2 : 1);
    if (need > u->arena_floats) {
        if (u->arena) cudaFree(u->arena);
        u->arena = nullptr;
        u->arena_floats = 0;
        if (cudaMalloc(&u->arena, need * sizeof(float)) != cudaSuccess) return GRBK_ENOMEM;
        u->arena_floats = need;
    }
    // weight-gradient slices: 128 slices of the largest layer (+ bias)
    size_t wp = 0;
    for (int l = 0; l < NLAYERS; ++l)
        wp = std::max(wp, (size_t)128 * (u->L[l].cout * (size_t)u->L[l].cin * 9 + u->L[l].cout));
    if (wp > u->wpart_floats) {
        if (u->wpart) cudaFree(u->wpart);
        u->wpart = nullptr;
        u->wpart_floats = 0;
        if (cudaMalloc(&u->wpart, wp * sizeof(float)) != cudaSuccess) return GRBK_ENOMEM;
        u->wpart_floats = wp;
    }
    return GRBK_OK;
}

// GRBK_ETIMEOUT when a bounded wait of the tensor-core convolution expired (the
// flag stays set: later convolutions leave at once, so the network's outputs
// are not trusted until the handle is destroyed)
static grbk_status tc_check(grbk_unet* u)
{
    if (!u->tc_err) return GRBK_OK;
    int h = 0;
    GRBK_CK(cudaMemcpyAsync(&h, u->tc_err, sizeof(int), cudaMemcpyDeviceToHost, u->stream));
    GRBK_CK(cudaStreamSynchronize(u->stream));
    return h ? GRBK_ETIMEOUT : GRBK_OK;
}

static cudaError_t forward(grbk_unet* u, const Acts& a, const float* C, int N, int H, int W)
{
    const int w = u->w, H2 = H / 2, W2 = W / 2, H4 = H / 4, W4 = W / 4;
    cudaError_t e;
    if (u->use_tc && tc_prepare(u, N, H, W) != GRBK_OK) return cudaErrorMemoryAllocation;
    if ((e = conv(u, ENC1A, V((float*)C, 1), V(a.a1, w), N, H, W)) != cudaSuccess) return e;
    if ((e = conv(u, ENC1B, V(a.a1, w), V(a.D1, 3 * w, 2 * w), N, H, W)) != cudaSuccess) return e;
    pool_fwd_kernel<<<plane_grid((int64_t)H2 * W2, w, N), 256, 0, u->stream>>>(V(a.D1, 3 * w, 2 * w), V(a.p1, w), w, N, H, W);
    if ((e = conv(u, ENC2A, V(a.p1, w), V(a.a2, 2 * w), N, H2, W2)) != cudaSuccess) return e;
    if ((e = conv(u, ENC2B, V(a.a2, 2 * w), V(a.D2, 6 * w, 4 * w), N, H2, W2)) != cudaSuccess) return e;
    pool_fwd_kernel<<<plane_grid((int64_t)H4 * W4, 2 * w, N), 256, 0, u->stream>>>(V(a.D2, 6 * w, 4 * w), V(a.p2, 2 * w),
                                                                                    2 * w, N, H2, W2);
    if ((e = conv(u, BOTA, V(a.p2, 2 * w), V(a.a3, 4 * w), N, H4, W4)) != cudaSuccess) return e;
    if ((e = conv(u, BOTB, V(a.a3, 4 * w), V(a.a3b, 4 * w), N, H4, W4)) != cudaSuccess) return e;
    up_fwd_kernel<<<plane_grid((int64_t)H2 * W2, 4 * w, N), 256, 0, u->stream>>>(V(a.a3b, 4 * w), V(a.D2, 6 * w, 0),
                                                                                  4 * w, N, H4, W4);
    if ((e = conv(u, DEC2A, V(a.D2, 6 * w), V(a.d2a, 2 * w), N, H2, W2)) != cudaSuccess) return e;
    if ((e = conv(u, DEC2B, V(a.d2a, 2 * w), V(a.d2b, 2 * w), N, H2, W2)) != cudaSuccess) return e;
    up_fwd_kernel<<<plane_grid((int64_t)H * W, 2 * w, N), 256, 0, u->stream>>>(V(a.d2b, 2 * w), V(a.D1, 3 * w, 0), 2 * w,
                                                                                N, H2, W2);
    if ((e = conv(u, DEC1A, V(a.D1, 3 * w), V(a.d1a, w), N, H, W)) != cudaSuccess) return e;
    if ((e = conv(u, DEC1B, V(a.d1a, w), V(a.d1b, w), N, H, W)) != cudaSuccess) return e;
    if ((e = conv(u, OUTL, V(a.d1b, w), V(a.y, 1), N, H, W)) != cudaSuccess) return e;
    return cudaGetLastError();
}

// gradients of all parameters for the loss already differentiated into g.y
static cudaError_t backward(grbk_unet* u, const Acts& a, const Acts& g, const float* C, int N, int H, int W)
{
    const int w = u->w, H2 = H / 2, W2 = W / 2, H4 = H / 4, W4 = W / 4;
    cudaError_t e;
    if ((e = conv_bwd(u, OUTL, V(a.d1b, w), V(a.y, 1), V(g.y, 1), V(g.d1b, w), 0, N, H, W)) != cudaSuccess) return e;
    if ((e = conv_bwd(u, DEC1B, V(a.d1a, w), V(a.d1b, w), V(g.d1b, w), V(g.d1a, w), 0, N, H, W)) != cudaSuccess) return e;
    if ((e = conv_bwd(u, DEC1A, V(a.D1, 3 * w), V(a.d1a, w), V(g.d1a, w), V(g.D1, 3 * w), 0, N, H, W)) != cudaSuccess) return e;
    up_bwd_kernel<<<plane_grid((int64_t)H2 * W2, 2 * w, N), 256, 0, u->stream>>>(V(g.D1, 3 * w, 0), V(g.d2b, 2 * w), 2 * w,
                                                                                  N, H2, W2);
    if ((e = conv_bwd(u, DEC2B, V(a.d2a, 2 * w), V(a.d2b, 2 * w), V(g.d2b, 2 * w), V(g.d2a, 2 * w), 0, N, H2, W2)) != cudaSuccess)
        return e;
    if ((e = conv_bwd(u, DEC2A, V(a.D2, 6 * w), V(a.d2a, 2 * w), V(g.d2a, 2 * w), V(g.D2, 6 * w), 0, N, H2, W2)) != cudaSuccess)
        return e;
    up_bwd_kernel<<<plane_grid((int64_t)H4 * W4, 4 * w, N), 256, 0, u->stream>>>(V(g.D2, 6 * w, 0), V(g.a3b, 4 * w), 4 * w,
                                                                                  N, H4, W4);
    if ((e = conv_bwd(u, BOTB, V(a.a3, 4 * w), V(a.a3b, 4 * w), V(g.a3b, 4 * w), V(g.a3, 4 * w), 0, N, H4, W4)) != cudaSuccess)
        return e;
    if ((e = conv_bwd(u, BOTA, V(a.p2, 2 * w), V(a.a3, 4 * w), V(g.a3, 4 * w), V(g.p2, 2 * w), 0, N, H4, W4)) != cudaSuccess)
        return e;
    pool_bwd_kernel<<<plane_grid((int64_t)H2 * W2, 2 * w, N), 256, 0, u->stream>>>(V(g.p2, 2 * w), V(g.D2, 6 * w, 4 * w),
                                                                                    2 * w, N, H2, W2, 1);
    if ((e = conv_bwd(u, ENC2B, V(a.a2, 2 * w), V(a.D2, 6 * w, 4 * w), V(g.D2, 6 * w, 4 * w), V(g.a2, 2 * w), 0, N, H2, W2)) !=
        cudaSuccess)
        return e;
    if ((e = conv_bwd(u, ENC2A, V(a.p1, w), V(a.a2, 2 * w), V(g.a2, 2 * w), V(g.p1, w), 0, N, H2, W2)) != cudaSuccess) return e;
    pool_bwd_kernel<<<plane_grid((int64_t)H * W, w, N), 256, 0, u->stream>>>(V(g.p1, w), V(g.D1, 3 * w, 2 * w), w, N, H, W,
                                                                              1);
    if ((e = conv_bwd(u, ENC1B, V(a.a1, w), V(a.D1, 3 * w, 2 * w), V(g.D1, 3 * w, 2 * w), V(g.a1, w), 0, N, H, W)) !=
        cudaSuccess)
        return e;
    if ((e = conv_bwd(u, ENC1A, V((float*)C, 1), V(a.a1, w), V(g.a1, w), kNone, 0, N, H, W)) != cudaSuccess) return e;
    return cudaGetLastError();
}

static bool shape_ok(int n, int h, int w) { return n > 0 && h >= 4 && w >= 4 && h % 4 == 0 && w % 4 == 0; }

extern "C" grbk_status grbk_unet_create(grbk_unet** out, int32_t width, void* stream)
{
    if (!out || width < 1 || width > 256) return GRBK_EINVAL;
    *out = nullptr;
    grbk_unet* u = new grbk_unet();
    memset(u, 0, sizeof(*u));
    u->w = width;
    u->stream = (cudaStream_t)stream;
    u->use_tc = 1;
    unet_layers(u);
    const size_t np = (size_t)u->nparams;
    if (cudaMalloc(&u->params, np * 4) != cudaSuccess || cudaMalloc(&u->wb, np * 2) != cudaSuccess ||
        cudaMalloc(&u->grad, np * 4) != cudaSuccess || cudaMalloc(&u->m1, np * 4) != cudaSuccess ||
        cudaMalloc(&u->m2, np * 4) != cudaSuccess || cudaMalloc(&u->lpart, 1024 * 8) != cudaSuccess ||
        cudaMallocHost(&u->lpart_host, 1024 * 8) != cudaSuccess) {
        grbk_unet_destroy(u);
        return GRBK_ENOMEM;
    }
    if (cudaMemsetAsync(u->params, 0, np * 4, u->stream) != cudaSuccess ||
        cudaMemsetAsync(u->wb, 0, np * 2, u->stream) != cudaSuccess ||
        cudaMemsetAsync(u->m1, 0, np * 4, u->stream) != cudaSuccess ||
        cudaMemsetAsync(u->m2, 0, np * 4, u->stream) != cudaSuccess) {
        grbk_unet_destroy(u);
        return GRBK_ECUDA;
    }
    *out = u;
    return GRBK_OK;
}

extern "C" int64_t grbk_unet_num_params(const grbk_unet* u) { return u ? u->nparams : -1; }

extern "C" grbk_status grbk_unet_set_params(grbk_unet* u, const float* params, int32_t on_device)
{
    if (!u || !params) return GRBK_EINVAL;
    GRBK_CK(cudaMemcpyAsync(u->params, params, u->nparams * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            u->stream));
    to_bf16_kernel<<<blocks_for(u->nparams), 256, 0, u->stream>>>(u->params, u->wb, u->nparams);
    GRBK_CK(cudaGetLastError());
    GRBK_CK(cudaMemsetAsync(u->m1, 0, u->nparams * 4, u->stream));
    GRBK_CK(cudaMemsetAsync(u->m2, 0, u->nparams * 4, u->stream));
    u->step = 0;
    GRBK_CK(cudaStreamSynchronize(u->stream));
    return GRBK_OK;
}

extern "C" grbk_status grbk_unet_get_params(grbk_unet* u, float* params, int32_t on_device)
{
    if (!u || !params) return GRBK_EINVAL;
    GRBK_CK(cudaMemcpyAsync(params, u->params, u->nparams * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            u->stream));
    GRBK_CK(cudaStreamSynchronize(u->stream));
    return GRBK_OK;
}

extern "C" grbk_status grbk_unet_forward(grbk_unet* u, const float* C, int32_t n, int32_t h, int32_t w, float* X0)
{
    if (!u || !C || !X0 || !shape_ok(n, h, w)) return GRBK_EINVAL;
    // sub-batches bounded to about 2^30 activation floats
    const size_t per = acts_floats(u->w, h, w);
    const int nb = (int)std::max<size_t>(1, std::min<size_t>((size_t)n, ((size_t)1 << 30) / per));
    grbk_status s = ensure_arena(u, nb, h, w, false);
    if (s != GRBK_OK) return s;
    for (int i0 = 0; i0 < n; i0 += nb) {
        const int N = std::min(nb, n - i0);
        float* p = u->arena;
        const Acts a = carve(p, u->w, N, h, w);
        const float* Ci = C + (size_t)i0 * h * w;
        GRBK_CK(forward(u, a, Ci, N, h, w));
        const int64_t tot = (int64_t)N * h * w;
        residual_out_kernel<<<blocks_for(tot), 256, 0, u->stream>>>(Ci, a.y, X0 + (size_t)i0 * h * w, tot);
        GRBK_CK(cudaGetLastError());
    }
    GRBK_CK(cudaStreamSynchronize(u->stream));
    return tc_check(u);
}

static grbk_status loss_and_grad(grbk_unet* u, const float* C, const float* T, int n, int h, int w, double* loss)
{
    const grbk_status tcs = tc_check(u);
    if (tcs != GRBK_OK) return tcs;
    grbk_status s = ensure_arena(u, n, h, w, true);
    if (s != GRBK_OK) return s;
    float* p = u->arena;
    const Acts a = carve(p, u->w, n, h, w);
    const Acts g = carve(p, u->w, n, h, w);
    GRBK_CK(forward(u, a, C, n, h, w));
    const int64_t tot = (int64_t)n * h * w;
    const unsigned nbk = std::min<unsigned>(blocks_for(tot), 1024);
    loss_kernel<<<nbk, 256, 0, u->stream>>>(C, a.y, T, g.y, tot, u->lpart);
    GRBK_CK(cudaGetLastError());
    GRBK_CK(backward(u, a, g, C, n, h, w));
    GRBK_CK(cudaMemcpyAsync(u->lpart_host, u->lpart, nbk * 8, cudaMemcpyDeviceToHost, u->stream));
    GRBK_CK(cudaStreamSynchronize(u->stream));
    double t = 0.0;
    for (unsigned i = 0; i < nbk; ++i) t += u->lpart_host[i];
    *loss = t / (double)tot;
    return tc_check(u);
}

extern "C" grbk_status grbk_unet_loss_grad(grbk_unet* u, const float* C, const float* T, int32_t n, int32_t h, int32_t w,
                                           double* loss, float* grad, int32_t grad_on_device)
{
    if (!u || !C || !T || !loss || !shape_ok(n, h, w)) return GRBK_EINVAL;
    grbk_status s = loss_and_grad(u, C, T, n, h, w, loss);
    if (s != GRBK_OK) return s;
    if (grad) {
        GRBK_CK(cudaMemcpyAsync(grad, u->grad, u->nparams * 4,
                                grad_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, u->stream));
        GRBK_CK(cudaStreamSynchronize(u->stream));
    }
    return GRBK_OK;
}

extern "C" grbk_status grbk_unet_train_step(grbk_unet* u, const float* C, const float* T, int32_t n, int32_t h, int32_t w,
                                            float lr, double* loss)
{
    if (!u || !C || !T || !shape_ok(n, h, w) || !(lr > 0.f)) return GRBK_EINVAL;
    double l = 0.0;
    grbk_status s = loss_and_grad(u, C, T, n, h, w, &l);
    if (s != GRBK_OK) return s;
    u->step += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, (float)u->step), c2 = 1.f - powf(b2, (float)u->step);
    adam_kernel<<<blocks_for(u->nparams), 256, 0, u->stream>>>(u->params, u->wb, u->grad, u->m1, u->m2, u->nparams, lr, b1,
                                                               b2, eps, c1, c2);
    GRBK_CK(cudaGetLastError());
    GRBK_CK(cudaStreamSynchronize(u->stream));
    if (loss) *loss = l;
    return GRBK_OK;
}

extern "C" grbk_status grbk_unet_use_tensor_cores(grbk_unet* u, int32_t on)
{
    if (!u) return GRBK_EINVAL;
    if (on < 0 || on > 2) return GRBK_EINVAL;
    u->use_tc = on;
    return GRBK_OK;
}

extern "C" void grbk_unet_destroy(grbk_unet* u)
{
    if (!u) return;
    void* bufs[] = {u->params, u->wb, u->grad, u->m1, u->m2, u->arena, u->wpart, u->lpart, u->xs, u->wtc, u->tc_err};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (u->lpart_host) cudaFreeHost(u->lpart_host);
    delete u;
}
