// Learned structure classifier: MLP 30 -> 64 -> 64 -> 4 (ReLU, softmax) on
// BF16 tensor cores (mma.sync m16n8k16, FP32 accumulation), its training
// (fused forward/backward, split-K weight gradients, AdamW) and the
// classification pipeline with exact-CNA fallback.
//
// Parameters are one FP32 vector (PPMD_MLP_NPARAM values):
//   mu[30] | isd[30] | W1[30][64] | b1[64] | W2[64][64] | b2[64] | W3[64][4] | b3[4]
// with x' = (x - mu) isd (input standardisation, fitted to the training
// features, not trained) and y = x' W + b (input-major weights).  Each call packs BF16 copies of
// the weights in the operand layouts the MMAs read.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>

#include "analysis.cuh"
#include "mlp_layout.cuh"
#include "mlp_tc.cuh"

namespace ppmd {

static_assert(NPARAM == PPMD_MLP_NPARAM, "parameter count");

// BF16 operand images (row strides padded so that fragment loads are free of
// shared-memory bank conflicts):
//   W1T[64][40]  W1T[n][k] = W1[k][n] (k < 30)      layer 1, B(k, n)
//   W2T[64][72]  W2T[n][k] = W2[k][n]               layer 2
//   W3T[8][72]   W3T[n][k] = W3[k][n] (n < 4)       layer 3
//   W2R[64][72]  W2R[n][k] = W2[n][k]               back-propagation through layer 2
//   W3R[64][24]  W3R[n][k] = W3[n][k] (k < 4)       back-propagation through layer 3
constexpr int S1 = 40, S2 = 72, S3 = 72, SR2 = 72, SR3 = 24;
constexpr int IMG_W1T = 0, IMG_W2T = IMG_W1T + 64 * S1, IMG_W3T = IMG_W2T + 64 * S2, IMG_W2R = IMG_W3T + 8 * S3,
              IMG_W3R = IMG_W2R + 64 * SR2, IMG_END = IMG_W3R + 64 * SR3;  // bf16 elements
constexpr int IMG_BYTES = IMG_END * 2;
constexpr int BIAS_FLOATS = 64 + 64 + 8;

__global__ void k_pack_weights(const float *__restrict__ p, __nv_bfloat16 *__restrict__ img) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < IMG_END; e += gridDim.x * blockDim.x) {
        float v = 0.0f;
        if (e < IMG_W2T) {
            const int n = e / S1, k = e % S1;
            v = k < 30 ? p[OFF_W1 + k * 64 + n] : 0.0f;
        } else if (e < IMG_W3T) {
            const int q = e - IMG_W2T, n = q / S2, k = q % S2;
            v = k < 64 ? p[OFF_W2 + k * 64 + n] : 0.0f;
        } else if (e < IMG_W2R) {
            const int q = e - IMG_W3T, n = q / S3, k = q % S3;
            v = (k < 64 && n < 4) ? p[OFF_W3 + k * 4 + n] : 0.0f;
        } else if (e < IMG_W3R) {
            const int q = e - IMG_W2R, n = q / SR2, k = q % SR2;
            v = k < 64 ? p[OFF_W2 + n * 64 + k] : 0.0f;
        } else {
            const int q = e - IMG_W3R, n = q / SR3, k = q % SR3;
            v = k < 4 ? p[OFF_W3 + n * 4 + k] : 0.0f;
        }
        img[e] = __float2bfloat16_rn(v);
    }
}

// ---------------------------------------------------------------------
// Tensor-core fragments (m16n8k16, row.col).  g = lane / 4, t = lane % 4.
// A (16x16): a0 = (g, 2t..2t+1) a1 = (g+8, 2t..) a2 = (g, 2t+8..) a3 = (g+8, 2t+8..)
// B (16x8):  b0 = (k 2t..2t+1, n g)  b1 = (k 2t+8..2t+9, n g)
// C (16x8):  c0,c1 = (g, 2t..2t+1)   c2,c3 = (g+8, 2t..2t+1)
// ---------------------------------------------------------------------
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}
__device__ __forceinline__ uint32_t lds32(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }
__device__ __forceinline__ uint32_t ldg32(const __nv_bfloat16 *p) { return __ldg(reinterpret_cast<const unsigned int *>(p)); }
// Two adjacent input features (columns c, c+1) standardised and repacked.
__device__ __forceinline__ uint32_t norm2(uint32_t raw, const float *mu, const float *isd, int c) {
    __nv_bfloat162 v = *reinterpret_cast<__nv_bfloat162 *>(&raw);
    return pack2((__low2float(v) - mu[c]) * isd[c], (__high2float(v) - mu[c + 1]) * isd[c + 1]);
}

struct MlpSmem {
    __nv_bfloat16 img[IMG_END];
    float bias[BIAS_FLOATS];  // b1[64] | b2[64] | b3[4] + 4 zeros
    float mu[32], isd[32];    // input standardisation (columns 30, 31: 0)
};

__device__ __forceinline__ void load_mlp_smem(MlpSmem &sm, const __nv_bfloat16 *img, const float *p) {
    const uint32_t *src = reinterpret_cast<const uint32_t *>(img);
    uint32_t *dst = reinterpret_cast<uint32_t *>(sm.img);
    for (int e = threadIdx.x; e < IMG_END / 2; e += blockDim.x) dst[e] = src[e];
    for (int e = threadIdx.x; e < BIAS_FLOATS; e += blockDim.x)
        sm.bias[e] = e < 64 ? p[OFF_B1 + e] : (e < 128 ? p[OFF_B2 + e - 64] : (e < 132 ? p[OFF_B3 + e - 128] : 0.0f));
    for (int e = threadIdx.x; e < 32; e += blockDim.x) {
        sm.mu[e] = e < 30 ? p[OFF_MU + e] : 0.0f;
        sm.isd[e] = e < 30 ? p[OFF_ISD + e] : 0.0f;
    }
    __syncthreads();
}

// Forward of one 16-row tile.  xrow(r) gives the bf16 input row r (30 used,
// 32 stored) or null past the end.  Returns the pre-activations z1, z2 and
// the logits as C fragments.
struct Fwd {
    float z1[8][4], z2[8][4], z3[4];
};

__device__ __forceinline__ void mlp_forward_tile(const MlpSmem &sm, const __nv_bfloat16 *x0, const __nv_bfloat16 *x1,
                                                 Fwd &f) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    // layer 1: x [16 x 32] . W1 [32 x 64]
    uint32_t a[2][4];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int c0 = 16 * s + 2 * t, c1 = c0 + 8;
        a[s][0] = x0 ? norm2(ldg32(x0 + c0), sm.mu, sm.isd, c0) : 0u;
        a[s][1] = x1 ? norm2(ldg32(x1 + c0), sm.mu, sm.isd, c0) : 0u;
        a[s][2] = x0 ? norm2(ldg32(x0 + c1), sm.mu, sm.isd, c1) : 0u;
        a[s][3] = x1 ? norm2(ldg32(x1 + c1), sm.mu, sm.isd, c1) : 0u;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float b0 = sm.bias[8 * j + 2 * t], b1 = sm.bias[8 * j + 2 * t + 1];
        f.z1[j][0] = b0;
        f.z1[j][1] = b1;
        f.z1[j][2] = b0;
        f.z1[j][3] = b1;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const __nv_bfloat16 *w = sm.img + IMG_W1T + (8 * j + g) * S1 + 16 * s + 2 * t;
            mma_bf16(f.z1[j], a[s], lds32(w), lds32(w + 8));
        }
    }
    // layer 2: relu(z1) [16 x 64] . W2 [64 x 64]
    uint32_t h[4][4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        h[s][0] = pack2(fmaxf(f.z1[2 * s][0], 0.f), fmaxf(f.z1[2 * s][1], 0.f));
        h[s][1] = pack2(fmaxf(f.z1[2 * s][2], 0.f), fmaxf(f.z1[2 * s][3], 0.f));
        h[s][2] = pack2(fmaxf(f.z1[2 * s + 1][0], 0.f), fmaxf(f.z1[2 * s + 1][1], 0.f));
        h[s][3] = pack2(fmaxf(f.z1[2 * s + 1][2], 0.f), fmaxf(f.z1[2 * s + 1][3], 0.f));
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float b0 = sm.bias[64 + 8 * j + 2 * t], b1 = sm.bias[64 + 8 * j + 2 * t + 1];
        f.z2[j][0] = b0;
        f.z2[j][1] = b1;
        f.z2[j][2] = b0;
        f.z2[j][3] = b1;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const __nv_bfloat16 *w = sm.img + IMG_W2T + (8 * j + g) * S2 + 16 * s + 2 * t;
            mma_bf16(f.z2[j], h[s], lds32(w), lds32(w + 8));
        }
    }
    // layer 3: relu(z2) [16 x 64] . W3 [64 x 8 (4 used)]
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        h[s][0] = pack2(fmaxf(f.z2[2 * s][0], 0.f), fmaxf(f.z2[2 * s][1], 0.f));
        h[s][1] = pack2(fmaxf(f.z2[2 * s][2], 0.f), fmaxf(f.z2[2 * s][3], 0.f));
        h[s][2] = pack2(fmaxf(f.z2[2 * s + 1][0], 0.f), fmaxf(f.z2[2 * s + 1][1], 0.f));
        h[s][3] = pack2(fmaxf(f.z2[2 * s + 1][2], 0.f), fmaxf(f.z2[2 * s + 1][3], 0.f));
    }
    {
        const float b0 = sm.bias[128 + 2 * t], b1 = sm.bias[128 + 2 * t + 1];
        f.z3[0] = b0;
        f.z3[1] = b1;
        f.z3[2] = b0;
        f.z3[3] = b1;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const __nv_bfloat16 *w = sm.img + IMG_W3T + g * S3 + 16 * s + 2 * t;
            mma_bf16(f.z3, h[s], lds32(w), lds32(w + 8));
        }
    }
}

// The four logits of the rows g and g+8 of a tile, in every lane of the quad.
__device__ __forceinline__ void quad_logits(const float (&z3)[4], float (&la)[4], float (&lb)[4]) {
    const int base = (threadIdx.x & 31) & ~3;
    la[0] = __shfl_sync(0xffffffffu, z3[0], base);
    la[1] = __shfl_sync(0xffffffffu, z3[1], base);
    la[2] = __shfl_sync(0xffffffffu, z3[0], base + 1);
    la[3] = __shfl_sync(0xffffffffu, z3[1], base + 1);
    lb[0] = __shfl_sync(0xffffffffu, z3[2], base);
    lb[1] = __shfl_sync(0xffffffffu, z3[3], base);
    lb[2] = __shfl_sync(0xffffffffu, z3[2], base + 1);
    lb[3] = __shfl_sync(0xffffffffu, z3[3], base + 1);
}

__device__ __forceinline__ void softmax4(const float (&l)[4], float (&p)[4]) {
    const float m = fmaxf(fmaxf(l[0], l[1]), fmaxf(l[2], l[3]));
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        p[c] = __expf(l[c] - m);
        s += p[c];
    }
    const float is = 1.0f / s;
#pragma unroll
    for (int c = 0; c < 4; ++c) p[c] *= is;
}

constexpr int MLP_WARPS = 4;

// ---------------------------------------------------------------------
// Training: forward and back-propagation of one tile per warp.  Stores, per
// sample, h1 = relu(z1), h2 = relu(z2), d1 = dL/dz1, d2 = dL/dz2 (bf16
// [B][64]) and d3 = dL/dz3 (bf16 [B][8], 4 used), L = mean cross entropy.
// ---------------------------------------------------------------------
__device__ __forceinline__ void store_tile64(__nv_bfloat16 *dst, int64_t r0, int64_t r1, int64_t B, const float (&c)[8][4],
                                             bool relu) {
    const int t = threadIdx.x & 3;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float v0 = c[j][0], v1 = c[j][1], v2 = c[j][2], v3 = c[j][3];
        if (relu) {
            v0 = fmaxf(v0, 0.f);
            v1 = fmaxf(v1, 0.f);
            v2 = fmaxf(v2, 0.f);
            v3 = fmaxf(v3, 0.f);
        }
        if (r0 < B) *reinterpret_cast<uint32_t *>(dst + r0 * 64 + 8 * j + 2 * t) = pack2(v0, v1);
        if (r1 < B) *reinterpret_cast<uint32_t *>(dst + r1 * 64 + 8 * j + 2 * t) = pack2(v2, v3);
    }
}

__global__ void __launch_bounds__(MLP_WARPS * 32) k_mlp_fwd_bwd(int64_t B, const __nv_bfloat16 *__restrict__ x,
                                                                const int8_t *__restrict__ y,
                                                                const __nv_bfloat16 *__restrict__ img,
                                                                const float *__restrict__ p,
                                                                __nv_bfloat16 *__restrict__ H1, __nv_bfloat16 *__restrict__ H2,
                                                                __nv_bfloat16 *__restrict__ D1, __nv_bfloat16 *__restrict__ D2,
                                                                __nv_bfloat16 *__restrict__ D3, double *__restrict__ loss_part) {
    __shared__ MlpSmem sm;
    __shared__ double s_loss[MLP_WARPS];
    load_mlp_smem(sm, img, p);
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, w = threadIdx.x >> 5;
    const int64_t ntile = (B + 15) / 16;
    const float invB = 1.0f / (float)B;
    double loss = 0.0;
    for (int64_t tile = (int64_t)blockIdx.x * MLP_WARPS + w; tile < ntile; tile += (int64_t)gridDim.x * MLP_WARPS) {
        const int64_t r0 = tile * 16 + g, r1 = r0 + 8;
        Fwd f;
        mlp_forward_tile(sm, r0 < B ? x + r0 * 32 : nullptr, r1 < B ? x + r1 * 32 : nullptr, f);
        store_tile64(H1, r0, r1, B, f.z1, true);
        store_tile64(H2, r0, r1, B, f.z2, true);
        // dL/dz3 = (softmax - onehot) / B for the rows g (lanes t=0) and g+8
        float la[4], lb[4], pa[4], pb[4];
        quad_logits(f.z3, la, lb);
        softmax4(la, pa);
        softmax4(lb, pb);
        const int ya = r0 < B ? y[r0] : -1, yb = r1 < B ? y[r1] : -1;
        if (t == 0) {
            if (ya >= 0) loss -= log((double)pa[ya]) / (double)B;
            if (yb >= 0) loss -= log((double)pb[yb]) / (double)B;
        }
        // this thread's C-layout columns of d3: 2t, 2t+1 (valid for t < 2)
        float d3[4] = {0.f, 0.f, 0.f, 0.f};
        if (t < 2) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int c = 2 * t + q;
                d3[q] = ya >= 0 ? (pa[c] - (c == ya ? 1.0f : 0.0f)) * invB : 0.f;
                d3[2 + q] = yb >= 0 ? (pb[c] - (c == yb ? 1.0f : 0.0f)) * invB : 0.f;
            }
        }
        if (t < 4) {
            if (r0 < B) *reinterpret_cast<uint32_t *>(D3 + r0 * 8 + 2 * t) = pack2(d3[0], d3[1]);
            if (r1 < B) *reinterpret_cast<uint32_t *>(D3 + r1 * 8 + 2 * t) = pack2(d3[2], d3[3]);
        }
        // dL/dh2 = d3 . W3^T (K = 4, padded to 16), masked by z2 > 0
        uint32_t a3[4] = {pack2(d3[0], d3[1]), pack2(d3[2], d3[3]), 0u, 0u};
        float d2[8][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            d2[j][0] = d2[j][1] = d2[j][2] = d2[j][3] = 0.f;
            const __nv_bfloat16 *wr = sm.img + IMG_W3R + (8 * j + g) * SR3 + 2 * t;
            mma_bf16(d2[j], a3, lds32(wr), lds32(wr + 8));
#pragma unroll
            for (int e = 0; e < 4; ++e) d2[j][e] = f.z2[j][e] > 0.f ? d2[j][e] : 0.f;
        }
        store_tile64(D2, r0, r1, B, d2, false);
        // dL/dh1 = d2 . W2^T, masked by z1 > 0
        uint32_t a2[4][4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            a2[s][0] = pack2(d2[2 * s][0], d2[2 * s][1]);
            a2[s][1] = pack2(d2[2 * s][2], d2[2 * s][3]);
            a2[s][2] = pack2(d2[2 * s + 1][0], d2[2 * s + 1][1]);
            a2[s][3] = pack2(d2[2 * s + 1][2], d2[2 * s + 1][3]);
        }
        float d1[8][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            d1[j][0] = d1[j][1] = d1[j][2] = d1[j][3] = 0.f;
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const __nv_bfloat16 *wr = sm.img + IMG_W2R + (8 * j + g) * SR2 + 16 * s + 2 * t;
                mma_bf16(d1[j], a2[s], lds32(wr), lds32(wr + 8));
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) d1[j][e] = f.z1[j][e] > 0.f ? d1[j][e] : 0.f;
        }
        store_tile64(D1, r0, r1, B, d1, false);
    }
    loss = warp_sum(loss);
    if (lane == 0) s_loss[w] = loss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < MLP_WARPS; ++q) s += s_loss[q];
        loss_part[blockIdx.x] = s;
    }
}

// ---------------------------------------------------------------------
// Weight gradients, split over the batch: block b sums its chunk of
// samples.  dW1 = x^T d1 (32 x 64), dW2 = h1^T d2 (64 x 64), dW3 = h2^T d3
// (64 x 8), on tensor cores with the samples as the contraction index;
// bias gradients are column sums of d1, d2, d3.  Warp 0/1: dW2 rows 0-31 /
// 32-63; warp 2: dW1; warp 3: dW3 and the biases.  Partials [blocks][NPARAM].
// ---------------------------------------------------------------------
constexpr int WG_ROWS = 64;  // samples staged per step

// A(m, k) = act[k][m] for m-tile mt, k-step rows kk (smem, row stride ld)
__device__ __forceinline__ void frag_At(uint32_t (&a)[4], const __nv_bfloat16 *act, int ld, int mt, int kk) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int m0 = 16 * mt + g, k0 = kk + 2 * t;
    auto e = [&](int k, int m) { return act[k * ld + m]; };
    __nv_bfloat162 v;
    v.x = e(k0, m0);
    v.y = e(k0 + 1, m0);
    a[0] = *reinterpret_cast<uint32_t *>(&v);
    v.x = e(k0, m0 + 8);
    v.y = e(k0 + 1, m0 + 8);
    a[1] = *reinterpret_cast<uint32_t *>(&v);
    v.x = e(k0 + 8, m0);
    v.y = e(k0 + 9, m0);
    a[2] = *reinterpret_cast<uint32_t *>(&v);
    v.x = e(k0 + 8, m0 + 8);
    v.y = e(k0 + 9, m0 + 8);
    a[3] = *reinterpret_cast<uint32_t *>(&v);
}
// B(k, n) = d[k][n] for n-tile nt
__device__ __forceinline__ void frag_B(uint32_t &b0, uint32_t &b1, const __nv_bfloat16 *d, int ld, int nt, int kk) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int n = 8 * nt + g, k0 = kk + 2 * t;
    __nv_bfloat162 v;
    v.x = d[k0 * ld + n];
    v.y = d[(k0 + 1) * ld + n];
    b0 = *reinterpret_cast<uint32_t *>(&v);
    v.x = d[(k0 + 8) * ld + n];
    v.y = d[(k0 + 9) * ld + n];
    b1 = *reinterpret_cast<uint32_t *>(&v);
}

__global__ void __launch_bounds__(128) k_mlp_wgrad(int64_t B, int64_t chunk, const __nv_bfloat16 *__restrict__ x,
                                                   const __nv_bfloat16 *__restrict__ H1,
                                                   const __nv_bfloat16 *__restrict__ H2,
                                                   const __nv_bfloat16 *__restrict__ D1,
                                                   const __nv_bfloat16 *__restrict__ D2,
                                                   const __nv_bfloat16 *__restrict__ D3, const float *__restrict__ p,
                                                   float *__restrict__ part) {
    // staged rows (padded strides against bank conflicts)
    __shared__ __nv_bfloat16 sx[WG_ROWS][40], sh1[WG_ROWS][72], sh2[WG_ROWS][72], sd1[WG_ROWS][72], sd2[WG_ROWS][72],
        sd3[WG_ROWS][8];
    __shared__ float smu[32], sisd[32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int64_t s0 = (int64_t)blockIdx.x * chunk, s1 = min(B, s0 + chunk);
    if (threadIdx.x < 32) {
        smu[threadIdx.x] = threadIdx.x < 30 ? p[OFF_MU + threadIdx.x] : 0.0f;
        sisd[threadIdx.x] = threadIdx.x < 30 ? p[OFF_ISD + threadIdx.x] : 0.0f;
    }
    float acc[16][4];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
    float bsum[5] = {0.f, 0.f, 0.f, 0.f, 0.f};  // warp 3: bias columns lane, lane+32 of d1, d2; lane < 4 of d3
    for (int64_t base = s0; base < s1; base += WG_ROWS) {
        __syncthreads();
        for (int e = threadIdx.x; e < WG_ROWS * 32; e += blockDim.x) {
            const int r = e / 32, c = e % 32;
            const int64_t row = base + r;
            const bool ok = row < s1;
            // 32-bit words: x row = 16 words, 64-wide rows = 32 words, d3 row = 4 words
            if (c < 16)
                *reinterpret_cast<uint32_t *>(&sx[r][2 * c]) = ok ? norm2(ldg32(x + row * 32 + 2 * c), smu, sisd, 2 * c) : 0u;
            *reinterpret_cast<uint32_t *>(&sh1[r][2 * c]) = ok ? ldg32(H1 + row * 64 + 2 * c) : 0u;
            *reinterpret_cast<uint32_t *>(&sh2[r][2 * c]) = ok ? ldg32(H2 + row * 64 + 2 * c) : 0u;
            *reinterpret_cast<uint32_t *>(&sd1[r][2 * c]) = ok ? ldg32(D1 + row * 64 + 2 * c) : 0u;
            *reinterpret_cast<uint32_t *>(&sd2[r][2 * c]) = ok ? ldg32(D2 + row * 64 + 2 * c) : 0u;
            if (c < 4) *reinterpret_cast<uint32_t *>(&sd3[r][2 * c]) = ok ? ldg32(D3 + row * 8 + 2 * c) : 0u;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < WG_ROWS; kk += 16) {
            if (w < 2) {  // dW2 rows 32w .. 32w+31
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    uint32_t a[4];
                    frag_At(a, &sh1[0][0], 72, 2 * w + mt, kk);
#pragma unroll
                    for (int nt = 0; nt < 8; ++nt) {
                        uint32_t b0, b1;
                        frag_B(b0, b1, &sd2[0][0], 72, nt, kk);
                        mma_bf16(acc[mt * 8 + nt], a, b0, b1);
                    }
                }
            } else if (w == 2) {  // dW1 (32 x 64)
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    uint32_t a[4];
                    frag_At(a, &sx[0][0], 40, mt, kk);
#pragma unroll
                    for (int nt = 0; nt < 8; ++nt) {
                        uint32_t b0, b1;
                        frag_B(b0, b1, &sd1[0][0], 72, nt, kk);
                        mma_bf16(acc[mt * 8 + nt], a, b0, b1);
                    }
                }
            } else {  // dW3 (64 x 8)
#pragma unroll
                for (int mt = 0; mt < 4; ++mt) {
                    uint32_t a[4];
                    frag_At(a, &sh2[0][0], 72, mt, kk);
                    uint32_t b0, b1;
                    frag_B(b0, b1, &sd3[0][0], 8, 0, kk);
                    mma_bf16(acc[mt], a, b0, b1);
                }
            }
        }
        if (w == 3) {
            const int rows = (int)min((int64_t)WG_ROWS, s1 - base);
            for (int r = 0; r < rows; ++r) {
                bsum[0] += __bfloat162float(sd1[r][lane]);
                bsum[1] += __bfloat162float(sd1[r][lane + 32]);
                bsum[2] += __bfloat162float(sd2[r][lane]);
                bsum[3] += __bfloat162float(sd2[r][lane + 32]);
                if (lane < 4) bsum[4] += __bfloat162float(sd3[r][lane]);
            }
        }
    }
    float *out = part + (int64_t)blockIdx.x * NPARAM;
    // C fragment (row m, col n) of tile (mt, nt) -> parameter W[m][n]
    if (w < 2) {
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const int m = 32 * w + 16 * mt + g, n = 8 * nt + 2 * t;
                out[OFF_W2 + m * 64 + n] = acc[mt * 8 + nt][0];
                out[OFF_W2 + m * 64 + n + 1] = acc[mt * 8 + nt][1];
                out[OFF_W2 + (m + 8) * 64 + n] = acc[mt * 8 + nt][2];
                out[OFF_W2 + (m + 8) * 64 + n + 1] = acc[mt * 8 + nt][3];
            }
    } else if (w == 2) {
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const int m = 16 * mt + g, n = 8 * nt + 2 * t;
                if (m < 30) {
                    out[OFF_W1 + m * 64 + n] = acc[mt * 8 + nt][0];
                    out[OFF_W1 + m * 64 + n + 1] = acc[mt * 8 + nt][1];
                }
                if (m + 8 < 30) {
                    out[OFF_W1 + (m + 8) * 64 + n] = acc[mt * 8 + nt][2];
                    out[OFF_W1 + (m + 8) * 64 + n + 1] = acc[mt * 8 + nt][3];
                }
            }
    } else {
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) {
            const int m = 16 * mt + g, n = 2 * t;
            if (n < 4) {
                out[OFF_W3 + m * 4 + n] = acc[mt][0];
                out[OFF_W3 + m * 4 + n + 1] = acc[mt][1];
                out[OFF_W3 + (m + 8) * 4 + n] = acc[mt][2];
                out[OFF_W3 + (m + 8) * 4 + n + 1] = acc[mt][3];
            }
        }
        out[OFF_B1 + lane] = bsum[0];
        out[OFF_B1 + lane + 32] = bsum[1];
        out[OFF_B2 + lane] = bsum[2];
        out[OFF_B2 + lane + 32] = bsum[3];
        if (lane < 4) out[OFF_B3 + lane] = bsum[4];
        for (int e = lane; e < OFF_W1; e += 32) out[e] = 0.0f;  // the standardisation is not trained
    }
}

// Fixed-order sum of the per-block partials.
__global__ void k_sum_partials(const float *__restrict__ part, int nblk, float *__restrict__ grad) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NPARAM) return;
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * NPARAM + e];
    grad[e] = s;
}

// AdamW (decoupled weight decay on the weight matrices only), step t >= 1.
__global__ void k_adamw(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v, const float *__restrict__ g,
                        float lr, float wd, float b1, float b2, float eps, float c1, float c2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NPARAM) return;
    if (e < OFF_W1) return;  // input standardisation: fitted, not trained
    const bool weight = (e < OFF_B1) || (e >= OFF_W2 && e < OFF_B2) || (e >= OFF_W3 && e < OFF_B3);
    const float gr = g[e];
    const float mm = b1 * m[e] + (1.0f - b1) * gr;
    const float vv = b2 * v[e] + (1.0f - b2) * gr * gr;
    m[e] = mm;
    v[e] = vv;
    float pe = p[e];
    if (weight) pe -= lr * wd * pe;
    pe -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    p[e] = pe;
}

__global__ void k_sum_loss(const double *part, int nblk, float *loss) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[b];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = (float)sh[0];
}

// Input standardisation from n feature rows: per feature (thread f of 32)
// sums of x and x^2 over rows, compensated (Kahan) in FP32 per thread (FP64
// arithmetic is slow on this part), then in FP64 across threads and blocks;
// one partial per block.
__global__ void k_feat_stats(int64_t n, const __nv_bfloat16 *__restrict__ x, double *__restrict__ part) {
    __shared__ double sh[8][32][2];
    const int f = threadIdx.x & 31, rl = threadIdx.x >> 5;
    float a = 0.0f, ac = 0.0f, b = 0.0f, bc = 0.0f;  // sums and their compensations
    for (int64_t r = (int64_t)blockIdx.x * 8 + rl; r < n; r += (int64_t)gridDim.x * 8) {
        const float v = __bfloat162float(x[r * 32 + f]);
        const float y1 = v - ac, t1 = a + y1;
        ac = (t1 - a) - y1;
        a = t1;
        const float y2 = fmaf(v, v, -bc), t2 = b + y2;
        bc = (t2 - b) - y2;
        b = t2;
    }
    double s = (double)a - (double)ac, s2 = (double)b - (double)bc;
    sh[rl][f][0] = s;
    sh[rl][f][1] = s2;
    __syncthreads();
    if (rl == 0) {
        for (int q = 1; q < 8; ++q) {
            s += sh[q][f][0];
            s2 += sh[q][f][1];
        }
        part[(blockIdx.x * 32 + f) * 2] = s;
        part[(blockIdx.x * 32 + f) * 2 + 1] = s2;
    }
}

__global__ void k_feat_norm(const double *__restrict__ part, int nblk, int64_t n, float *__restrict__ p) {
    const int f = threadIdx.x;
    if (f >= 30) return;
    double s = 0.0, s2 = 0.0;
    for (int b = 0; b < nblk; ++b) {
        s += part[(b * 32 + f) * 2];
        s2 += part[(b * 32 + f) * 2 + 1];
    }
    const double mu = s / (double)n, var = fmax(s2 / (double)n - mu * mu, 0.0);
    p[OFF_MU + f] = (float)mu;
    p[OFF_ISD + f] = var > 1e-12 ? (float)(1.0 / sqrt(var)) : 1.0f;
}

int pack_weights(ppmd_ctx *ctx, const float *params, __nv_bfloat16 **img) {
    *img = (__nv_bfloat16 *)scratch(ctx, S_AUX3, IMG_BYTES);
    if (!*img) return PPMD_ERR_NOMEM;
    PPMD_LAUNCH(ctx, k_pack_weights, div_up(IMG_END, 256), 256, 0, params, *img);
    return check_launch(ctx, "pack_weights");
}

int mlp_grid(int64_t tiles) {
    int64_t b = (tiles + MLP_WARPS - 1) / MLP_WARPS;
    return (int)std::min<int64_t>(b, 148 * 16);
}

}  // namespace ppmd

using namespace ppmd;

extern "C" int ppmd_mlp_forward(ppmd_ctx *ctx, const float *params, const uint16_t *x, int64_t n, float *logits) {
    if (!ctx || !params || n < 0 || (n > 0 && (!x || !logits))) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_mlp_forward: bad argument");
    cudaSetDevice(ctx->device);
    return mlp_infer_tc(ctx, n, (const __nv_bfloat16 *)x, params, logits, nullptr, nullptr, 0.0f, nullptr, nullptr);
}

extern "C" int ppmd_mlp_grad(ppmd_ctx *ctx, const float *params, const uint16_t *x, const int8_t *y, int64_t batch,
                             float *grad, float *loss) {
    if (!ctx || !params || batch < 1 || !x || !y || !grad) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_mlp_grad: bad argument");
    cudaSetDevice(ctx->device);
    __nv_bfloat16 *img;
    PPMD_TRY(pack_weights(ctx, params, &img));
    const size_t rows = (size_t)batch;
    __nv_bfloat16 *act = (__nv_bfloat16 *)scratch(ctx, S_AUX1, sizeof(__nv_bfloat16) * rows * (4 * 64 + 8));
    if (!act) return PPMD_ERR_NOMEM;
    __nv_bfloat16 *H1 = act, *H2 = H1 + rows * 64, *D1 = H2 + rows * 64, *D2 = D1 + rows * 64, *D3 = D2 + rows * 64;
    const int fb_grid = mlp_grid((batch + 15) / 16);
    const int64_t chunk = std::max<int64_t>(WG_ROWS, ((batch + 255) / 256 + WG_ROWS - 1) / WG_ROWS * WG_ROWS);
    const int wg_grid = (int)((batch + chunk - 1) / chunk);
    double *lpart = (double *)scratch(ctx, S_AUX2, sizeof(double) * fb_grid + sizeof(float) * (size_t)wg_grid * NPARAM + 64);
    if (!lpart) return PPMD_ERR_NOMEM;
    float *wpart = (float *)(lpart + fb_grid);
    PPMD_LAUNCH(ctx, k_mlp_fwd_bwd, fb_grid, MLP_WARPS * 32, 0, batch, (const __nv_bfloat16 *)x, y, img, params, H1, H2, D1, D2,
                D3, lpart);
    PPMD_LAUNCH(ctx, k_mlp_wgrad, wg_grid, 128, 0, batch, chunk, (const __nv_bfloat16 *)x, H1, H2, D1, D2, D3, params,
                wpart);
    PPMD_LAUNCH(ctx, k_sum_partials, div_up(NPARAM, 256), 256, 0, wpart, wg_grid, grad);
    if (loss) PPMD_LAUNCH(ctx, k_sum_loss, 1, 256, 0, lpart, fb_grid, loss);
    return check_launch(ctx, "ppmd_mlp_grad");
}

extern "C" int ppmd_mlp_fit_input_norm(ppmd_ctx *ctx, float *params, const uint16_t *x, int64_t n) {
    if (!ctx || !params || n < 1 || !x) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_mlp_fit_input_norm: bad argument");
    cudaSetDevice(ctx->device);
    const int nblk = 256;
    double *part = (double *)scratch(ctx, S_AUX2, sizeof(double) * nblk * 64);
    if (!part) return PPMD_ERR_NOMEM;
    PPMD_LAUNCH(ctx, k_feat_stats, nblk, 256, 0, n, (const __nv_bfloat16 *)x, part);
    PPMD_LAUNCH(ctx, k_feat_norm, 1, 32, 0, part, nblk, n, params);
    return check_launch(ctx, "ppmd_mlp_fit_input_norm");
}

extern "C" int ppmd_mlp_adamw(ppmd_ctx *ctx, float *params, float *m, float *v, const float *grad, int64_t step, float lr,
                              float wd, float beta1, float beta2, float eps) {
    if (!ctx || !params || !m || !v || !grad || step < 1) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_mlp_adamw: bad argument");
    cudaSetDevice(ctx->device);
    const float c1 = (float)(1.0 - pow((double)beta1, (double)step)), c2 = (float)(1.0 - pow((double)beta2, (double)step));
    PPMD_LAUNCH(ctx, k_adamw, div_up(NPARAM, 256), 256, 0, params, m, v, grad, lr, wd, beta1, beta2, eps, c1, c2);
    return check_launch(ctx, "ppmd_mlp_adamw");
}

extern "C" int ppmd_mlp_train_step(ppmd_ctx *ctx, float *params, float *m, float *v, int64_t step, const uint16_t *x,
                                   const int8_t *y, int64_t batch, float lr, float wd, float *loss) {
    float *grad = (float *)scratch(ctx, S_AUX0, sizeof(float) * NPARAM);
    if (!grad) return PPMD_ERR_NOMEM;
    PPMD_TRY(ppmd_mlp_grad(ctx, params, x, y, batch, grad, loss));
    return ppmd_mlp_adamw(ctx, params, m, v, grad, step, lr, wd, 0.9f, 0.999f, 1e-8f);
}

// ---------------------------------------------------------------------
// Classification pipeline: features, MLP class and confidence written in
// the caller's order, exact CNA over the low-confidence atoms written over
// their class.
// ---------------------------------------------------------------------
extern "C" int ppmd_classify_boxes(ppmd_ctx *ctx, int mode, const double *pos, int64_t nbox, const int64_t *atom_off,
                                   const ppmd_box *boxes, double r_feat, double r_cna, const float *params, float threshold,
                                   int8_t *label, float *confidence, int64_t *n_fallback) {
    if (!ctx) return PPMD_ERR_INVALID;
    PPMD_TRY(check_boxes(ctx, nbox, atom_off, boxes, "ppmd_classify"));
    const int64_t n = atom_off[nbox];
    if ((n > 0 && (!pos || !label)) || mode < 0 || mode > 2 || (mode == 1 && !params) ||
        (mode != 2 && !(r_cna > 0)) || (mode == 1 && !(r_feat >= r_cna)) || (mode == 2 && !(r_feat > 0)) ||
        (mode == 2 && !(threshold >= 0.0f)))
        return set_error(ctx, PPMD_ERR_INVALID, "ppmd_classify: bad argument");
    cudaSetDevice(ctx->device);
    if (mode == 0) {
        if (n_fallback) *n_fallback = n;
        return ppmd_analyze_boxes(ctx, pos, nbox, atom_off, boxes, 0.0, r_cna, nullptr, nullptr, nullptr, label);
    }
    const size_t nn = (size_t)(n > 0 ? n : 1);
    if (mode == 2) {
        // bond order within a tolerance: Q4, Q6 over r_feat, nearest table value
        float *q = (float *)scratch(ctx, S_TMP0, sizeof(float) * 2 * nn);
        if (!q) return PPMD_ERR_NOMEM;
        int32_t max_nbr = snapshot_capacity_boxes(nbox, atom_off, boxes, r_feat);
        for (int attempt = 0;; ++attempt) {
            Snapshot s;
            PPMD_TRY(sorted_snapshot_boxes(ctx, pos, nbox, atom_off, boxes, r_feat, max_nbr, s));
            PPMD_TRY(boa_launch(ctx, n, s.xq, s.pos, s.st, s.nbr, s.cnt, s.max_nbr, s.ld, r_feat, s.Lmax, s.perm, q, q + nn,
                                nullptr));
            PPMD_TRY(boa_tolerance_launch(ctx, n, q, q + nn, threshold, label, confidence));
            if (!n_fallback) return check_launch(ctx, "ppmd_classify");
            const int rc = end_pipeline(ctx, attempt, max_nbr);
            if (rc == PIPELINE_RETRY) continue;
            *n_fallback = 0;
            return rc;
        }
    }
    int32_t max_nbr = snapshot_capacity_boxes(nbox, atom_off, boxes, r_feat);
    for (int attempt = 0;; ++attempt) {
        Snapshot s;
        PPMD_TRY(sorted_snapshot_boxes(ctx, pos, nbox, atom_off, boxes, r_feat, max_nbr, s));
        __nv_bfloat16 *feat = (__nv_bfloat16 *)scratch(ctx, S_TMP0, sizeof(__nv_bfloat16) * 32 * nn);
        int32_t *fb = (int32_t *)scratch(ctx, S_AUX1, sizeof(int32_t) * nn);
        if (!feat || !fb) return PPMD_ERR_NOMEM;
        int32_t *nfb = ctx->d_status + 4;  // the fallback count, read back with the status
        PPMD_TRY(features_launch(ctx, n, s.xq, s.pos, s.st, s.nbr, s.cnt, s.max_nbr, s.ld, r_feat, r_cna, s.Lmax, nullptr,
                                 nullptr, feat));
        // MLP class and confidence of every atom, in the caller's order
        PPMD_TRY(mlp_infer_tc(ctx, n, feat, params, nullptr, label, confidence, threshold, fb, nfb, s.perm));
        // exact CNA for the low-confidence atoms (as many as the device
        // found), written over their MLP class
        PPMD_TRY(cna_subset_launch(ctx, n, nfb, fb, s.xq, s.pos, s.st, s.nbr, s.cnt, s.max_nbr, s.ld, r_cna, s.Lmax,
                                   s.perm, label));
        PPMD_TRY(check_launch(ctx, "ppmd_classify"));
        if (!n_fallback) return PPMD_OK;  // asynchronous: an overflow stays latched
        int32_t hfb = 0;
        const int rc = end_pipeline(ctx, attempt, max_nbr, &hfb);
        if (rc == PIPELINE_RETRY) continue;
        *n_fallback = hfb;
        return rc;
    }
}

extern "C" int ppmd_classify(ppmd_ctx *ctx, int mode, const double *pos, int64_t n, const ppmd_box *box, double r_feat,
                             double r_cna, const float *params, float threshold, int8_t *label, float *confidence,
                             int64_t *n_fallback) {
    if (!ctx || !box || n < 0) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_classify: bad argument");
    const int64_t off[2] = {0, n};
    return ppmd_classify_boxes(ctx, mode, pos, 1, off, box, r_feat, r_cna, params, threshold, label, confidence,
                               n_fallback);
}
