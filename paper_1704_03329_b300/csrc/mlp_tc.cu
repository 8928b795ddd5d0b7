// Classifier MLP inference (30 -> 64 -> 64 -> 4, ReLU, softmax) on the
// tcgen05 tensor cores.
//
// One CTA of 128 threads handles 128-row tiles (persistent over the tiles):
// thread t owns row t of a tile, which is also lane t of the tile's
// accumulators in tensor memory.  Per tile:
//   1. every thread standardises its feature row, converts it to BF16 and
//      writes it to shared memory (operand A of layer 1);
//   2. one thread issues the layer's tcgen05.mma instructions (M = 128,
//      K = 16 each, BF16 inputs, FP32 accumulation into tensor memory) and
//      commits them to an mbarrier; every thread waits on it (bounded);
//   3. every warp reads its 32 lanes of the accumulator (tcgen05.ld), adds
//      the bias, applies ReLU and writes the BF16 activations back to shared
//      memory as operand A of the next layer;
//   4. after layer 3 (N padded to 16) the logits give class, confidence and
//      the fallback list.
// Each thread loads its feature row of the next tile while the current one
// is processed; up to seven CTAs share an SM.
// The weights (operand B), biases and standardisation are packed once per
// call and brought into each CTA by one bulk copy (cp.async.bulk).
//
// Operands use the non-swizzled K-major layout of the tensor cores: 8-row x
// 16-byte core matrices (8 BF16 values of K per row, rows 16 bytes apart);
// the core matrix holding (row r, k) of an R-row operand sits at
// ((k / 8) * (R / 8) + r / 8) * 128 bytes, so consecutive core matrices
// along K are R * 16 bytes apart (the descriptor's leading-dimension offset)
// and consecutive 8-row groups 128 bytes apart (its stride-dimension offset).
#include <cuda_bf16.h>

#include "mlp_layout.cuh"
#include "mlp_tc.cuh"

namespace ppmd {
namespace {

constexpr int TC_ROWS = 128;
// shared-memory map (bytes from the 1024-aligned dynamic base)
// X (A of layer 1, 128 x 32 BF16) and H (A of layers 2 and 3, 128 x 64)
// share one region: each is written only after the tensor cores finished
// reading the other.
constexpr uint32_t SM_X = 0;
constexpr uint32_t SM_H = 0;
constexpr uint32_t SM_W1 = 16384;         // B of layer 1: 64 x 32 (n x k)
constexpr uint32_t SM_W2 = SM_W1 + 4096;  // B of layer 2: 64 x 64
constexpr uint32_t SM_W3 = SM_W2 + 8192;  // B of layer 3: 16 x 64 (n >= 4 zero)
constexpr uint32_t SM_BIAS = SM_W3 + 2048;    // b1[64] b2[64] b3[16] (floats)
constexpr uint32_t SM_NORM = SM_BIAS + 576;   // mu[32] isd[32]
constexpr uint32_t SM_BAR = SM_NORM + 256;    // mbarrier (8 bytes) + tensor-memory address (4 bytes)
constexpr uint32_t SM_USED = SM_BAR + 16;
// Requested dynamic shared memory: at most seven CTAs per SM, so that their
// tensor memory (64 columns each) stays within the SM's 512 columns.
constexpr uint32_t SM_REQUEST = 32 * 1024;
static_assert(SM_USED <= SM_REQUEST, "shared memory map");
constexpr uint32_t TMEM_COLS = 64;  // every layer's accumulator at column 0, read before the next layer
constexpr int TC_CTAS_PER_SM = 7;
constexpr uint32_t WAIT_LIMIT = 1u << 22;

__device__ __forceinline__ uint32_t core_off(int r, int k, int R) {
    return (uint32_t)((((k >> 3) * (R >> 3)) + (r >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor: start address, leading-dimension (K)
// byte offset, stride-dimension byte offset (each encoded >> 4), the fixed
// version bits 0b001 at bit 46, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B,
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t instr_desc(int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TC_ROWS >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16_tc(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n"
            ".reg .pred p;\n"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n"
            "}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r[c]);
}

__device__ __forceinline__ uint32_t pk_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

// Eight BF16 values of K (one 16-byte row of a core matrix).
__device__ __forceinline__ void st_chunk(uint8_t *smem, uint32_t off, const float (&v)[8]) {
    uint4 q;
    q.x = pk_bf16(v[0], v[1]);
    q.y = pk_bf16(v[2], v[3]);
    q.z = pk_bf16(v[4], v[5]);
    q.w = pk_bf16(v[6], v[7]);
    *reinterpret_cast<uint4 *>(smem + off) = q;
}

// Layer output of this thread's row: bias + ReLU, BF16, into operand H.
__device__ __forceinline__ void relu_to_h(uint8_t *smem, uint32_t t_lane, const float *bias) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float v[16];
        tmem_ld16(t_lane + 16 * q, v);
        float lo[8], hi[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            lo[c] = fmaxf(v[c] + bias[16 * q + c], 0.0f);
            hi[c] = fmaxf(v[8 + c] + bias[16 * q + 8 + c], 0.0f);
        }
        const int r = threadIdx.x;
        st_chunk(smem, SM_H + core_off(r, 16 * q, TC_ROWS), lo);
        st_chunk(smem, SM_H + core_off(r, 16 * q + 8, TC_ROWS), hi);
    }
}

// The shared-memory image from SM_W1 on (weights as operand B in BF16,
// biases, standardisation), built once per call in global memory and
// copied into each CTA by one bulk copy.
constexpr uint32_t IMG_TC_BYTES = SM_BAR - SM_W1;
static_assert(IMG_TC_BYTES % 16 == 0, "bulk copies move multiples of 16 bytes");

__global__ void k_pack_tc(const float *__restrict__ p, uint8_t *__restrict__ img) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 64 * 32 + 64 * 64 + 16 * 64 + 144 + 64;
         e += gridDim.x * blockDim.x) {
        if (e < 64 * 32) {
            const int nn = e >> 5, k = e & 31;
            *reinterpret_cast<__nv_bfloat16 *>(img + (SM_W1 - SM_W1) + core_off(nn, k, 64)) =
                __float2bfloat16_rn(k < 30 ? p[OFF_W1 + k * 64 + nn] : 0.0f);
        } else if (e < 64 * 32 + 64 * 64) {
            const int q = e - 64 * 32, nn = q >> 6, k = q & 63;
            *reinterpret_cast<__nv_bfloat16 *>(img + (SM_W2 - SM_W1) + core_off(nn, k, 64)) =
                __float2bfloat16_rn(p[OFF_W2 + k * 64 + nn]);
        } else if (e < 64 * 32 + 64 * 64 + 16 * 64) {
            const int q = e - 64 * 32 - 64 * 64, nn = q >> 6, k = q & 63;
            *reinterpret_cast<__nv_bfloat16 *>(img + (SM_W3 - SM_W1) + core_off(nn, k, 16)) =
                __float2bfloat16_rn(nn < 4 ? p[OFF_W3 + k * 4 + nn] : 0.0f);
        } else if (e < 64 * 32 + 64 * 64 + 16 * 64 + 144) {
            const int b = e - (64 * 32 + 64 * 64 + 16 * 64);
            reinterpret_cast<float *>(img + (SM_BIAS - SM_W1))[b] =
                b < 64 ? p[OFF_B1 + b] : (b < 128 ? p[OFF_B2 + b - 64] : (b < 132 ? p[OFF_B3 + b - 128] : 0.0f));
        } else {
            const int q = e - (64 * 32 + 64 * 64 + 16 * 64 + 144);  // mu[32] then isd[32]
            reinterpret_cast<float *>(img + (SM_NORM - SM_W1))[q] =
                q < 32 ? (q < 30 ? p[OFF_MU + q] : 0.0f) : (q - 32 < 30 ? p[OFF_ISD + q - 32] : 0.0f);
        }
    }
}

__global__ void __launch_bounds__(TC_ROWS, 1) k_mlp_infer_tc(int64_t n, const __nv_bfloat16 *__restrict__ x,
                                                             const uint8_t *__restrict__ img, float *__restrict__ logits,
                                                             int8_t *__restrict__ cls, float *__restrict__ conf,
                                                             float threshold, int32_t *__restrict__ fallback,
                                                             int32_t *__restrict__ n_fallback, int32_t *status) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const uint32_t sb = (uint32_t)__cvta_generic_to_shared(smem);
    const int tid = threadIdx.x, warp = tid >> 5;
    float *bias = reinterpret_cast<float *>(smem + SM_BIAS);
    float *mu = reinterpret_cast<float *>(smem + SM_NORM), *isd = mu + 32;
    const uint32_t bar = sb + SM_BAR;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + SM_BAR + 8);

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // the packed weights, biases and standardisation: one bulk copy (TMA)
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(IMG_TC_BYTES) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         sb + SM_W1),
                     "l"(img), "r"(IMG_TC_BYTES), "r"(bar)
                     : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sb + SM_BAR + 8),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t t_lane = tmem + ((uint32_t)(warp * 32) << 16);  // this warp's 32 lanes
    bool ok = __syncthreads_and(bar_wait(bar, 0) ? 1 : 0) != 0;  // the weights have arrived
    uint32_t phase = 1;

    const uint64_t ntile = (uint64_t)((n + TC_ROWS - 1) / TC_ROWS);
    // this thread's feature row of the next tile, loaded one tile ahead
    auto load_row = [&](uint64_t tl, uint4 (&q4)[4]) {
        const int64_t rr = (int64_t)tl * TC_ROWS + tid;
        if (tl < ntile && rr < n) {
            const uint4 *src = reinterpret_cast<const uint4 *>(x + rr * 32);
#pragma unroll
            for (int q = 0; q < 4; ++q) q4[q] = __ldg(src + q);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) q4[q] = make_uint4(0u, 0u, 0u, 0u);
        }
    };
    uint4 cur[4];
    load_row(blockIdx.x, cur);
    for (uint64_t tile = blockIdx.x; tile < ntile && ok; tile += gridDim.x) {
        const int64_t r = (int64_t)tile * TC_ROWS + tid;
        uint4 nxt[4];
        load_row(tile + gridDim.x, nxt);
        // 1. standardised BF16 row into operand A of layer 1
        {
            float xv[32];
            {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint4 w4 = cur[q];
                    const uint32_t w[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        __nv_bfloat162 b2 = *reinterpret_cast<const __nv_bfloat162 *>(&w[h]);
                        xv[8 * q + 2 * h] = __low2float(b2);
                        xv[8 * q + 2 * h + 1] = __high2float(b2);
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float v[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int kk = 8 * c + k;
                    v[k] = (xv[kk] - mu[kk]) * isd[kk];  // columns 30, 31: isd = 0
                }
                st_chunk(smem, SM_X + core_off(tid, 8 * c, TC_ROWS), v);
            }
        }
        // layers 1..3
#pragma unroll 1
        for (int layer = 0; layer < 3 && ok; ++layer) {
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                const uint32_t a_base = sb + (layer == 0 ? SM_X : SM_H);
                const int nk = layer == 0 ? 2 : 4;         // K / 16
                const int N = layer == 2 ? 16 : 64;
                const uint32_t b_base = sb + (layer == 0 ? SM_W1 : (layer == 1 ? SM_W2 : SM_W3));
                const uint32_t d = tmem;
                for (int s = 0; s < nk; ++s) {
                    const uint64_t da = smem_desc(a_base + (uint32_t)(2 * s) * (TC_ROWS / 8) * 128, (TC_ROWS / 8) * 128, 128);
                    const uint64_t db = smem_desc(b_base + (uint32_t)(2 * s) * (N / 8) * 128, (N / 8) * 128, 128);
                    mma_bf16_tc(d, da, db, instr_desc(N), s > 0 ? 1u : 0u);
                }
                mma_commit(bar);
            }
            // a timed-out wait ends the loop on every thread together
            ok = __syncthreads_and(bar_wait(bar, phase) ? 1 : 0) != 0;
            phase ^= 1u;
            tc_fence_after();
            if (!ok) break;
            if (layer < 2) {
                relu_to_h(smem, t_lane, bias + 64 * layer);
            } else {
                float v[16];
                tmem_ld16(t_lane, v);
                if (r < n) {
                    float l[4], mx = -3.4e38f;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        l[c] = v[c] + bias[128 + c];
                        mx = fmaxf(mx, l[c]);
                    }
                    float e[4], sum = 0.0f;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        e[c] = expf(l[c] - mx);
                        sum += e[c];
                    }
                    int best = 0;  // the first largest logit
#pragma unroll
                    for (int c = 1; c < 4; ++c)
                        if (l[c] > l[best]) best = c;
                    const float pb = e[best] / sum;
                    if (logits)
#pragma unroll
                        for (int c = 0; c < 4; ++c) logits[r * 4 + c] = l[c];
                    if (cls) cls[r] = (int8_t)best;
                    if (conf) conf[r] = pb;
                    if (fallback && pb < threshold) fallback[atomicAdd(n_fallback, 1)] = (int32_t)r;
                }
            }
        }
        tc_fence_before();
        __syncthreads();  // the next tile overwrites the operands and accumulators
        tc_fence_after();
#pragma unroll
        for (int q = 0; q < 4; ++q) cur[q] = nxt[q];
    }
    if (!ok && tid == 0) latch_status(status, PPMD_ERR_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

}  // namespace

int mlp_infer_tc(ppmd_ctx *ctx, int64_t n, const __nv_bfloat16 *x, const float *params, float *logits, int8_t *cls,
                 float *conf, float threshold, int32_t *fallback, int32_t *n_fallback) {
    if (n <= 0) return PPMD_OK;
    static bool attr = false;
    if (!attr) {
        PPMD_TRY(cuda_check(ctx, cudaFuncSetAttribute(k_mlp_infer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      (int)SM_REQUEST),
                            "cudaFuncSetAttribute"));
        attr = true;
    }
    uint8_t *img = (uint8_t *)scratch(ctx, S_MLPTC, IMG_TC_BYTES);
    if (!img) return PPMD_ERR_NOMEM;
    PPMD_LAUNCH(ctx, k_pack_tc, 32, 256, 0, params, img);
    const int64_t ntile = (n + TC_ROWS - 1) / TC_ROWS;
    const int64_t grid = ntile < 148 * TC_CTAS_PER_SM ? ntile : 148 * TC_CTAS_PER_SM;
    PPMD_LAUNCH(ctx, k_mlp_infer_tc, grid, TC_ROWS, SM_REQUEST, n, x, img, logits, cls, conf, threshold, fallback,
                n_fallback, ctx->d_status);
    return check_launch(ctx, "mlp_infer_tc");
}

}  // namespace ppmd
