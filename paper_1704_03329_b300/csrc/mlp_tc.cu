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
// Two tiles are in flight per CTA (two operand slots, two accumulator
// regions, two mbarriers): while the tensor cores work on one, the threads
// prepare or finish the other; up to four CTAs share an SM.
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
// Two tiles are in flight per CTA (slots 0 and 1).  In each slot X (A of
// layer 1, 128 x 32 BF16) and H (A of layers 2 and 3, 128 x 64) share one
// 16 KB region: each is written only after the tensor cores finished
// reading the other.
constexpr uint32_t SM_SLOT = 16384;
constexpr uint32_t SM_W1 = 2 * SM_SLOT;   // B of layer 1: 64 x 32 (n x k)
constexpr uint32_t SM_W2 = SM_W1 + 4096;  // B of layer 2: 64 x 64
constexpr uint32_t SM_W3 = SM_W2 + 8192;  // B of layer 3: 16 x 64 (n >= 4 zero)
constexpr uint32_t SM_BIAS = SM_W3 + 2048;    // b1[64] b2[64] b3[16] (floats)
constexpr uint32_t SM_NORM = SM_BIAS + 576;   // mu[32] isd[32]
constexpr uint32_t SM_BAR = SM_NORM + 256;    // mbarriers of slots 0, 1 (8 bytes each) + tensor-memory address
constexpr uint32_t SM_USED = SM_BAR + 32;
// Requested dynamic shared memory: at most four CTAs per SM, so that their
// tensor memory (128 columns each) stays within the SM's 512 columns.
constexpr uint32_t SM_REQUEST = 48 * 1024;
static_assert(SM_USED <= SM_REQUEST, "shared memory map");
constexpr uint32_t TMEM_COLS = 128;  // slot s: columns 64 s .. 64 s + 63, every layer's accumulator
constexpr int TC_CTAS_PER_SM = 4;
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

// 16 consecutive FP32 columns of this thread's lane (issued; complete
// after tmem_wait).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Two FP32 values (first in the low half) as packed BF16, rounded to
// nearest, negatives to zero (ReLU) when RELU.
template <bool RELU>
__device__ __forceinline__ uint32_t pk_bf16x2(unsigned long long v) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
    uint32_t d;
    if (RELU) asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    else asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
__device__ __forceinline__ unsigned long long pk2(uint32_t lo, uint32_t hi) {
    unsigned long long v;
    asm("mov.b64 %0, {%1, %2};" : "=l"(v) : "r"(lo), "r"(hi));
    return v;
}
// packed FP32 pairs (round to nearest, as the scalar operations)
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Layer output of this thread's row: bias + ReLU, BF16, into operand H
// (the four loads of the 64 columns complete on one wait; bias pairs added
// as packed FP32, ReLU folded into the BF16 conversion).
__device__ __forceinline__ void relu_to_h(uint8_t *smem, uint32_t h_base, uint32_t t_lane, const float *bias) {
    uint32_t raw[4][16];
#pragma unroll
    for (int q = 0; q < 4; ++q) tmem_ld16(t_lane + 16 * q, raw[q]);
    tmem_wait();
    const ulonglong2 *b4 = reinterpret_cast<const ulonglong2 *>(bias);
    const int r = threadIdx.x;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t w[8];
#pragma unroll
        for (int p = 0; p < 8; p += 2) {
            const ulonglong2 bb = b4[4 * q + p / 2];  // bias of columns 16 q + 2 p .. + 3
            w[p] = pk_bf16x2<true>(add2(pk2(raw[q][2 * p], raw[q][2 * p + 1]), bb.x));
            w[p + 1] = pk_bf16x2<true>(add2(pk2(raw[q][2 * p + 2], raw[q][2 * p + 3]), bb.y));
        }
        *reinterpret_cast<uint4 *>(smem + h_base + core_off(r, 16 * q, TC_ROWS)) = make_uint4(w[0], w[1], w[2], w[3]);
        *reinterpret_cast<uint4 *>(smem + h_base + core_off(r, 16 * q + 8, TC_ROWS)) = make_uint4(w[4], w[5], w[6], w[7]);
    }
}

// The shared-memory image from SM_W1 on (weights as operand B in BF16,
// biases, standardisation), built once per call in global memory and
// copied into each CTA by one bulk copy.
constexpr uint32_t IMG_TC_BYTES = SM_BAR - SM_W1;
static_assert(IMG_TC_BYTES % 16 == 0, "bulk copies move multiples of 16 bytes");

__global__ void k_pack_tc(const float *__restrict__ p, uint8_t *__restrict__ img, int32_t *n_fallback) {
    if (n_fallback && blockIdx.x == 0 && threadIdx.x == 0) *n_fallback = 0;  // before the inference kernel runs
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
                                                             int32_t *__restrict__ n_fallback,
                                                             const int32_t *__restrict__ out_idx, int32_t *status) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const uint32_t sb = (uint32_t)__cvta_generic_to_shared(smem);
    const int tid = threadIdx.x, warp = tid >> 5;
    float *bias = reinterpret_cast<float *>(smem + SM_BIAS);
    float *mu = reinterpret_cast<float *>(smem + SM_NORM), *isd = mu + 32;
    const uint32_t bar0 = sb + SM_BAR, bar1 = sb + SM_BAR + 8;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + SM_BAR + 16);

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // the packed weights, biases and standardisation: one bulk copy (TMA)
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar0), "r"(IMG_TC_BYTES) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         sb + SM_W1),
                     "l"(img), "r"(IMG_TC_BYTES), "r"(bar0)
                     : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sb + SM_BAR + 16),
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
    bool ok = __syncthreads_and(bar_wait(bar0, 0) ? 1 : 0) != 0;  // the weights have arrived
    uint32_t ph[2] = {1u, 0u};  // next phase to wait for, per slot

    const int64_t ntile = (n + TC_ROWS - 1) / TC_ROWS;
    auto load_row = [&](int64_t tl, uint4 (&q4)[4]) {
        const int64_t rr = tl * TC_ROWS + tid;
        if (tl < ntile && rr < n) {
            const uint4 *src = reinterpret_cast<const uint4 *>(x + rr * 32);
#pragma unroll
            for (int q = 0; q < 4; ++q) q4[q] = __ldg(src + q);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) q4[q] = make_uint4(0u, 0u, 0u, 0u);
        }
    };
    // standardised BF16 row into slot s as operand A of layer 1: (x - mu) isd
    // on packed FP32 pairs (columns 30, 31: isd = 0), rounded to BF16
    const unsigned long long *mu2 = reinterpret_cast<const unsigned long long *>(mu);
    const unsigned long long *isd2 = reinterpret_cast<const unsigned long long *>(isd);
    auto stage = [&](int sl, const uint4 (&q4)[4]) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const uint32_t w[4] = {q4[c].x, q4[c].y, q4[c].z, q4[c].w};
            uint32_t o[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int kk2 = 4 * c + h;  // the pair of columns 2 kk2, 2 kk2 + 1
                const unsigned long long x2 = pk2(w[h] << 16, w[h] & 0xFFFF0000u);  // BF16 -> FP32, exact
                o[h] = pk_bf16x2<false>(mul2(sub2(x2, mu2[kk2]), isd2[kk2]));
            }
            *reinterpret_cast<uint4 *>(smem + sl * SM_SLOT + core_off(tid, 8 * c, TC_ROWS)) =
                make_uint4(o[0], o[1], o[2], o[3]);
        }
    };
    // operands of slot s visible to the tensor cores, then one thread issues
    // layer `layer` of slot s and commits it to the slot's mbarrier
    auto issue = [&](int sl, int layer) {
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a_base = sb + sl * SM_SLOT;
            const int nk = layer == 0 ? 2 : 4;  // K / 16
            const int N = layer == 2 ? 16 : 64;
            const uint32_t b_base = sb + (layer == 0 ? SM_W1 : (layer == 1 ? SM_W2 : SM_W3));
            for (int k = 0; k < nk; ++k) {
                const uint64_t da = smem_desc(a_base + (uint32_t)(2 * k) * (TC_ROWS / 8) * 128, (TC_ROWS / 8) * 128, 128);
                const uint64_t db = smem_desc(b_base + (uint32_t)(2 * k) * (N / 8) * 128, (N / 8) * 128, 128);
                mma_bf16_tc(tmem + 64u * sl, da, db, instr_desc(N), k > 0 ? 1u : 0u);
            }
            mma_commit(sl == 0 ? bar0 : bar1);
        }
    };
    // wait for slot s (a timed-out wait ends the work on every thread together)
    auto wait_slot = [&](int sl) {
        ok = __syncthreads_and(ok && bar_wait(sl == 0 ? bar0 : bar1, ph[sl]) ? 1 : 0) != 0;
        ph[sl] ^= 1u;
        tc_fence_after();
        return ok;
    };
    auto finish = [&](int sl, int64_t tl) {
        uint32_t raw[16];
        tmem_ld16(t_lane + 64u * sl, raw);
        tmem_wait();
        const int64_t r = tl * TC_ROWS + tid;
        if (tl < ntile && r < n) {
            float l[4], mx = -3.4e38f;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                l[c] = __uint_as_float(raw[c]) + bias[128 + c];
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
            const int64_t o = out_idx ? out_idx[r] : r;
            if (cls) cls[o] = (int8_t)best;
            if (conf) conf[o] = pb;
            if (fallback && pb < threshold) fallback[atomicAdd(n_fallback, 1)] = (int32_t)r;
        }
    };
    // pairs of tiles: while the tensor cores work on one slot, the threads
    // prepare or finish the other
    for (int64_t t0 = 2 * (int64_t)blockIdx.x; t0 < ntile && ok; t0 += 2 * (int64_t)gridDim.x) {
        const int64_t t1 = t0 + 1;
        uint4 q0[4], q1[4];
        load_row(t0, q0);
        load_row(t1, q1);
        stage(0, q0);
        issue(0, 0);
        stage(1, q1);
        issue(1, 0);
#pragma unroll 1
        for (int layer = 1; layer < 3 && ok; ++layer) {
            if (!wait_slot(0)) break;
            relu_to_h(smem, 0, t_lane, bias + 64 * (layer - 1));
            issue(0, layer);
            if (!wait_slot(1)) break;
            relu_to_h(smem, SM_SLOT, t_lane + 64u, bias + 64 * (layer - 1));
            issue(1, layer);
        }
        if (ok && wait_slot(0)) finish(0, t0);
        if (ok && wait_slot(1)) finish(1, t1);
        tc_fence_before();
        __syncthreads();  // the next pair overwrites the operands and accumulators
        tc_fence_after();
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
                 float *conf, float threshold, int32_t *fallback, int32_t *n_fallback, const int32_t *out_idx) {
    if (n <= 0) return n_fallback ? cuda_check(ctx, cudaMemsetAsync(n_fallback, 0, sizeof(int32_t), ctx->stream), "memset")
                                  : PPMD_OK;
    // (a per-device setting: set on every call, on the context's device)
    PPMD_TRY(cuda_check(ctx, cudaFuncSetAttribute(k_mlp_infer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)SM_REQUEST),
                        "cudaFuncSetAttribute"));
    uint8_t *img = (uint8_t *)scratch(ctx, S_MLPTC, IMG_TC_BYTES);
    if (!img) return PPMD_ERR_NOMEM;
    PPMD_LAUNCH(ctx, k_pack_tc, 32, 256, 0, params, img, fallback ? n_fallback : nullptr);
    const int64_t ntile = (n + TC_ROWS - 1) / TC_ROWS;
    const int64_t npair = (ntile + 1) / 2;
    const int64_t grid = npair < 148 * TC_CTAS_PER_SM ? npair : 148 * TC_CTAS_PER_SM;
    PPMD_LAUNCH(ctx, k_mlp_infer_tc, grid, TC_ROWS, SM_REQUEST, n, x, img, logits, cls, conf, threshold, fallback,
                n_fallback, out_idx, ctx->d_status);
    return check_launch(ctx, "mlp_infer_tc");
}

}  // namespace ppmd
