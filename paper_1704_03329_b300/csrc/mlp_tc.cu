// Classifier MLP (30 -> 64 -> 64 -> 4, ReLU, softmax) on the tcgen05 tensor
// cores: inference, and the forward and back-propagation of training.
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

// ---------------------------------------------------------------------
// Training: forward and back-propagation of 128-row tiles on tcgen05.
// Per tile (thread t = row t = tensor-memory lane t), five chained groups
// of MMAs into tensor memory:
//   z1 = x' W1 (N 64), z2 = h1 W2 (N 64), z3 = h2 W3 (N 16, 4 used),
//   dh2 = d3 W3^T (K 16, 4 used), dh1 = d2 W2^T (K 64);
// between them every thread turns its row of the accumulator into the next
// operand: h = relu(z + b) (BF16, with the sign of z kept as a bit mask),
// d3 = (softmax(z3 + b3) - onehot(y)) / B, d2 = dh2 masked by z2 > 0,
// d1 = dh1 masked by z1 > 0.  h1, h2, d1, d2 (BF16 [B][64]) and d3 (BF16
// [B][8], 4 used) go to global memory for the weight gradients; the mean
// cross entropy as one FP64 partial per block.
// ---------------------------------------------------------------------
constexpr uint32_t TR_A1 = 0;                // x' (A of layer 1): 128 x 32
constexpr uint32_t TR_H = 8192;              // h1, then h2, then d2 (A of layers 2, 3, back 2): 128 x 64
constexpr uint32_t TR_A4 = 24576;            // d3 (A of back 1): 128 x 16
constexpr uint32_t TR_W1 = 28672;            // B of layer 1: 64 x 32 (the image starts here)
constexpr uint32_t TR_W2 = TR_W1 + 4096;     // B of layer 2: 64 x 64
constexpr uint32_t TR_W3 = TR_W2 + 8192;     // B of layer 3: 16 x 64
constexpr uint32_t TR_W3T = TR_W3 + 2048;    // B of back 1: n = j (64) x k = class (16)
constexpr uint32_t TR_W2T = TR_W3T + 2048;   // B of back 2: n = i (64) x k = j (64)
constexpr uint32_t TR_BIAS = TR_W2T + 8192;  // b1[64] b2[64] b3[16]
constexpr uint32_t TR_NORM = TR_BIAS + 576;  // mu[32] isd[32]
constexpr uint32_t TR_BAR = TR_NORM + 256;   // mbarriers: image, MMA; tensor-memory address
constexpr uint32_t TR_USED = TR_BAR + 32;
constexpr uint32_t TR_IMG_BYTES = TR_BAR - TR_W1;
static_assert(TR_IMG_BYTES % 16 == 0, "bulk copies move multiples of 16 bytes");
// at most two CTAs per SM (256 tensor-memory columns each)
constexpr uint32_t TR_REQUEST = 100 * 1024;
static_assert(TR_USED <= TR_REQUEST, "shared memory map");
constexpr uint32_t TR_TMEM_COLS = 256;  // z1 / dh2: 0-63, z2 / dh1: 64-127, z3: 128-143
constexpr int TR_CTAS_PER_SM = 2;

__global__ void k_pack_train_tc(const float *__restrict__ p, uint8_t *__restrict__ img) {
    constexpr int E1 = 64 * 32, E2 = E1 + 64 * 64, E3 = E2 + 16 * 64, E4 = E3 + 64 * 16, E5 = E4 + 64 * 64,
                  E6 = E5 + 144, E7 = E6 + 64;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E7; e += gridDim.x * blockDim.x) {
        __nv_bfloat16 *bf = nullptr;
        float v = 0.0f;
        if (e < E1) {  // W1B[n][k] = W1[k][n]
            const int nn = e >> 5, k = e & 31;
            bf = reinterpret_cast<__nv_bfloat16 *>(img + (TR_W1 - TR_W1) + core_off(nn, k, 64));
            v = k < 30 ? p[OFF_W1 + k * 64 + nn] : 0.0f;
        } else if (e < E2) {  // W2B[n][k] = W2[k][n]
            const int q = e - E1, nn = q >> 6, k = q & 63;
            bf = reinterpret_cast<__nv_bfloat16 *>(img + (TR_W2 - TR_W1) + core_off(nn, k, 64));
            v = p[OFF_W2 + k * 64 + nn];
        } else if (e < E3) {  // W3B[n][k] = W3[k][n], n < 4
            const int q = e - E2, nn = q >> 6, k = q & 63;
            bf = reinterpret_cast<__nv_bfloat16 *>(img + (TR_W3 - TR_W1) + core_off(nn, k, 16));
            v = nn < 4 ? p[OFF_W3 + k * 4 + nn] : 0.0f;
        } else if (e < E4) {  // W3T[n = j][k = c] = W3[j][c], c < 4
            const int q = e - E3, nn = q >> 4, k = q & 15;
            bf = reinterpret_cast<__nv_bfloat16 *>(img + (TR_W3T - TR_W1) + core_off(nn, k, 64));
            v = k < 4 ? p[OFF_W3 + nn * 4 + k] : 0.0f;
        } else if (e < E5) {  // W2T[n = i][k = j] = W2[i][j]
            const int q = e - E4, nn = q >> 6, k = q & 63;
            bf = reinterpret_cast<__nv_bfloat16 *>(img + (TR_W2T - TR_W1) + core_off(nn, k, 64));
            v = p[OFF_W2 + nn * 64 + k];
        } else if (e < E6) {
            const int b = e - E5;
            reinterpret_cast<float *>(img + (TR_BIAS - TR_W1))[b] =
                b < 64 ? p[OFF_B1 + b] : (b < 128 ? p[OFF_B2 + b - 64] : (b < 132 ? p[OFF_B3 + b - 128] : 0.0f));
        } else {
            const int q = e - E6;  // mu[32] then isd[32]
            reinterpret_cast<float *>(img + (TR_NORM - TR_W1))[q] =
                q < 32 ? (q < 30 ? p[OFF_MU + q] : 0.0f) : (q - 32 < 30 ? p[OFF_ISD + q - 32] : 0.0f);
        }
        if (bf) *bf = __float2bfloat16_rn(v);
    }
}

__global__ void __launch_bounds__(TC_ROWS, 1) k_mlp_train_tc(int64_t B, const __nv_bfloat16 *__restrict__ x,
                                                             const int8_t *__restrict__ y,
                                                             const uint8_t *__restrict__ img,
                                                             __nv_bfloat16 *__restrict__ H1, __nv_bfloat16 *__restrict__ H2,
                                                             __nv_bfloat16 *__restrict__ D1, __nv_bfloat16 *__restrict__ D2,
                                                             __nv_bfloat16 *__restrict__ D3,
                                                             double *__restrict__ loss_part, int32_t *status) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ double s_loss[TC_ROWS / 32];
    const uint32_t sb = (uint32_t)__cvta_generic_to_shared(smem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float *bias = reinterpret_cast<float *>(smem + TR_BIAS);
    float *mu = reinterpret_cast<float *>(smem + TR_NORM), *isd = mu + 32;
    const uint32_t bar_img = sb + TR_BAR, bar_mma = sb + TR_BAR + 8;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + TR_BAR + 16);

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_img) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_mma) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_img), "r"(TR_IMG_BYTES) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         sb + TR_W1),
                     "l"(img), "r"(TR_IMG_BYTES), "r"(bar_img)
                     : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sb + TR_BAR + 16),
                     "r"(TR_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t t_lane = tmem + ((uint32_t)(warp * 32) << 16);
    bool ok = __syncthreads_and(bar_wait(bar_img, 0) ? 1 : 0) != 0;
    uint32_t ph = 0;  // next phase of the MMA barrier
    const float invB = 1.0f / (float)B;
    const unsigned long long *mu2 = reinterpret_cast<const unsigned long long *>(mu);
    const unsigned long long *isd2 = reinterpret_cast<const unsigned long long *>(isd);
    double loss = 0.0;

    // one group of MMAs: A (128 rows) at a_off, B (N rows) at b_off, K = 16 nk,
    // into columns col; committed to the MMA barrier, then waited for by all
    auto mma = [&](uint32_t a_off, uint32_t b_off, int nk, int N, uint32_t col) {
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            for (int k = 0; k < nk; ++k) {
                const uint64_t da = smem_desc(sb + a_off + (uint32_t)(2 * k) * (TC_ROWS / 8) * 128, (TC_ROWS / 8) * 128, 128);
                const uint64_t db = smem_desc(sb + b_off + (uint32_t)(2 * k) * (N / 8) * 128, (N / 8) * 128, 128);
                mma_bf16_tc(tmem + col, da, db, instr_desc(N), k > 0 ? 1u : 0u);
            }
            mma_commit(bar_mma);
        }
        ok = __syncthreads_and(ok && bar_wait(bar_mma, ph) ? 1 : 0) != 0;
        ph ^= 1u;
        tc_fence_after();
        return ok;
    };
    // this thread's 64 accumulator columns from col (complete on return)
    auto load64 = [&](uint32_t col, uint32_t (&raw)[4][16]) {
#pragma unroll
        for (int q = 0; q < 4; ++q) tmem_ld16(t_lane + col + 16 * q, raw[q]);
        tmem_wait();
    };
    // 64 BF16 values of the row (pairs w[32]) into operand TR_H and, for
    // a valid row, into row r of dst
    auto put64 = [&](const uint32_t (&w)[32], __nv_bfloat16 *dst, int64_t r, bool valid) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 lo = make_uint4(w[8 * q], w[8 * q + 1], w[8 * q + 2], w[8 * q + 3]);
            const uint4 hi = make_uint4(w[8 * q + 4], w[8 * q + 5], w[8 * q + 6], w[8 * q + 7]);
            *reinterpret_cast<uint4 *>(smem + TR_H + core_off(tid, 16 * q, TC_ROWS)) = lo;
            *reinterpret_cast<uint4 *>(smem + TR_H + core_off(tid, 16 * q + 8, TC_ROWS)) = hi;
            if (valid) {
                uint4 *g = reinterpret_cast<uint4 *>(dst + r * 64) + 2 * q;
                g[0] = lo;
                g[1] = hi;
            }
        }
    };
    // h = relu(z + b) of the accumulator at col into operand TR_H and dst; the
    // sign bits of z + b as a mask
    auto hidden = [&](uint32_t col, const float *b, __nv_bfloat16 *dst, int64_t r, bool valid) {
        uint32_t raw[4][16];
        load64(col, raw);
        uint32_t w[32];
        unsigned long long m = 0ull;
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int p = 0; p < 16; p += 2) {
                const int c = 16 * q + p;
                const unsigned long long z = add2(pk2(raw[q][p], raw[q][p + 1]),
                                                  *reinterpret_cast<const unsigned long long *>(b + c));
                float z0, z1;
                asm("mov.b64 {%0, %1}, %2;" : "=f"(z0), "=f"(z1) : "l"(z));
                m |= (unsigned long long)(z0 > 0.0f) << c;
                m |= (unsigned long long)(z1 > 0.0f) << (c + 1);
                w[c / 2] = pk_bf16x2<true>(z);
            }
        put64(w, dst, r, valid);
        return m;
    };
    // d = dh masked by the sign bits of z, into dst (and operand TR_H when
    // to_smem)
    auto masked = [&](uint32_t col, unsigned long long m, __nv_bfloat16 *dst, int64_t r, bool valid, bool to_smem) {
        uint32_t raw[4][16];
        load64(col, raw);
        uint32_t w[32];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int p = 0; p < 16; p += 2) {
                const int c = 16 * q + p;
                const uint32_t a = (m >> c) & 1ull ? raw[q][p] : 0u, bb = (m >> (c + 1)) & 1ull ? raw[q][p + 1] : 0u;
                w[c / 2] = pk_bf16x2<false>(pk2(a, bb));
            }
        if (to_smem) {
            put64(w, dst, r, valid);
        } else if (valid) {
#pragma unroll
            for (int q = 0; q < 8; ++q)
                reinterpret_cast<uint4 *>(dst + r * 64)[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
        }
    };

    const int64_t ntile = (B + TC_ROWS - 1) / TC_ROWS;
    for (int64_t tl = blockIdx.x; tl < ntile && ok; tl += gridDim.x) {
        const int64_t r = tl * TC_ROWS + tid;
        const bool valid = r < B;
        // x' = (x - mu) isd, BF16, as operand A of layer 1
        {
            uint4 q4[4];
            const uint4 *src = reinterpret_cast<const uint4 *>(x + (valid ? r : 0) * 32);
#pragma unroll
            for (int q = 0; q < 4; ++q) q4[q] = valid ? __ldg(src + q) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const uint32_t wv[4] = {q4[c].x, q4[c].y, q4[c].z, q4[c].w};
                uint32_t o[4];
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int kk2 = 4 * c + h;
                    const unsigned long long x2 = pk2(wv[h] << 16, wv[h] & 0xFFFF0000u);
                    o[h] = pk_bf16x2<false>(mul2(sub2(x2, mu2[kk2]), isd2[kk2]));
                }
                *reinterpret_cast<uint4 *>(smem + TR_A1 + core_off(tid, 8 * c, TC_ROWS)) = make_uint4(o[0], o[1], o[2], o[3]);
            }
        }
        if (!mma(TR_A1, TR_W1, 2, 64, 0)) break;
        const unsigned long long m1 = hidden(0, bias, H1, r, valid);
        if (!mma(TR_H, TR_W2, 4, 64, 64)) break;
        const unsigned long long m2 = hidden(64, bias + 64, H2, r, valid);
        if (!mma(TR_H, TR_W3, 4, 16, 128)) break;
        {
            // d3 = (softmax - onehot) / B (zero for rows past the batch)
            uint32_t raw[16];
            tmem_ld16(t_lane + 128, raw);
            tmem_wait();
            float l[4], pr[4], mx = -3.4e38f, s = 0.0f;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                l[c] = __uint_as_float(raw[c]) + bias[128 + c];
                mx = fmaxf(mx, l[c]);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                pr[c] = __expf(l[c] - mx);
                s += pr[c];
            }
            const float is = 1.0f / s;
            const int yc = valid ? (int)y[r] : -1;
            float d3[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                pr[c] *= is;
                d3[c] = yc >= 0 ? (pr[c] - (c == yc ? 1.0f : 0.0f)) * invB : 0.0f;
            }
            if (yc >= 0) loss -= log((double)pr[yc]) / (double)B;
            const uint32_t w0 = pk_bf16x2<false>(pk2(__float_as_uint(d3[0]), __float_as_uint(d3[1])));
            const uint32_t w1 = pk_bf16x2<false>(pk2(__float_as_uint(d3[2]), __float_as_uint(d3[3])));
            *reinterpret_cast<uint4 *>(smem + TR_A4 + core_off(tid, 0, TC_ROWS)) = make_uint4(w0, w1, 0u, 0u);
            *reinterpret_cast<uint4 *>(smem + TR_A4 + core_off(tid, 8, TC_ROWS)) = make_uint4(0u, 0u, 0u, 0u);
            if (valid) *reinterpret_cast<uint4 *>(D3 + r * 8) = make_uint4(w0, w1, 0u, 0u);
        }
        if (!mma(TR_A4, TR_W3T, 1, 64, 0)) break;
        masked(0, m2, D2, r, valid, true);
        if (!mma(TR_H, TR_W2T, 4, 64, 64)) break;
        masked(64, m1, D1, r, valid, false);
        tc_fence_before();
        __syncthreads();  // the next tile overwrites the operands and accumulators
        tc_fence_after();
    }
    if (!ok && tid == 0) latch_status(status, PPMD_ERR_TIMEOUT);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
    if (lane == 0) s_loss[warp] = loss;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) loss_part[blockIdx.x] = s_loss[0] + s_loss[1] + s_loss[2] + s_loss[3];
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TR_TMEM_COLS) : "memory");
}

// ---------------------------------------------------------------------
// Training: weight and bias gradients on tcgen05, the samples as the
// contraction index.  A CTA takes a chunk of whole 128-sample blocks; per
// block every thread (one sample) writes its sample's values transposed
// into two operand pairs (K-major, K = the block's 128 samples):
//   G1: A = [h1^T ; h2^T] (M 128) against B = [d2^T | d3^T] (N 80)
//       -> rows 0-63: dW2 = h1^T d2 (columns 0-63);
//          rows 64-127: dW3 = h2^T d3 (columns 64-67);
//   G2: A = [x'^T ; 1 ; 0] (M 128) against B = [d2^T | d3^T | 0 | d1^T] (N 144)
//       -> rows 0-29: dW1 = x'^T d1 (columns 80-143);
//          row 32: the bias gradients, column sums of d2 (0-63), d3 (64-67)
//          and d1 (80-143).
// The two B operands share one array (G1 reads its first 80 rows).  The
// products accumulate in tensor memory over the chunk; the CTA then writes
// its partial gradient row, summed over CTAs in a fixed order afterwards.
// ---------------------------------------------------------------------
constexpr uint32_t WG_A1 = 0;                           // 128 x 128 (m x k)
constexpr uint32_t WG_A2 = WG_A1 + 128 * 128 * 2;       // 128 x 128
constexpr uint32_t WG_B = WG_A2 + 128 * 128 * 2;        // 144 x 128 (n x k)
constexpr uint32_t WG_NORM = WG_B + 144 * 128 * 2;      // mu[32] isd[32]
constexpr uint32_t WG_BAR = WG_NORM + 256;              // mbarrier, tensor-memory address
constexpr uint32_t WG_USED = WG_BAR + 16;
constexpr uint32_t WG_REQUEST = 120 * 1024;  // one CTA per SM
static_assert(WG_USED <= WG_REQUEST, "shared memory map");
constexpr uint32_t WG_TMEM_COLS = 256;  // G1: columns 0-79, G2: 96-239
constexpr uint32_t WG_G2 = 96;

__global__ void __launch_bounds__(TC_ROWS, 1) k_mlp_wgrad_tc(int64_t B, int64_t chunk, const __nv_bfloat16 *__restrict__ x,
                                                             const __nv_bfloat16 *__restrict__ H1,
                                                             const __nv_bfloat16 *__restrict__ H2,
                                                             const __nv_bfloat16 *__restrict__ D1,
                                                             const __nv_bfloat16 *__restrict__ D2,
                                                             const __nv_bfloat16 *__restrict__ D3,
                                                             const float *__restrict__ p, float *__restrict__ part,
                                                             int32_t *status) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const uint32_t sb = (uint32_t)__cvta_generic_to_shared(smem);
    const int tid = threadIdx.x, warp = tid >> 5;
    float *mu = reinterpret_cast<float *>(smem + WG_NORM), *isd = mu + 32;
    const uint32_t bar = sb + WG_BAR;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + WG_BAR + 8);
    __nv_bfloat16 *a1 = reinterpret_cast<__nv_bfloat16 *>(smem + WG_A1);
    __nv_bfloat16 *a2 = reinterpret_cast<__nv_bfloat16 *>(smem + WG_A2);
    __nv_bfloat16 *bb = reinterpret_cast<__nv_bfloat16 *>(smem + WG_B);
    auto el = [](__nv_bfloat16 *base, int m, int k, int R) -> __nv_bfloat16 & {
        return *reinterpret_cast<__nv_bfloat16 *>(reinterpret_cast<uint8_t *>(base) + core_off(m, k, R));
    };

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < 32) {
        mu[tid] = tid < 30 ? p[OFF_MU + tid] : 0.0f;
        isd[tid] = tid < 30 ? p[OFF_ISD + tid] : 0.0f;
    }
    // the constant parts: A2 rows 33-127 and B rows 72-79 stay zero
    for (int e = tid; e < 128 * 128 / 8; e += TC_ROWS) reinterpret_cast<uint4 *>(a2)[e] = make_uint4(0u, 0u, 0u, 0u);
    for (int e = tid; e < 144 * 128 / 8; e += TC_ROWS) reinterpret_cast<uint4 *>(bb)[e] = make_uint4(0u, 0u, 0u, 0u);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sb + WG_BAR + 8),
                     "r"(WG_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    bool ok = true;
    uint32_t ph = 0;
    const int64_t s0 = (int64_t)blockIdx.x * chunk, s1 = min(B, s0 + chunk);
    int nblk = 0;
    for (int64_t base = s0; base < s1 && ok; base += TC_ROWS, ++nblk) {
        const int64_t r = base + tid;
        const bool valid = r < s1;
        const int k = tid;  // this sample's place along K
        {
            const uint4 *h1 = reinterpret_cast<const uint4 *>(H1 + r * 64), *h2 = reinterpret_cast<const uint4 *>(H2 + r * 64);
            const uint4 *d1 = reinterpret_cast<const uint4 *>(D1 + r * 64), *d2 = reinterpret_cast<const uint4 *>(D2 + r * 64);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
                const uint4 vh1 = valid ? h1[q] : zero, vh2 = valid ? h2[q] : zero;
                const uint4 vd1 = valid ? d1[q] : zero, vd2 = valid ? d2[q] : zero;
                const uint32_t w[4][4] = {{vh1.x, vh1.y, vh1.z, vh1.w}, {vh2.x, vh2.y, vh2.z, vh2.w},
                                          {vd1.x, vd1.y, vd1.z, vd1.w}, {vd2.x, vd2.y, vd2.z, vd2.w}};
#pragma unroll
                for (int h = 0; h < 4; ++h)
#pragma unroll
                    for (int half = 0; half < 2; ++half) {
                        const int c = 8 * q + 2 * h + half;  // column of the 64
                        __nv_bfloat16_raw v[4];
#pragma unroll
                        for (int mtx = 0; mtx < 4; ++mtx) v[mtx].x = (unsigned short)(w[mtx][h] >> (16 * half));
                        el(a1, c, k, 128) = v[0];
                        el(a1, 64 + c, k, 128) = v[1];
                        el(bb, 80 + c, k, 144) = v[2];
                        el(bb, c, k, 144) = v[3];
                    }
            }
            const uint4 vd3 = valid ? *reinterpret_cast<const uint4 *>(D3 + r * 8) : make_uint4(0u, 0u, 0u, 0u);
            const uint32_t w3[4] = {vd3.x, vd3.y, vd3.z, vd3.w};
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                __nv_bfloat16_raw v;
                v.x = (unsigned short)(w3[c >> 1] >> (16 * (c & 1)));
                el(bb, 64 + c, k, 144) = v;
            }
            // x' = (x - mu) isd in BF16, as in the forward pass; the ones row
            const uint4 *xs = reinterpret_cast<const uint4 *>(x + r * 32);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint4 vx = valid ? __ldg(xs + q) : make_uint4(0u, 0u, 0u, 0u);
                const uint32_t wx[4] = {vx.x, vx.y, vx.z, vx.w};
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int c = 8 * q + 2 * h;
                    const unsigned long long x2 = pk2(wx[h] << 16, wx[h] & 0xFFFF0000u);
                    const uint32_t o = valid ? pk_bf16x2<false>(mul2(sub2(x2, *reinterpret_cast<const unsigned long long *>(mu + c)),
                                                                     *reinterpret_cast<const unsigned long long *>(isd + c)))
                                             : 0u;
                    __nv_bfloat16_raw lo, hi;
                    lo.x = (unsigned short)(o & 0xFFFFu);
                    hi.x = (unsigned short)(o >> 16);
                    el(a2, c, k, 128) = lo;
                    el(a2, c + 1, k, 128) = hi;
                }
            }
            __nv_bfloat16_raw one;
            one.x = valid ? (unsigned short)0x3F80u : (unsigned short)0u;  // 1.0 in BF16
            el(a2, 32, k, 128) = one;
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            for (int kk = 0; kk < 8; ++kk) {  // K = 128 samples, 16 per instruction
                const uint32_t ko = (uint32_t)(2 * kk);
                const uint64_t da1 = smem_desc(sb + WG_A1 + ko * (128 / 8) * 128, (128 / 8) * 128, 128);
                const uint64_t da2 = smem_desc(sb + WG_A2 + ko * (128 / 8) * 128, (128 / 8) * 128, 128);
                const uint64_t db = smem_desc(sb + WG_B + ko * (144 / 8) * 128, (144 / 8) * 128, 128);
                const uint32_t acc = (nblk > 0 || kk > 0) ? 1u : 0u;
                mma_bf16_tc(tmem, da1, db, instr_desc(80), acc);
                mma_bf16_tc(tmem + WG_G2, da2, db, instr_desc(144), acc);
            }
            mma_commit(bar);
        }
        // the operands are rewritten by the next block only after this
        ok = __syncthreads_and(ok && bar_wait(bar, ph) ? 1 : 0) != 0;
        ph ^= 1u;
        tc_fence_after();
    }
    if (!ok && tid == 0) latch_status(status, PPMD_ERR_TIMEOUT);
    // the CTA's partial gradient: row m of both accumulators in thread m,
    // 16 columns at a time (loads by whole warps, writes by the rows that
    // hold parameters)
    float *out = part + (int64_t)blockIdx.x * NPARAM;
    const uint32_t t_lane = tmem + ((uint32_t)(warp * 32) << 16);
    const int m = tid;
    const bool have = nblk > 0 && ok;
    for (int q = 0; q < 5; ++q) {  // G1: dW2 (rows 0-63), dW3 (rows 64-127, columns 64-67)
        uint32_t v[16];
        tmem_ld16(t_lane + 16 * q, v);
        tmem_wait();
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const int c = 16 * q + e;
            const float g = have ? __uint_as_float(v[e]) : 0.0f;
            if (m < 64 && c < 64) out[OFF_W2 + m * 64 + c] = g;
            if (m >= 64 && c >= 64 && c < 68) out[OFF_W3 + (m - 64) * 4 + (c - 64)] = g;
        }
    }
    for (int q = 0; q < 9; ++q) {  // G2: dW1 (rows 0-29, columns 80-143), biases (row 32)
        uint32_t v[16];
        tmem_ld16(t_lane + WG_G2 + 16 * q, v);
        tmem_wait();
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const int c = 16 * q + e;
            const float g = have ? __uint_as_float(v[e]) : 0.0f;
            if (m < 30 && c >= 80) out[OFF_W1 + m * 64 + (c - 80)] = g;
            if (m == 32) {
                if (c < 64) out[OFF_B2 + c] = g;
                else if (c < 68) out[OFF_B3 + c - 64] = g;
                else if (c >= 80) out[OFF_B1 + c - 80] = g;
            }
        }
    }
    if (m < OFF_W1 / 2) {  // the standardisation is not trained
        out[2 * m] = 0.0f;
        out[2 * m + 1] = 0.0f;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(WG_TMEM_COLS) : "memory");
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

int64_t mlp_train_tc_blocks(int64_t batch) {
    const int64_t ntile = (batch + TC_ROWS - 1) / TC_ROWS;
    return ntile < 148 * TR_CTAS_PER_SM ? ntile : 148 * TR_CTAS_PER_SM;
}

int64_t mlp_wgrad_tc_chunk(int64_t batch) {
    const int64_t blocks = (batch + TC_ROWS - 1) / TC_ROWS;
    return (blocks + 147) / 148 * TC_ROWS;  // whole 128-sample blocks, at most 148 CTAs
}

int mlp_wgrad_tc(ppmd_ctx *ctx, int64_t batch, const __nv_bfloat16 *x, const __nv_bfloat16 *H1, const __nv_bfloat16 *H2,
                 const __nv_bfloat16 *D1, const __nv_bfloat16 *D2, const __nv_bfloat16 *D3, const float *params,
                 float *part, int64_t *nblk) {
    const int64_t chunk = mlp_wgrad_tc_chunk(batch);
    *nblk = (batch + chunk - 1) / chunk;
    if (batch <= 0) return PPMD_OK;
    PPMD_TRY(cuda_check(ctx, cudaFuncSetAttribute(k_mlp_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)WG_REQUEST),
                        "cudaFuncSetAttribute"));
    PPMD_LAUNCH(ctx, k_mlp_wgrad_tc, *nblk, TC_ROWS, WG_REQUEST, batch, chunk, x, H1, H2, D1, D2, D3, params, part,
                ctx->d_status);
    return check_launch(ctx, "mlp_wgrad_tc");
}

int mlp_train_tc(ppmd_ctx *ctx, int64_t batch, const __nv_bfloat16 *x, const int8_t *y, const float *params,
                 __nv_bfloat16 *H1, __nv_bfloat16 *H2, __nv_bfloat16 *D1, __nv_bfloat16 *D2, __nv_bfloat16 *D3,
                 double *loss_part) {
    if (batch <= 0) return PPMD_OK;
    PPMD_TRY(cuda_check(ctx, cudaFuncSetAttribute(k_mlp_train_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)TR_REQUEST),
                        "cudaFuncSetAttribute"));
    uint8_t *img = (uint8_t *)scratch(ctx, S_AUX3, TR_IMG_BYTES);
    if (!img) return PPMD_ERR_NOMEM;
    PPMD_LAUNCH(ctx, k_pack_train_tc, 32, 256, 0, params, img);
    PPMD_LAUNCH(ctx, k_mlp_train_tc, mlp_train_tc_blocks(batch), TC_ROWS, TR_REQUEST, batch, x, y, img, H1, H2, D1, D2, D3,
                loss_part, ctx->d_status);
    return check_launch(ctx, "mlp_train_tc");
}

}  // namespace ppmd
