// Classifier MLP inference and training forward/backward on the
// fifth-generation tensor cores (tcgen05): 128-row tiles, operands in shared
// memory, accumulators in tensor memory.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace ppmd {

// Logits (may be null), class = argmax, confidence = largest softmax
// probability (may be null) of the BF16 feature rows x [n][32]; rows with
// confidence < threshold are appended (as row numbers) to fallback (when
// given), their count kept at *n_fallback (zeroed first).  Class and
// confidence of row r are written at out_idx[r] (r when out_idx is null).
// params: the FP32 parameter vector (device).
int mlp_infer_tc(ppmd_ctx *ctx, int64_t n, const __nv_bfloat16 *x, const float *params, float *logits, int8_t *cls,
                 float *conf, float threshold, int32_t *fallback, int32_t *n_fallback, const int32_t *out_idx = nullptr);

// Training forward and back-propagation of a batch of BF16 feature rows x
// [batch][32] with labels y: h1, h2, d1 = dL/dz1, d2 = dL/dz2 (BF16
// [batch][64]) and d3 = dL/dz3 (BF16 [batch][8], 4 used), L = mean cross
// entropy; loss_part[b] (b < mlp_train_tc_blocks(batch)) the loss of block b.
int64_t mlp_train_tc_blocks(int64_t batch);
int mlp_train_tc(ppmd_ctx *ctx, int64_t batch, const __nv_bfloat16 *x, const int8_t *y, const float *params,
                 __nv_bfloat16 *H1, __nv_bfloat16 *H2, __nv_bfloat16 *D1, __nv_bfloat16 *D2, __nv_bfloat16 *D3,
                 double *loss_part);

// Weight and bias gradients from the activations and derivatives above (the
// samples as the contraction index): per CTA one partial parameter-gradient
// row part[b][PPMD_MLP_NPARAM], b < *nblk (sum them in a fixed order).
int64_t mlp_wgrad_tc_chunk(int64_t batch);
int mlp_wgrad_tc(ppmd_ctx *ctx, int64_t batch, const __nv_bfloat16 *x, const __nv_bfloat16 *H1, const __nv_bfloat16 *H2,
                 const __nv_bfloat16 *D1, const __nv_bfloat16 *D2, const __nv_bfloat16 *D3, const float *params,
                 float *part, int64_t *nblk);

}  // namespace ppmd
