// Classifier MLP inference on the fifth-generation tensor cores (tcgen05):
// 128-row tiles, operands in shared memory, accumulators in tensor memory.
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

}  // namespace ppmd
