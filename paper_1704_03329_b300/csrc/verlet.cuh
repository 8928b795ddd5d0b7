// Integrator kernels shared with the time-stepping driver.
#pragma once
#include "common.cuh"

namespace ppmd {
int md_kick_drift(ppmd_ctx *ctx, int64_t n, double *pos, double *vel, const float4 *f4, const double *f64, int4 *xq,
                  const int4 *xq_ref, const SegTable &st, double h, double dt, unsigned int *max_disp_bits);
int64_t kick_blocks(int64_t n);
int md_kick(ppmd_ctx *ctx, int64_t n, double *vel, const float4 *f4, const double *f64, double h, double half_m,
            double *partials);
int gather_sorted(ppmd_ctx *ctx, int64_t n, const int32_t *perm, const double *pos, const double *vel, const int4 *xq,
                  const int32_t *orig, const int32_t *cell_of, double *pos_o, double *vel_o, int4 *xq_o,
                  int32_t *orig_o, int32_t *cell_o);
int scatter_vec3(ppmd_ctx *ctx, int64_t n, const int32_t *orig, const double *in, double *out);
int scatter_f4(ppmd_ctx *ctx, int64_t n, const int32_t *orig, const float4 *in, double *out);
}  // namespace ppmd
