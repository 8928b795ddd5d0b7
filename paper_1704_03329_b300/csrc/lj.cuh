// Lennard-Jones pair loop shared by the entry point and the integrator.
#pragma once
#include "common.cuh"
#include "neighbours.cuh"

namespace ppmd {
struct LJConst {
    double rc2, s2d, f48d, e2d, shiftd;  // rc^2, sigma^2, 48 eps / sigma^2, 2 eps, shift
    float rc2_lo, rc2_hi;                // FP32 decision band around rc^2
    float s2, f48, e2, shift;            // sigma^2, 48 eps, 2 eps, shift
};
LJConst make_ljconst(const ppmd_lj_params &p, double Lmax);
int64_t lj_blocks(int64_t n);
// Forces of n atoms (positions xq / pos64 in list order).  FP32 path: into f4
// (Fx, Fy, Fz, e_i) when f4 != null, else into f64/e64; FP64 path into
// f64/e64.  partials (may be null): per-block (U, W) FP64 sums, lj_blocks(n) rows.
int lj_launch(ppmd_ctx *ctx, int64_t n, const int4 *xq, const double *pos64, const SegTable &st, const LJConst &c,
              const int32_t *nbr, const int32_t *cnt, int32_t max_nbr, int prec, float4 *f4, double *f64, double *e64,
              double *partials);
}  // namespace ppmd
