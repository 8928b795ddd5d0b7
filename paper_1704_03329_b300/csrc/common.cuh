// Shared definitions of the ppmd CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "ppmd.h"

namespace ppmd {

// ---------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------
struct Scratch {
    void *ptr = nullptr;
    size_t bytes = 0;
};

enum ScratchSlot {
    S_STATUS = 0,  // device status word + needed capacity (never regrown)
    S_XQ,          // int4 fixed-point positions (granular calls)
    S_COUNT,       // per-cell counters
    S_SCAN,        // scan block sums
    S_PARTIAL,     // per-block FP64 partial sums
    S_TMP0,
    S_TMP1,
    S_TMP2,
    S_SORTPOS,  // analysis: sorted positions
    S_SORTIDX,
    S_CELLKEY,
    S_CELLTMP,
    S_MLPTC,
    S_CELLS0,
    S_CELLS1,
    S_CELLS2,
    S_NBR,
    S_NBRCNT,
    S_AUX0,
    S_AUX1,
    S_AUX2,
    S_AUX3,
    S_SEGS,    // analysis of several boxes: segment table, atom offsets,
    S_SEGOFF,  // segment of each atom, bricks
    S_SEGOF,
    S_BRICKS,
    S_NSLOTS
};

}  // namespace ppmd

struct ppmd_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int32_t *d_status = nullptr;             // [0] latched status
    unsigned long long *d_needed = nullptr;  // largest capacity asked for
    int32_t *h_status = nullptr;             // pinned mirror
    unsigned long long *h_needed = nullptr;
    int64_t launches = 0;
    int64_t host_needed = 0;  // capacity asked for by a host-side check
    char err[512] = {0};
    ppmd::Scratch scratch[ppmd::S_NSLOTS];
    void *h_stage = nullptr;           // pinned staging of host tables (stage_host)
    size_t h_stage_bytes = 0;
    cudaEvent_t stage_ev = nullptr;    // recorded after the last copy out of h_stage
};

namespace ppmd {

int set_error(ppmd_ctx *ctx, int code, const char *fmt, ...);
int cuda_check(ppmd_ctx *ctx, cudaError_t e, const char *what);
// Scratch buffer of at least `bytes` (grows; contents not preserved on growth).
void *scratch(ppmd_ctx *ctx, int slot, size_t bytes);
int check_launch(ppmd_ctx *ctx, const char *what);
// Pinned host buffer of at least `bytes` for tables that are then copied to
// the device with cudaMemcpyAsync (which does not wait for the stream when
// the source is pinned); waits until the copies of the previous use have
// run.  After issuing the copies, call stage_done.
void *stage_host(ppmd_ctx *ctx, size_t bytes);
int stage_done(ppmd_ctx *ctx);

#define PPMD_LAUNCH(ctx, kernel, grid, block, smem, ...)                           \
    do {                                                                           \
        kernel<<<(grid), (block), (smem), (ctx)->stream>>>(__VA_ARGS__);           \
        (ctx)->launches += 1;                                                      \
    } while (0)

#define PPMD_TRY(expr)              \
    do {                            \
        int _rc = (expr);           \
        if (_rc < 0) return _rc;    \
    } while (0)

// ---------------------------------------------------------------------
// Device-side status latch: errors (< 0) replace warnings (> 0); the first
// error is kept.
// ---------------------------------------------------------------------
__device__ __forceinline__ void latch_status(int32_t *st, int32_t code) {
    int32_t old = *((volatile int32_t *)st);
    while (old == 0 || (old > 0 && code < 0)) {
        int32_t prev = atomicCAS(st, old, code);
        if (prev == old) break;
        old = prev;
    }
}
__device__ __forceinline__ void latch_needed(unsigned long long *nd, unsigned long long v) { atomicMax(nd, v); }

// ---------------------------------------------------------------------
// Box segments.  A segment is one periodic box with its atoms and its
// cell grid; a batch of independent replicas is a table of segments.
// ---------------------------------------------------------------------
struct Seg {
    double L[3];
    double w[3];      // cell edge L/n
    double inv_w[3];  // 1/w (fast binning)
    double fxs[3];    // 2^32 / L  (coordinate -> fixed point)
    double inv_L[3];  // 1/L
    float sx[3];      // L / 2^32  (fixed point -> length)
    int32_t nc[3];
    int32_t cell0;    // first global cell index of the segment
    double rl2;       // list cutoff squared (FP64)
    float rl2_lo, rl2_hi;  // FP32 decision band around rl2
    int64_t atom0, atom1;
};

struct SegTable {
    const Seg *d;  // device table (nseg > 1)
    Seg one;       // the segment when nseg == 1
    int32_t nseg;
};

__device__ __forceinline__ const Seg &seg_ref(const SegTable &t, int32_t s) { return t.nseg == 1 ? t.one : t.d[s]; }

// Host: fill a segment for box L, cell grid for min_cell_width (0 = none).
int make_seg(ppmd_ctx *ctx, Seg &s, const double L[3], double min_cell_width, double r_list);
// Wait for the stream and read the latched status (as ppmd_status); with
// aux, also the int32 result word that kernels may leave at d_status[4].
int status_sync(ppmd_ctx *ctx, int64_t *needed, int32_t *aux);
// FP32 decision band for a squared cutoff rc2 in a box of largest edge Lmax.
void cutoff_band(double rc2, double Lmax, float *lo, float *hi);

// ---------------------------------------------------------------------
// Fixed-point coordinates.  x in [0, L) is stored as round(x 2^32 / L)
// modulo 2^32; the difference of two such words, read as a signed 32-bit
// integer, is the minimum-image separation in units of L / 2^32.
// ---------------------------------------------------------------------
__device__ __forceinline__ uint32_t to_fixed(double x, double fxs) {
    unsigned long long q = __double2ull_rn(x * fxs);
    return (uint32_t)q;  // 2^32 (x rounding up to L) wraps to 0
}

__device__ __forceinline__ float fixed_delta(uint32_t a, uint32_t b, float s) {
    return __int2float_rn((int32_t)(a - b)) * s;
}

// Wrap into [0, L): x - L floor(x / L), an exact L mapping to 0.  The
// operations are the IEEE ones (no contraction) so that the result equals
// the plain C evaluation bit for bit.
__device__ __forceinline__ double wrap_exact(double x, double L) {
    double y = __dsub_rn(x, __dmul_rn(L, floor(__ddiv_rn(x, L))));
    if (y >= L || y < 0.0) y = 0.0;
    return y;
}

// Cheap wrap for a coordinate already within one box length of [0, L).
__device__ __forceinline__ double wrap_near(double x, double L) {
    if (x >= L) x = __dsub_rn(x, L);
    else if (x < 0.0) x = __dadd_rn(x, L);
    if (x >= L || x < 0.0) x = 0.0;
    return x;
}

// Minimum-image squared distance in FP64, evaluated exactly as
// d = a - b; d = d - L rint(d / L); r2 = dx*dx + dy*dy + dz*dz.
// rint(d/L) is computed as rint(d * (1/L)): for |d| < L/2 + r with r < L/2
// both give the same integer.
__device__ __forceinline__ double min_image_r2(const double *a, const double *b, const Seg &s, double dr[3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double t = __dsub_rn(a[k], b[k]);
        double m = rint(__dmul_rn(t, s.inv_L[k]));
        dr[k] = __dsub_rn(t, __dmul_rn(s.L[k], m));
    }
    return __dadd_rn(__dadd_rn(__dmul_rn(dr[0], dr[0]), __dmul_rn(dr[1], dr[1])), __dmul_rn(dr[2], dr[2]));
}

// ---------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Reciprocal: hardware approximation refined by one Newton-Raphson step
// (r' = r + r (1 - x r)), accurate to about one unit in the last place for
// normal x.
__device__ __forceinline__ float recip(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    float e = fmaf(-x, r, 1.0f);
    return fmaf(r, e, r);
}

// Kahan-compensated accumulator: value = s - c.
struct Kahan {
    float s, c;
    __device__ __forceinline__ void init() { s = 0.f; c = 0.f; }
    __device__ __forceinline__ void add(float v) {
        float y = v - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// Merge of two compensated sums (hi, lo) with an error-free TwoSum of the
// leading parts.
__device__ __forceinline__ void two_sum_merge(float &hi, float &lo, float hi2, float lo2) {
    float s = hi + hi2;
    float bp = s - hi;
    float err = (hi - (s - bp)) + (hi2 - bp);
    hi = s;
    lo = lo + lo2 + err;
}

inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Exclusive scan of n int32 counts into out[0..n] (out[n] = total), in place
// allowed.  Uses scratch slot S_SCAN.
int exclusive_scan(ppmd_ctx *ctx, const int32_t *in, int32_t *out, int64_t n);

// Fixed-order sum of `nparts` rows of `width` doubles into dst[width].
int reduce_partials(ppmd_ctx *ctx, const double *parts, int64_t nparts, int width, double *dst);

}  // namespace ppmd
