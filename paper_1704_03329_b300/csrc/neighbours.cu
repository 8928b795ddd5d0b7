// Neighbour-list build (Sec. 3.5, Eq. (3)): one warp per atom sweeps the 27
// cells around its cell, tests every candidate in single precision from
// fixed-point coordinates, re-tests pairs near the cutoff in double
// precision, and compacts the hits with a warp ballot into the atom's row.
#include "cells.cuh"
#include "neighbours.cuh"

namespace ppmd {

// Fixed-point copy of positions (and, optionally, the exact cell of each
// atom for a grid of n_d cells per edge).
__global__ void k_prep_fixed(const double *__restrict__ pos, int64_t n, SegTable st, const int32_t *__restrict__ seg_of,
                             int4 *__restrict__ xq, int32_t *__restrict__ cell_of, int32_t *status) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t sid = seg_of ? seg_of[i] : 0;
    const Seg &S = seg_ref(st, sid);
    uint32_t q[3];
    int32_t c[3];
    bool bad = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double x = pos[3 * i + d];
        if (!isfinite(x)) {
            bad = true;
            x = 0.0;
        }
        // the fixed-point word only needs x modulo L; the exact cell (when
        // asked for) follows the documented wrap
        const double xw = cell_of ? wrap_exact(x, S.L[d]) : ((x >= 0.0 && x < S.L[d]) ? x : wrap_exact(x, S.L[d]));
        q[d] = to_fixed(xw, S.fxs[d]);
        if (cell_of) {
            int32_t cd = (int32_t)floor(__ddiv_rn(xw, S.w[d]));
            c[d] = cd < 0 ? 0 : (cd > S.nc[d] - 1 ? S.nc[d] - 1 : cd);
        }
    }
    if (bad) latch_status(status, PPMD_ERR_NONFINITE);
    xq[i] = make_int4((int)q[0], (int)q[1], (int)q[2], sid);
    if (cell_of) cell_of[i] = S.cell0 + (c[2] * S.nc[1] + c[1]) * S.nc[0] + c[0];
}

int prep_fixed(ppmd_ctx *ctx, const double *pos, int64_t n, const SegTable &st, const int32_t *seg_of, int4 *xq,
               int32_t *cell_of) {
    if (n > 0) PPMD_LAUNCH(ctx, k_prep_fixed, div_up(n, 256), 256, 0, pos, n, st, seg_of, xq, cell_of, ctx->d_status);
    return check_launch(ctx, "prep_fixed");
}

// pos64: double positions in the same order as xq (for the exact re-test).
// Candidate k of a cell range is atom cell_atoms[k] (or k itself when
// cell_atoms is null: atoms stored in cell order).
__global__ void __launch_bounds__(256) k_neigh(int64_t n, const int4 *__restrict__ xq, const double *__restrict__ pos64,
                                               SegTable st, const int32_t *__restrict__ cell_of,
                                               const int32_t *__restrict__ cell_start,
                                               const int32_t *__restrict__ cell_atoms, int32_t *__restrict__ nbr,
                                               int32_t *__restrict__ cnt, int32_t max_nbr, int32_t *status,
                                               unsigned long long *needed) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;
    const int4 xi = __ldg(&xq[i]);
    const Seg &S = seg_ref(st, xi.w);
    const int32_t nx = S.nc[0], ny = S.nc[1], nz = S.nc[2];
    int32_t c = cell_of[i] - S.cell0;
    const int32_t cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
    const float sx = S.sx[0], sy = S.sx[1], sz = S.sx[2];
    const float lo = S.rl2_lo, hi = S.rl2_hi;
    int32_t count = 0;
    int32_t *row = nbr + i * (int64_t)max_nbr;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int dz = -1; dz <= 1; ++dz) {
        int32_t z = cz + dz;
        z = z < 0 ? z + nz : (z >= nz ? z - nz : z);
        for (int dy = -1; dy <= 1; ++dy) {
            int32_t y = cy + dy;
            y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
            const int32_t rowc = S.cell0 + (z * ny + y) * nx;
            // the three cells x-1, x, x+1 of this row as one or two index ranges
            int32_t a0, b0, a1 = 0, b1 = 0;
            if (nx == 3) {
                a0 = cell_start[rowc];
                b0 = cell_start[rowc + 3];
            } else if (cx == 0) {
                a0 = cell_start[rowc];
                b0 = cell_start[rowc + 2];
                a1 = cell_start[rowc + nx - 1];
                b1 = cell_start[rowc + nx];
            } else if (cx == nx - 1) {
                a0 = cell_start[rowc + nx - 2];
                b0 = cell_start[rowc + nx];
                a1 = cell_start[rowc];
                b1 = cell_start[rowc + 1];
            } else {
                a0 = cell_start[rowc + cx - 1];
                b0 = cell_start[rowc + cx + 2];
            }
#pragma unroll 1
            for (int part = 0; part < 2; ++part) {
                const int32_t a = part ? a1 : a0, b = part ? b1 : b0;
                for (int32_t base = a; base < b; base += 32) {
                    const int32_t k = base + lane;
                    bool hit = false;
                    int32_t j = -1;
                    if (k < b) {
                        j = cell_atoms ? cell_atoms[k] : k;
                        if (j != (int32_t)i) {
                            const int4 xj = __ldg(&xq[j]);
                            float dx = fixed_delta((uint32_t)xi.x, (uint32_t)xj.x, sx);
                            float dy_ = fixed_delta((uint32_t)xi.y, (uint32_t)xj.y, sy);
                            float dz_ = fixed_delta((uint32_t)xi.z, (uint32_t)xj.z, sz);
                            float r2 = fmaf(dx, dx, fmaf(dy_, dy_, dz_ * dz_));
                            if (r2 < lo) {
                                hit = true;
                            } else if (r2 < hi) {
                                double dr[3];
                                hit = min_image_r2(pos64 + 3 * i, pos64 + 3 * (int64_t)j, S, dr) < S.rl2;
                            }
                        }
                    }
                    const unsigned ball = __ballot_sync(0xffffffffu, hit);
                    if (hit) {
                        const int32_t slot = count + __popc(ball & lt_mask);
                        if (slot < max_nbr) row[slot] = j;
                    }
                    count += __popc(ball);
                }
            }
        }
    }
    if (lane == 0) {
        cnt[i] = count;
        if (count > max_nbr) {
            latch_status(status, PPMD_ERR_CAPACITY);
            latch_needed(needed, (unsigned long long)count);
        }
    }
}

int build_list(ppmd_ctx *ctx, int64_t n, const int4 *xq, const double *pos64, const SegTable &st, const int32_t *cell_of,
               const int32_t *cell_start, const int32_t *cell_atoms, int32_t *nbr, int32_t *cnt, int32_t max_nbr) {
    if (n > 0)
        PPMD_LAUNCH(ctx, k_neigh, div_up(n * 32, 256), 256, 0, n, xq, pos64, st, cell_of, cell_start, cell_atoms, nbr, cnt,
                    max_nbr, ctx->d_status, ctx->d_needed);
    return check_launch(ctx, "build_list");
}

__global__ void k_max_count(const int32_t *cnt, int64_t n, unsigned long long *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int32_t v = i < n ? cnt[i] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0 && v > 0) atomicMax(out, (unsigned long long)v);
}

}  // namespace ppmd

using namespace ppmd;

extern "C" int ppmd_build_neighbours(ppmd_ctx *ctx, const double *pos, int64_t n, const ppmd_box *box, double r_list,
                                     const int32_t *cell_start, const int32_t *cell_atoms, const int32_t ncell[3],
                                     int32_t *nbr, int32_t *nbr_count, int32_t max_nbr, int32_t *needed_max_nbr) {
    if (!ctx || !box || !ncell || n < 0 || max_nbr < 0 || !(r_list > 0))
        return set_error(ctx, PPMD_ERR_INVALID, "ppmd_build_neighbours: bad argument");
    if (n > 0 && (!pos || !cell_start || !cell_atoms || !nbr_count || (max_nbr > 0 && !nbr)))
        return set_error(ctx, PPMD_ERR_INVALID, "ppmd_build_neighbours: null array");
    cudaSetDevice(ctx->device);
    SegTable st;
    st.d = nullptr;
    st.nseg = 1;
    PPMD_TRY(make_seg(ctx, st.one, box->L, 0.0, r_list));
    for (int d = 0; d < 3; ++d) {
        if (ncell[d] < 3) return set_error(ctx, PPMD_ERR_BOX, "fewer than 3 cells along edge %d", d);
        st.one.nc[d] = ncell[d];
        st.one.w[d] = box->L[d] / ncell[d];
        st.one.inv_w[d] = 1.0 / st.one.w[d];
        if (st.one.w[d] < r_list) return set_error(ctx, PPMD_ERR_BOX, "cell edge %g is below the cutoff %g", st.one.w[d], r_list);
    }
    int4 *xq = (int4 *)scratch(ctx, S_XQ, sizeof(int4) * (size_t)(n > 0 ? n : 1));
    int32_t *cell_of = (int32_t *)scratch(ctx, S_TMP0, sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!xq || !cell_of) return PPMD_ERR_NOMEM;
    PPMD_TRY(prep_fixed(ctx, pos, n, st, nullptr, xq, cell_of));
    PPMD_TRY(build_list(ctx, n, xq, pos, st, cell_of, cell_start, cell_atoms, nbr, nbr_count, max_nbr));
    if (needed_max_nbr) {
        unsigned long long *d = (unsigned long long *)scratch(ctx, S_TMP1, 8);
        if (!d) return PPMD_ERR_NOMEM;
        PPMD_TRY(cuda_check(ctx, cudaMemsetAsync(d, 0, 8, ctx->stream), "memset"));
        if (n > 0) PPMD_LAUNCH(ctx, k_max_count, div_up(n, 256), 256, 0, nbr_count, n, d);
        unsigned long long h = 0;
        PPMD_TRY(cuda_check(ctx, cudaMemcpyAsync(&h, d, 8, cudaMemcpyDeviceToHost, ctx->stream), "copy"));
        int rc = ppmd_sync(ctx);
        *needed_max_nbr = (int32_t)h;
        return rc;
    }
    return PPMD_OK;
}
