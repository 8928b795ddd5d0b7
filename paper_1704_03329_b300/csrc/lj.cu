// Lennard-Jones pair loop over a neighbour list (Eqs. (9) and (12), Listing
// "LJ-kernel"): every ordered pair (i, j) writes to i only (Sec. 2).  A group
// of G lanes handles one atom, each lane a strided share of its neighbours;
// the G partial sums are merged with warp shuffles.
#include "cells.cuh"
#include "lj.cuh"

namespace ppmd {

struct OutF64 {
    double *force;   // [n][3]
    double *e_atom;  // [n] or null
    __device__ __forceinline__ void store(int64_t i, double fx, double fy, double fz, double e) const {
        force[3 * i + 0] = fx;
        force[3 * i + 1] = fy;
        force[3 * i + 2] = fz;
        if (e_atom) e_atom[i] = e;
    }
};

struct OutF4 {
    float4 *f;  // (Fx, Fy, Fz, e_i)
    __device__ __forceinline__ void store(int64_t i, double fx, double fy, double fz, double e) const {
        f[i] = make_float4((float)fx, (float)fy, (float)fz, (float)e);
    }
};

template <int G>
__device__ __forceinline__ void group_merge(float &hi, float &lo) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        two_sum_merge(hi, lo, h2, l2);
    }
}

template <int G>
__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-level FP64 sum of (U, W) into partials[2 * blockIdx.x].
__device__ __forceinline__ void block_partials(double u, double w, double *partials) {
    __shared__ double su[32], sw[32];
    u = warp_sum(u);
    w = warp_sum(w);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        su[wid] = u;
        sw[wid] = w;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            a += su[k];
            b += sw[k];
        }
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = b;
    }
}

// Single-precision pair arithmetic with compensated sums.
template <int G, class Out>
__global__ void __launch_bounds__(256) k_lj_fp32(int64_t n, const int4 *__restrict__ xq, const double *__restrict__ pos64,
                                                 SegTable st, LJConst c, const int32_t *__restrict__ nbr,
                                                 const int32_t *__restrict__ cnt, int32_t max_nbr, Out out,
                                                 double *__restrict__ partials) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = t / G;
    const int sub = threadIdx.x % G;
    const bool active = i < n;
    Kahan fx, fy, fz, ea, vir;
    fx.init();
    fy.init();
    fz.init();
    ea.init();
    vir.init();
    if (active) {
        const int4 xi = __ldg(&xq[i]);
        const Seg &S = seg_ref(st, xi.w);
        const float sx = S.sx[0], sy = S.sx[1], sz = S.sx[2];
        const int32_t m = min(cnt[i], max_nbr);
        const int32_t *row = nbr + i * (int64_t)max_nbr;
        for (int32_t k = sub; k < m; k += G) {
            const int32_t j = __ldg(&row[k]);
            const int4 xj = __ldg(&xq[j]);
            const float dx = fixed_delta((uint32_t)xi.x, (uint32_t)xj.x, sx);
            const float dy = fixed_delta((uint32_t)xi.y, (uint32_t)xj.y, sy);
            const float dz = fixed_delta((uint32_t)xi.z, (uint32_t)xj.z, sz);
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            bool inside = r2 < c.rc2_lo;
            if (!inside && r2 < c.rc2_hi) {
                double dr[3];
                inside = min_image_r2(pos64 + 3 * i, pos64 + 3 * (int64_t)j, S, dr) < c.rc2;
            }
            const float ir2 = recip(r2);
            const float sr2 = c.s2 * ir2;
            const float sr6 = sr2 * sr2 * sr2;
            float fmag = c.f48 * sr6 * (sr6 - 0.5f) * ir2;
            float v = c.e2 * fmaf(sr6, sr6 - 1.0f, c.shift);
            fmag = inside ? fmag : 0.0f;
            v = inside ? v : 0.0f;
            fx.add(fmag * dx);
            fy.add(fmag * dy);
            fz.add(fmag * dz);
            ea.add(v);
            vir.add(fmag * r2);
        }
    }
    float hx = fx.s, lx = -fx.c, hy = fy.s, ly = -fy.c, hz = fz.s, lz = -fz.c, he = ea.s, le = -ea.c, hv = vir.s,
          lv = -vir.c;
    group_merge<G>(hx, lx);
    group_merge<G>(hy, ly);
    group_merge<G>(hz, lz);
    group_merge<G>(he, le);
    group_merge<G>(hv, lv);
    const double e_i = (double)he + (double)le;
    if (active && sub == 0) out.store(i, (double)hx + (double)lx, (double)hy + (double)ly, (double)hz + (double)lz, e_i);
    if (partials) {
        const bool lead = active && sub == 0;
        block_partials(lead ? e_i : 0.0, lead ? 0.5 * ((double)hv + (double)lv) : 0.0, partials);
    }
}

// Double-precision pair arithmetic (the plain FP64 path).
template <int G, class Out>
__global__ void __launch_bounds__(256) k_lj_fp64(int64_t n, const int4 *__restrict__ xq, const double *__restrict__ pos64,
                                                 SegTable st, LJConst c, const int32_t *__restrict__ nbr,
                                                 const int32_t *__restrict__ cnt, int32_t max_nbr, Out out,
                                                 double *__restrict__ partials) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = t / G;
    const int sub = threadIdx.x % G;
    const bool active = i < n;
    double fx = 0.0, fy = 0.0, fz = 0.0, ea = 0.0, vir = 0.0;
    if (active) {
        const int32_t sid = xq[i].w;
        const Seg &S = seg_ref(st, sid);
        const int32_t m = min(cnt[i], max_nbr);
        const int32_t *row = nbr + i * (int64_t)max_nbr;
        const double *pi = pos64 + 3 * i;
        for (int32_t k = sub; k < m; k += G) {
            const int32_t j = __ldg(&row[k]);
            double dr[3];
            const double r2 = min_image_r2(pi, pos64 + 3 * (int64_t)j, S, dr);
            if (r2 < c.rc2) {
                const double sr2 = c.s2d / r2;
                const double sr6 = sr2 * sr2 * sr2;
                const double sr8 = sr6 * sr2;
                const double sr12 = sr6 * sr6;
                const double sr14 = sr12 * sr2;
                const double fmag = c.f48d * (sr14 - 0.5 * sr8);
                fx += fmag * dr[0];
                fy += fmag * dr[1];
                fz += fmag * dr[2];
                ea += c.e2d * (sr12 - sr6 + c.shiftd);
                vir += fmag * r2;
            }
        }
    }
    fx = group_sum<G>(fx);
    fy = group_sum<G>(fy);
    fz = group_sum<G>(fz);
    ea = group_sum<G>(ea);
    vir = group_sum<G>(vir);
    if (active && sub == 0) out.store(i, fx, fy, fz, ea);
    if (partials) {
        const bool lead = active && sub == 0;
        block_partials(lead ? ea : 0.0, lead ? 0.5 * vir : 0.0, partials);
    }
}

// ---------------------------------------------------------------------
// List-free pair loop: the cell structure of Sec. 3.5 used directly, with
// no neighbour matrix W built or read (the role of the layer algorithm the
// paper cites for cell-based codes).  Atoms are sorted by cell (edge >= rc,
// at least three cells per axis); G lanes of one atom sweep the nine rows
// of three cells around its own, each row one range of the sorted order or
// two where it wraps in x.  Pair arithmetic, cutoff decisions and sums as
// in k_lj_fp32 (F32) or k_lj_fp64; results are stored at the caller's
// index perm[i].
// ---------------------------------------------------------------------
template <bool F32>
__global__ void __launch_bounds__(256) k_lj_cells(int64_t n, const int4 *__restrict__ xq, const double *__restrict__ pos64,
                                                  Seg S, LJConst c, const int32_t *__restrict__ cell_of,
                                                  const int32_t *__restrict__ perm,
                                                  const int32_t *__restrict__ cell_start, OutF64 out,
                                                  double *__restrict__ partials) {
    constexpr int G = 8;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = t / G;
    const int sub = threadIdx.x % G;
    const bool active = i < n;
    Kahan fx, fy, fz, ea, vir;  // F32
    fx.init();
    fy.init();
    fz.init();
    ea.init();
    vir.init();
    double dfx = 0.0, dfy = 0.0, dfz = 0.0, dea = 0.0, dvir = 0.0;  // !F32
    int64_t orig = 0;
    if (active) {
        orig = perm[i];
        const int32_t nx = S.nc[0], ny = S.nc[1], nz = S.nc[2];
        const int32_t cell = cell_of[orig] - S.cell0;
        const int32_t cx = cell % nx, cy = (cell / nx) % ny, cz = cell / (nx * ny);
        const int4 xi = __ldg(&xq[i]);
        const double *pi = pos64 + 3 * i;
        for (int dz = -1; dz <= 1; ++dz) {
            const int32_t zz = cz + dz < 0 ? nz - 1 : (cz + dz >= nz ? 0 : cz + dz);
            for (int dy = -1; dy <= 1; ++dy) {
                const int32_t yy = cy + dy < 0 ? ny - 1 : (cy + dy >= ny ? 0 : cy + dy);
                const int32_t rb = S.cell0 + (zz * ny + yy) * nx;
                // cells cx - 1, cx, cx + 1 of the row as sorted ranges [a0, b0) and [a1, b1)
                int32_t a0, b0, a1 = 0, b1 = 0;
                if (cx >= 1 && cx <= nx - 2) {
                    a0 = cell_start[rb + cx - 1];
                    b0 = cell_start[rb + cx + 2];
                } else if (cx == 0) {
                    a0 = cell_start[rb];
                    b0 = cell_start[rb + 2];
                    a1 = cell_start[rb + nx - 1];
                    b1 = cell_start[rb + nx];
                } else {
                    a0 = cell_start[rb + nx - 2];
                    b0 = cell_start[rb + nx];
                    a1 = cell_start[rb];
                    b1 = cell_start[rb + 1];
                }
                for (int part = 0; part < 2; ++part) {
                    const int32_t a = part ? a1 : a0, b = part ? b1 : b0;
                    for (int32_t j = a + sub; j < b; j += G) {
                        if (j == i) continue;
                        const int4 xj = __ldg(&xq[j]);
                        const float dx = fixed_delta((uint32_t)xi.x, (uint32_t)xj.x, S.sx[0]);
                        const float dy = fixed_delta((uint32_t)xi.y, (uint32_t)xj.y, S.sx[1]);
                        const float dzf = fixed_delta((uint32_t)xi.z, (uint32_t)xj.z, S.sx[2]);
                        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dzf * dzf));
                        if (!(r2 < c.rc2_hi)) continue;  // outside the cutoff for certain
                        if (F32) {
                            bool inside = r2 < c.rc2_lo;
                            if (!inside) {
                                double dr[3];
                                inside = min_image_r2(pi, pos64 + 3 * (int64_t)j, S, dr) < c.rc2;
                            }
                            if (!inside) continue;
                            const float ir2 = recip(r2);
                            const float sr2 = c.s2 * ir2;
                            const float sr6 = sr2 * sr2 * sr2;
                            const float fmag = c.f48 * sr6 * (sr6 - 0.5f) * ir2;
                            fx.add(fmag * dx);
                            fy.add(fmag * dy);
                            fz.add(fmag * dzf);
                            ea.add(c.e2 * fmaf(sr6, sr6 - 1.0f, c.shift));
                            vir.add(fmag * r2);
                        } else {
                            double dr[3];
                            const double r2d = min_image_r2(pi, pos64 + 3 * (int64_t)j, S, dr);
                            if (!(r2d < c.rc2)) continue;
                            const double sr2 = c.s2d / r2d;
                            const double sr6 = sr2 * sr2 * sr2;
                            const double sr8 = sr6 * sr2;
                            const double sr12 = sr6 * sr6;
                            const double sr14 = sr12 * sr2;
                            const double fmag = c.f48d * (sr14 - 0.5 * sr8);
                            dfx += fmag * dr[0];
                            dfy += fmag * dr[1];
                            dfz += fmag * dr[2];
                            dea += c.e2d * (sr12 - sr6 + c.shiftd);
                            dvir += fmag * r2d;
                        }
                    }
                }
            }
        }
    }
    double e_i, v_i;
    if (F32) {
        float hx = fx.s, lx = -fx.c, hy = fy.s, ly = -fy.c, hz = fz.s, lz = -fz.c, he = ea.s, le = -ea.c, hv = vir.s,
              lv = -vir.c;
        group_merge<G>(hx, lx);
        group_merge<G>(hy, ly);
        group_merge<G>(hz, lz);
        group_merge<G>(he, le);
        group_merge<G>(hv, lv);
        e_i = (double)he + (double)le;
        v_i = (double)hv + (double)lv;
        if (active && sub == 0) out.store(orig, (double)hx + (double)lx, (double)hy + (double)ly, (double)hz + (double)lz, e_i);
    } else {
        dfx = group_sum<G>(dfx);
        dfy = group_sum<G>(dfy);
        dfz = group_sum<G>(dfz);
        e_i = group_sum<G>(dea);
        v_i = group_sum<G>(dvir);
        if (active && sub == 0) out.store(orig, dfx, dfy, dfz, e_i);
    }
    if (partials) {
        const bool lead = active && sub == 0;
        block_partials(lead ? e_i : 0.0, lead ? 0.5 * v_i : 0.0, partials);
    }
}

__global__ void k_gather_sorted3(int64_t n, const int32_t *__restrict__ perm, const double *__restrict__ pos,
                                 double *__restrict__ out) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t o = perm[k];
    out[3 * k] = pos[3 * o];
    out[3 * k + 1] = pos[3 * o + 1];
    out[3 * k + 2] = pos[3 * o + 2];
}

LJConst make_ljconst(const ppmd_lj_params &p, double Lmax) {
    LJConst c;
    c.rc2 = p.rc * p.rc;
    cutoff_band(c.rc2, Lmax, &c.rc2_lo, &c.rc2_hi);
    c.s2d = p.sigma * p.sigma;
    c.f48d = 48.0 * p.eps / c.s2d;
    c.e2d = 2.0 * p.eps;
    c.shiftd = p.shift;
    c.s2 = (float)c.s2d;
    c.f48 = (float)(48.0 * p.eps);
    c.e2 = (float)c.e2d;
    c.shift = (float)p.shift;
    return c;
}

constexpr int LJ_G = 8;
constexpr int LJ_BLOCK = 256;

int64_t lj_blocks(int64_t n) { return div_up(n * LJ_G, LJ_BLOCK); }

int lj_launch(ppmd_ctx *ctx, int64_t n, const int4 *xq, const double *pos64, const SegTable &st, const LJConst &c,
              const int32_t *nbr, const int32_t *cnt, int32_t max_nbr, int prec, float4 *f4, double *f64, double *e64,
              double *partials) {
    if (n <= 0) return PPMD_OK;
    int64_t nb = lj_blocks(n);
    if (prec == PPMD_FP32) {
        if (f4) {
            OutF4 o{f4};
            PPMD_LAUNCH(ctx, (k_lj_fp32<LJ_G, OutF4>), nb, LJ_BLOCK, 0, n, xq, pos64, st, c, nbr, cnt, max_nbr, o, partials);
        } else {
            OutF64 o{f64, e64};
            PPMD_LAUNCH(ctx, (k_lj_fp32<LJ_G, OutF64>), nb, LJ_BLOCK, 0, n, xq, pos64, st, c, nbr, cnt, max_nbr, o, partials);
        }
    } else {
        OutF64 o{f64, e64};
        PPMD_LAUNCH(ctx, (k_lj_fp64<LJ_G, OutF64>), nb, LJ_BLOCK, 0, n, xq, pos64, st, c, nbr, cnt, max_nbr, o, partials);
    }
    return check_launch(ctx, "lj");
}

}  // namespace ppmd

using namespace ppmd;

extern "C" int ppmd_lj_forces(ppmd_ctx *ctx, const double *pos, int64_t n, const ppmd_box *box, const ppmd_lj_params *lj,
                              const int32_t *nbr, const int32_t *nbr_count, int32_t max_nbr, ppmd_prec prec,
                              double *force, double *e_atom, double *e_total, double *virial) {
    if (!ctx || !box || !lj || n < 0 || max_nbr < 0 || (prec != PPMD_FP32 && prec != PPMD_FP64))
        return set_error(ctx, PPMD_ERR_INVALID, "ppmd_lj_forces: bad argument");
    if (n > 0 && (!pos || !nbr_count || !force || (max_nbr > 0 && !nbr)))
        return set_error(ctx, PPMD_ERR_INVALID, "ppmd_lj_forces: null array");
    if (!(lj->rc > 0) || !(lj->sigma > 0)) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_lj_forces: bad parameters");
    cudaSetDevice(ctx->device);
    SegTable st;
    st.d = nullptr;
    st.nseg = 1;
    PPMD_TRY(make_seg(ctx, st.one, box->L, 0.0, lj->rc));
    double Lmax = fmax(box->L[0], fmax(box->L[1], box->L[2]));
    LJConst c = make_ljconst(*lj, Lmax);
    int4 *xq = (int4 *)scratch(ctx, S_XQ, sizeof(int4) * (size_t)(n > 0 ? n : 1));
    if (!xq) return PPMD_ERR_NOMEM;
    PPMD_TRY(prep_fixed(ctx, pos, n, st, nullptr, xq, nullptr));
    double *partials = nullptr;
    int64_t nb = lj_blocks(n);
    if (e_total || virial) {
        partials = (double *)scratch(ctx, S_PARTIAL, sizeof(double) * 2 * (size_t)(nb + 1));
        if (!partials) return PPMD_ERR_NOMEM;
    }
    PPMD_TRY(lj_launch(ctx, n, xq, pos, st, c, nbr, nbr_count, max_nbr, prec, nullptr, force, e_atom, partials));
    if (partials) {
        double *tot = (double *)scratch(ctx, S_TMP1, 2 * sizeof(double));
        if (!tot) return PPMD_ERR_NOMEM;
        PPMD_TRY(reduce_partials(ctx, partials, nb, 2, tot));
        if (e_total) PPMD_TRY(cuda_check(ctx, cudaMemcpyAsync(e_total, tot, 8, cudaMemcpyDeviceToDevice, ctx->stream), "copy"));
        if (virial) PPMD_TRY(cuda_check(ctx, cudaMemcpyAsync(virial, tot + 1, 8, cudaMemcpyDeviceToDevice, ctx->stream), "copy"));
    }
    return PPMD_OK;
}

extern "C" int ppmd_lj_forces_cells(ppmd_ctx *ctx, const double *pos, int64_t n, const ppmd_box *box,
                                    const ppmd_lj_params *lj, ppmd_prec prec, double *force, double *e_atom,
                                    double *e_total, double *virial) {
    if (!ctx || !box || !lj || n < 0 || (prec != PPMD_FP32 && prec != PPMD_FP64))
        return set_error(ctx, PPMD_ERR_INVALID, "ppmd_lj_forces_cells: bad argument");
    if (n > 0 && (!pos || !force)) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_lj_forces_cells: null array");
    if (n >= (int64_t)1 << 31) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_lj_forces_cells: n too large");
    if (!(lj->rc > 0) || !(lj->sigma > 0)) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_lj_forces_cells: bad parameters");
    cudaSetDevice(ctx->device);
    SegTable st;
    st.d = nullptr;
    st.nseg = 1;
    PPMD_TRY(make_seg(ctx, st.one, box->L, lj->rc, lj->rc));  // cells of edge >= rc, at least three per axis
    st.one.atom0 = 0;
    st.one.atom1 = n;
    const double Lmax = fmax(box->L[0], fmax(box->L[1], box->L[2]));
    const LJConst c = make_ljconst(*lj, Lmax);
    const int64_t ncell = (int64_t)st.one.nc[0] * st.one.nc[1] * st.one.nc[2];
    const size_t nn = (size_t)(n > 0 ? n : 1);
    int32_t *cell_of = (int32_t *)scratch(ctx, S_CELLS0, sizeof(int32_t) * nn);
    int32_t *cell_start = (int32_t *)scratch(ctx, S_CELLS1, sizeof(int32_t) * (size_t)(ncell + 1));
    int32_t *perm = (int32_t *)scratch(ctx, S_CELLS2, sizeof(int32_t) * nn);
    double *spos = (double *)scratch(ctx, S_SORTPOS, sizeof(double) * 3 * nn);
    int4 *xq = (int4 *)scratch(ctx, S_AUX0, sizeof(int4) * nn);
    if (!cell_of || !cell_start || !perm || !spos || !xq) return PPMD_ERR_NOMEM;
    PPMD_TRY(bin_atoms(ctx, pos, n, st, nullptr, ncell, false, cell_of, cell_start, perm));
    if (n > 0) PPMD_LAUNCH(ctx, k_gather_sorted3, div_up(n, 256), 256, 0, n, perm, pos, spos);
    PPMD_TRY(prep_fixed(ctx, spos, n, st, nullptr, xq, nullptr));
    const int64_t nb = div_up(n * 8, 256);
    double *partials = nullptr;
    if (e_total || virial) {
        partials = (double *)scratch(ctx, S_PARTIAL, sizeof(double) * 2 * (size_t)(nb + 1));
        if (!partials) return PPMD_ERR_NOMEM;
    }
    OutF64 o{force, e_atom};
    if (n > 0) {
        if (prec == PPMD_FP32)
            PPMD_LAUNCH(ctx, k_lj_cells<true>, nb, 256, 0, n, xq, spos, st.one, c, cell_of, perm, cell_start, o, partials);
        else
            PPMD_LAUNCH(ctx, k_lj_cells<false>, nb, 256, 0, n, xq, spos, st.one, c, cell_of, perm, cell_start, o, partials);
    }
    PPMD_TRY(check_launch(ctx, "lj_cells"));
    if (partials) {
        double *tot = (double *)scratch(ctx, S_TMP1, 2 * sizeof(double));
        if (!tot) return PPMD_ERR_NOMEM;
        if (n > 0) {
            PPMD_TRY(reduce_partials(ctx, partials, nb, 2, tot));
        } else {
            PPMD_TRY(cuda_check(ctx, cudaMemsetAsync(tot, 0, 2 * sizeof(double), ctx->stream), "memset"));
        }
        if (e_total) PPMD_TRY(cuda_check(ctx, cudaMemcpyAsync(e_total, tot, 8, cudaMemcpyDeviceToDevice, ctx->stream), "copy"));
        if (virial) PPMD_TRY(cuda_check(ctx, cudaMemcpyAsync(virial, tot + 1, 8, cudaMemcpyDeviceToDevice, ctx->stream), "copy"));
    }
    return PPMD_OK;
}
