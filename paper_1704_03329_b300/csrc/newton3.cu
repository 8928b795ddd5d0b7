// Lennard-Jones pair loop over a half neighbour list (Newton's third law):
// every unordered pair {i, j} is evaluated once, by the atom whose row
// holds it, and its force is added to that atom and, with the opposite
// sign, to the other.  Sec. 2 evaluates every ordered pair and writes to i
// only; the half list halves the pair arithmetic and the list bytes and
// pays for it with one atomic update of the other atom per interacting pair
// (the write conflicts the paper's design avoids).
//
// FP32 path: the pair terms of Eqs. (9) and (12) in single precision; each
// atom's own share in compensated (Kahan) sums, the shares received from
// other atoms through float4 atomic adds (x, y, z, energy) into an FP32
// buffer, so the order of those additions, and with it the last bits of
// the result, varies from run to run.  FP64 path: double-precision terms,
// own shares summed in order, received shares through double atomic adds.
#include "lj.cuh"

namespace ppmd {
namespace {

constexpr int N3_G = 8;  // lanes per atom
constexpr int N3_BLOCK = 256;

// Half list from a full row-major list: the entries j of row i whose
// minimum-image displacement r_j - r_i, taken in the 32-bit fixed-point box
// coordinates, is positive in the order (z, y, x) (the first non-zero
// component decides).  The wrapping integer differences are exactly
// antisymmetric, so every pair is kept by exactly one of its two atoms and
// rows hold about half of the full length whatever the atom order.  Rows
// longer than max_half latch PPMD_ERR_CAPACITY with the length needed.
__global__ void k_half_list(int64_t n, const int4 *__restrict__ xq, const int32_t *__restrict__ nbr,
                            const int32_t *__restrict__ cnt, int32_t max_nbr, int32_t *__restrict__ half,
                            int32_t *__restrict__ hcnt, int32_t max_half, int32_t *status,
                            unsigned long long *needed) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int4 xi = xq[i];
    const int32_t m = min(cnt[i], max_nbr);
    const int32_t *row = nbr + i * (int64_t)max_nbr;
    int32_t *out = half + i * (int64_t)max_half;
    int32_t k = 0;
    for (int32_t e = 0; e < m; ++e) {
        const int32_t j = row[e];
        const int4 xj = xq[j];
        const int32_t dx = (int32_t)((uint32_t)xj.x - (uint32_t)xi.x), dy = (int32_t)((uint32_t)xj.y - (uint32_t)xi.y),
                      dz = (int32_t)((uint32_t)xj.z - (uint32_t)xi.z);
        const bool upper = dz > 0 || (dz == 0 && (dy > 0 || (dy == 0 && dx > 0)));
        if (upper) {
            if (k < max_half) out[k] = j;
            ++k;
        }
    }
    hcnt[i] = k;
    if (k > max_half) {
        latch_status(status, PPMD_ERR_CAPACITY);
        latch_needed(needed, (unsigned long long)k);
    }
}

template <int G>
__device__ __forceinline__ void n3_merge(float &hi, float &lo) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        two_sum_merge(hi, lo, h2, l2);
    }
}

template <int G>
__device__ __forceinline__ double n3_sum(double v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block sums of (U, W) into partials[2 * blockIdx.x].
__device__ __forceinline__ void n3_partials(double u, double w, double *partials) {
    __shared__ double su[N3_BLOCK / 32], sw[N3_BLOCK / 32];
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
        for (int k = 0; k < N3_BLOCK / 32; ++k) {
            a += su[k];
            b += sw[k];
        }
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = b;
    }
}

// FP32: acc[i] = (Fx, Fy, Fz, e_i) accumulated by atomics (zeroed before).
__global__ void __launch_bounds__(N3_BLOCK) k_lj_n3_fp32(int64_t n, const int4 *__restrict__ xq,
                                                         const double *__restrict__ pos64, SegTable st, LJConst c,
                                                         const int32_t *__restrict__ half,
                                                         const int32_t *__restrict__ hcnt, int32_t max_half,
                                                         float4 *__restrict__ acc, double *__restrict__ partials) {
    constexpr int G = N3_G;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = t / G;
    const int sub = threadIdx.x % G;
    const bool active = i < n;
    Kahan fx, fy, fz, ea, vir;  // own force, own half of the pair energies, pair virial
    fx.init();
    fy.init();
    fz.init();
    ea.init();
    vir.init();
    if (active) {
        const int4 xi = __ldg(&xq[i]);
        const Seg &S = seg_ref(st, xi.w);
        const int32_t m = min(hcnt[i], max_half);
        const int32_t *row = half + i * (int64_t)max_half;
        for (int32_t k = sub; k < m; k += G) {
            const int32_t j = __ldg(&row[k]);
            const int4 xj = __ldg(&xq[j]);
            const float dx = fixed_delta((uint32_t)xi.x, (uint32_t)xj.x, S.sx[0]);
            const float dy = fixed_delta((uint32_t)xi.y, (uint32_t)xj.y, S.sx[1]);
            const float dz = fixed_delta((uint32_t)xi.z, (uint32_t)xj.z, S.sx[2]);
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            bool inside = r2 < c.rc2_lo;
            if (!inside && r2 < c.rc2_hi) {
                double dr[3];
                inside = min_image_r2(pos64 + 3 * i, pos64 + 3 * (int64_t)j, S, dr) < c.rc2;
            }
            if (!inside) continue;
            const float ir2 = recip(r2);
            const float sr2 = c.s2 * ir2;
            const float sr6 = sr2 * sr2 * sr2;
            const float fmag = c.f48 * sr6 * (sr6 - 0.5f) * ir2;
            const float vh = c.e2 * fmaf(sr6, sr6 - 1.0f, c.shift);  // half of V(r)
            const float gx = fmag * dx, gy = fmag * dy, gz = fmag * dz;
            fx.add(gx);
            fy.add(gy);
            fz.add(gz);
            ea.add(vh);
            vir.add(fmag * r2);
            atomicAdd(&acc[j], make_float4(-gx, -gy, -gz, vh));
        }
    }
    float hx = fx.s, lx = -fx.c, hy = fy.s, ly = -fy.c, hz = fz.s, lz = -fz.c, he = ea.s, le = -ea.c, hv = vir.s,
          lv = -vir.c;
    n3_merge<G>(hx, lx);
    n3_merge<G>(hy, ly);
    n3_merge<G>(hz, lz);
    n3_merge<G>(he, le);
    n3_merge<G>(hv, lv);
    const double e_own = (double)he + (double)le;
    if (active && sub == 0) atomicAdd(&acc[i], make_float4(hx + lx, hy + ly, hz + lz, (float)e_own));
    if (partials) {
        const bool lead = active && sub == 0;
        // U: every pair once, V = twice the half kept by i; W: every pair once
        n3_partials(lead ? 2.0 * e_own : 0.0, lead ? (double)hv + (double)lv : 0.0, partials);
    }
}

// FP64: acc[4 i + (0..3)] = (Fx, Fy, Fz, e_i) accumulated by atomics.
__global__ void __launch_bounds__(N3_BLOCK) k_lj_n3_fp64(int64_t n, const int4 *__restrict__ xq,
                                                         const double *__restrict__ pos64, SegTable st, LJConst c,
                                                         const int32_t *__restrict__ half,
                                                         const int32_t *__restrict__ hcnt, int32_t max_half,
                                                         double *__restrict__ acc, double *__restrict__ partials) {
    constexpr int G = N3_G;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = t / G;
    const int sub = threadIdx.x % G;
    const bool active = i < n;
    double fx = 0.0, fy = 0.0, fz = 0.0, ea = 0.0, vir = 0.0;
    if (active) {
        const Seg &S = seg_ref(st, xq[i].w);
        const int32_t m = min(hcnt[i], max_half);
        const int32_t *row = half + i * (int64_t)max_half;
        const double *pi = pos64 + 3 * i;
        for (int32_t k = sub; k < m; k += G) {
            const int32_t j = __ldg(&row[k]);
            double dr[3];
            const double r2 = min_image_r2(pi, pos64 + 3 * (int64_t)j, S, dr);
            if (!(r2 < c.rc2)) continue;
            const double sr2 = c.s2d / r2;
            const double sr6 = sr2 * sr2 * sr2;
            const double sr8 = sr6 * sr2;
            const double sr12 = sr6 * sr6;
            const double sr14 = sr12 * sr2;
            const double fmag = c.f48d * (sr14 - 0.5 * sr8);
            const double vh = c.e2d * (sr12 - sr6 + c.shiftd);
            const double gx = fmag * dr[0], gy = fmag * dr[1], gz = fmag * dr[2];
            fx += gx;
            fy += gy;
            fz += gz;
            ea += vh;
            vir += fmag * r2;
            atomicAdd(&acc[4 * (int64_t)j + 0], -gx);
            atomicAdd(&acc[4 * (int64_t)j + 1], -gy);
            atomicAdd(&acc[4 * (int64_t)j + 2], -gz);
            atomicAdd(&acc[4 * (int64_t)j + 3], vh);
        }
    }
    fx = n3_sum<G>(fx);
    fy = n3_sum<G>(fy);
    fz = n3_sum<G>(fz);
    ea = n3_sum<G>(ea);
    vir = n3_sum<G>(vir);
    if (active && sub == 0) {
        atomicAdd(&acc[4 * i + 0], fx);
        atomicAdd(&acc[4 * i + 1], fy);
        atomicAdd(&acc[4 * i + 2], fz);
        atomicAdd(&acc[4 * i + 3], ea);
    }
    if (partials) {
        const bool lead = active && sub == 0;
        n3_partials(lead ? 2.0 * ea : 0.0, lead ? vir : 0.0, partials);
    }
}

__global__ void k_n3_out_f32(int64_t n, const float4 *__restrict__ acc, double *__restrict__ force,
                             double *__restrict__ e_atom) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 a = acc[i];
    force[3 * i] = a.x;
    force[3 * i + 1] = a.y;
    force[3 * i + 2] = a.z;
    if (e_atom) e_atom[i] = a.w;
}

__global__ void k_n3_out_f64(int64_t n, const double *__restrict__ acc, double *__restrict__ force,
                             double *__restrict__ e_atom) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    force[3 * i] = acc[4 * i];
    force[3 * i + 1] = acc[4 * i + 1];
    force[3 * i + 2] = acc[4 * i + 2];
    if (e_atom) e_atom[i] = acc[4 * i + 3];
}

}  // namespace
}  // namespace ppmd

using namespace ppmd;

extern "C" int ppmd_half_list(ppmd_ctx *ctx, const double *pos, int64_t n, const ppmd_box *box, const int32_t *nbr,
                              const int32_t *nbr_count, int32_t max_nbr, int32_t *half, int32_t *half_count,
                              int32_t max_half) {
    if (!ctx || !box || n < 0 || max_nbr < 0 || max_half < 0)
        return set_error(ctx, PPMD_ERR_INVALID, "ppmd_half_list: bad argument");
    if (n > 0 && (!pos || !nbr_count || !half_count || (max_nbr > 0 && !nbr) || (max_half > 0 && !half)))
        return set_error(ctx, PPMD_ERR_INVALID, "ppmd_half_list: null array");
    cudaSetDevice(ctx->device);
    SegTable st;
    st.d = nullptr;
    st.nseg = 1;
    PPMD_TRY(make_seg(ctx, st.one, box->L, 0.0, 0.0));
    int4 *xq = (int4 *)scratch(ctx, S_XQ, sizeof(int4) * (size_t)(n > 0 ? n : 1));
    if (!xq) return PPMD_ERR_NOMEM;
    PPMD_TRY(prep_fixed(ctx, pos, n, st, nullptr, xq, nullptr));
    if (n > 0)
        PPMD_LAUNCH(ctx, k_half_list, div_up(n, 256), 256, 0, n, xq, nbr, nbr_count, max_nbr, half, half_count, max_half,
                    ctx->d_status, ctx->d_needed);
    return check_launch(ctx, "half_list");
}

extern "C" int ppmd_lj_forces_newton3(ppmd_ctx *ctx, const double *pos, int64_t n, const ppmd_box *box,
                                      const ppmd_lj_params *lj, const int32_t *half, const int32_t *half_count,
                                      int32_t max_half, ppmd_prec prec, double *force, double *e_atom, double *e_total,
                                      double *virial) {
    if (!ctx || !box || !lj || n < 0 || max_half < 0 || (prec != PPMD_FP32 && prec != PPMD_FP64))
        return set_error(ctx, PPMD_ERR_INVALID, "ppmd_lj_forces_newton3: bad argument");
    if (n > 0 && (!pos || !half_count || !force || (max_half > 0 && !half)))
        return set_error(ctx, PPMD_ERR_INVALID, "ppmd_lj_forces_newton3: null array");
    if (!(lj->rc > 0) || !(lj->sigma > 0))
        return set_error(ctx, PPMD_ERR_INVALID, "ppmd_lj_forces_newton3: bad parameters");
    cudaSetDevice(ctx->device);
    SegTable st;
    st.d = nullptr;
    st.nseg = 1;
    PPMD_TRY(make_seg(ctx, st.one, box->L, 0.0, lj->rc));
    const double Lmax = fmax(box->L[0], fmax(box->L[1], box->L[2]));
    const LJConst c = make_ljconst(*lj, Lmax);
    const size_t nn = (size_t)(n > 0 ? n : 1);
    int4 *xq = (int4 *)scratch(ctx, S_XQ, sizeof(int4) * nn);
    void *acc = scratch(ctx, S_TMP0, (prec == PPMD_FP32 ? sizeof(float4) : 4 * sizeof(double)) * nn);
    if (!xq || !acc) return PPMD_ERR_NOMEM;
    const int64_t nb = div_up(n * N3_G, N3_BLOCK);
    double *partials = nullptr;
    if (e_total || virial) {
        partials = (double *)scratch(ctx, S_PARTIAL, sizeof(double) * 2 * (size_t)(nb + 1));
        if (!partials) return PPMD_ERR_NOMEM;
    }
    PPMD_TRY(prep_fixed(ctx, pos, n, st, nullptr, xq, nullptr));
    if (n > 0) {
        PPMD_TRY(cuda_check(ctx, cudaMemsetAsync(acc, 0, (prec == PPMD_FP32 ? sizeof(float4) : 4 * sizeof(double)) * nn,
                                                 ctx->stream),
                            "memset"));
        if (prec == PPMD_FP32) {
            PPMD_LAUNCH(ctx, k_lj_n3_fp32, nb, N3_BLOCK, 0, n, xq, pos, st, c, half, half_count, max_half, (float4 *)acc,
                        partials);
            PPMD_LAUNCH(ctx, k_n3_out_f32, div_up(n, 256), 256, 0, n, (const float4 *)acc, force, e_atom);
        } else {
            PPMD_LAUNCH(ctx, k_lj_n3_fp64, nb, N3_BLOCK, 0, n, xq, pos, st, c, half, half_count, max_half, (double *)acc,
                        partials);
            PPMD_LAUNCH(ctx, k_n3_out_f64, div_up(n, 256), 256, 0, n, (const double *)acc, force, e_atom);
        }
    }
    PPMD_TRY(check_launch(ctx, "lj_newton3"));
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
