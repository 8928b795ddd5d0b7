// Velocity Verlet particle loops (Algorithm 6, Listings "position_update"
// and "velocity_update") and the kinetic-energy particle loop (Sec. 2).
#include "verlet.cuh"

namespace ppmd {

// Entry-point form: IEEE operations without contraction, in the order
// v = v + (dt/2m) F, r = r + dt v, r = r - L floor(r / L).
__global__ void k_vv_plain(int phase, double *__restrict__ pos, double *__restrict__ vel, const double *__restrict__ F,
                           int64_t n, double L0, double L1, double L2, double h, double dt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double L[3] = {L0, L1, L2};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double v = __dadd_rn(vel[3 * i + d], __dmul_rn(h, F[3 * i + d]));
        vel[3 * i + d] = v;
        if (phase == 1) pos[3 * i + d] = wrap_exact(__dadd_rn(pos[3 * i + d], __dmul_rn(dt, v)), L[d]);
    }
}

// Block sums of m |v|^2 / 2 into partials[blockIdx.x].
__device__ __forceinline__ void block_sum1(double v, double *partials) {
    __shared__ double sh[32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) a += sh[k];
        partials[blockIdx.x] = a;
    }
}

__global__ void k_kinetic(const double *__restrict__ vel, int64_t n, double half_m, double *partials) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double k = 0.0;
    if (i < n) {
        double vx = vel[3 * i], vy = vel[3 * i + 1], vz = vel[3 * i + 2];
        k = half_m * (vx * vx + vy * vy + vz * vz);
    }
    block_sum1(k, partials);
}

// ---------------------------------------------------------------------
// Integrator kernels (atoms in cell order, forces as float4 or double[3]).
// ---------------------------------------------------------------------
template <class F>
__device__ __forceinline__ void load_force(const F *f, int64_t i, double out[3]);
template <>
__device__ __forceinline__ void load_force<float4>(const float4 *f, int64_t i, double out[3]) {
    float4 v = f[i];
    out[0] = v.x;
    out[1] = v.y;
    out[2] = v.z;
}
template <>
__device__ __forceinline__ void load_force<double>(const double *f, int64_t i, double out[3]) {
    out[0] = f[3 * i];
    out[1] = f[3 * i + 1];
    out[2] = f[3 * i + 2];
}

// Kick + drift + wrap; refresh the fixed-point copy; track the largest
// displacement since the last list build (as a float bit pattern).
template <class F>
__global__ void __launch_bounds__(256) k_md_kick_drift(int64_t n, double *__restrict__ pos, double *__restrict__ vel,
                                                       const F *__restrict__ force, int4 *__restrict__ xq,
                                                       const int4 *__restrict__ xq_ref, SegTable st, double h, double dt,
                                                       unsigned int *max_disp_bits) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float d2 = 0.0f;
    if (i < n) {
        double f[3];
        load_force<F>(force, i, f);
        const int4 old = xq[i];
        const Seg &S = seg_ref(st, old.w);
        uint32_t q[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double v = fma(h, f[d], vel[3 * i + d]);
            vel[3 * i + d] = v;
            double r = wrap_near(fma(dt, v, pos[3 * i + d]), S.L[d]);
            pos[3 * i + d] = r;
            q[d] = to_fixed(r, S.fxs[d]);
        }
        xq[i] = make_int4((int)q[0], (int)q[1], (int)q[2], old.w);
        const int4 ref = xq_ref[i];
        float ex = fixed_delta(q[0], (uint32_t)ref.x, S.sx[0]);
        float ey = fixed_delta(q[1], (uint32_t)ref.y, S.sx[1]);
        float ez = fixed_delta(q[2], (uint32_t)ref.z, S.sx[2]);
        d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d2 = fmaxf(d2, __shfl_xor_sync(0xffffffffu, d2, o));
    if ((threadIdx.x & 31) == 0 && d2 > 0.0f) atomicMax(max_disp_bits, __float_as_uint(d2));
}

// Kick; on energy steps also the block sums of the kinetic energy.
template <class F>
__global__ void __launch_bounds__(256) k_md_kick(int64_t n, double *__restrict__ vel, const F *__restrict__ force, double h,
                                                 double half_m, double *partials) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double k = 0.0;
    if (i < n) {
        double f[3];
        load_force<F>(force, i, f);
        double vx = fma(h, f[0], vel[3 * i]);
        double vy = fma(h, f[1], vel[3 * i + 1]);
        double vz = fma(h, f[2], vel[3 * i + 2]);
        vel[3 * i] = vx;
        vel[3 * i + 1] = vy;
        vel[3 * i + 2] = vz;
        k = half_m * (vx * vx + vy * vy + vz * vz);
    }
    if (partials) block_sum1(k, partials);
}

int md_kick_drift(ppmd_ctx *ctx, int64_t n, double *pos, double *vel, const float4 *f4, const double *f64, int4 *xq,
                  const int4 *xq_ref, const SegTable &st, double h, double dt, unsigned int *max_disp_bits) {
    if (n <= 0) return PPMD_OK;
    if (f4)
        PPMD_LAUNCH(ctx, k_md_kick_drift<float4>, div_up(n, 256), 256, 0, n, pos, vel, f4, xq, xq_ref, st, h, dt, max_disp_bits);
    else
        PPMD_LAUNCH(ctx, k_md_kick_drift<double>, div_up(n, 256), 256, 0, n, pos, vel, f64, xq, xq_ref, st, h, dt, max_disp_bits);
    return check_launch(ctx, "md_kick_drift");
}

int64_t kick_blocks(int64_t n) { return div_up(n, 256); }

int md_kick(ppmd_ctx *ctx, int64_t n, double *vel, const float4 *f4, const double *f64, double h, double half_m,
            double *partials) {
    if (n <= 0) return PPMD_OK;
    if (f4)
        PPMD_LAUNCH(ctx, k_md_kick<float4>, div_up(n, 256), 256, 0, n, vel, f4, h, half_m, partials);
    else
        PPMD_LAUNCH(ctx, k_md_kick<double>, div_up(n, 256), 256, 0, n, vel, f64, h, half_m, partials);
    return check_launch(ctx, "md_kick");
}

// ---------------------------------------------------------------------
// Reordering by cell: gather every per-atom array through `perm`
// (new position k holds old atom perm[k]).
// ---------------------------------------------------------------------
__global__ void k_gather(int64_t n, const int32_t *__restrict__ perm, const double *__restrict__ pos,
                         const double *__restrict__ vel, const int4 *__restrict__ xq, const int32_t *__restrict__ orig,
                         const int32_t *__restrict__ cell_of, double *__restrict__ pos_o, double *__restrict__ vel_o,
                         int4 *__restrict__ xq_o, int32_t *__restrict__ orig_o, int32_t *__restrict__ cell_o) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t j = perm[k];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        pos_o[3 * k + d] = pos[3 * j + d];
        vel_o[3 * k + d] = vel[3 * j + d];
    }
    xq_o[k] = xq[j];
    orig_o[k] = orig[j];
    cell_o[k] = cell_of[j];
}

int gather_sorted(ppmd_ctx *ctx, int64_t n, const int32_t *perm, const double *pos, const double *vel, const int4 *xq,
                  const int32_t *orig, const int32_t *cell_of, double *pos_o, double *vel_o, int4 *xq_o,
                  int32_t *orig_o, int32_t *cell_o) {
    if (n > 0)
        PPMD_LAUNCH(ctx, k_gather, div_up(n, 256), 256, 0, n, perm, pos, vel, xq, orig, cell_of, pos_o, vel_o, xq_o, orig_o,
                    cell_o);
    return check_launch(ctx, "gather_sorted");
}

// Export in caller order: out[orig[k]] = in[k].
template <class T, int W>
__global__ void k_scatter_rows(int64_t n, const int32_t *__restrict__ orig, const T *__restrict__ in, T *__restrict__ out) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t o = orig[k];
#pragma unroll
    for (int d = 0; d < W; ++d) out[W * o + d] = in[W * k + d];
}

__global__ void k_scatter_f4(int64_t n, const int32_t *__restrict__ orig, const float4 *__restrict__ in,
                             double *__restrict__ out) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t o = orig[k];
    float4 v = in[k];
    out[3 * o] = v.x;
    out[3 * o + 1] = v.y;
    out[3 * o + 2] = v.z;
}

int scatter_vec3(ppmd_ctx *ctx, int64_t n, const int32_t *orig, const double *in, double *out) {
    if (n > 0) PPMD_LAUNCH(ctx, (k_scatter_rows<double, 3>), div_up(n, 256), 256, 0, n, orig, in, out);
    return check_launch(ctx, "scatter_vec3");
}

int scatter_f4(ppmd_ctx *ctx, int64_t n, const int32_t *orig, const float4 *in, double *out) {
    if (n > 0) PPMD_LAUNCH(ctx, k_scatter_f4, div_up(n, 256), 256, 0, n, orig, in, out);
    return check_launch(ctx, "scatter_f4");
}

}  // namespace ppmd

using namespace ppmd;

extern "C" int ppmd_verlet_step(ppmd_ctx *ctx, int phase, double *pos, double *vel, const double *force, int64_t n,
                                const ppmd_box *box, double mass, double dt) {
    if (!ctx || !box || n < 0 || (phase != 1 && phase != 2) || !(mass > 0))
        return set_error(ctx, PPMD_ERR_INVALID, "ppmd_verlet_step: bad argument");
    if (n > 0 && (!vel || !force || (phase == 1 && !pos))) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_verlet_step: null array");
    for (int d = 0; d < 3; ++d)
        if (!(box->L[d] > 0)) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_verlet_step: bad box");
    cudaSetDevice(ctx->device);
    double h = dt / (2.0 * mass);
    if (n > 0) PPMD_LAUNCH(ctx, k_vv_plain, div_up(n, 256), 256, 0, phase, pos, vel, force, n, box->L[0], box->L[1], box->L[2], h, dt);
    return check_launch(ctx, "ppmd_verlet_step");
}

extern "C" int ppmd_kinetic_energy(ppmd_ctx *ctx, const double *vel, int64_t n, double mass, double *ke) {
    if (!ctx || n < 0 || !ke || (n > 0 && !vel)) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_kinetic_energy: bad argument");
    cudaSetDevice(ctx->device);
    int64_t nb = div_up(n, 256);
    double *parts = (double *)scratch(ctx, S_PARTIAL, sizeof(double) * (size_t)(nb + 1));
    if (!parts) return PPMD_ERR_NOMEM;
    if (n > 0) PPMD_LAUNCH(ctx, k_kinetic, nb, 256, 0, vel, n, 0.5 * mass, parts);
    return reduce_partials(ctx, parts, nb, 1, ke);
}
