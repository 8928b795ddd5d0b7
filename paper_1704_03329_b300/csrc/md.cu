// Time stepping: Algorithm 6 with the list-reuse policy of Sec. 3.5 and
// Eq. (3) (the paper's IntegratorRange), for one box or a batch of
// independent boxes.  Particles are kept in device memory sorted by cell;
// every list rebuild re-sorts them (the periodic reordering the paper's
// conclusions call for), and whole rebuild periods are replayed as CUDA
// graphs.
#include <algorithm>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string>

#include "analysis.cuh"
#include "cells.cuh"
#include "lj.cuh"
#include "neighbours.cuh"
#include "md_kernels.cuh"
#include "verlet.cuh"

using namespace ppmd;

struct ppmd_md {
    ppmd_ctx *ctx = nullptr;
    int64_t n = 0, nbox = 0, ncell = 0;
    ppmd_md_params p{};
    LJConst c{};
    double h = 0, half_m = 0, skin_half = 0;
    std::vector<Seg> segs;
    Seg *d_segs = nullptr;
    SegTable st{};
    int64_t *d_atom_off = nullptr;
    // particle state in cell order
    double *pos = nullptr, *vel = nullptr, *f64 = nullptr;
    float4 *f4 = nullptr;
    int4 *xq = nullptr, *xq_ref = nullptr;
    // pos and xq point at buffer `cur` of two: a pair loop with the next
    // drift fused in writes the other one.  Rebuilds and set-up return to
    // buffer 0, so a captured rebuild period starts and ends there.
    double *pos_buf[2] = {nullptr, nullptr};
    int4 *xq_buf[2] = {nullptr, nullptr};
    int cur = 0;
    bool half_kicked = false;  // positions already at step+1 (velocities at step+1/2)
    int32_t *orig = nullptr, *seg_of = nullptr, *cell_of = nullptr, *cell_start = nullptr, *cell_atoms = nullptr;
    int32_t *W = nullptr, *cnt = nullptr;  // column-major neighbour matrix W[m * ld + i]
    int64_t ld = 0;
    // FP32 runs keep the list as brick-stage slots (slots.cu) instead of W;
    // on-the-fly analysis and the FP64 path use W
    bool slots = false;
    uint16_t *W16 = nullptr;
    // optional CUDA events around the pair loops of a captured unit (their
    // durations in the last replay): begin/end of the launch of step k at
    // ev[2 (k - 1)], ev[2 (k - 1) + 1]; ev_fused[k - 1]: that launch also
    // made the next step's kick and drift
    bool time_pair = false;
    bool rec_events = false;  // capturing the graph with the events
    std::vector<cudaEvent_t> ev;
    std::vector<char> ev_fused;
    int32_t ev_steps = 0;
    int32_t *stage_need = nullptr;  // largest neighbourhood met by a slot-list build
    Brick *bricks = nullptr;
    int32_t stage_cap = 0;  // shared-memory stage of a list-build block (atoms)
    int64_t nbricks = 0, bricks_alloc = 0;
    // launch shapes (ppmd_md_set_shape / ppmd_md_tune): the FP32 pair loop's
    // and the expected home atoms of a list-build brick
    ColShape col;
    int32_t brick_home = BRICK_THREADS;
    int32_t shape = 0;
    double *tune_buf = nullptr;  // the state (caller order) while shapes are timed
    // reorder temporaries
    double *pos_t = nullptr, *vel_t = nullptr;
    int4 *xq_t = nullptr;
    int32_t *orig_t = nullptr, *cell_t = nullptr, *seg_t = nullptr;
    // reductions
    double *part_f = nullptr, *part_k = nullptr, *red = nullptr, *ebuf = nullptr;
    unsigned int *max_disp_bits = nullptr;
    // missed-pair check at every rebuild (optional): the reference words of
    // the previous build gathered into the new order, and the running count
    bool check = false, have_ref = false;
    int4 *xq_old = nullptr;
    unsigned long long *missed = nullptr;
    int64_t step = 0, rebuilds = 0;
    bool ready = false;
    // graphs
    cudaStream_t cap_stream = nullptr;
    // exec: the unit's graph; exec_ev: the same with the pair-loop events
    // (replayed only as the last unit of a run, so that the event-record
    // nodes leave the other replays undisturbed)
    cudaGraphExec_t exec = nullptr, exec_ev = nullptr;
    int32_t graph_steps = 0;
    int64_t graph_kernels = 0, graph_kernels_ev = 0;
    // on-the-fly analysis run (Sec. 5.2): Andersen thermostat and Q4/Q5/Q6
    uint64_t thermo_thr = 0, thermo_seed = 0;
    double thermo_sd = 0.0, Lmax = 0.0;
    int32_t boa_every = 0;
    double r_boa = 0.0;
    float *q3 = nullptr;  // [3][n] of the last analysis step, caller order
    double *part_q = nullptr, *red_q = nullptr, *qbuf = nullptr;
    int64_t *d_base = nullptr;  // step number before a replayed unit
    bool have_q = false;
    // short list for the analysis: pairs of W closer than r_boa + skin at
    // the last build (they stay a superset of the bonds until the next one)
    int32_t *W2 = nullptr, *cnt2 = nullptr;
    int32_t max2 = 64;
    int32_t *coll_list = nullptr, *coll_count = nullptr;  // this step's colliding atoms
    std::vector<void *> allocs;
};

namespace {

int64_t force_blocks(const ppmd_md *m) {
    if (m->slots) return m->nbricks;
    return m->p.prec == PPMD_FP32 ? lj_columns_blocks(m->n, m->col) : div_up(m->n, lj_col64_atoms_per_block(m->n));
}

template <class T>
int md_alloc(ppmd_md *m, T **p, size_t count) {
    void *q = nullptr;
    if (cudaMalloc(&q, sizeof(T) * (count > 0 ? count : 1)) != cudaSuccess) {
        cudaGetLastError();
        return set_error(m->ctx, PPMD_ERR_NOMEM, "integrator allocation of %zu bytes failed", sizeof(T) * count);
    }
    m->allocs.push_back(q);
    *p = (T *)q;
    return PPMD_OK;
}

__global__ void k_init_state(int64_t n, double *pos, const int64_t *atom_off, int64_t nbox, SegTable st, int4 *xq,
                             int32_t *orig, int32_t *seg_of, int32_t *status) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // box of atom i: the last b with atom_off[b] <= i
    int64_t lo = 0, hi = nbox - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if (atom_off[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    const int32_t sid = (int32_t)lo;
    const Seg &S = seg_ref(st, sid);
    uint32_t q[3];
    bool bad = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double x = pos[3 * i + d];
        if (!isfinite(x)) {
            bad = true;
            x = 0.0;
        }
        x = wrap_exact(x, S.L[d]);
        pos[3 * i + d] = x;
        q[d] = to_fixed(x, S.fxs[d]);
    }
    if (bad) latch_status(status, PPMD_ERR_NONFINITE);
    xq[i] = make_int4((int)q[0], (int)q[1], (int)q[2], sid);
    orig[i] = (int32_t)i;
    seg_of[i] = sid;
}

__global__ void k_gather_i32(int64_t n, const int32_t *perm, const int32_t *in, int32_t *out) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = in[perm[k]];
}

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64
// products by 0xD2511F53 and 0xCD9E8D57 with the counter words permuted
// and mixed with the key; the key advances by 0x9E3779B9, 0xBB67AE85 before
// every round but the first.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

// Andersen collisions at the end of step (*base + step_off) (base may be
// null): atom i (caller index orig[i]) collides when the first Philox word
// at counter (orig[i], step mod 2^32, step / 2^32, 0), key (seed mod 2^32,
// seed / 2^32) is below thr; its velocity is then drawn from N(0, sd^2)
// per component by Box-Muller on U(u) = (u + 1/2) 2^-32: (v_x, v_y) from
// words 1, 2, v_z from word 3 and word 0 of the draw at counter word 3 = 1.
// The decision (integer work for every atom) and the draw (FP64
// transcendentals, slow on this part) run as two kernels: the colliding
// atoms are first collected in a list so that the draw runs on full warps.
__global__ void k_andersen_decide(int64_t n, const int32_t *__restrict__ orig, uint64_t seed, uint64_t thr,
                                  const int64_t *__restrict__ base, int64_t step_off, int32_t *__restrict__ list,
                                  int32_t *__restrict__ count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool hit = false;
    if (i < n) {
        const int64_t step = (base ? *base : 0) + step_off;
        uint32_t u[4] = {(uint32_t)orig[i], (uint32_t)step, (uint32_t)((uint64_t)step >> 32), 0u};
        philox4x32_10(u, (uint32_t)seed, (uint32_t)(seed >> 32));
        hit = (uint64_t)u[0] < thr;
    }
    const unsigned b = __ballot_sync(0xffffffffu, hit);
    if (!b) return;
    const int lane = threadIdx.x & 31, leader = __ffs(b) - 1;
    int32_t at = 0;
    if (lane == leader) at = atomicAdd(count, __popc(b));
    at = __shfl_sync(0xffffffffu, at, leader);
    if (hit) list[at + __popc(b & ((1u << lane) - 1u))] = (int32_t)i;
}

// The new velocity of a collider (atom orig_id, step): Maxwell-Boltzmann
// components of standard deviation sd by Box-Muller in FP64 from the
// Philox4x32-10 words of the counters (orig_id, step, 0) and (orig_id,
// step, 1).
__device__ __forceinline__ void andersen_draw(int32_t orig_id, int64_t step, uint64_t seed, double sd, double (&v)[3]) {
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    uint32_t u[4] = {(uint32_t)orig_id, (uint32_t)step, (uint32_t)((uint64_t)step >> 32), 0u};
    philox4x32_10(u, k0, k1);
    uint32_t w[4] = {(uint32_t)orig_id, (uint32_t)step, (uint32_t)((uint64_t)step >> 32), 1u};
    philox4x32_10(w, k0, k1);
    const double two_pi = 6.283185307179586, inv32 = 2.3283064365386962890625e-10;
    const double U1 = __dmul_rn(__dadd_rn((double)u[1], 0.5), inv32);
    const double U2 = __dmul_rn(__dadd_rn((double)u[2], 0.5), inv32);
    const double U3 = __dmul_rn(__dadd_rn((double)u[3], 0.5), inv32);
    const double U4 = __dmul_rn(__dadd_rn((double)w[0], 0.5), inv32);
    const double r1 = sqrt(__dmul_rn(-2.0, log(U1))), t1 = __dmul_rn(two_pi, U2);
    const double r2 = sqrt(__dmul_rn(-2.0, log(U3))), t2 = __dmul_rn(two_pi, U4);
    v[0] = __dmul_rn(sd, __dmul_rn(r1, cos(t1)));
    v[1] = __dmul_rn(sd, __dmul_rn(r1, sin(t1)));
    v[2] = __dmul_rn(sd, __dmul_rn(r2, cos(t2)));
}

__global__ void k_andersen(const int32_t *__restrict__ list, const int32_t *__restrict__ count,
                           double *__restrict__ vel, const int32_t *__restrict__ orig, uint64_t seed, double sd,
                           const int64_t *__restrict__ base, int64_t step_off) {
    const int32_t m = *count;
    for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += gridDim.x * blockDim.x) {
        const int64_t i = list[t];
        double v[3];
        andersen_draw(orig[i], (base ? *base : 0) + step_off, seed, sd, v);
        vel[3 * i] = v[0];
        vel[3 * i + 1] = v[1];
        vel[3 * i + 2] = v[2];
    }
}

// The collisions of a step whose pair loop already made the next step's
// kick and drift: each collider gets its new velocity (the draw of
// k_andersen), and its next kick, drift, fixed-point word and displacement
// are made again from it in the same arithmetic as the pair loop's
// epilogue, so the state equals that of the separate kick and drift.
// pos: the step's positions; pos_next, xq_next: those the pair loop wrote.
__global__ void k_andersen_fused(const int32_t *__restrict__ list, const int32_t *__restrict__ count,
                                 double *__restrict__ vel, const int32_t *__restrict__ orig, uint64_t seed, double sd,
                                 const int64_t *__restrict__ base, int64_t step_off, const float4 *__restrict__ f4,
                                 const double *__restrict__ pos, double *__restrict__ pos_next,
                                 int4 *__restrict__ xq_next, const int4 *__restrict__ xq_ref, SegTable st, double h,
                                 double dt, unsigned int *max_disp_bits) {
    const int32_t m = *count;
    for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += gridDim.x * blockDim.x) {
        const int64_t i = list[t];
        double vn[3];
        andersen_draw(orig[i], (base ? *base : 0) + step_off, seed, sd, vn);
        const float4 fq = f4[i];
        const double f[3] = {(double)fq.x, (double)fq.y, (double)fq.z};
        const int4 ref = xq_ref[i];
        const Seg &S = seg_ref(st, ref.w);
        uint32_t q[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double v = fma(h, f[d], vn[d]);
            const double r = fma(dt, v, pos[3 * i + d]);
            vel[3 * i + d] = v;
            pos_next[3 * i + d] = r;
            q[d] = (uint32_t)(unsigned long long)__double2ll_rn(r * S.fxs[d]);
        }
        xq_next[i] = make_int4((int)q[0], (int)q[1], (int)q[2], ref.w);
        const float ex = fixed_delta(q[0], (uint32_t)ref.x, S.sx[0]);
        const float ey = fixed_delta(q[1], (uint32_t)ref.y, S.sx[1]);
        const float ez = fixed_delta(q[2], (uint32_t)ref.z, S.sx[2]);
        const float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
        if (d2 > 0.0f) atomicMax(max_disp_bits, __float_as_uint(d2));
    }
}

// Entries of the list W (column-major) closer than r_short (FP32 test
// with a small margin: extra entries are harmless, the analysis decides
// exactly) into W2 (column-major, capacity max2; more: PPMD_ERR_CAPACITY).
__global__ void k_short_list(int64_t n, const int4 *__restrict__ xq, SegTable st, const int32_t *__restrict__ W,
                             const int32_t *__restrict__ cnt, int32_t max_nbr, int64_t ld, float r2_short,
                             int32_t *__restrict__ W2, int32_t *__restrict__ cnt2, int32_t max2, int32_t *status,
                             unsigned long long *needed) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int4 xi = xq[i];
    const Seg &S = seg_ref(st, xi.w);
    const int32_t deg = min(cnt[i], max_nbr);
    int32_t c = 0;
    for (int32_t k0 = 0; k0 < deg; k0 += 4) {  // four loads in flight per thread
        int32_t jv[4];
        int4 xv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) jv[q] = k0 + q < deg ? __ldg(W + (((int64_t)(k0 >> 2) * ld + i) << 2) + q) : (int32_t)i;
#pragma unroll
        for (int q = 0; q < 4; ++q) xv[q] = __ldg(&xq[jv[q]]);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (k0 + q >= deg) break;
            const float dx = fixed_delta((uint32_t)xi.x, (uint32_t)xv[q].x, S.sx[0]);
            const float dy = fixed_delta((uint32_t)xi.y, (uint32_t)xv[q].y, S.sx[1]);
            const float dz = fixed_delta((uint32_t)xi.z, (uint32_t)xv[q].z, S.sx[2]);
            if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < r2_short) {
                if (c < max2) W2[(int64_t)c * ld + i] = jv[q];
                ++c;
            }
        }
    }
    cnt2[i] = c;
    if (c > max2) {
        latch_status(status, PPMD_ERR_CAPACITY);
        latch_needed(needed, (unsigned long long)c);
    }
}

int build_short_list(ppmd_md *m) {
    if (m->boa_every <= 0 || m->n <= 0) return PPMD_OK;
    const double rs = (m->r_boa + (m->p.r_list - m->p.lj.rc)) * (1.0 + 1e-5);
    PPMD_LAUNCH(m->ctx, k_short_list, div_up(m->n, 256), 256, 0, m->n, m->xq, m->st, m->W, m->cnt, m->p.max_nbr,
                m->ld, (float)(rs * rs), m->W2, m->cnt2, m->max2, m->ctx->d_status, m->ctx->d_needed);
    return check_launch(m->ctx, "short list");
}

__global__ void k_q_row(const double *red, double n, double *row) {
    if (threadIdx.x < 3) row[threadIdx.x] = __ddiv_rn(red[threadIdx.x], n);
}

__global__ void k_set_i64(int64_t *p, int64_t v) { *p = v; }

__global__ void k_energy_row(const double *red, double *row) {
    // red = (potential U, virial W, kinetic K)
    row[0] = red[2];
    row[1] = red[0];
}

void use_buffer(ppmd_md *m, int b) {
    m->cur = b;
    m->pos = m->pos_buf[b];
    m->xq = m->xq_buf[b];
}

// Pairs of the new list (built from the current positions) that are now
// closer than r_c although they were at least r_list apart at the previous
// build, i.e. missing from the list the pair loop used since then.  xq: the
// current words, xq_old: the previous build's words in the same (new)
// order.  FP32 tests on the fixed-point differences, FP64 inside the bands
// of both cutoffs (exact up to the fixed-point quantum, L 2^-32).
__global__ void k_missed_pairs(int64_t n, int64_t ld, const int4 *__restrict__ xq, const int4 *__restrict__ xq_old,
                               const double *__restrict__ pos64, SegTable st, const int32_t *__restrict__ W,
                               const int32_t *__restrict__ cnt, int32_t max_nbr, double rc2, float rc2_lo, float rc2_hi,
                               unsigned long long *missed) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long c = 0;
    if (i < n) {
        const int4 a = xq[i], ao = xq_old[i];
        const Seg &S = seg_ref(st, a.w);
        const int32_t m = min(cnt[i], max_nbr);
        for (int32_t k = 0; k < m; ++k) {
            const int32_t j = W[(((int64_t)(k >> 2) * ld + i) << 2) + (k & 3)];
            const int4 b = xq[j];
            const float dx = fixed_delta((uint32_t)a.x, (uint32_t)b.x, S.sx[0]);
            const float dy = fixed_delta((uint32_t)a.y, (uint32_t)b.y, S.sx[1]);
            const float dz = fixed_delta((uint32_t)a.z, (uint32_t)b.z, S.sx[2]);
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            bool inside = r2 < rc2_lo;
            if (!inside && r2 < rc2_hi) {
                double dr[3];
                inside = min_image_r2(pos64 + 3 * i, pos64 + 3 * (int64_t)j, S, dr) < rc2;
            }
            if (!inside) continue;
            const int4 bo = xq_old[j];
            const int32_t q[3] = {(int32_t)((uint32_t)ao.x - (uint32_t)bo.x), (int32_t)((uint32_t)ao.y - (uint32_t)bo.y),
                                  (int32_t)((uint32_t)ao.z - (uint32_t)bo.z)};
            const float fo = fmaf((float)q[0] * S.sx[0], (float)q[0] * S.sx[0],
                                  fmaf((float)q[1] * S.sx[1], (float)q[1] * S.sx[1], (float)q[2] * S.sx[2] * (float)q[2] * S.sx[2]));
            bool was_listed = fo < S.rl2_lo;
            if (!was_listed && fo < S.rl2_hi) {
                double r2o = 0.0;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const double x = (double)q[d] * (S.L[d] * 2.3283064365386962890625e-10);
                    r2o += x * x;
                }
                was_listed = r2o < S.rl2;
            }
            if (!was_listed) ++c;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(missed, c);
}

__global__ void k_gather_xq(int64_t n, const int32_t *__restrict__ perm, const int4 *__restrict__ in, int4 *__restrict__ out) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = in[perm[k]];
}

int rebuild(ppmd_md *m) {
    ppmd_ctx *ctx = m->ctx;
    cudaStream_t s = ctx->stream;
    const int64_t n = m->n;
    // the fixed-point words are current here (set-up, the kick and drift,
    // or a pair loop with the drift fused in made them)
    PPMD_TRY(bin_atoms_md(ctx, m->xq, m->pos, n, m->st, m->seg_of, m->ncell, m->cell_of, m->cell_start, m->cell_atoms));
    const bool check = m->check && m->have_ref && n > 0;
    // the previous build's words in the new order, before they are replaced
    if (check) PPMD_LAUNCH(ctx, k_gather_xq, div_up(n, 256), 256, 0, n, m->cell_atoms, m->xq_ref, m->xq_old);
    // The sorted state goes to buffer 0.  With the positions in buffer 1
    // (the fused steps of a rebuild period of even length flip the buffers an
    // odd number of times; a captured period finds the same buffer at every
    // replay) the gather writes buffer 0 directly, otherwise through the
    // temporaries.
    const bool direct = m->cur == 1;
    PPMD_TRY(md_gather(ctx, n, m->cell_atoms, m->st, m->pos, m->vel, m->orig, m->seg_of, m->xq,
                       direct ? m->pos_buf[0] : m->pos_t, m->vel_t, direct ? m->xq_buf[0] : m->xq_t, m->xq_ref,
                       m->orig_t, m->seg_t));
    use_buffer(m, 0);
    if (n > 0) {
        if (!direct) {
            PPMD_TRY(cuda_check(
                ctx, cudaMemcpyAsync(m->pos, m->pos_t, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s), "copy"));
            PPMD_TRY(
                cuda_check(ctx, cudaMemcpyAsync(m->xq, m->xq_t, sizeof(int4) * n, cudaMemcpyDeviceToDevice, s), "copy"));
        }
        PPMD_TRY(
            cuda_check(ctx, cudaMemcpyAsync(m->vel, m->vel_t, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s), "copy"));
        PPMD_TRY(
            cuda_check(ctx, cudaMemcpyAsync(m->orig, m->orig_t, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s), "copy"));
        PPMD_TRY(cuda_check(ctx, cudaMemcpyAsync(m->seg_of, m->seg_t, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s),
                            "copy"));
    }
    m->have_ref = true;
    if (m->slots) {
        PPMD_TRY(build_slot_list(ctx, m->nbricks, m->bricks, m->xq, m->pos, m->st, m->cell_start, m->W16, m->ld, m->cnt,
                                 m->p.max_nbr, m->stage_cap, m->stage_need, m->n));
        if (check)
            PPMD_TRY(slots_to_atoms(ctx, m->nbricks, m->bricks, m->st, m->cell_start, m->W16, m->ld, m->cnt,
                                    m->p.max_nbr, m->stage_cap, m->W, m->n));
    } else {
        PPMD_TRY(build_list_bricks(ctx, m->nbricks, m->bricks, BrickShape{1, 1, 1}, m->xq, m->pos, m->st, m->cell_start,
                                   m->W, m->ld, m->cnt, m->p.max_nbr, m->stage_cap, true));
    }
    if (check)
        PPMD_LAUNCH(ctx, k_missed_pairs, div_up(n, 256), 256, 0, n, m->ld, m->xq, m->xq_old, m->pos, m->st, m->W, m->cnt,
                    m->p.max_nbr, m->c.rc2, m->c.rc2_lo, m->c.rc2_hi, m->missed);
    return m->slots ? check_launch(ctx, "rebuild") : build_short_list(m);
}

// Pair loop; with kick = true also the second kick of the step, with
// drift = true (FP32) also the next step's kick and drift; on energy steps
// the per-block (U, W, K) sums.
int forces(ppmd_md *m, bool energy, bool kick, bool drift = false) {
    const bool f32 = m->p.prec == PPMD_FP32;
    Drift d;
    if (drift) {
        d.pos_next = m->pos_buf[m->cur ^ 1];
        d.xq_next = m->xq_buf[m->cur ^ 1];
        d.xq_ref = m->xq_ref;
        d.dt = m->p.dt;
        d.max_disp_bits = m->max_disp_bits;
    }
    if (m->slots)
        PPMD_TRY(lj_slots(m->ctx, m->nbricks, m->bricks, m->xq, m->pos, m->st, m->cell_start, m->c, m->W16, m->ld, m->cnt,
                          m->p.max_nbr, m->stage_cap, m->f4, kick ? m->vel : nullptr, m->h, m->half_m,
                          energy ? m->part_f : nullptr, d, m->n));
    else
        PPMD_TRY(lj_columns(m->ctx, m->n, m->ld, m->xq, m->pos, m->st, m->c, m->W, m->cnt, m->p.max_nbr, m->p.prec,
                            f32 ? m->f4 : nullptr, f32 ? nullptr : m->f64, kick ? m->vel : nullptr, m->h, m->half_m,
                            energy ? m->part_f : nullptr, d, f32 ? m->col : ColShape()));
    if (drift) {
        use_buffer(m, m->cur ^ 1);
        m->half_kicked = true;
    }
    return PPMD_OK;
}

// One step of Algorithm 6.  erow: device row receiving (KE, PE) on energy
// steps; qrow: (mean Q4, Q5, Q6) on analysis steps.  The step's kick and
// drift are skipped when the previous pair loop already made them; with
// fuse_next (FP32) this step's pair loop makes the next step's (thermostat
// collisions then make them again for the colliders, the analysis reads the
// step's positions from the other buffer).  base: device step number to add
// to s (graph capture), else null.
int one_step(ppmd_md *m, int64_t s, double *erow, bool fuse_next, double *qrow = nullptr,
             const int64_t *base = nullptr) {
    ppmd_ctx *ctx = m->ctx;
    const bool f32 = m->p.prec == PPMD_FP32;
    const bool energy = m->p.energy_every > 0 && (s % m->p.energy_every) == 0 && erow;
    const bool thermo = m->thermo_thr > 0;
    const bool analyse = m->boa_every > 0 && (s % m->boa_every) == 0;
    if (!m->half_kicked)
        PPMD_TRY(md_kick_drift2(ctx, m->n, m->pos, m->vel, f32 ? m->f4 : nullptr, f32 ? nullptr : m->f64, m->xq,
                                m->xq_ref, m->st, m->h, m->p.dt, m->max_disp_bits));
    m->half_kicked = false;
    if (m->p.rebuild_every > 0 && s % m->p.rebuild_every == 0) {
        PPMD_TRY(rebuild(m));
    }
    // with the next step's kick and drift fused in, the step's positions
    // stay in the other buffer (prev) for the thermostat and the analysis
    const bool fused = fuse_next && f32;
    const bool timed = m->rec_events && base && s >= 1 && 2 * s <= (int64_t)m->ev.size();
    // during stream capture, only an external record becomes an event-record node
    if (timed)
        PPMD_TRY(cuda_check(ctx, cudaEventRecordWithFlags(m->ev[2 * (s - 1)], ctx->stream, cudaEventRecordExternal),
                            "event"));
    PPMD_TRY(forces(m, energy, true, fused));
    if (timed) {
        PPMD_TRY(cuda_check(ctx, cudaEventRecordWithFlags(m->ev[2 * (s - 1) + 1], ctx->stream, cudaEventRecordExternal),
                            "event"));
        m->ev_fused[s - 1] = fused ? 1 : 0;
    }
    const int prev = fused ? m->cur ^ 1 : m->cur;
    if (energy) {
        PPMD_TRY(reduce_partials(ctx, m->part_f, force_blocks(m), 3, m->red));
        PPMD_LAUNCH(ctx, k_energy_row, 1, 1, 0, m->red, erow);
    }
    if (thermo && m->n > 0) {
        PPMD_TRY(cuda_check(ctx, cudaMemsetAsync(m->coll_count, 0, sizeof(int32_t), ctx->stream), "memset"));
        PPMD_LAUNCH(ctx, k_andersen_decide, div_up(m->n, 256), 256, 0, m->n, m->orig, m->thermo_seed, m->thermo_thr,
                    base, s, m->coll_list, m->coll_count);
        if (fused)
            PPMD_LAUNCH(ctx, k_andersen_fused, std::min<int64_t>(div_up(m->n, 128), 148 * 4), 128, 0, m->coll_list,
                        m->coll_count, m->vel, m->orig, m->thermo_seed, m->thermo_sd, base, s, m->f4,
                        m->pos_buf[prev], m->pos, m->xq, m->xq_ref, m->st, m->h, m->p.dt, m->max_disp_bits);
        else
            PPMD_LAUNCH(ctx, k_andersen, std::min<int64_t>(div_up(m->n, 128), 148 * 4), 128, 0, m->coll_list,
                        m->coll_count, m->vel, m->orig, m->thermo_seed, m->thermo_sd, base, s);
    }
    if (analyse) {
        PPMD_TRY(boa_otf_launch(ctx, m->n, m->xq_buf[prev], m->pos_buf[prev], m->st, m->W2, m->cnt2, m->max2, m->ld,
                                m->r_boa, m->Lmax, m->orig, m->q3, m->part_q));
        PPMD_TRY(reduce_partials(ctx, m->part_q, boa_otf_blocks(m->n), 3, m->red_q));
        if (qrow) PPMD_LAUNCH(ctx, k_q_row, 1, 32, 0, m->red_q, (double)(m->n > 0 ? m->n : 1), qrow);
        m->have_q = true;
    }
    return check_launch(ctx, "one_step");
}

}  // namespace

extern "C" int ppmd_md_create(ppmd_ctx *ctx, ppmd_md **out, int64_t nbox, const int64_t *atom_off, const ppmd_box *boxes,
                              const double *box_r_list, const ppmd_md_params *params) {
    if (!ctx || !out || nbox < 1 || !atom_off || !boxes || !params) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_md_create: bad argument");
    *out = nullptr;
    const ppmd_md_params &p = *params;
    if (!(p.r_list >= p.lj.rc) || !(p.lj.rc > 0) || !(p.mass > 0) || !(p.dt > 0) || p.max_nbr < 1 || p.rebuild_every < 1 ||
        (p.prec != PPMD_FP32 && p.prec != PPMD_FP64) || p.energy_every < 0)
        return set_error(ctx, PPMD_ERR_INVALID, "ppmd_md_create: bad parameters");
    if (atom_off[0] != 0) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_md_create: atom_off[0] must be 0");
    for (int64_t b = 0; b < nbox; ++b)
        if (atom_off[b + 1] < atom_off[b]) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_md_create: atom_off not increasing");
    if (atom_off[nbox] >= ((int64_t)1 << 31)) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_md_create: too many atoms");
    cudaSetDevice(ctx->device);
    ppmd_md *m = new ppmd_md();
    m->ctx = ctx;
    m->n = atom_off[nbox];
    m->nbox = nbox;
    m->p = p;
    // the atom-index list is stored in groups of four; FP32 rows are rounded
    // to eight so that the brick-staged mechanism can use the same capacity
    m->p.max_nbr = p.prec == PPMD_FP32 ? (p.max_nbr + 7) & ~7 : (p.max_nbr + 3) & ~3;
    m->h = p.dt / (2.0 * p.mass);
    m->half_m = 0.5 * p.mass;
    m->segs.resize(nbox);
    double Lmax = 0;
    int64_t cell0 = 0;
    double min_skin = 1e300;
    for (int64_t b = 0; b < nbox; ++b) {
        double rl = p.r_list;
        if (box_r_list && box_r_list[b] < rl) rl = box_r_list[b];
        if (!(rl >= p.lj.rc)) {
            ppmd_md_destroy(m);
            return set_error(ctx, PPMD_ERR_INVALID, "box %lld: list cutoff %g below rc", (long long)b, rl);
        }
        int rc = make_seg(ctx, m->segs[b], boxes[b].L, rl, rl);
        if (rc != PPMD_OK) {
            ppmd_md_destroy(m);
            return rc;
        }
        Seg &S = m->segs[b];
        S.cell0 = (int32_t)cell0;
        S.atom0 = atom_off[b];
        S.atom1 = atom_off[b + 1];
        cell0 += (int64_t)S.nc[0] * S.nc[1] * S.nc[2];
        for (int d = 0; d < 3; ++d) Lmax = fmax(Lmax, boxes[b].L[d]);
        min_skin = fmin(min_skin, rl - p.lj.rc);
        if (cell0 >= ((int64_t)1 << 31)) {
            ppmd_md_destroy(m);
            return set_error(ctx, PPMD_ERR_BOX, "too many cells");
        }
    }
    m->ncell = cell0;
    m->skin_half = 0.5 * min_skin;
    m->Lmax = Lmax;
    m->c = make_ljconst(p.lj, Lmax);
    const int64_t n = m->n;
    int rc = PPMD_OK;
    if (nbox > 1) {
        rc = md_alloc(m, &m->d_segs, nbox);
        if (rc == PPMD_OK) rc = cuda_check(ctx, cudaMemcpy(m->d_segs, m->segs.data(), sizeof(Seg) * nbox, cudaMemcpyHostToDevice), "copy");
        m->st.d = m->d_segs;
        m->st.nseg = (int32_t)nbox;
    } else {
        m->st.d = nullptr;
        m->st.one = m->segs[0];
        m->st.nseg = 1;
    }
    if (rc == PPMD_OK) rc = md_alloc(m, &m->d_atom_off, nbox + 1);
    if (rc == PPMD_OK)
        rc = cuda_check(ctx, cudaMemcpy(m->d_atom_off, atom_off, sizeof(int64_t) * (nbox + 1), cudaMemcpyHostToDevice), "copy");
    if (rc == PPMD_OK) rc = md_alloc(m, &m->pos_buf[0], 3 * n);
    if (rc == PPMD_OK && p.prec == PPMD_FP32) rc = md_alloc(m, &m->pos_buf[1], 3 * n);
    if (rc == PPMD_OK) rc = md_alloc(m, &m->vel, 3 * n);
    if (rc == PPMD_OK) rc = md_alloc(m, &m->pos_t, 3 * n);
    if (rc == PPMD_OK) rc = md_alloc(m, &m->vel_t, 3 * n);
    if (rc == PPMD_OK) {
        if (p.prec == PPMD_FP32) rc = md_alloc(m, &m->f4, n);
        else rc = md_alloc(m, &m->f64, 3 * n);
    }
    if (rc == PPMD_OK) rc = md_alloc(m, &m->xq_buf[0], n);
    if (rc == PPMD_OK && p.prec == PPMD_FP32) rc = md_alloc(m, &m->xq_buf[1], n);
    use_buffer(m, 0);
    if (rc == PPMD_OK) rc = md_alloc(m, &m->xq_ref, n);
    if (rc == PPMD_OK) rc = md_alloc(m, &m->xq_t, n);
    if (rc == PPMD_OK) rc = md_alloc(m, &m->orig, n);
    if (rc == PPMD_OK) rc = md_alloc(m, &m->orig_t, n);
    if (rc == PPMD_OK) rc = md_alloc(m, &m->seg_of, n);
    if (rc == PPMD_OK) rc = md_alloc(m, &m->seg_t, n);
    if (rc == PPMD_OK) rc = md_alloc(m, &m->cell_of, n);
    if (rc == PPMD_OK) rc = md_alloc(m, &m->cell_t, n);
    if (rc == PPMD_OK) rc = md_alloc(m, &m->cell_atoms, n);
    if (rc == PPMD_OK) rc = md_alloc(m, &m->cell_start, m->ncell + 1);
    m->ld = (n + 31) / 32 * 32;
    if (rc == PPMD_OK) rc = md_alloc(m, &m->W, (size_t)m->ld * m->p.max_nbr);
    if (rc == PPMD_OK) rc = md_alloc(m, &m->stage_need, 1);
    if (rc == PPMD_OK) rc = cuda_check(ctx, cudaMemset(m->stage_need, 0, sizeof(int32_t)), "memset");
    if (rc == PPMD_OK) {
        std::vector<Brick> bl;
        m->stage_cap = make_bricks(m->segs, bl);
        m->nbricks = m->bricks_alloc = (int64_t)bl.size();
        rc = md_alloc(m, &m->bricks, bl.size());
        if (rc == PPMD_OK && !bl.empty())
            rc = cuda_check(ctx, cudaMemcpy(m->bricks, bl.data(), sizeof(Brick) * bl.size(), cudaMemcpyHostToDevice), "copy");
    }
    if (rc == PPMD_OK) rc = neigh_brick_setup(ctx, m->p.max_nbr);
    if (rc == PPMD_OK) rc = md_alloc(m, &m->cnt, n);
    // partial rows: the most blocks of any pair-loop shape or brick table
    if (rc == PPMD_OK)
        rc = md_alloc(m, &m->part_f, 3 * std::max<int64_t>(div_up(n, 8), m->nbricks) + 3);
    if (rc == PPMD_OK) rc = md_alloc(m, &m->part_k, kick_blocks(n) + 1);
    if (rc == PPMD_OK) rc = md_alloc(m, &m->red, 4);
    if (rc == PPMD_OK) rc = md_alloc(m, &m->ebuf, 2 * 1024);
    if (rc == PPMD_OK) rc = md_alloc(m, &m->q3, 3 * n);
    if (rc == PPMD_OK) rc = md_alloc(m, &m->part_q, 3 * boa_otf_blocks(n) + 3);
    if (rc == PPMD_OK) rc = md_alloc(m, &m->red_q, 3);
    if (rc == PPMD_OK) rc = md_alloc(m, &m->qbuf, 3 * 1024);
    if (rc == PPMD_OK) rc = md_alloc(m, &m->d_base, 1);
    if (rc == PPMD_OK) rc = md_alloc(m, &m->W2, (size_t)m->ld * (size_t)m->max2);
    if (rc == PPMD_OK) rc = md_alloc(m, &m->cnt2, n);
    if (rc == PPMD_OK) rc = md_alloc(m, &m->coll_list, n);
    if (rc == PPMD_OK) rc = md_alloc(m, &m->coll_count, 1);
    if (rc == PPMD_OK) rc = md_alloc(m, &m->max_disp_bits, 1);
    if (rc == PPMD_OK) rc = cuda_check(ctx, cudaMemset(m->max_disp_bits, 0, sizeof(unsigned int)), "memset");
    if (rc != PPMD_OK) {
        ppmd_md_destroy(m);
        return rc;
    }
    *out = m;
    return PPMD_OK;
}

extern "C" int ppmd_md_destroy(ppmd_md *m) {
    if (!m) return PPMD_OK;
    if (m->ctx) {
        cudaSetDevice(m->ctx->device);
        cudaStreamSynchronize(m->ctx->stream);
    }
    if (m->exec) cudaGraphExecDestroy(m->exec);
    if (m->exec_ev) cudaGraphExecDestroy(m->exec_ev);
    if (m->cap_stream) cudaStreamDestroy(m->cap_stream);
    for (cudaEvent_t e : m->ev) cudaEventDestroy(e);
    for (void *q : m->allocs) cudaFree(q);
    delete m;
    return PPMD_OK;
}

namespace {
void drop_graph(ppmd_md *m);

// After the set-up list build: if a brick's neighbourhood did not fit the
// shared-memory stage, grow the stage (up to what a block may use) and build
// again.  This reads one device word (a synchronisation, at set-up only).
int fit_stage(ppmd_md *m) {
    ppmd_ctx *ctx = m->ctx;
    int32_t need = 0, st = 0;
    PPMD_TRY(cuda_check(ctx, cudaMemcpyAsync(&need, m->stage_need, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream),
                        "copy"));
    PPMD_TRY(cuda_check(ctx, cudaMemcpyAsync(&st, ctx->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream),
                        "copy"));
    PPMD_TRY(cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "sync"));
    if (need <= m->stage_cap) return PPMD_OK;
    const int32_t cap = (int32_t)(((int64_t)need * 5 / 4 + 63) / 64 * 64);
    if (slot_list_smem(cap, m->p.max_nbr) > 200 * 1024 || cap >= 65535)
        return set_error(ctx, PPMD_ERR_CAPACITY, "a brick neighbourhood of %d atoms exceeds the shared-memory stage", need);
    if (st == PPMD_ERR_CAPACITY) {
        // the overflow latched by the first build; the build below latches
        // again if a row still overflows the list capacity
        int32_t zero = 0;
        PPMD_TRY(cuda_check(ctx, cudaMemcpyAsync(ctx->d_status, &zero, sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream),
                            "copy"));
    }
    drop_graph(m);
    m->stage_cap = cap;
    PPMD_TRY(slots_setup(ctx, m->stage_cap, m->p.max_nbr));
    use_buffer(m, 0);
    return build_slot_list(ctx, m->nbricks, m->bricks, m->xq, m->pos, m->st, m->cell_start, m->W16, m->ld, m->cnt,
                           m->p.max_nbr, m->stage_cap, m->stage_need, m->n);
}
}  // namespace

extern "C" int ppmd_md_set_state(ppmd_md *m, const double *pos, const double *vel) {
    if (!m || (m->n > 0 && (!pos || !vel))) return PPMD_ERR_INVALID;
    ppmd_ctx *ctx = m->ctx;
    cudaSetDevice(ctx->device);
    const int64_t n = m->n;
    cudaStream_t s = ctx->stream;
    use_buffer(m, 0);
    m->half_kicked = false;
    if (n > 0) {
        PPMD_TRY(cuda_check(ctx, cudaMemcpyAsync(m->pos, pos, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s), "copy"));
        PPMD_TRY(cuda_check(ctx, cudaMemcpyAsync(m->vel, vel, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s), "copy"));
    }
    if (n > 0)
        PPMD_LAUNCH(ctx, k_init_state, div_up(n, 256), 256, 0, n, m->pos, m->d_atom_off, m->nbox, m->st, m->xq, m->orig,
                    m->seg_of, ctx->d_status);
    m->have_ref = false;  // the first build of a state has no previous list
    if (m->missed) PPMD_TRY(cuda_check(ctx, cudaMemsetAsync(m->missed, 0, sizeof(unsigned long long), s), "memset"));
    PPMD_TRY(rebuild(m));
    if (m->slots) PPMD_TRY(fit_stage(m));
    PPMD_TRY(forces(m, false, false));
    m->step = 0;
    m->rebuilds = 1;
    m->ready = true;
    return check_launch(ctx, "ppmd_md_set_state");
}

extern "C" int ppmd_md_run(ppmd_md *m, int32_t nsteps, double *energies, int use_graph) {
    return ppmd_md_run_analysed(m, nsteps, energies, nullptr, use_graph);
}

extern "C" int ppmd_md_run_analysed(ppmd_md *m, int32_t nsteps, double *energies, double *qrows, int use_graph) {
    if (!m || nsteps < 0) return PPMD_ERR_INVALID;
    ppmd_ctx *ctx = m->ctx;
    if (!m->ready) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_md_run: state not set");
    cudaSetDevice(ctx->device);
    const int32_t P = m->p.rebuild_every;
    const int32_t E = m->p.energy_every;
    const int32_t B = m->boa_every;
    int32_t unit = P * std::max(1, 10 / P);
    const bool graph_ok = use_graph && unit <= 1024 && (E == 0 || unit % E == 0) && (B == 0 || unit % B == 0);
    int32_t done = 0;
    while (done < nsteps) {
        const int64_t s0 = m->step;
        if (graph_ok && s0 % unit == 0 && nsteps - done >= unit) {
            // with pair-loop timing on, the run's last whole unit replays the
            // graph that records the events
            const bool with_ev = m->time_pair && nsteps - done < 2 * unit;
            cudaGraphExec_t &exec = with_ev ? m->exec_ev : m->exec;
            int64_t &graph_kernels = with_ev ? m->graph_kernels_ev : m->graph_kernels;
            if (!exec) {
                // capture one unit of whole rebuild periods on a private stream
                if (!m->cap_stream)
                    PPMD_TRY(cuda_check(ctx, cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking), "stream"));
                PPMD_TRY(cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "sync"));
                cudaStream_t user = ctx->stream;
                ctx->stream = m->cap_stream;
                int64_t k0 = ctx->launches;
                cudaGraph_t g = nullptr;
                int rc = cuda_check(ctx, cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal), "capture");
                // a unit starts and ends with full-step velocities; inside it
                // each pair loop makes the next step's kick and drift
                m->rec_events = with_ev;
                for (int32_t k = 1; rc == PPMD_OK && k <= unit; ++k)
                    rc = one_step(m, k, m->ebuf + 2 * (k - 1), k < unit, m->qbuf + 3 * (k - 1), m->d_base);
                m->rec_events = false;
                cudaError_t e = cudaStreamEndCapture(m->cap_stream, &g);
                ctx->stream = user;
                if (rc != PPMD_OK) {
                    if (g) cudaGraphDestroy(g);
                    return rc;
                }
                PPMD_TRY(cuda_check(ctx, e, "end capture"));
                e = cudaGraphInstantiate(&exec, g, 0);
                cudaGraphDestroy(g);
                PPMD_TRY(cuda_check(ctx, e, "graph instantiate"));
                m->graph_steps = unit;
                graph_kernels = ctx->launches - k0;
                ctx->launches = k0;
            }
            PPMD_LAUNCH(ctx, k_set_i64, 1, 1, 0, m->d_base, s0);  // step numbers of the replayed unit
            PPMD_TRY(cuda_check(ctx, cudaGraphLaunch(exec, ctx->stream), "graph launch"));
            ctx->launches += graph_kernels;
            if (qrows && B > 0) {
                for (int32_t k = 1; k <= unit; ++k)
                    if ((k % B) == 0)
                        PPMD_TRY(cuda_check(ctx, cudaMemcpyAsync(qrows + 3 * (done + k - 1), m->qbuf + 3 * (k - 1),
                                                                 3 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream),
                                            "copy"));
            }
            if (energies && E > 0) {
                for (int32_t k = 1; k <= unit; ++k)
                    if ((k % E) == 0)
                        PPMD_TRY(cuda_check(ctx, cudaMemcpyAsync(energies + 2 * (done + k - 1), m->ebuf + 2 * (k - 1),
                                                                 2 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream),
                                            "copy"));
            }
            m->rebuilds += unit / P;
            m->step += unit;
            done += unit;
        } else {
            const int64_t s = s0 + 1;
            // fuse the next step's kick and drift unless this is the run's
            // last step or the next one is a graph replay
            const bool next_graph = graph_ok && s % unit == 0 && nsteps - (done + 1) >= unit;
            PPMD_TRY(one_step(m, s, energies ? energies + 2 * done : nullptr, done + 1 < nsteps && !next_graph,
                              qrows ? qrows + 3 * done : nullptr, nullptr));
            if (s % P == 0) m->rebuilds += 1;
            m->step = s;
            done += 1;
        }
    }
    return check_launch(ctx, "ppmd_md_run");
}

extern "C" int ppmd_md_get_state(ppmd_md *m, double *pos, double *vel, double *force) {
    if (!m) return PPMD_ERR_INVALID;
    ppmd_ctx *ctx = m->ctx;
    cudaSetDevice(ctx->device);
    if (pos) PPMD_TRY(scatter_vec3(ctx, m->n, m->orig, m->pos, pos));
    if (vel) PPMD_TRY(scatter_vec3(ctx, m->n, m->orig, m->vel, vel));
    if (force) {
        if (m->p.prec == PPMD_FP32) PPMD_TRY(scatter_f4(ctx, m->n, m->orig, m->f4, force));
        else PPMD_TRY(scatter_vec3(ctx, m->n, m->orig, m->f64, force));
    }
    return PPMD_OK;
}

extern "C" int ppmd_md_info(ppmd_md *m, int64_t *steps, int64_t *rebuilds, double *max_disp) {
    if (!m) return PPMD_ERR_INVALID;
    ppmd_ctx *ctx = m->ctx;
    cudaSetDevice(ctx->device);
    unsigned int bits = 0;
    PPMD_TRY(cuda_check(ctx, cudaMemcpyAsync(&bits, m->max_disp_bits, 4, cudaMemcpyDeviceToHost, ctx->stream), "copy"));
    int rc = ppmd_sync(ctx);
    float d2;
    memcpy(&d2, &bits, 4);
    double md = sqrt((double)d2);
    if (steps) *steps = m->step;
    if (rebuilds) *rebuilds = m->rebuilds;
    if (max_disp) *max_disp = md;
    if (rc == PPMD_OK && md > m->skin_half) rc = PPMD_WARN_SKIN;
    return rc;
}

namespace {
// Row orig[k] of out (caller order) gets the caller indices of sorted atom
// k's neighbours, from the grouped column-major atom-index list W.
__global__ void k_list_out(int64_t n, const int32_t *__restrict__ orig, const int32_t *__restrict__ W,
                           const int32_t *__restrict__ cnt, int32_t max_nbr, int64_t ld, int32_t *__restrict__ out,
                           int32_t *__restrict__ out_cnt, int32_t max_out) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t o = orig[k];
    const int32_t c = cnt[k];
    out_cnt[o] = c;
    const int32_t m = min(min(c, max_nbr), max_out);
    for (int32_t e = 0; e < m; ++e) out[o * max_out + e] = orig[W[(((int64_t)(e >> 2) * ld + k) << 2) + (e & 3)]];
}
}  // namespace

extern "C" int ppmd_md_get_list(ppmd_md *m, int32_t *nbr, int32_t *nbr_count, int32_t max_nbr) {
    if (!m || !m->ready || max_nbr < 0 || (m->n > 0 && (!nbr_count || (max_nbr > 0 && !nbr))))
        return m ? set_error(m->ctx, PPMD_ERR_INVALID, "ppmd_md_get_list: bad argument") : PPMD_ERR_INVALID;
    ppmd_ctx *ctx = m->ctx;
    cudaSetDevice(ctx->device);
    if (m->n == 0) return PPMD_OK;
    const int32_t *W = m->W;
    if (m->slots) {
        int32_t *w = (int32_t *)scratch(ctx, S_TMP2, sizeof(int32_t) * (size_t)m->ld * (size_t)m->p.max_nbr);
        if (!w) return PPMD_ERR_NOMEM;
        PPMD_TRY(slots_to_atoms(ctx, m->nbricks, m->bricks, m->st, m->cell_start, m->W16, m->ld, m->cnt, m->p.max_nbr,
                                m->stage_cap, w, m->n));
        W = w;
    }
    if (m->n > 0)
        PPMD_LAUNCH(ctx, k_list_out, div_up(m->n, 256), 256, 0, m->n, m->orig, W, m->cnt, m->p.max_nbr, m->ld, nbr,
                    nbr_count, max_nbr);
    return check_launch(ctx, "ppmd_md_get_list");
}

namespace {
__global__ void k_list_stats(const int32_t *cnt, int64_t n, unsigned long long *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int32_t v = i < n ? cnt[i] : 0;
    unsigned long long s = (unsigned long long)v;
    int32_t mx = v;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&out[0], s);
        atomicMax(&out[1], (unsigned long long)mx);
    }
}
}  // namespace

namespace {
void drop_graph(ppmd_md *m) {
    for (cudaGraphExec_t *x : {&m->exec, &m->exec_ev}) {
        if (*x) {
            cudaStreamSynchronize(m->ctx->stream);
            cudaGraphExecDestroy(*x);
            *x = nullptr;
        }
    }
}
}  // namespace

extern "C" int ppmd_md_set_thermostat(ppmd_md *m, double T, double nu, uint64_t seed) {
    if (!m) return PPMD_ERR_INVALID;
    if (!(T >= 0.0) || !(nu >= 0.0) || !isfinite(T) || !isfinite(nu))
        return set_error(m->ctx, PPMD_ERR_INVALID, "ppmd_md_set_thermostat: bad temperature or rate");
    cudaSetDevice(m->ctx->device);
    drop_graph(m);
    const double p = nu * m->p.dt;
    m->thermo_thr = !(p > 0.0) ? 0 : (p >= 1.0 ? ((uint64_t)1 << 32) : (uint64_t)floor(p * 4294967296.0));
    m->thermo_sd = sqrt(T / m->p.mass);
    m->thermo_seed = seed;
    return PPMD_OK;
}

extern "C" int ppmd_md_set_boa(ppmd_md *m, int32_t every, double r_boa) {
    if (!m) return PPMD_ERR_INVALID;
    if (every < 0 || (every > 0 && !(r_boa > 0.0 && r_boa <= m->p.lj.rc)))
        return set_error(m->ctx, PPMD_ERR_INVALID, "ppmd_md_set_boa: need every >= 0 and 0 < r_boa <= rc");
    cudaSetDevice(m->ctx->device);
    drop_graph(m);
    if (every > 0 && m->slots) {
        // the analysis reads the atom-index list W: convert the current slot
        // list (same entries, same order) and build W from now on
        if (!m->W) PPMD_TRY(md_alloc(m, &m->W, (size_t)m->ld * m->p.max_nbr));
        if (m->ready)
            PPMD_TRY(slots_to_atoms(m->ctx, m->nbricks, m->bricks, m->st, m->cell_start, m->W16, m->ld, m->cnt,
                                    m->p.max_nbr, m->stage_cap, m->W, m->n));
        m->slots = false;
    }
    m->boa_every = every;
    m->r_boa = r_boa;
    // the short list of the current build (later builds make their own)
    return m->ready ? build_short_list(m) : PPMD_OK;
}

extern "C" int ppmd_md_set_pair_loop(ppmd_md *m, int mechanism) {
    if (!m) return PPMD_ERR_INVALID;
    ppmd_ctx *ctx = m->ctx;
    if (mechanism != PPMD_PAIR_COLUMNS && mechanism != PPMD_PAIR_BRICKS)
        return set_error(ctx, PPMD_ERR_INVALID, "ppmd_md_set_pair_loop: unknown mechanism %d", mechanism);
    if (m->ready) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_md_set_pair_loop: call it before ppmd_md_set_state");
    if (mechanism == PPMD_PAIR_BRICKS && (m->p.prec != PPMD_FP32 || m->boa_every > 0 || m->shape != 0))
        return set_error(ctx, PPMD_ERR_INVALID,
                         "ppmd_md_set_pair_loop: bricks need FP32, no on-the-fly analysis and the default shape");
    cudaSetDevice(ctx->device);
    drop_graph(m);
    if (mechanism == PPMD_PAIR_BRICKS) {
        if (!m->W16) PPMD_TRY(md_alloc(m, &m->W16, (size_t)m->ld * m->p.max_nbr));
        PPMD_TRY(slots_setup(ctx, m->stage_cap, m->p.max_nbr));
    }
    m->slots = mechanism == PPMD_PAIR_BRICKS;
    return PPMD_OK;
}

extern "C" int ppmd_md_set_check(ppmd_md *m, int on) {
    if (!m) return PPMD_ERR_INVALID;
    cudaSetDevice(m->ctx->device);
    drop_graph(m);
    if (on && !m->xq_old) {
        PPMD_TRY(md_alloc(m, &m->xq_old, (size_t)m->n));
        PPMD_TRY(md_alloc(m, &m->missed, 1));
        PPMD_TRY(cuda_check(m->ctx, cudaMemset(m->missed, 0, sizeof(unsigned long long)), "memset"));
    }
    m->check = on != 0;
    return PPMD_OK;
}

extern "C" int ppmd_md_missed_pairs(ppmd_md *m, int64_t *missed) {
    if (!m || !missed) return PPMD_ERR_INVALID;
    ppmd_ctx *ctx = m->ctx;
    *missed = 0;
    if (!m->missed) return PPMD_OK;
    cudaSetDevice(ctx->device);
    unsigned long long h = 0;
    PPMD_TRY(cuda_check(ctx, cudaMemcpyAsync(&h, m->missed, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream), "copy"));
    const int rc = ppmd_sync(ctx);
    *missed = (int64_t)h;
    return rc;
}

extern "C" int ppmd_md_time_pair_loops(ppmd_md *m, int on) {
    if (!m) return PPMD_ERR_INVALID;
    cudaSetDevice(m->ctx->device);
    drop_graph(m);
    m->time_pair = on != 0;
    if (m->time_pair && m->ev.empty()) {
        const int32_t P = m->p.rebuild_every, unit = P * std::max(1, 10 / P);
        m->ev.resize(2 * (size_t)std::min(unit, 1024));
        m->ev_fused.assign(m->ev.size() / 2, 0);
        for (cudaEvent_t &e : m->ev) PPMD_TRY(cuda_check(m->ctx, cudaEventCreate(&e), "event"));
    }
    return PPMD_OK;
}

extern "C" int ppmd_md_pair_loop_times(ppmd_md *m, double *ms_fused, int32_t *n_fused, double *ms_other,
                                       int32_t *n_other) {
    if (!m) return PPMD_ERR_INVALID;
    ppmd_ctx *ctx = m->ctx;
    if (!m->time_pair || !m->exec_ev)
        return set_error(ctx, PPMD_ERR_INVALID, "ppmd_md_pair_loop_times: no timed graph replay yet");
    cudaSetDevice(ctx->device);
    PPMD_TRY(cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "sync"));
    double sf = 0, so = 0;
    int32_t nf = 0, no = 0;
    for (int32_t k = 0; k < m->graph_steps && 2 * k + 1 < (int32_t)m->ev.size(); ++k) {
        float t = 0.0f;
        PPMD_TRY(cuda_check(ctx, cudaEventElapsedTime(&t, m->ev[2 * k], m->ev[2 * k + 1]), "event time"));
        if (m->ev_fused[k]) {
            sf += t;
            ++nf;
        } else {
            so += t;
            ++no;
        }
    }
    if (ms_fused) *ms_fused = nf ? sf / nf : 0.0;
    if (n_fused) *n_fused = nf;
    if (ms_other) *ms_other = no ? so / no : 0.0;
    if (n_other) *n_other = no;
    return PPMD_OK;
}

extern "C" int ppmd_md_get_q(ppmd_md *m, float *q4, float *q5, float *q6) {
    if (!m) return PPMD_ERR_INVALID;
    ppmd_ctx *ctx = m->ctx;
    if (!m->have_q) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_md_get_q: no analysis step yet");
    cudaSetDevice(ctx->device);
    float *out[3] = {q4, q5, q6};
    for (int l = 0; l < 3; ++l)
        if (out[l])
            PPMD_TRY(cuda_check(ctx, cudaMemcpyAsync(out[l], m->q3 + (size_t)l * m->n, sizeof(float) * (size_t)m->n,
                                                     cudaMemcpyDeviceToDevice, ctx->stream),
                                "copy"));
    return PPMD_OK;
}

extern "C" int ppmd_md_forces(ppmd_md *m) {
    if (!m || !m->ready) return PPMD_ERR_INVALID;
    cudaSetDevice(m->ctx->device);
    return forces(m, false, false);
}

extern "C" int ppmd_md_list_stats(ppmd_md *m, int64_t *pairs, int32_t *max_row) {
    if (!m || !m->ready) return PPMD_ERR_INVALID;
    ppmd_ctx *ctx = m->ctx;
    cudaSetDevice(ctx->device);
    unsigned long long *d = (unsigned long long *)scratch(ctx, S_TMP1, 16);
    if (!d) return PPMD_ERR_NOMEM;
    PPMD_TRY(cuda_check(ctx, cudaMemsetAsync(d, 0, 16, ctx->stream), "memset"));
    if (m->n > 0) PPMD_LAUNCH(ctx, k_list_stats, div_up(m->n, 256), 256, 0, m->cnt, m->n, d);
    unsigned long long h[2] = {0, 0};
    PPMD_TRY(cuda_check(ctx, cudaMemcpyAsync(h, d, 16, cudaMemcpyDeviceToHost, ctx->stream), "copy"));
    int rc = ppmd_sync(ctx);
    if (pairs) *pairs = (int64_t)h[0];
    if (max_row) *max_row = (int32_t)h[1];
    return rc;
}

// ---------------------------------------------------------------------
// Launch shapes and their tuning.
// ---------------------------------------------------------------------
namespace {

// Candidates: (FP32 pair-loop threads per block, persistent blocks per SM
// (0: one thread per atom), expected home atoms of a list-build brick).
struct ShapeCand {
    int32_t block, per_sm, home;
};
constexpr ShapeCand SHAPES[PPMD_MD_SHAPES] = {{128, 0, 128}, {256, 0, 128}, {128, 8, 128}, {256, 4, 128},
                                              {128, 0, 64},  {256, 0, 64},  {128, 8, 64},  {256, 4, 64}};

int apply_shape(ppmd_md *m, int32_t k) {
    ppmd_ctx *ctx = m->ctx;
    const ShapeCand &c = SHAPES[k];
    int sms = 0;
    PPMD_TRY(cuda_check(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device), "attribute"));
    drop_graph(m);
    m->col.block = c.block;
    m->col.grid_cap = c.per_sm > 0 ? (int64_t)c.per_sm * sms : 0;
    if (c.home != m->brick_home) {
        std::vector<Brick> bl;
        const int32_t cap = make_bricks(m->segs, bl, c.home);
        if ((int64_t)bl.size() > m->bricks_alloc) {
            PPMD_TRY(md_alloc(m, &m->bricks, bl.size()));  // (the smaller table stays allocated until destroy)
            m->bricks_alloc = (int64_t)bl.size();
        }
        if (!bl.empty())
            PPMD_TRY(cuda_check(ctx, cudaMemcpy(m->bricks, bl.data(), sizeof(Brick) * bl.size(), cudaMemcpyHostToDevice),
                                "copy"));
        m->nbricks = (int64_t)bl.size();
        m->stage_cap = cap;
        m->brick_home = c.home;
    }
    m->shape = k;
    return PPMD_OK;
}

// The workload's shape as a cache key: atoms, boxes, cells, cutoffs, list
// policy, the device and the candidate table (an entry written for another
// table never matches).
std::string shape_key(const ppmd_md *m) {
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, m->ctx->device);
    std::string table;
    for (const ShapeCand &c : SHAPES)
        table += std::to_string(c.block) + "/" + std::to_string(c.per_sm) + "/" + std::to_string(c.home) + ",";
    char buf[512];
    snprintf(buf, sizeof(buf), "n=%lld;boxes=%lld;cells=%lld;r_list=%.9g;rc=%.9g;max_nbr=%d;every=%d;dev=%s;sms=%d;shapes=",
             (long long)m->n, (long long)m->nbox, (long long)m->ncell, m->p.r_list, m->p.lj.rc, m->p.max_nbr,
             m->p.rebuild_every, prop.name, prop.multiProcessorCount);
    std::string key = buf + table;
    for (char &c : key)
        if (c == '\t' || c == '\n') c = ' ';
    return key;
}

}  // namespace

extern "C" int ppmd_md_set_shape(ppmd_md *m, int32_t shape) {
    if (!m) return PPMD_ERR_INVALID;
    ppmd_ctx *ctx = m->ctx;
    if (shape < 0 || shape >= PPMD_MD_SHAPES) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_md_set_shape: shape %d", shape);
    if (shape != 0 && (m->p.prec != PPMD_FP32 || m->slots))
        return set_error(ctx, PPMD_ERR_INVALID, "ppmd_md_set_shape: shapes are for the FP32 atom-index pair loop");
    cudaSetDevice(ctx->device);
    return apply_shape(m, shape);
}

extern "C" int ppmd_md_get_shape(ppmd_md *m, int32_t *shape, int32_t *block, int32_t *per_sm, int32_t *brick_home) {
    if (!m) return PPMD_ERR_INVALID;
    const ShapeCand &c = SHAPES[m->shape];
    if (shape) *shape = m->shape;
    if (block) *block = c.block;
    if (per_sm) *per_sm = c.per_sm;
    if (brick_home) *brick_home = c.home;
    return PPMD_OK;
}

extern "C" int ppmd_md_tune(ppmd_md *m, int32_t steps, const char *cache_path, int32_t *shape, double *ms_per_step,
                            int *timed) {
    if (!m || steps < 1) return PPMD_ERR_INVALID;
    ppmd_ctx *ctx = m->ctx;
    if (!m->ready) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_md_tune: state not set");
    cudaSetDevice(ctx->device);
    if (timed) *timed = 0;
    if (ms_per_step)
        for (int k = 0; k < PPMD_MD_SHAPES; ++k) ms_per_step[k] = -1.0;
    if (m->p.prec != PPMD_FP32 || m->slots) {  // nothing to choose
        if (shape) *shape = m->shape;
        return PPMD_OK;
    }
    const std::string key = shape_key(m);
    if (cache_path) {
        FILE *f = fopen(cache_path, "r");
        int32_t found = -1;
        if (f) {
            char line[1024];
            while (fgets(line, sizeof(line), f)) {
                char *tab = strchr(line, '\t');
                if (!tab) continue;
                *tab = 0;
                if (key == line) {
                    const int32_t k = (int32_t)strtol(tab + 1, nullptr, 10);
                    if (k >= 0 && k < PPMD_MD_SHAPES) found = k;  // the last entry of the key counts
                }
            }
            fclose(f);
        }
        if (found >= 0) {
            PPMD_TRY(apply_shape(m, found));
            if (shape) *shape = found;
            return PPMD_OK;
        }
    }
    // time every candidate from the present state, then start again from it
    const int64_t n = m->n;
    if (!m->tune_buf) PPMD_TRY(md_alloc(m, &m->tune_buf, 6 * (size_t)std::max<int64_t>(n, 1)));
    double *tp = m->tune_buf, *tv = m->tune_buf + 3 * n;
    PPMD_TRY(ppmd_md_get_state(m, tp, tv, nullptr));
    const int32_t P = m->p.rebuild_every, unit = P * std::max(1, 10 / P);
    const int32_t timed_steps = (steps + unit - 1) / unit * unit;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PPMD_TRY(cuda_check(ctx, cudaEventCreate(&e0), "event"));
    int rc = cuda_check(ctx, cudaEventCreate(&e1), "event");
    double t[PPMD_MD_SHAPES];
    int32_t best = 0;
    for (int32_t k = 0; rc == PPMD_OK && k < PPMD_MD_SHAPES; ++k) {
        rc = apply_shape(m, k);
        if (rc == PPMD_OK) rc = ppmd_md_set_state(m, tp, tv);
        if (rc == PPMD_OK) rc = ppmd_md_run(m, unit, nullptr, 1);  // warm-up, graph capture
        if (rc == PPMD_OK) rc = cuda_check(ctx, cudaEventRecord(e0, ctx->stream), "event");
        if (rc == PPMD_OK) rc = ppmd_md_run(m, timed_steps, nullptr, 1);
        if (rc == PPMD_OK) rc = cuda_check(ctx, cudaEventRecord(e1, ctx->stream), "event");
        if (rc == PPMD_OK) rc = cuda_check(ctx, cudaEventSynchronize(e1), "event");
        float ms = 0.0f;
        if (rc == PPMD_OK) rc = cuda_check(ctx, cudaEventElapsedTime(&ms, e0, e1), "event time");
        t[k] = ms / timed_steps;
        if (ms_per_step) ms_per_step[k] = t[k];
        if (rc == PPMD_OK && t[k] < t[best]) best = k;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != PPMD_OK) return rc;
    PPMD_TRY(apply_shape(m, best));
    PPMD_TRY(ppmd_md_set_state(m, tp, tv));
    if (shape) *shape = best;
    if (timed) *timed = 1;
    if (cache_path) {
        FILE *f = fopen(cache_path, "a");
        if (!f) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_md_tune: cannot write %s", cache_path);
        fprintf(f, "%s\t%d\t%.6f\n", key.c_str(), best, t[best]);
        fclose(f);
    }
    return PPMD_OK;
}
