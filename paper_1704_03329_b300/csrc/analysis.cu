// Structure analysis over a neighbour list:
//  - bond order parameters Q4, Q6 (Eqs. (4)-(5), Algorithms 1-2), one thread
//    per atom accumulating the spherical-harmonic moments of its bonds;
//  - common neighbour analysis (Eqs. (6)-(8), Algorithms 3-5 and 7), one warp
//    per atom on 64-bit adjacency masks of the atom's bonded neighbours;
//  - an analysis pipeline that bins and sorts the atoms by cell, builds the
//    list and runs either analysis, returning results in caller order.
#include <cuda_bf16.h>
#include <math.h>

#include "analysis.cuh"
#include "cells.cuh"
#include "md_kernels.cuh"
#include "neighbours.cuh"

namespace ppmd {

// ---------------------------------------------------------------------
// Spherical harmonics for l = 4 and l = 6.
// For a unit vector u = (x, y, z):  Y_l^m(u) = N_lm P_l^m(z) e^{i m phi} and
// P_l^m(z) e^{i m phi} = Pr_l^m(z) (x + i y)^m with Pr_l^m = P_l^m / (1-z^2)^{m/2},
// a polynomial obtained from the three-term recurrence
//   Pr_m^m = (-1)^m (2m-1)!!,  Pr_{m+1}^m = (2m+1) z Pr_m^m,
//   (l-m) Pr_l^m = (2l-1) z Pr_{l-1}^m - (l+m-1) Pr_{l-2}^m.
// Q_l^2 = 4 pi/(2l+1) sum_{m=-l..l} |q_lm|^2 = sum_{m=0..l} c_lm |S_lm|^2 / nu^2 with
// S_lm = sum_j Pr_l^m(z_j) (x_j + i y_j)^m, c_l0 = 1, c_lm = 2 (l-m)!/(l+m)! (m > 0)
// (the Y_l^{-m} terms equal the Y_l^m ones in modulus).  sqrt(c_lm) is folded
// into each term so that every partial sum stays of order one.
// ---------------------------------------------------------------------
// The polynomials sqrt(c_lm) Pr_l^m(z) have the parity of l - m, so each is
// stored as z^((l-m) mod 2) times a polynomial in z^2 (ascending
// coefficients), built on the host from the recurrence above in FP64.
struct YlmCoef {
    float c4[5][3];  // l = 4: degree (4-m)/2 in z^2
    float c5[6][3];  // l = 5: degree (5-m)/2 in z^2
    float c6[7][4];  // l = 6: degree (6-m)/2 in z^2
};

static YlmCoef make_coef() {
    YlmCoef k;
    memset(&k, 0, sizeof(k));
    auto fact = [](int q) {
        double f = 1.0;
        for (int i = 2; i <= q; ++i) f *= i;
        return f;
    };
    for (int m = 0; m <= 6; ++m) {
        // polynomials in z as coefficient arrays (index = power)
        double pm2[8] = {0}, pm1[8] = {0}, pl[8] = {0};
        double df = 1.0;
        for (int q = 1; q <= m; ++q) df *= (2.0 * q - 1.0);
        pm1[0] = (m % 2 ? -1.0 : 1.0) * df;  // Pr_m^m
        auto store = [&](int l, const double *poly) {
            if (l < 4) return;
            const double sc = sqrt((m ? 2.0 : 1.0) * fact(l - m) / fact(l + m));
            const int par = (l - m) & 1;
            for (int e = 0; e <= (l - m) / 2; ++e) {
                const float v = (float)(sc * poly[2 * e + par]);
                if (l == 4) k.c4[m][e] = v;
                else if (l == 5) k.c5[m][e] = v;
                else k.c6[m][e] = v;
            }
        };
        store(m, pm1);
        if (m + 1 <= 6) {
            for (int e = 0; e < 7; ++e) pl[e + 1] = (2.0 * m + 1.0) * pm1[e];  // Pr_{m+1}^m
            memcpy(pm2, pm1, sizeof(pm1));
            memcpy(pm1, pl, sizeof(pl));
            store(m + 1, pm1);
        }
        for (int l = m + 2; l <= 6; ++l) {
            double nx[8] = {0};
            for (int e = 0; e < 8; ++e) {
                const double zt = e > 0 ? pm1[e - 1] : 0.0;
                nx[e] = ((2.0 * l - 1.0) * zt - (l + m - 1.0) * pm2[e]) / (l - m);
            }
            memcpy(pm2, pm1, sizeof(pm1));
            memcpy(pm1, nx, sizeof(nx));
            store(l, pm1);
        }
    }
    return k;
}

// Adds the moments of one bond direction (x, y, z) (unit vector):
// r_lm + i i_lm += sqrt(c_lm) Pr_l^m(z) (x + i y)^m, l = 4, 6 (and 5 with
// Q5), m = 0..l.
template <bool Q5>
__device__ __forceinline__ void boa_moments(const YlmCoef &K, float x, float y, float z, float (&r4)[5],
                                            float (&i4)[5], float (&r5)[6], float (&i5)[6], float (&r6)[7],
                                            float (&i6)[7]) {
    const float z2 = z * z;
    float pr = 1.0f, pi = 0.0f;  // (x + i y)^m
#pragma unroll
    for (int m = 0; m <= 6; ++m) {
        if (m > 0) {
            const float t = fmaf(pr, x, -pi * y);
            pi = fmaf(pr, y, pi * x);
            pr = t;
        }
        if (m <= 4) {
            float w = K.c4[m][(4 - m) / 2];
#pragma unroll
            for (int e = (4 - m) / 2 - 1; e >= 0; --e) w = fmaf(w, z2, K.c4[m][e]);
            if ((4 - m) & 1) w *= z;
            r4[m] = fmaf(w, pr, r4[m]);
            if (m > 0) i4[m] = fmaf(w, pi, i4[m]);
        }
        if (Q5 && m <= 5) {
            float w = K.c5[m][(5 - m) / 2];
#pragma unroll
            for (int e = (5 - m) / 2 - 1; e >= 0; --e) w = fmaf(w, z2, K.c5[m][e]);
            if ((5 - m) & 1) w *= z;
            r5[m] = fmaf(w, pr, r5[m]);
            if (m > 0) i5[m] = fmaf(w, pi, i5[m]);
        }
        float w6 = K.c6[m][(6 - m) / 2];
#pragma unroll
        for (int e = (6 - m) / 2 - 1; e >= 0; --e) w6 = fmaf(w6, z2, K.c6[m][e]);
        if ((6 - m) & 1) w6 *= z;
        r6[m] = fmaf(w6, pr, r6[m]);
        if (m > 0) i6[m] = fmaf(w6, pi, i6[m]);
    }
}

__device__ __forceinline__ void boa_accumulate(const YlmCoef &K, float x, float y, float z, float (&r4)[5],
                                               float (&i4)[5], float (&r6)[7], float (&i6)[7]) {
    float r5[6], i5[6];  // unused
    boa_moments<false>(K, x, y, z, r4, i4, r5, i5, r6, i6);
}

// One thread per atom.  Bonds: list entries with r < r_cut (exact decision).
// out_idx (may be null): write the results of atom i at out_idx[i].
__global__ void __launch_bounds__(256) k_boa(int64_t n, const int4 *__restrict__ xq, const double *__restrict__ pos64,
                                             SegTable st, const int32_t *__restrict__ nbr, const int32_t *__restrict__ cnt,
                                             int32_t max_nbr, int64_t si, int64_t sm, double rc2, float rc2_lo,
                                             float rc2_hi, YlmCoef K,
                                             const int32_t *__restrict__ out_idx, float *__restrict__ q4,
                                             float *__restrict__ q6, int32_t *__restrict__ nnb) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int4 xi = xq[i];
    const Seg &S = seg_ref(st, xi.w);
    float r4[5], i4[5], r6[7], i6[7];
#pragma unroll
    for (int m = 0; m < 7; ++m) {
        if (m < 5) r4[m] = i4[m] = 0.0f;
        r6[m] = i6[m] = 0.0f;
    }
    const int32_t deg = min(cnt[i], max_nbr);
    const int32_t *row = nbr + i * si;
    int32_t nu = 0;
    for (int32_t k = 0; k < deg; ++k) {
        const int32_t j = row[k * sm];
        const int4 xj = __ldg(&xq[j]);
        float dx = fixed_delta((uint32_t)xi.x, (uint32_t)xj.x, S.sx[0]);
        float dy = fixed_delta((uint32_t)xi.y, (uint32_t)xj.y, S.sx[1]);
        float dz = fixed_delta((uint32_t)xi.z, (uint32_t)xj.z, S.sx[2]);
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        bool in = r2 < rc2_lo;
        if (!in && r2 < rc2_hi) {
            double dr[3];
            in = min_image_r2(pos64 + 3 * i, pos64 + 3 * (int64_t)j, S, dr) < rc2;
        }
        if (!in) continue;
        const float ir = rsqrtf(r2);
        boa_accumulate(K, dx * ir, dy * ir, dz * ir, r4, i4, r6, i6);
        ++nu;
    }
    float s4 = 0.0f, s6 = 0.0f;
#pragma unroll
    for (int m = 0; m < 7; ++m) {
        if (m < 5) s4 = fmaf(r4[m], r4[m], fmaf(i4[m], i4[m], s4));
        s6 = fmaf(r6[m], r6[m], fmaf(i6[m], i6[m], s6));
    }
    const float inv = nu > 0 ? 1.0f / (float)nu : 0.0f;
    const int64_t o = out_idx ? out_idx[i] : i;
    if (q4) q4[o] = sqrtf(s4) * inv;
    if (q6) q6[o] = sqrtf(s6) * inv;
    if (nnb) nnb[o] = nu;
}

// ---------------------------------------------------------------------
// Common neighbour analysis, one warp per atom.
// Bonded neighbours of i (list entries with r < r_cut) get local indices
// 0..nu-1; A[a] is the 64-bit set of local indices bonded to neighbour a.
// For the bond (i, a):  C = A[a] (common neighbours of i and a),
//   n_cn = |C|,  n_b = sum_{b in C} |A[b] & C| / 2,
//   n_lcb = edges of the largest connected component of (C, A restricted to C),
// found by growing each component from its lowest member.
// Triplets: trip[i*max_nbr + m] for list slot m (0xFFFFFFFF: not bonded).
// ---------------------------------------------------------------------
// CNA: a group of CNA_G = 16 lanes per atom (two atoms per warp: the
// 12-14 bonds of a crystal atom fill most of a group).
constexpr int CNA_WARPS = 4, CNA_G = 16, CNA_GROUPS = CNA_WARPS * 32 / CNA_G;
constexpr uint32_t NOT_BONDED = 0xFFFFFFFFu;

__device__ __forceinline__ bool bonded(const int4 &a, const int4 &b, const double *pa, const double *pb, const Seg &S,
                                       double rc2, float lo, float hi) {
    float dx = fixed_delta((uint32_t)a.x, (uint32_t)b.x, S.sx[0]);
    float dy = fixed_delta((uint32_t)a.y, (uint32_t)b.y, S.sx[1]);
    float dz = fixed_delta((uint32_t)a.z, (uint32_t)b.z, S.sx[2]);
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    if (r2 < lo) return true;
    if (r2 >= hi) return false;
    double dr[3];
    return min_image_r2(pa, pb, S, dr) < rc2;
}

__device__ __forceinline__ int32_t cna_label_of(int nu, int c421, int c422, int c444, int c666) {
    if (nu == 12 && c421 == 12) return PPMD_FCC;
    if (nu == 12 && c421 == 6 && c422 == 6) return PPMD_HCP;
    if (nu == 14 && c666 == 8 && c444 == 6) return PPMD_BCC;
    return PPMD_OTHER;
}

__device__ __forceinline__ void cna_atom(int64_t i, int lane, unsigned gmask, int shift, const int4 *__restrict__ xq,
                                         const double *__restrict__ pos64, const SegTable &st,
                                         const int32_t *__restrict__ nbr, const int32_t *__restrict__ cnt,
                                         int32_t max_nbr, int64_t si, int64_t sm, double rc2, float lo, float hi,
                                         const int32_t *__restrict__ out_idx, uint32_t *__restrict__ trip,
                                         int8_t *__restrict__ label, int32_t *status, unsigned long long *needed,
                                         int32_t *s_j, int32_t *s_slot, int4 *s_x, unsigned long long *s_A) {
    const int4 xi = xq[i];
    const Seg &S = seg_ref(st, xi.w);
    const int32_t deg = min(cnt[i], max_nbr);
    const int32_t *row = nbr + i * si;
    uint32_t *trow = trip ? trip + i * (int64_t)max_nbr : nullptr;
    const unsigned lt = (1u << lane) - 1u;
    // bonded neighbours, compacted in list order
    int32_t nu = 0;
    for (int32_t base = 0; base < deg; base += CNA_G) {
        const int32_t k = base + lane;
        bool b = false;
        int32_t j = 0;
        int4 xj = make_int4(0, 0, 0, 0);
        if (k < deg) {
            j = row[k * sm];
            xj = xq[j];
            b = bonded(xi, xj, pos64 + 3 * i, pos64 + 3 * (int64_t)j, S, rc2, lo, hi);
            if (!b && trow) trow[k] = NOT_BONDED;
        }
        const unsigned ball = __ballot_sync(gmask, b) >> shift;
        if (b) {
            const int32_t a = nu + __popc(ball & lt);
            if (a < 64) {
                s_j[a] = j;
                s_slot[a] = k;
                s_x[a] = xj;
            }
        }
        nu += __popc(ball);
    }
    __syncwarp(gmask);
    if (nu > 64) {
        // more bonded neighbours than the 64-bit masks hold
        if (lane == 0) {
            latch_status(status, PPMD_ERR_CAPACITY);
            latch_needed(needed, (unsigned long long)nu);
            if (label) label[out_idx ? out_idx[i] : i] = PPMD_OTHER;
        }
        return;
    }
    if (!trow && nu != 12 && nu != 14) {
        // labels only: no signature with this many bonds (cna_label_of)
        if (lane == 0 && label) label[out_idx ? out_idx[i] : i] = PPMD_OTHER;
        return;
    }
    // adjacency among the bonded neighbours, each pair tested once: lane a
    // takes the pairs (a, a + o mod nu) for o = 1 .. nu/2 (o = nu/2 of an
    // even nu only for a < nu/2), so every lane has about nu/2 tests
    for (int a = lane; a < nu; a += CNA_G) s_A[a] = 0ull;
    __syncwarp(gmask);
    for (int a = lane; a < nu; a += CNA_G) {
        unsigned long long m = 0ull;
        const int4 xa = s_x[a];
        const int32_t ja = s_j[a];
        const int half = nu >> 1;
        const int last = ((nu & 1) == 0 && a >= half) ? half - 1 : half;
        for (int o = 1; o <= last; ++o) {
            const int b = a + o < nu ? a + o : a + o - nu;
            if (bonded(xa, s_x[b], pos64 + 3 * (int64_t)ja, pos64 + 3 * (int64_t)s_j[b], S, rc2, lo, hi)) {
                m |= 1ull << b;
                atomicOr(&s_A[b], 1ull << a);
            }
        }
        atomicOr(&s_A[a], m);
    }
    __syncwarp(gmask);
    int c421 = 0, c422 = 0, c444 = 0, c666 = 0;
    for (int a = lane; a < nu; a += CNA_G) {
        const unsigned long long C = s_A[a];
        const int ncn = __popcll(C);
        int twice_nb = 0;
        for (unsigned long long r = C; r; r &= r - 1) twice_nb += __popcll(s_A[__ffsll((long long)r) - 1] & C);
        // components of the common-neighbour graph
        int best = 0;
        unsigned long long rest = C;
        while (rest) {
            unsigned long long comp = rest & (~rest + 1ull);
            unsigned long long frontier = comp;
            while (frontier) {
                unsigned long long grow = 0ull;
                for (unsigned long long f = frontier; f; f &= f - 1) grow |= s_A[__ffsll((long long)f) - 1];
                grow &= C & ~comp;
                comp |= grow;
                frontier = grow;
            }
            int twice_e = 0;
            for (unsigned long long f = comp; f; f &= f - 1) twice_e += __popcll(s_A[__ffsll((long long)f) - 1] & comp);
            best = max(best, twice_e >> 1);
            rest &= ~comp;
        }
        const uint32_t t = ((uint32_t)ncn << 16) | ((uint32_t)(twice_nb >> 1) << 8) | (uint32_t)best;
        if (trow) trow[s_slot[a]] = t;
        c421 += t == ((4u << 16) | (2u << 8) | 1u);
        c422 += t == ((4u << 16) | (2u << 8) | 2u);
        c444 += t == ((4u << 16) | (4u << 8) | 4u);
        c666 += t == ((6u << 16) | (6u << 8) | 6u);
    }
    c421 = __reduce_add_sync(gmask, c421);
    c422 = __reduce_add_sync(gmask, c422);
    c444 = __reduce_add_sync(gmask, c444);
    c666 = __reduce_add_sync(gmask, c666);
    if (lane == 0 && label) label[out_idx ? out_idx[i] : i] = (int8_t)cna_label_of(nu, c421, c422, c444, c666);
}

__global__ void __launch_bounds__(CNA_WARPS * 32) k_cna(int64_t n, const int4 *__restrict__ xq,
                                                        const double *__restrict__ pos64, SegTable st,
                                                        const int32_t *__restrict__ nbr, const int32_t *__restrict__ cnt,
                                                        int32_t max_nbr, int64_t si, int64_t sm, double rc2, float lo,
                                                        float hi,
                                                        const int32_t *__restrict__ out_idx, uint32_t *__restrict__ trip,
                                                        int8_t *__restrict__ label, int32_t *status,
                                                        unsigned long long *needed, const int32_t *__restrict__ which,
                                                        const int32_t *__restrict__ n_dev) {
    __shared__ int32_t s_j[CNA_GROUPS][64];
    __shared__ int32_t s_slot[CNA_GROUPS][64];
    __shared__ int4 s_x[CNA_GROUPS][64];
    __shared__ unsigned long long s_A[CNA_GROUPS][64];
    const int lane = threadIdx.x & (CNA_G - 1), g = threadIdx.x / CNA_G, shift = threadIdx.x & 31 & ~(CNA_G - 1);
    const unsigned gmask = ((1u << CNA_G) - 1u) << shift;
    // the count comes from the device when the subset was chosen there
    const int64_t m = n_dev ? (int64_t)*n_dev : n;
    for (int64_t gi = (int64_t)blockIdx.x * CNA_GROUPS + g; gi < m; gi += (int64_t)gridDim.x * CNA_GROUPS) {
        const int64_t i = which ? (int64_t)which[gi] : gi;  // a subset of the atoms when `which` is given
        cna_atom(i, lane, gmask, shift, xq, pos64, st, nbr, cnt, max_nbr, si, sm, rc2, lo, hi, out_idx, trip, label, status,
                 needed, s_j[g], s_slot[g], s_x[g], s_A[g]);
        __syncwarp(gmask);
    }
}

// ---------------------------------------------------------------------
// Adaptive CNA (the extension the CNA section cites): per-atom cutoffs
// from the 12 (fcc/hcp test) or 14 (bcc test) nearest neighbours,
//   r_12 = f (d_1 + ... + d_12) / 12,  r_14 = f (c (d_1 + ... + d_8) + d_9 + ... + d_14) / 14,
// f = (1 + sqrt 2)/2, c = 2/sqrt 3; only those neighbours take part, two of
// them bonded when closer than the cutoff; CNA triplets over them.  One warp
// per atom, up to 64 list entries (two per lane).  Every decision is the
// FP64 one: the nearest neighbours are ranked in FP32 and the candidates
// that could sit at the N-th place within FP32 error are ranked again by
// their FP64 distance (ties by index); the cutoff is summed in FP64 in rank
// order with IEEE operations; bond tests take FP32 outside a band around
// the cutoff and FP64 inside it.
// ---------------------------------------------------------------------
constexpr int ACNA_WARPS = 4;

__global__ void __launch_bounds__(ACNA_WARPS * 32) k_acna(int64_t n, const int4 *__restrict__ xq,
                                                          const double *__restrict__ pos64, SegTable st,
                                                          const int32_t *__restrict__ nbr,
                                                          const int32_t *__restrict__ cnt, int32_t max_nbr, int64_t si,
                                                          int64_t sm, double f, double c,
                                                          const int32_t *__restrict__ out_idx, int8_t *__restrict__ label,
                                                          double *__restrict__ rcut, int32_t *status,
                                                          unsigned long long *needed) {
    __shared__ int32_t s_j[ACNA_WARPS][16];
    __shared__ int4 s_x[ACNA_WARPS][16];
    __shared__ unsigned s_A[ACNA_WARPS][16];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * ACNA_WARPS + w;
    if (i >= n) return;
    const int4 xi = xq[i];
    const Seg &S = seg_ref(st, xi.w);
    const int32_t deg = min(cnt[i], max_nbr);
    const int64_t o = out_idx ? out_idx[i] : i;
    if (deg > 64) {
        if (lane == 0) {
            latch_status(status, PPMD_ERR_CAPACITY);
            latch_needed(needed, (unsigned long long)deg);
            label[o] = PPMD_OTHER;
            if (rcut) rcut[2 * o] = rcut[2 * o + 1] = 0.0;
        }
        return;
    }
    const int32_t *row = nbr + i * si;
    // candidates k = lane and lane + 32
    int32_t jj[2];
    int4 xj[2];
    float r2f[2];
    double d64[2];
    bool have64[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int32_t k = lane + 32 * q;
        have64[q] = false;
        d64[q] = 0.0;
        if (k < deg) {
            jj[q] = row[k * sm];
            xj[q] = xq[jj[q]];
            const float dx = fixed_delta((uint32_t)xi.x, (uint32_t)xj[q].x, S.sx[0]);
            const float dy = fixed_delta((uint32_t)xi.y, (uint32_t)xj[q].y, S.sx[1]);
            const float dz = fixed_delta((uint32_t)xi.z, (uint32_t)xj[q].z, S.sx[2]);
            r2f[q] = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        } else {
            jj[q] = 0x7fffffff;
            xj[q] = make_int4(0, 0, 0, 0);
            r2f[q] = __int_as_float(0x7f800000);  // +inf
        }
    }
    // FP32 rank by (r2, index) among the deg candidates (slots past the row
    // hold +inf and never come first)
    int rk[2] = {0, 0};
    const int d0 = min(deg, 32), d1 = deg - 32;  // sources in the first and second slot of each lane
    for (int src = 0; src < d0; ++src) {
        const float r = __shfl_sync(0xffffffffu, r2f[0], src);
        const int32_t jv = __shfl_sync(0xffffffffu, jj[0], src);
        rk[0] += (r < r2f[0]) || (r == r2f[0] && jv < jj[0]);
        if (d1 > 0) rk[1] += (r < r2f[1]) || (r == r2f[1] && jv < jj[1]);
    }
    for (int src = 0; src < d1; ++src) {
        const float r = __shfl_sync(0xffffffffu, r2f[1], src);
        const int32_t jv = __shfl_sync(0xffffffffu, jj[1], src);
        rk[0] += (r < r2f[0]) || (r == r2f[0] && jv < jj[0]);
        rk[1] += (r < r2f[1]) || (r == r2f[1] && jv < jj[1]);
    }
    int8_t lab = PPMD_OTHER;
    double rc12 = 0.0, rc14 = 0.0;
    for (int test = 0; test < 2; ++test) {
        const int N = test == 0 ? 12 : 14;
        if (deg < N || (test == 1 && lab != PPMD_OTHER)) break;
        // FP32 distances of the N-th and (N+1)-th candidates (inf when none)
        float tN = __int_as_float(0x7f800000), tN1 = 0.0f;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const bool v = lane + 32 * q < deg;
            const unsigned b = __ballot_sync(0xffffffffu, rk[q] == N && v);
            if (b) tN = __shfl_sync(0xffffffffu, r2f[q], __ffs(b) - 1);
            const unsigned b1 = __ballot_sync(0xffffffffu, rk[q] == N - 1 && v);
            if (b1) tN1 = __shfl_sync(0xffffffffu, r2f[q], __ffs(b1) - 1);
        }
        // FP32 r^2 is within ~3e-7 r^2 + 1e-7 of the FP64 value: with a
        // wider gap between the N-th and the (N+1)-th the FP32 ranks select
        // the same N atoms as the FP64 ones
        const float tol = 2e-6f * tN + 1e-6f;
        const bool ambiguous = deg > N && tN - tN1 <= 2.0f * tol;
        bool sel[2];
        int ex[2];
        if (!ambiguous) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                sel[q] = lane + 32 * q < deg && rk[q] < N;
                ex[q] = rk[q];
            }
        } else {
            // every candidate that can be among the N nearest lies below
            // tN + tol: rank those by (FP64 r^2, index)
            const float lim = tN + tol;
            bool near[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                near[q] = (lane + 32 * q < deg) && r2f[q] <= lim;
                if (near[q] && !have64[q]) {
                    double dr[3];
                    d64[q] = min_image_r2(pos64 + 3 * i, pos64 + 3 * (int64_t)jj[q], S, dr);
                    have64[q] = true;
                }
            }
            ex[0] = ex[1] = 0;
#pragma unroll
            for (int q2 = 0; q2 < 2; ++q2)
                for (int src = 0; src < (q2 ? d1 : d0); ++src) {
                    const bool nv = __shfl_sync(0xffffffffu, near[q2], src);
                    const double dv = __shfl_sync(0xffffffffu, d64[q2], src);
                    const int32_t jv = __shfl_sync(0xffffffffu, jj[q2], src);
#pragma unroll
                    for (int q = 0; q < 2; ++q) ex[q] += nv && ((dv < d64[q]) || (dv == d64[q] && jv < jj[q]));
                }
#pragma unroll
            for (int q = 0; q < 2; ++q) sel[q] = near[q] && ex[q] < N;
        }
#pragma unroll
        for (int q = 0; q < 2; ++q)
            if (sel[q]) {
                s_j[w][ex[q]] = jj[q];
                s_x[w][ex[q]] = xj[q];
            }
        // FP32 cutoff: within ~3e-6 r^2 of the FP64 one (the selected set is exact)
        float part = 0.0f, part6 = 0.0f;
#pragma unroll
        for (int q = 0; q < 2; ++q)
            if (sel[q]) {
                const float d = sqrtf(r2f[q]);
                if (test == 0 || ex[q] < 8) part += d;
                else part6 += d;
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            part += __shfl_xor_sync(0xffffffffu, part, o);
            part6 += __shfl_xor_sync(0xffffffffu, part6, o);
        }
        const float rcf = test == 0 ? (float)f * (part / 12.0f) : (float)f * (((float)c * part + part6) / 14.0f);
        float rc2f = rcf * rcf;
        // the exact FP64 cutoff: the sum of the FP64 distances in FP64 rank
        // order, needed for the cutoff output and for bond tests within the
        // band (computed only then)
        double rc2 = 0.0;
        auto exact_cutoff = [&]() {
#pragma unroll
            for (int q = 0; q < 2; ++q)
                if (sel[q] && !have64[q]) {
                    double dr[3];
                    d64[q] = min_image_r2(pos64 + 3 * i, pos64 + 3 * (int64_t)jj[q], S, dr);
                    have64[q] = true;
                }
            int er[2] = {0, 0};  // FP64 rank among the selected
#pragma unroll
            for (int q2 = 0; q2 < 2; ++q2)
                for (int src = 0; src < (q2 ? d1 : d0); ++src) {
                    const bool sv = __shfl_sync(0xffffffffu, sel[q2], src);
                    const double dv = __shfl_sync(0xffffffffu, d64[q2], src);
                    const int32_t jv = __shfl_sync(0xffffffffu, jj[q2], src);
#pragma unroll
                    for (int q = 0; q < 2; ++q) er[q] += sv && ((dv < d64[q]) || (dv == d64[q] && jv < jj[q]));
                }
            double sq[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) sq[q] = sel[q] ? __dsqrt_rn(d64[q]) : 0.0;
            double s8 = 0.0, s6 = 0.0;
            for (int r = 0; r < N; ++r) {
                double v = 0.0;
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const unsigned bb = __ballot_sync(0xffffffffu, sel[q] && er[q] == r);
                    if (bb) v = __shfl_sync(0xffffffffu, sq[q], __ffs(bb) - 1);
                }
                if (test == 0 || r < 8) s8 = __dadd_rn(s8, v);
                else s6 = __dadd_rn(s6, v);
            }
            const double rc = test == 0 ? __dmul_rn(f, __ddiv_rn(s8, 12.0))
                                        : __dmul_rn(f, __ddiv_rn(__dadd_rn(__dmul_rn(c, s8), s6), 14.0));
            rc2 = __dmul_rn(rc, rc);
            if (test == 0) rc12 = rc;
            else rc14 = rc;
        };
        if (rcut) exact_cutoff();
        __syncwarp();
        // bonds among the N selected (bit b of s_A[a]: a and b closer than
        // rc): FP32 against the FP32 cutoff outside a band that covers both
        // errors, the FP64 test against the exact cutoff inside it
        // (each pair tested once, both bits set: lane a takes the pairs
        // (a, a + o mod N), o = 1 .. N/2, o = N/2 only for a < N/2)
        const float bandb = 2e-5f * rc2f + 1e-6f;
        if (lane < N) s_A[w][lane] = 0u;
        __syncwarp();
        unsigned m = 0u, und = 0u;
        if (lane < N) {
            const int4 xa = s_x[w][lane];
            const int half = N >> 1, last = lane >= half ? half - 1 : half;  // N is even
            for (int o = 1; o <= last; ++o) {
                const int b = lane + o < N ? lane + o : lane + o - N;
                const int4 xb = s_x[w][b];
                const float dx = fixed_delta((uint32_t)xa.x, (uint32_t)xb.x, S.sx[0]);
                const float dy = fixed_delta((uint32_t)xa.y, (uint32_t)xb.y, S.sx[1]);
                const float dz = fixed_delta((uint32_t)xa.z, (uint32_t)xb.z, S.sx[2]);
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                if (r2 < rc2f - bandb) {
                    m |= 1u << b;
                    atomicOr(&s_A[w][b], 1u << lane);
                } else if (r2 <= rc2f + bandb) {
                    und |= 1u << b;
                }
            }
        }
        if (__any_sync(0xffffffffu, und != 0u)) {
            if (!rcut) exact_cutoff();
            if (lane < N) {
                const double *pa = pos64 + 3 * (int64_t)s_j[w][lane];
                for (unsigned u = und; u; u &= u - 1) {
                    const int b = __ffs(u) - 1;
                    double dr[3];
                    if (min_image_r2(pa, pos64 + 3 * (int64_t)s_j[w][b], S, dr) < rc2) {
                        m |= 1u << b;
                        atomicOr(&s_A[w][b], 1u << lane);
                    }
                }
            }
        }
        if (lane < N) atomicOr(&s_A[w][lane], m);
        __syncwarp();
        int c421 = 0, c422 = 0, c444 = 0, c666 = 0;
        if (lane < N) {
            const unsigned C = s_A[w][lane];
            const int ncn = __popc(C);
            int twice_nb = 0;
            for (unsigned r = C; r; r &= r - 1) twice_nb += __popc(s_A[w][__ffs(r) - 1] & C);
            int best = 0;
            unsigned rest = C;
            while (rest) {
                unsigned comp = rest & (~rest + 1u), frontier = comp;
                while (frontier) {
                    unsigned grow = 0u;
                    for (unsigned fr = frontier; fr; fr &= fr - 1) grow |= s_A[w][__ffs(fr) - 1];
                    grow &= C & ~comp;
                    comp |= grow;
                    frontier = grow;
                }
                int twice_e = 0;
                for (unsigned fr = comp; fr; fr &= fr - 1) twice_e += __popc(s_A[w][__ffs(fr) - 1] & comp);
                best = max(best, twice_e >> 1);
                rest &= ~comp;
            }
            const uint32_t t = ((uint32_t)ncn << 16) | ((uint32_t)(twice_nb >> 1) << 8) | (uint32_t)best;
            c421 = t == ((4u << 16) | (2u << 8) | 1u);
            c422 = t == ((4u << 16) | (2u << 8) | 2u);
            c444 = t == ((4u << 16) | (4u << 8) | 4u);
            c666 = t == ((6u << 16) | (6u << 8) | 6u);
        }
        c421 = __reduce_add_sync(0xffffffffu, c421);
        c422 = __reduce_add_sync(0xffffffffu, c422);
        c444 = __reduce_add_sync(0xffffffffu, c444);
        c666 = __reduce_add_sync(0xffffffffu, c666);
        if (test == 0) {
            if (c421 == 12) lab = PPMD_FCC;
            else if (c421 == 6 && c422 == 6) lab = PPMD_HCP;
        } else if (c666 == 8 && c444 == 6) {
            lab = PPMD_BCC;
        }
        __syncwarp();
    }
    if (lane == 0) {
        label[o] = lab;
        if (rcut) {
            rcut[2 * o] = rc12;
            rcut[2 * o + 1] = rc14;
        }
    }
}

int acna_launch(ppmd_ctx *ctx, int64_t n, const int4 *xq, const double *pos64, const SegTable &st, const int32_t *nbr,
                const int32_t *cnt, int32_t max_nbr, int64_t ld, const int32_t *out_idx, int8_t *label, double *rcut) {
    const double f = (1.0 + sqrt(2.0)) * 0.5, c = 2.0 / sqrt(3.0);
    if (n > 0)
        PPMD_LAUNCH(ctx, k_acna, div_up(n, ACNA_WARPS), ACNA_WARPS * 32, 0, n, xq, pos64, st, nbr, cnt, max_nbr,
                    ld ? 1 : (int64_t)max_nbr, ld ? ld : 1, f, c, out_idx, label, rcut, ctx->d_status, ctx->d_needed);
    return check_launch(ctx, "acna");
}

// A list entry, read once per analysis: not kept in L1, which then holds
// the neighbour positions.
__device__ __forceinline__ int32_t ld_once_i32(const int32_t *p) {
    int32_t v;
    asm("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// Q4, Q5, Q6 of the integrator's atoms (the on-the-fly analysis of
// Sec. 5.2) over its column-major list W[m * ld + i], bonds r < r_cut:
// per atom into q3 [3][n] at out_idx[i] (the caller's order) and per block
// the three sums into partials[3 * block + l - 4] (FP64).
constexpr int BOA_OTF_BLOCK = 128;

__global__ void __launch_bounds__(BOA_OTF_BLOCK) k_boa_otf(int64_t n, const int4 *__restrict__ xq,
                                                           const double *__restrict__ pos64, SegTable st,
                                                           const int32_t *__restrict__ W,
                                                           const int32_t *__restrict__ cnt, int32_t max_nbr,
                                                           int64_t ld, double rc2, float rc2_lo, float rc2_hi,
                                                           YlmCoef K, const int32_t *__restrict__ out_idx,
                                                           float *__restrict__ q3, double *__restrict__ partials) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float qs[3] = {0.0f, 0.0f, 0.0f};
    if (i < n) {
        const int4 xi = xq[i];
        const Seg &S = seg_ref(st, xi.w);
        float r4[5], i4[5], r5[6], i5[6], r6[7], i6[7];
#pragma unroll
        for (int m = 0; m < 7; ++m) {
            if (m < 5) r4[m] = i4[m] = 0.0f;
            if (m < 6) r5[m] = i5[m] = 0.0f;
            r6[m] = i6[m] = 0.0f;
        }
        const int32_t deg = min(cnt[i], max_nbr);
        int32_t nu = 0;
        // four entries per pass: their list words and positions are loaded
        // together, so four loads are in flight per thread
        for (int32_t k0 = 0; k0 < deg; k0 += 4) {
            int32_t jv[4];
            int4 xv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) jv[q] = k0 + q < deg ? ld_once_i32(W + (int64_t)(k0 + q) * ld + i) : (int32_t)i;
#pragma unroll
            for (int q = 0; q < 4; ++q) xv[q] = __ldg(&xq[jv[q]]);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (k0 + q >= deg) break;
                const float dx = fixed_delta((uint32_t)xi.x, (uint32_t)xv[q].x, S.sx[0]);
                const float dy = fixed_delta((uint32_t)xi.y, (uint32_t)xv[q].y, S.sx[1]);
                const float dz = fixed_delta((uint32_t)xi.z, (uint32_t)xv[q].z, S.sx[2]);
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                bool in = r2 < rc2_lo;
                if (!in && r2 < rc2_hi) {
                    double dr[3];
                    in = min_image_r2(pos64 + 3 * i, pos64 + 3 * (int64_t)jv[q], S, dr) < rc2;
                }
                if (!in) continue;
                const float ir = rsqrtf(r2);
                boa_moments<true>(K, dx * ir, dy * ir, dz * ir, r4, i4, r5, i5, r6, i6);
                ++nu;
            }
        }
        float s4 = 0.0f, s5 = 0.0f, s6 = 0.0f;
#pragma unroll
        for (int m = 0; m < 7; ++m) {
            if (m < 5) s4 = fmaf(r4[m], r4[m], fmaf(i4[m], i4[m], s4));
            if (m < 6) s5 = fmaf(r5[m], r5[m], fmaf(i5[m], i5[m], s5));
            s6 = fmaf(r6[m], r6[m], fmaf(i6[m], i6[m], s6));
        }
        const float inv = nu > 0 ? 1.0f / (float)nu : 0.0f;
        const float Q4 = sqrtf(s4) * inv, Q5 = sqrtf(s5) * inv, Q6 = sqrtf(s6) * inv;
        const int64_t o = out_idx ? out_idx[i] : i;
        q3[o] = Q4;
        q3[n + o] = Q5;
        q3[2 * n + o] = Q6;
        qs[0] = Q4;
        qs[1] = Q5;
        qs[2] = Q6;
    }
    // warp sums in FP32 (32 values of order one), block and grid sums in
    // FP64 (FP64 arithmetic on every lane is slow on this part)
    __shared__ double sh[3][BOA_OTF_BLOCK / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        float v = qs[l];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sh[l][w] = (double)v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double v = 0.0;
        for (int q = 0; q < BOA_OTF_BLOCK / 32; ++q) v += sh[threadIdx.x][q];
        partials[3 * blockIdx.x + threadIdx.x] = v;
    }
}

int64_t boa_otf_blocks(int64_t n) { return div_up(n, BOA_OTF_BLOCK); }

int boa_otf_launch(ppmd_ctx *ctx, int64_t n, const int4 *xq, const double *pos64, const SegTable &st, const int32_t *W,
                   const int32_t *cnt, int32_t max_nbr, int64_t ld, double r_cut, double Lmax, const int32_t *out_idx,
                   float *q3, double *partials) {
    static const YlmCoef K = make_coef();
    float lo, hi;
    cutoff_band(r_cut * r_cut, Lmax, &lo, &hi);
    if (n > 0)
        PPMD_LAUNCH(ctx, k_boa_otf, boa_otf_blocks(n), BOA_OTF_BLOCK, 0, n, xq, pos64, st, W, cnt, max_nbr, ld,
                    r_cut * r_cut, lo, hi, K, out_idx, q3, partials);
    return check_launch(ctx, "boa_otf");
}

int boa_launch(ppmd_ctx *ctx, int64_t n, const int4 *xq, const double *pos64, const SegTable &st, const int32_t *nbr,
               const int32_t *cnt, int32_t max_nbr, int64_t ld, double r_cut, double Lmax, const int32_t *out_idx, float *q4,
               float *q6, int32_t *nnb) {
    static const YlmCoef K = make_coef();
    float lo, hi;
    cutoff_band(r_cut * r_cut, Lmax, &lo, &hi);
    if (n > 0)
        PPMD_LAUNCH(ctx, k_boa, div_up(n, 256), 256, 0, n, xq, pos64, st, nbr, cnt, max_nbr, ld ? 1 : (int64_t)max_nbr,
                    ld ? ld : 1, r_cut * r_cut, lo, hi, K, out_idx,
                    q4, q6, nnb);
    return check_launch(ctx, "boa");
}

// Structure by bond order within a tolerance (Sec. 4.1: Q_l compared with
// the perfect-lattice values of the table of Q4, Q5, Q6, "within some
// tolerance"): the lattice whose (Q4, Q6) of that table is nearest in the
// plane, in the order fcc, hcp, bcc on ties, if its distance is below tol;
// else other.  dist (may be null): that smallest distance.
__global__ void k_boa_tolerance(int64_t n, const float *__restrict__ q4, const float *__restrict__ q6, float tol,
                                int8_t *__restrict__ label, float *__restrict__ dist) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // (Q4, Q6) of perfect fcc, hcp and bcc as the table prints them
    const float ref4[3] = {0.191f, 0.097f, 0.036f}, ref6[3] = {0.575f, 0.485f, 0.511f};
    const int8_t code[3] = {1, 2, 3};
    const float a = q4[i], b = q6[i];
    float best = 3.4e38f;
    int8_t lab = 0;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        const float d4 = a - ref4[s], d6 = b - ref6[s];
        const float d2 = fmaf(d4, d4, d6 * d6);
        if (d2 < best) {
            best = d2;
            lab = code[s];
        }
    }
    const float d = sqrtf(best);
    label[i] = d < tol ? lab : (int8_t)0;
    if (dist) dist[i] = d;
}

int boa_tolerance_launch(ppmd_ctx *ctx, int64_t n, const float *q4, const float *q6, float tol, int8_t *label,
                         float *dist) {
    if (n > 0) PPMD_LAUNCH(ctx, k_boa_tolerance, div_up(n, 256), 256, 0, n, q4, q6, tol, label, dist);
    return check_launch(ctx, "boa_tolerance");
}

int cna_launch(ppmd_ctx *ctx, int64_t n, const int4 *xq, const double *pos64, const SegTable &st, const int32_t *nbr,
               const int32_t *cnt, int32_t max_nbr, int64_t ld, double r_cut, double Lmax, const int32_t *out_idx, uint32_t *trip,
               int8_t *label) {
    float lo, hi;
    cutoff_band(r_cut * r_cut, Lmax, &lo, &hi);
    if (n > 0)
        PPMD_LAUNCH(ctx, k_cna, div_up(n, CNA_GROUPS), CNA_WARPS * 32, 0, n, xq, pos64, st, nbr, cnt, max_nbr,
                    ld ? 1 : (int64_t)max_nbr, ld ? ld : 1, r_cut * r_cut,
                    lo, hi, out_idx, trip, label, ctx->d_status, ctx->d_needed, nullptr, nullptr);
    return check_launch(ctx, "cna");
}

int cna_subset_launch(ppmd_ctx *ctx, int64_t m_max, const int32_t *m_dev, const int32_t *which, const int4 *xq,
                      const double *pos64, const SegTable &st, const int32_t *nbr, const int32_t *cnt, int32_t max_nbr,
                      int64_t ld, double r_cut, double Lmax, const int32_t *out_idx, int8_t *label) {
    float lo, hi;
    cutoff_band(r_cut * r_cut, Lmax, &lo, &hi);
    // a grid of a few blocks per SM strides over however many atoms the
    // device chose
    const int64_t grid = std::min<int64_t>(div_up(m_max, CNA_GROUPS), 148 * 8);
    if (m_max > 0)
        PPMD_LAUNCH(ctx, k_cna, grid, CNA_WARPS * 32, 0, m_max, xq, pos64, st, nbr, cnt, max_nbr,
                    ld ? 1 : (int64_t)max_nbr, ld ? ld : 1, r_cut * r_cut,
                    lo, hi, out_idx, nullptr, label, ctx->d_status, ctx->d_needed, which, m_dev);
    return check_launch(ctx, "cna_subset");
}


// ---------------------------------------------------------------------
// Local-environment features of the learned classifier, eight lanes per
// atom.  With nu bonds (r < r_feat) of unit vectors u_a and lengths d_a,
// and the nbd bonded neighbours (r < r_ref) at r_i - r_j = v_a:
//   f[0], f[1]   Q4, Q6 (as k_boa);
//   f[2..15]     the 14 smallest d_a, ascending, as (d_a - r_ref) / (r_feat - r_ref)
//                (missing: 1);
//   f[16..29]    histogram of the chords |v_a - v_b| over the pairs a < b of
//                bonded neighbours: 14 bins of width 0.05 centred at
//                r_ref - 0.35 + 0.05 (k + 1/2), linear weights between bin
//                centres (clamped at both ends), divided by 24.
// Output: f32 [n][30] and/or bf16 [n][32] (f[30], f[31] = 0).
// ---------------------------------------------------------------------
constexpr int FEAT_WARPS = 4, FEAT_G = 8, FEAT_GROUPS = FEAT_WARPS * 32 / FEAT_G, FEAT_CAP = 64, FEAT_PF = 3;

__global__ void __launch_bounds__(FEAT_WARPS * 32, 8) k_features(int64_t n, const int4 *__restrict__ xq,
                                                                 const double *__restrict__ pos64, SegTable st,
                                                                 const int32_t *__restrict__ nbr,
                                                                 const int32_t *__restrict__ cnt, int32_t max_nbr,
                                                                 int64_t si, int64_t sm, double rc2, float lo, float hi,
                                                                 double rb2, float blo, float bhi, float r_ref,
                                                                 float inv_span, YlmCoef K,
                                                                 const int32_t *__restrict__ out_idx,
                                                                 float *__restrict__ f32, __nv_bfloat16 *__restrict__ fb16,
                                                                 int32_t *status, unsigned long long *needed) {
    // The bonds of each group as (v_a, d_a), one 16-byte entry each (the
    // eight lanes of a group read eight entries in one conflict-free phase):
    // the bonded neighbours (r < r_ref) from the front, the other bonds from
    // the back.
    __shared__ float4 s_e[FEAT_GROUPS][FEAT_CAP];
    __shared__ float s_h[15][FEAT_WARPS * 32];  // private histogram of each lane, bin-major (no bank conflicts); row 14 a guard
    __shared__ float s_f[FEAT_GROUPS][32];
    const int gl = threadIdx.x & (FEAT_G - 1), g = threadIdx.x / FEAT_G, shift = threadIdx.x & 31 & ~(FEAT_G - 1);
    const unsigned gmask = 0xffu << shift;
    const int64_t i = (int64_t)blockIdx.x * FEAT_GROUPS + g;
    if (i >= n) return;  // whole groups leave together
    const int4 xi = xq[i];
    const Seg &S = seg_ref(st, xi.w);
    const int32_t deg = min(cnt[i], max_nbr);
    const int32_t *row = nbr + i * si;
    const int64_t o = out_idx ? out_idx[i] : i;
    const unsigned lt = (1u << gl) - 1u;
    float *hist = &s_h[0][threadIdx.x];  // bin k at hist[k * FEAT_WARPS * 32]
#pragma unroll
    for (int k = 0; k < 15; ++k) hist[k * FEAT_WARPS * 32] = 0.0f;
#pragma unroll
    for (int c = gl; c < 32; c += FEAT_G) s_f[g][c] = (c >= 2 && c < 16) ? 1.0f : 0.0f;
    int32_t nu = 0, nbd = 0;  // bonds, bonded neighbours among them
    // FEAT_PF list entries per lane in flight (one round trip for up to
    // FEAT_G * FEAT_PF neighbours), then taken in list order
    for (int32_t base0 = 0; base0 < deg; base0 += FEAT_G * FEAT_PF) {
        int32_t jj[FEAT_PF];
        int4 xx[FEAT_PF];
#pragma unroll
        for (int u = 0; u < FEAT_PF; ++u) {
            const int32_t k = base0 + u * FEAT_G + gl;
            jj[u] = k < deg ? row[k * sm] : -1;
        }
#pragma unroll
        for (int u = 0; u < FEAT_PF; ++u) xx[u] = jj[u] >= 0 ? xq[jj[u]] : make_int4(0, 0, 0, 0);
#pragma unroll
        for (int u = 0; u < FEAT_PF; ++u) {
            if (base0 + u * FEAT_G >= deg) break;  // (uniform over the group)
            const int32_t j = jj[u];
            bool b = false, bb = false;
            float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 0.f;
            if (j >= 0) {
                const int4 xj = xx[u];
                dx = fixed_delta((uint32_t)xi.x, (uint32_t)xj.x, S.sx[0]);
                dy = fixed_delta((uint32_t)xi.y, (uint32_t)xj.y, S.sx[1]);
                dz = fixed_delta((uint32_t)xi.z, (uint32_t)xj.z, S.sx[2]);
                r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                double r2x = -1.0;  // exact r^2 when needed
                b = r2 < lo;
                if (!b && r2 < hi) {
                    double dr[3];
                    r2x = min_image_r2(pos64 + 3 * i, pos64 + 3 * (int64_t)j, S, dr);
                    b = r2x < rc2;
                }
                bb = r2 < blo;
                if (!bb && r2 < bhi) {
                    if (r2x < 0.0) {
                        double dr[3];
                        r2x = min_image_r2(pos64 + 3 * i, pos64 + 3 * (int64_t)j, S, dr);
                    }
                    bb = r2x < rb2;
                }
                bb = bb && b;
            }
            const unsigned ball = __ballot_sync(gmask, b) >> shift, bbal = __ballot_sync(gmask, bb) >> shift;
            if (b) {
                const float ir = rsqrtf(r2), r = r2 * ir;  // hardware estimates (~2 ulp)
                const int32_t a = bb ? nbd + __popc(bbal & lt) : FEAT_CAP - 1 - (nu - nbd) - __popc(ball & ~bbal & lt);
                if (a >= 0 && a < FEAT_CAP) s_e[g][a] = make_float4(dx, dy, dz, r);
            }
            nu += __popc(ball);
            nbd += __popc(bbal);
        }
    }
    if (nu > FEAT_CAP) {
        if (gl == 0) {
            latch_status(status, PPMD_ERR_CAPACITY);
            latch_needed(needed, (unsigned long long)nu);
        }
        nbd = min(nbd, FEAT_CAP);
        nu = FEAT_CAP;  // (entries overwritten; the call reports the error)
    }
    const int32_t back = FEAT_CAP - nu;  // bond number q >= nbd is at back + q
    __syncwarp(gmask);
    // Q4, Q6: each lane its bonds; unit vectors from the same r^2 and
    // reciprocal root as the stored length
    float r4[5], i4[5], r6[7], i6[7];
#pragma unroll
    for (int m = 0; m < 7; ++m) {
        if (m < 5) r4[m] = i4[m] = 0.0f;
        r6[m] = i6[m] = 0.0f;
    }
    for (int q = gl; q < nu; q += FEAT_G) {
        const float4 e = s_e[g][q < nbd ? q : back + q];
        const float ir = rsqrtf(fmaf(e.x, e.x, fmaf(e.y, e.y, e.z * e.z)));
        boa_accumulate(K, e.x * ir, e.y * ir, e.z * ir, r4, i4, r6, i6);
    }
    // group sums of the 22 moments (the imaginary parts of m = 0 vanish):
    // reduce-scatter over the eight lanes, lane gl ends with moments
    // 3 gl .. 3 gl + 2 of the list r4[0..4] i4[1..4] r6[0..6] i6[1..6] 0 0
    float v[24];
#pragma unroll
    for (int m = 0; m < 5; ++m) v[m] = r4[m];
#pragma unroll
    for (int m = 1; m < 5; ++m) v[4 + m] = i4[m];
#pragma unroll
    for (int m = 0; m < 7; ++m) v[9 + m] = r6[m];
#pragma unroll
    for (int m = 1; m < 7; ++m) v[15 + m] = i6[m];
    v[22] = v[23] = 0.0f;
#pragma unroll
    for (int h = 12; h >= 3; h >>= 1) {
        const bool up = (gl & (h / 3)) != 0;
#pragma unroll
        for (int k = 0; k < h; ++k) {
            const float keep = up ? v[k + h] : v[k], send = up ? v[k] : v[k + h];
            v[k] = keep + __shfl_xor_sync(gmask, send, h / 3);
        }
    }
    float s4 = 0.0f, s6 = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int idx = 3 * gl + k;
        const float sq = v[k] * v[k];
        if (idx < 9) s4 += sq;
        else s6 += sq;
    }
#pragma unroll
    for (int o = FEAT_G / 2; o > 0; o >>= 1) {
        s4 += __shfl_xor_sync(gmask, s4, o);
        s6 += __shfl_xor_sync(gmask, s6, o);
    }
    // chord histogram: the nbd (nbd - 1) / 2 pairs spread over the lanes,
    // tent weights added to the lane's own row
    const int npair = nbd * (nbd - 1) / 2;
    const float hlo = r_ref - 0.35f;
    // pair (a, b), a < b, numbered pidx = b (b - 1) / 2 + a: the lane's next
    // pair (pidx + FEAT_G) by carrying a into b
    int pa = gl, pb = 1;
    while (pa >= pb) {
        pa -= pb;
        ++pb;
    }
    for (int pidx = gl; pidx < npair; pidx += FEAT_G) {
        const float4 va = s_e[g][pa], vb = s_e[g][pb];
        pa += FEAT_G;
        while (pa >= pb) {
            pa -= pb;
            ++pb;
        }
        const float cx = va.x - vb.x, cy = va.y - vb.y, cz = va.z - vb.z;
        const float c2 = fmaxf(fmaf(cx, cx, fmaf(cy, cy, cz * cz)), 1e-30f);
        const float chord = c2 * rsqrtf(c2);
        // position among the bin centres, clamped to [0, 13]: a chord beyond
        // either end puts weight 1 on the end bin and 0 on its neighbour (the
        // guard row beyond bin 13)
        const float x = fminf(fmaxf((chord - hlo) * 20.0f - 0.5f, 0.0f), 13.0f);
        const float fl = floorf(x);
        const float t = x - fl;
        float *h0 = hist + (int)fl * (FEAT_WARPS * 32);
        h0[0] += 1.0f - t;
        h0[FEAT_WARPS * 32] += t;
    }
    // sorted bond lengths: the rank of each (ties ordered by slot), two
    // bonds per lane per pass over the others
    for (int q = gl; q < nu; q += 2 * FEAT_G) {
        const int q2 = q + FEAT_G;
        const int a1 = q < nbd ? q : back + q, a2 = q2 < nbd ? q2 : back + q2;
        const float d1 = s_e[g][a1].w, d2 = q2 < nu ? s_e[g][a2].w : 3.4e38f;
        int rank1 = 0, rank2 = 0;
        for (int c = 0; c < nu; ++c) {
            const int sl = c < nbd ? c : back + c;
            const float dc = s_e[g][sl].w;
            rank1 += (dc < d1) || (dc == d1 && sl < a1);
            rank2 += (dc < d2) || (dc == d2 && sl < a2);
        }
        if (rank1 < 14) s_f[g][2 + rank1] = (d1 - r_ref) * inv_span;
        if (q2 < nu && rank2 < 14) s_f[g][2 + rank2] = (d2 - r_ref) * inv_span;
    }
    __syncwarp(gmask);
    for (int c = gl; c < 14; c += FEAT_G) {
        // lanes start at different rows of the group (distinct banks); each
        // bin is always summed in the same order
        float acc = 0.0f;
#pragma unroll
        for (int l = 0; l < FEAT_G; ++l) acc += s_h[c][g * FEAT_G + ((l + gl) & (FEAT_G - 1))];
        s_f[g][16 + c] = acc * (1.0f / 24.0f);
    }
    if (gl == 0) {
        const float inv = nu > 0 ? 1.0f / (float)nu : 0.0f;
        s_f[g][0] = sqrtf(s4) * inv;
        s_f[g][1] = sqrtf(s6) * inv;
    }
    __syncwarp(gmask);
    const float4 fv = make_float4(s_f[g][4 * gl], s_f[g][4 * gl + 1], s_f[g][4 * gl + 2], s_f[g][4 * gl + 3]);
    if (f32) {
        float *dst = f32 + o * 30 + 4 * gl;
        dst[0] = fv.x;
        dst[1] = fv.y;
        if (gl < 7) {
            dst[2] = fv.z;
            dst[3] = fv.w;
        }
    }
    if (fb16) {
        const __nv_bfloat162 lo2 = __floats2bfloat162_rn(fv.x, fv.y), hi2 = __floats2bfloat162_rn(fv.z, fv.w);
        uint2 w2;
        w2.x = *reinterpret_cast<const uint32_t *>(&lo2);
        w2.y = *reinterpret_cast<const uint32_t *>(&hi2);
        *reinterpret_cast<uint2 *>(fb16 + o * 32 + 4 * gl) = w2;
    }
}

int features_launch(ppmd_ctx *ctx, int64_t n, const int4 *xq, const double *pos64, const SegTable &st,
                    const int32_t *nbr, const int32_t *cnt, int32_t max_nbr, int64_t ld, double r_feat, double r_ref,
                    double Lmax, const int32_t *out_idx, float *f32, __nv_bfloat16 *fb16) {
    static const YlmCoef K = make_coef();
    float lo, hi, blo, bhi;
    cutoff_band(r_feat * r_feat, Lmax, &lo, &hi);
    cutoff_band(r_ref * r_ref, Lmax, &blo, &bhi);
    if (n > 0)
        PPMD_LAUNCH(ctx, k_features, div_up(n, FEAT_GROUPS), FEAT_WARPS * 32, 0, n, xq, pos64, st, nbr, cnt, max_nbr,
                    ld ? 1 : (int64_t)max_nbr, ld ? ld : 1, r_feat * r_feat, lo, hi, r_ref * r_ref, blo, bhi, (float)r_ref, (float)(1.0 / (r_feat - r_ref)), K, out_idx, f32, fb16,
                    ctx->d_status, ctx->d_needed);
    return check_launch(ctx, "features");
}

// ---------------------------------------------------------------------
// Pipeline: sort by cell, list at r_list, analyses, results in caller order.
// ---------------------------------------------------------------------
// Sorted copies: positions and fixed-point words of the atoms perm[k].
__global__ void k_gather_pos_xq(int64_t n, const int32_t *__restrict__ perm, const double *__restrict__ pos,
                                const int4 *__restrict__ xq, double *__restrict__ pos_o, int4 *__restrict__ xq_o) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t o = perm[k];
    pos_o[3 * k] = pos[3 * o];
    pos_o[3 * k + 1] = pos[3 * o + 1];
    pos_o[3 * k + 2] = pos[3 * o + 2];
    xq_o[k] = xq[o];
}

int32_t snapshot_capacity(int64_t n, const ppmd_box *box, double r_list) {
    // 1.6 times the mean count within r_list plus 16, at least 48: an overflow
    // needs a local density far above the box's
    const double vol = box->L[0] * box->L[1] * box->L[2];
    const double mean = vol > 0 ? 4.18879020478639 * r_list * r_list * r_list * (double)n / vol : 0.0;
    const int64_t cap = ((int64_t)ceil(1.6 * mean + 16.0) + 15) / 16 * 16;
    return (int32_t)std::min<int64_t>(std::max<int64_t>(cap, 48), 1 << 20);
}

int end_pipeline(ppmd_ctx *ctx, int attempt, int32_t &max_nbr, int32_t *aux) {
    int64_t need = 0;
    const int rc = status_sync(ctx, &need, aux);
    if (rc == PPMD_ERR_CAPACITY && attempt == 0 && need > max_nbr) {
        max_nbr = (int32_t)((need + 15) / 16 * 16);
        return PIPELINE_RETRY;
    }
    return rc;
}

int sorted_snapshot(ppmd_ctx *ctx, const double *pos, int64_t n, const ppmd_box *box, double r_list, int32_t max_nbr,
                    Snapshot &s) {
    s.n = n;
    s.st.d = nullptr;
    s.st.nseg = 1;
    PPMD_TRY(make_seg(ctx, s.st.one, box->L, r_list, r_list));
    s.st.one.atom0 = 0;
    s.st.one.atom1 = n;
    s.Lmax = fmax(box->L[0], fmax(box->L[1], box->L[2]));
    const int64_t ncell = (int64_t)s.st.one.nc[0] * s.st.one.nc[1] * s.st.one.nc[2];
    const size_t nn = (size_t)(n > 0 ? n : 1);
    int32_t *cell0 = (int32_t *)scratch(ctx, S_CELLS0, sizeof(int32_t) * nn);
    s.cell_start = (int32_t *)scratch(ctx, S_CELLS1, sizeof(int32_t) * (size_t)(ncell + 1));
    s.perm = (int32_t *)scratch(ctx, S_CELLS2, sizeof(int32_t) * nn);
    s.pos = (double *)scratch(ctx, S_SORTPOS, sizeof(double) * 3 * nn);
    s.xq = (int4 *)scratch(ctx, S_AUX0, sizeof(int4) * nn);
    if (!cell0 || !s.cell_start || !s.perm || !s.pos || !s.xq) return PPMD_ERR_NOMEM;
    // one segment: bricks are cut from the grid inside the kernel
    s.st.one.atom1 = n;
    const BrickShape shape = brick_shape(s.st.one);
    const int64_t nbricks = brick_count(s.st.one, shape);
    // fixed point in the caller's order (positions need not be wrapped), bin
    // and sort by cell on the fixed-point words, gather both copies
    int4 *xq_c = (int4 *)scratch(ctx, S_XQ, sizeof(int4) * nn);
    if (!xq_c) return PPMD_ERR_NOMEM;
    PPMD_TRY(prep_fixed(ctx, pos, n, s.st, nullptr, xq_c, nullptr));
    PPMD_TRY(bin_atoms_fixed(ctx, xq_c, n, s.st, ncell, cell0, s.cell_start, s.perm));
    if (n > 0) PPMD_LAUNCH(ctx, k_gather_pos_xq, div_up(n, 256), 256, 0, n, s.perm, pos, xq_c, s.pos, s.xq);
    s.ld = (n + 31) / 32 * 32;
    PPMD_TRY(neigh_brick_setup(ctx, max_nbr));
    s.max_nbr = max_nbr;
    s.nbr = (int32_t *)scratch(ctx, S_NBR, sizeof(int32_t) * (size_t)s.ld * (size_t)max_nbr);
    s.cnt = (int32_t *)scratch(ctx, S_NBRCNT, sizeof(int32_t) * nn);
    if (!s.nbr || !s.cnt) return PPMD_ERR_NOMEM;
    PPMD_TRY(build_list_bricks(ctx, nbricks, nullptr, shape, s.xq, s.pos, s.st, s.cell_start, s.nbr, s.ld, s.cnt,
                               max_nbr, brick_stage_cap(s.st.one, shape)));
    return PPMD_OK;
}

__global__ void k_seg_of(int64_t n, const int64_t *__restrict__ off, int32_t nbox, int32_t *__restrict__ seg_of) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t lo = 0, hi = nbox - 1;  // the last box with off[b] <= i
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (off[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        seg_of[i] = lo;
    }
}

int check_boxes(ppmd_ctx *ctx, int64_t nbox, const int64_t *atom_off, const ppmd_box *boxes, const char *who) {
    if (nbox < 1 || nbox >= ((int64_t)1 << 31) || !atom_off || !boxes)
        return set_error(ctx, PPMD_ERR_INVALID, "%s: bad box set", who);
    if (atom_off[0] != 0) return set_error(ctx, PPMD_ERR_INVALID, "%s: atom_off[0] must be 0", who);
    for (int64_t b = 0; b < nbox; ++b)
        if (atom_off[b + 1] < atom_off[b]) return set_error(ctx, PPMD_ERR_INVALID, "%s: atom_off decreases at %lld", who, (long long)b);
    if (atom_off[nbox] >= (int64_t)1 << 31) return set_error(ctx, PPMD_ERR_INVALID, "%s: too many atoms", who);
    return PPMD_OK;
}

int32_t snapshot_capacity_boxes(int64_t nbox, const int64_t *atom_off, const ppmd_box *boxes, double r_list) {
    int32_t cap = 0;
    for (int64_t b = 0; b < nbox; ++b)
        cap = std::max(cap, snapshot_capacity(atom_off[b + 1] - atom_off[b], &boxes[b], r_list));
    return cap;
}

int sorted_snapshot_boxes(ppmd_ctx *ctx, const double *pos, int64_t nbox, const int64_t *atom_off,
                          const ppmd_box *boxes, double r_list, int32_t max_nbr, Snapshot &s) {
    if (nbox == 1) return sorted_snapshot(ctx, pos, atom_off[1], boxes, r_list, max_nbr, s);
    const int64_t n = atom_off[nbox];
    s.n = n;
    std::vector<Seg> segs((size_t)nbox);
    int64_t ncell = 0;
    double Lmax = 0;
    for (int64_t b = 0; b < nbox; ++b) {
        Seg &S = segs[(size_t)b];
        PPMD_TRY(make_seg(ctx, S, boxes[b].L, r_list, r_list));
        S.cell0 = (int32_t)ncell;
        S.atom0 = atom_off[b];
        S.atom1 = atom_off[b + 1];
        ncell += (int64_t)S.nc[0] * S.nc[1] * S.nc[2];
        if (ncell >= (int64_t)1 << 31) return set_error(ctx, PPMD_ERR_BOX, "too many cells");
        for (int d = 0; d < 3; ++d) Lmax = fmax(Lmax, boxes[b].L[d]);
    }
    s.Lmax = Lmax;
    std::vector<Brick> bl;
    const int32_t stage_cap = make_bricks(segs, bl);
    const size_t nn = (size_t)(n > 0 ? n : 1);
    Seg *d_segs = (Seg *)scratch(ctx, S_SEGS, sizeof(Seg) * (size_t)nbox);
    int64_t *d_off = (int64_t *)scratch(ctx, S_SEGOFF, sizeof(int64_t) * (size_t)(nbox + 1));
    int32_t *seg_of = (int32_t *)scratch(ctx, S_SEGOF, sizeof(int32_t) * nn);
    Brick *d_bricks = (Brick *)scratch(ctx, S_BRICKS, sizeof(Brick) * (bl.empty() ? 1 : bl.size()));
    int32_t *cell0 = (int32_t *)scratch(ctx, S_CELLS0, sizeof(int32_t) * nn);
    s.cell_start = (int32_t *)scratch(ctx, S_CELLS1, sizeof(int32_t) * (size_t)(ncell + 1));
    s.perm = (int32_t *)scratch(ctx, S_CELLS2, sizeof(int32_t) * nn);
    s.pos = (double *)scratch(ctx, S_SORTPOS, sizeof(double) * 3 * nn);
    s.xq = (int4 *)scratch(ctx, S_AUX0, sizeof(int4) * nn);
    if (!d_segs || !d_off || !seg_of || !d_bricks || !cell0 || !s.cell_start || !s.perm || !s.pos || !s.xq)
        return PPMD_ERR_NOMEM;
    // the three tables through the context's pinned staging buffer: the
    // copies queue behind the stream's work instead of waiting for it
    const size_t b_seg = sizeof(Seg) * (size_t)nbox, b_off = sizeof(int64_t) * (size_t)(nbox + 1),
                 b_brk = sizeof(Brick) * bl.size();
    const size_t o_off = (b_seg + 15) / 16 * 16, o_brk = o_off + (b_off + 15) / 16 * 16;
    char *h = (char *)stage_host(ctx, o_brk + b_brk);
    if (!h) return PPMD_ERR_NOMEM;
    memcpy(h, segs.data(), b_seg);
    memcpy(h + o_off, atom_off, b_off);
    if (b_brk) memcpy(h + o_brk, bl.data(), b_brk);
    cudaStream_t st = ctx->stream;
    PPMD_TRY(cuda_check(ctx, cudaMemcpyAsync(d_segs, h, b_seg, cudaMemcpyHostToDevice, st), "copy"));
    PPMD_TRY(cuda_check(ctx, cudaMemcpyAsync(d_off, h + o_off, b_off, cudaMemcpyHostToDevice, st), "copy"));
    if (b_brk) PPMD_TRY(cuda_check(ctx, cudaMemcpyAsync(d_bricks, h + o_brk, b_brk, cudaMemcpyHostToDevice, st), "copy"));
    PPMD_TRY(stage_done(ctx));
    s.st.d = d_segs;
    s.st.nseg = (int32_t)nbox;
    s.st.one = segs[0];
    if (n > 0) PPMD_LAUNCH(ctx, k_seg_of, div_up(n, 256), 256, 0, n, d_off, (int32_t)nbox, seg_of);
    // fixed point in the caller's order (the segment in .w), bin and sort by
    // cell on the fixed-point words (cells of box b follow those of box b -
    // 1, so the sorted atoms of box b keep the positions atom_off[b] ..
    // atom_off[b + 1] - 1), gather both copies
    int4 *xq_c = (int4 *)scratch(ctx, S_XQ, sizeof(int4) * nn);
    if (!xq_c) return PPMD_ERR_NOMEM;
    PPMD_TRY(prep_fixed(ctx, pos, n, s.st, seg_of, xq_c, nullptr));
    PPMD_TRY(bin_atoms_fixed(ctx, xq_c, n, s.st, ncell, cell0, s.cell_start, s.perm));
    if (n > 0) PPMD_LAUNCH(ctx, k_gather_pos_xq, div_up(n, 256), 256, 0, n, s.perm, pos, xq_c, s.pos, s.xq);
    s.ld = (n + 31) / 32 * 32;
    PPMD_TRY(neigh_brick_setup(ctx, max_nbr));
    s.max_nbr = max_nbr;
    s.nbr = (int32_t *)scratch(ctx, S_NBR, sizeof(int32_t) * (size_t)s.ld * (size_t)max_nbr);
    s.cnt = (int32_t *)scratch(ctx, S_NBRCNT, sizeof(int32_t) * nn);
    if (!s.nbr || !s.cnt) return PPMD_ERR_NOMEM;
    PPMD_TRY(build_list_bricks(ctx, (int64_t)bl.size(), d_bricks, BrickShape{1, 1, 1}, s.xq, s.pos, s.st, s.cell_start,
                               s.nbr, s.ld, s.cnt, max_nbr, stage_cap));
    return PPMD_OK;
}

}  // namespace ppmd

using namespace ppmd;

static int list_args_ok(ppmd_ctx *ctx, const double *pos, int64_t n, const ppmd_box *box, double r_cut, const int32_t *nbr,
                        const int32_t *cnt, int32_t max_nbr) {
    if (!ctx || !box || n < 0 || max_nbr < 0 || !(r_cut > 0)) return set_error(ctx, PPMD_ERR_INVALID, "bad argument");
    if (n > 0 && (!pos || !cnt || (max_nbr > 0 && !nbr))) return set_error(ctx, PPMD_ERR_INVALID, "null array");
    return PPMD_OK;
}

extern "C" int ppmd_boa_q46(ppmd_ctx *ctx, const double *pos, int64_t n, const ppmd_box *box, double r_cut,
                            const int32_t *nbr, const int32_t *nbr_count, int32_t max_nbr, float *q4, float *q6,
                            int32_t *n_nb) {
    PPMD_TRY(list_args_ok(ctx, pos, n, box, r_cut, nbr, nbr_count, max_nbr));
    cudaSetDevice(ctx->device);
    SegTable st;
    st.d = nullptr;
    st.nseg = 1;
    PPMD_TRY(make_seg(ctx, st.one, box->L, 0.0, r_cut));
    int4 *xq = (int4 *)scratch(ctx, S_XQ, sizeof(int4) * (size_t)(n > 0 ? n : 1));
    if (!xq) return PPMD_ERR_NOMEM;
    PPMD_TRY(prep_fixed(ctx, pos, n, st, nullptr, xq, nullptr));
    double Lmax = fmax(box->L[0], fmax(box->L[1], box->L[2]));
    return boa_launch(ctx, n, xq, pos, st, nbr, nbr_count, max_nbr, 0, r_cut, Lmax, nullptr, q4, q6, n_nb);
}

extern "C" int ppmd_cna(ppmd_ctx *ctx, const double *pos, int64_t n, const ppmd_box *box, double r_cut, const int32_t *nbr,
                        const int32_t *nbr_count, int32_t max_nbr, uint32_t *triplets, int8_t *label) {
    PPMD_TRY(list_args_ok(ctx, pos, n, box, r_cut, nbr, nbr_count, max_nbr));
    cudaSetDevice(ctx->device);
    SegTable st;
    st.d = nullptr;
    st.nseg = 1;
    PPMD_TRY(make_seg(ctx, st.one, box->L, 0.0, r_cut));
    int4 *xq = (int4 *)scratch(ctx, S_XQ, sizeof(int4) * (size_t)(n > 0 ? n : 1));
    if (!xq) return PPMD_ERR_NOMEM;
    PPMD_TRY(prep_fixed(ctx, pos, n, st, nullptr, xq, nullptr));
    double Lmax = fmax(box->L[0], fmax(box->L[1], box->L[2]));
    return cna_launch(ctx, n, xq, pos, st, nbr, nbr_count, max_nbr, 0, r_cut, Lmax, nullptr, triplets, label);
}

extern "C" int ppmd_analyze_boxes(ppmd_ctx *ctx, const double *pos, int64_t nbox, const int64_t *atom_off,
                                  const ppmd_box *boxes, double r_boa, double r_cna, float *q4, float *q6, int32_t *n_nb,
                                  int8_t *label) {
    if (!ctx) return PPMD_ERR_INVALID;
    PPMD_TRY(check_boxes(ctx, nbox, atom_off, boxes, "ppmd_analyze"));
    const int64_t n = atom_off[nbox];
    if (n > 0 && !pos) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_analyze: bad argument");
    const bool want_boa = q4 || q6 || n_nb;
    const bool want_cna = label != nullptr;
    if ((want_boa && !(r_boa > 0)) || (want_cna && !(r_cna > 0)))
        return set_error(ctx, PPMD_ERR_INVALID, "ppmd_analyze: bad cutoff");
    cudaSetDevice(ctx->device);
    double r_list = fmax(want_boa ? r_boa : 0.0, want_cna ? r_cna : 0.0);
    if (!(r_list > 0)) return PPMD_OK;
    // asynchronous: a list overflow stays latched for the next synchronising call
    Snapshot s;
    PPMD_TRY(sorted_snapshot_boxes(ctx, pos, nbox, atom_off, boxes, r_list,
                                   snapshot_capacity_boxes(nbox, atom_off, boxes, r_list), s));
    if (want_boa)
        PPMD_TRY(boa_launch(ctx, n, s.xq, s.pos, s.st, s.nbr, s.cnt, s.max_nbr, s.ld, r_boa, s.Lmax, s.perm, q4, q6, n_nb));
    if (want_cna)
        PPMD_TRY(cna_launch(ctx, n, s.xq, s.pos, s.st, s.nbr, s.cnt, s.max_nbr, s.ld, r_cna, s.Lmax, s.perm, nullptr, label));
    return check_launch(ctx, "ppmd_analyze");
}

extern "C" int ppmd_analyze(ppmd_ctx *ctx, const double *pos, int64_t n, const ppmd_box *box, double r_boa, double r_cna,
                            float *q4, float *q6, int32_t *n_nb, int8_t *label) {
    if (!ctx || !box || n < 0) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_analyze: bad argument");
    const int64_t off[2] = {0, n};
    return ppmd_analyze_boxes(ctx, pos, 1, off, box, r_boa, r_cna, q4, q6, n_nb, label);
}

extern "C" int ppmd_acna(ppmd_ctx *ctx, const double *pos, int64_t n, const ppmd_box *box, double r_list,
                         int8_t *label, double *rcut) {
    if (!ctx || !box || n < 0 || (n > 0 && (!pos || !label)) || !(r_list > 0))
        return set_error(ctx, PPMD_ERR_INVALID, "ppmd_acna: bad argument");
    cudaSetDevice(ctx->device);
    // asynchronous, as ppmd_analyze
    Snapshot s;
    PPMD_TRY(sorted_snapshot(ctx, pos, n, box, r_list, snapshot_capacity(n, box, r_list), s));
    PPMD_TRY(acna_launch(ctx, n, s.xq, s.pos, s.st, s.nbr, s.cnt, s.max_nbr, s.ld, s.perm, label, rcut));
    return PPMD_OK;
}

extern "C" int ppmd_features(ppmd_ctx *ctx, const double *pos, int64_t n, const ppmd_box *box, double r_feat,
                             double r_ref, float *feat, uint16_t *feat_bf16) {
    if (!ctx || !box || n < 0 || (n > 0 && !pos) || !(r_feat > 0) || !(r_ref < r_feat) || (!feat && !feat_bf16))
        return set_error(ctx, PPMD_ERR_INVALID, "ppmd_features: bad argument");
    cudaSetDevice(ctx->device);
    int32_t max_nbr = snapshot_capacity(n, box, r_feat);
    for (int attempt = 0;; ++attempt) {
        Snapshot s;
        PPMD_TRY(sorted_snapshot(ctx, pos, n, box, r_feat, max_nbr, s));
        PPMD_TRY(features_launch(ctx, n, s.xq, s.pos, s.st, s.nbr, s.cnt, s.max_nbr, s.ld, r_feat, r_ref, s.Lmax, s.perm,
                                 feat, (__nv_bfloat16 *)feat_bf16));
        const int rc = end_pipeline(ctx, attempt, max_nbr);
        if (rc != PIPELINE_RETRY) return rc;
    }
}
