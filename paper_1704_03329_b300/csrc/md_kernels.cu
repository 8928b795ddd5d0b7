// Kernels of the time-stepping driver.  Atoms are stored in cell order, so
// the atoms of consecutive cells of a row are contiguous.
//  - List build: one block per brick of cells stages the positions of the
//    brick's neighbourhood in shared memory; each home atom tests the
//    x-window of each of its nine rows of three cells; the rows are written
//    out as the paper's column-major neighbour matrix W[m][i].
//  - Pair loop: one thread per atom walks its column of W; the
//    single-precision arithmetic runs on packed pairs (f32x2: two neighbours
//    per instruction) with compensated sums, and the second kick of
//    Algorithm 6 is applied in the same thread.
#include <algorithm>

#include "md_kernels.cuh"
#include "pair32.cuh"

namespace ppmd {

// A 16-byte list word, read once per step: not kept in L1, which then holds
// the neighbour positions the loop gathers again and again.
__device__ __forceinline__ int4 ld_stream4(const int4 *p) {
    int4 v;
    asm("ld.global.nc.L1::no_allocate.v4.s32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

BrickShape brick_shape(const Seg &S, int32_t home_max) {
    // the neighbourhood spans bw + 2 cells of a row, bh + 2 rows and bd + 2
    // planes; they must be distinct cells of the periodic grid, and one cell
    // more must stay outside them along each axis for the staged FP32 path
    // of the list build (bw + 3 <= nx and so on; a grid of three cells per
    // axis always takes the other path)
    const double pc = (double)(S.atom1 - S.atom0) / ((double)S.nc[0] * S.nc[1] * S.nc[2]);
    const int32_t mw = std::max(1, std::min(BW_MAX, S.nc[0] - 3)), mh = std::max(1, std::min(BH_MAX, S.nc[1] - 3)),
                  md = std::max(1, std::min(BD_MAX, S.nc[2] - 3));
    BrickShape best{1, 1, 1};
    double best_home = -1.0, best_halo = 0.0;
    for (int32_t bd = 1; bd <= md; ++bd)
        for (int32_t bh = 1; bh <= mh; ++bh)
            for (int32_t bw = 1; bw <= mw; ++bw) {
                const double cells = (double)bw * bh * bd, hood = (double)(bw + 2) * (bh + 2) * (bd + 2);
                const double home = pc * cells;
                if (1.5 * pc * hood + (ROW_GAP + 1) * (bh + 2) * (bd + 2) > NB_MAX || home > home_max) continue;
                const double halo = hood / cells;
                if (home > best_home * (1.0 + 1e-9) || (home >= best_home * (1.0 - 1e-9) && halo < best_halo)) {
                    best = BrickShape{bw, bh, bd};
                    best_home = home;
                    best_halo = halo;
                }
            }
    return best;
}

int64_t brick_count(const Seg &S, BrickShape b) {
    return (int64_t)((S.nc[0] + b.bw - 1) / b.bw) * ((S.nc[1] + b.bh - 1) / b.bh) * ((S.nc[2] + b.bd - 1) / b.bd);
}

int32_t make_bricks(const std::vector<Seg> &segs, std::vector<Brick> &out, int32_t home_max) {
    home_max = std::max(1, std::min(home_max, BRICK_THREADS));
    out.clear();
    int32_t cap = 64;
    for (size_t s = 0; s < segs.size(); ++s) {
        const Seg &S = segs[s];
        const BrickShape b = brick_shape(S, home_max);
        cap = std::max(cap, brick_stage_cap(S, b));
        for (int32_t z0 = 0; z0 < S.nc[2]; z0 += b.bd)
            for (int32_t y0 = 0; y0 < S.nc[1]; y0 += b.bh)
                for (int32_t x0 = 0; x0 < S.nc[0]; x0 += b.bw) {
                    const int32_t x1 = std::min(x0 + b.bw, S.nc[0]), y1 = std::min(y0 + b.bh, S.nc[1]),
                                  z1 = std::min(z0 + b.bd, S.nc[2]);
                    out.push_back(Brick{(int32_t)s, x0 | (x1 << 16), y0 | (y1 << 16), z0 | (z1 << 16)});
                }
    }
    return cap;
}

size_t neigh_brick_smem(int32_t) { return (size_t)NB_MAX * sizeof(int4); }

// Staged atoms of a brick: the expected neighbourhood count with a 1.25x
// margin (for a neighbourhood of ~1200 atoms, a Poisson count would exceed
// it only ~9 standard deviations above its mean; denser bricks read the
// global arrays instead), so that six list-build blocks share an SM.
int32_t brick_stage_cap(const Seg &S, BrickShape b) {
    const double pc = (double)(S.atom1 - S.atom0) / ((double)S.nc[0] * S.nc[1] * S.nc[2]);
    const double need = 1.25 * pc * (b.bw + 2) * (b.bh + 2) * (b.bd + 2) + (ROW_GAP + 1) * (b.bh + 2) * (b.bd + 2);
    const int64_t cap = ((int64_t)ceil(need) + 63) / 64 * 64;
    return (int32_t)std::max<int64_t>(64, std::min<int64_t>(NB_MAX, cap));
}

__device__ __forceinline__ int32_t wrapi(int32_t v, int32_t n) { return v < 0 ? v + n : (v >= n ? v - n : v); }


// List build (Sec. 3.5: the 27 cells around each atom's cell), one block per
// brick of cells.  The brick's neighbourhood (its cells and one cell more on
// every side) is staged in shared memory as (bh + 2)(bd + 2) x-rows of
// bw + 2 consecutive cells: a row of the sorted order is contiguous up to the
// periodic wrap in x, so each staged row maps back to the sorted order by one
// or two offsets.  Each home atom's candidates are the nine rows around its
// cell, three cells of each; the output order is, per atom, the nine rows in
// order and in each row the candidates in stage order (the sorted order,
// x-ordered within a cell).
//
// Atoms are ordered by x within each cell, so the three cells of a row are
// ordered by x and only the window |dx| < r_list of a row can hold hits.  A
// thread owns one home atom; the 32 home atoms of a warp are consecutive in
// one x-row of home cells, so their windows have nearly the same length.  The
// warp walks row q of all its atoms together, four candidates per step (two
// packed pairs), for the longest window of the warp (a lane past its own
// window reads the row's sentinels).  A candidate's tests are the sign bits
// of two packed differences, r^2 - lo and r^2 - hi.  Hits go to a ring of
// RING entries per thread in shared memory and are written out in groups of
// four (one 16-byte store per group in the grouped layout) whenever a ring of
// the warp fills up: no per-hit branch.
constexpr int RING = 16;

// The FP32 stage holds slots in pairs: float4 s & ~1 is (x, x', y, y') and
// float4 s | 1 is (z, z', j, j') of slots s & ~1 and (s & ~1) + 1 (j: the
// atom's sorted index), so two candidates arrive as packed pairs.
__device__ __forceinline__ void pair_put(float4 *P, int32_t s, float x, float y, float z, int32_t j) {
    float *a = reinterpret_cast<float *>(P + (s & ~1)), *b = reinterpret_cast<float *>(P + (s | 1));
    const int h = s & 1;
    a[h] = x;
    a[2 + h] = y;
    b[h] = z;
    b[2 + h] = __int_as_float(j);
}
__device__ __forceinline__ float pair_x(const float4 *P, int32_t s) {
    return reinterpret_cast<const float *>(P + (s & ~1))[s & 1];
}

template <bool VEC4>
__device__ __forceinline__ void put_entry(int32_t *W, int64_t ld, int64_t i, int32_t e, int32_t j) {
    if (VEC4) W[(((int64_t)(e >> 2) * ld + i) << 2) + (e & 3)] = j;
    else W[(int64_t)e * ld + i] = j;
}

template <bool B>
struct Flag {
    static constexpr bool value = B;
};

template <bool VEC4>
__global__ void __launch_bounds__(BRICK_THREADS, 6) k_neigh_brick(const Brick *__restrict__ bricks, BrickShape shape,
                                                              const int4 *__restrict__ xq,
                                                              const double *__restrict__ pos64, SegTable st,
                                                              const int32_t *__restrict__ cs, int32_t *__restrict__ W,
                                                              int64_t ld, int32_t *__restrict__ cnt, int32_t max_nbr,
                                                              int32_t stage_cap, int32_t *status,
                                                              unsigned long long *needed) {
    constexpr int NROW = (BH_MAX + 2) * (BD_MAX + 2), NHOME = BH_MAX * BD_MAX;
    extern __shared__ __align__(16) unsigned char smem[];
    int4 *s_x = (int4 *)smem;
    float4 *P = (float4 *)smem;
    __shared__ int32_t s_cell[NROW][BW_MAX + 3];  // start of the row's cells t = 0 .. bw+2 in the stage
    __shared__ int32_t s_da[NROW], s_db[NROW], s_sw[NROW];  // global = local + (local < sw ? da : db)
    __shared__ int32_t s_home[NHOME][BW_MAX + 1];  // cell starts of the home cells of each home row
    __shared__ int32_t s_hoff[32];                 // first home index of each home row (then H)
    __shared__ int32_t s_total;
    __shared__ int32_t s_ring[RING * BRICK_THREADS];  // entry e of thread t at [e * BRICK_THREADS + t]

    Brick B;
    if (bricks) {
        B = bricks[blockIdx.x];
    } else {
        const Seg &S0 = seg_ref(st, 0);
        const int32_t nbx = (S0.nc[0] + shape.bw - 1) / shape.bw, nby = (S0.nc[1] + shape.bh - 1) / shape.bh;
        const int32_t bx = (int32_t)(blockIdx.x % nbx), by = (int32_t)((blockIdx.x / nbx) % nby),
                      bz = (int32_t)(blockIdx.x / ((int64_t)nbx * nby));
        const int32_t x0 = bx * shape.bw, y0 = by * shape.bh, z0 = bz * shape.bd;
        B.seg = 0;
        B.x01 = x0 | (min(x0 + shape.bw, S0.nc[0]) << 16);
        B.y01 = y0 | (min(y0 + shape.bh, S0.nc[1]) << 16);
        B.z01 = z0 | (min(z0 + shape.bd, S0.nc[2]) << 16);
    }
    const Seg &S = seg_ref(st, B.seg);
    const int32_t nx = S.nc[0], ny = S.nc[1], nz = S.nc[2];
    const int32_t x0 = B.x01 & 0xffff, x1 = B.x01 >> 16, y0 = B.y01 & 0xffff, y1 = B.y01 >> 16;
    const int32_t z0 = B.z01 & 0xffff, z1 = B.z01 >> 16;
    const int32_t bw = x1 - x0, bh = y1 - y0, bd = z1 - z0, nyr = bh + 2, nrow = nyr * (bd + 2), nhome = bh * bd;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid < 32) {
        // warp 0: the staged rows, their cell offsets and their mapping back
        // to the sorted order
        int32_t tot = 0, rb = 0;
        if (tid < nrow) {
            const int32_t yy = wrapi(y0 - 1 + tid % nyr, ny), zz = wrapi(z0 - 1 + tid / nyr, nz);
            rb = S.cell0 + (zz * ny + yy) * nx;
            for (int t = 0; t <= bw + 1; ++t) {
                const int32_t x = wrapi(x0 - 1 + t, nx);
                s_cell[tid][t] = tot;
                tot += cs[rb + x + 1] - cs[rb + x];
            }
            s_cell[tid][bw + 2] = tot;
        }
        // each staged row is followed by at least ROW_GAP far-away sentinels
        // (candidate reads may run past a row's end without bounds tests) and
        // starts on an even slot (a pair)
        const int32_t span = tid < nrow ? (tot + ROW_GAP + 1) & ~1 : 0;
        int32_t inc = span;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        const int32_t base = inc - span;
        if (tid < nrow) {
            for (int t = 0; t <= bw + 2; ++t) s_cell[tid][t] += base;
            const int32_t xa = x0 - 1, xb = x1;  // inclusive cell range of the row
            if (xa < 0) {  // cell nx-1 first, then cells 0 .. xb
                const int32_t len1 = cs[rb + nx] - cs[rb + nx - 1];
                s_da[tid] = cs[rb + nx - 1] - base;
                s_sw[tid] = base + len1;
                s_db[tid] = cs[rb] - (base + len1);
            } else if (xb >= nx) {  // cells xa .. nx-1, then cell 0
                const int32_t len1 = cs[rb + nx] - cs[rb + xa];
                s_da[tid] = cs[rb + xa] - base;
                s_sw[tid] = base + len1;
                s_db[tid] = cs[rb] - (base + len1);
            } else {
                s_da[tid] = cs[rb + xa] - base;
                s_sw[tid] = base + tot;
                s_db[tid] = s_da[tid];
            }
        }
        if (tid == 31) s_total = inc;
    } else if (tid < 64) {
        // warp 1: the home rows (home row l is row l % bh, plane l / bh)
        const int l = lane;
        int32_t c = 0;
        if (l < nhome) {
            const int32_t rm = S.cell0 + ((z0 + l / bh) * ny + y0 + l % bh) * nx;
            for (int t = 0; t <= bw; ++t) s_home[l][t] = cs[rm + x0 + t];
            c = s_home[l][bw] - s_home[l][0];
        }
        int32_t inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        s_hoff[l] = inc - c;  // rows past nhome hold H
    }
    __syncthreads();
    const int32_t T = s_total;
    const int32_t H = s_hoff[nhome];
    // a neighbourhood larger than the shared-memory stage is read from global
    // memory instead (same indices, slower)
    const bool staged = T <= stage_cap;
    // Where the neighbourhood leaves at least one cell of the periodic grid
    // outside it in every direction, positions are staged as FP32 offsets
    // from its centre (the signed fixed-point difference is then the
    // periodic image seen from the brick), so the candidate tests need no
    // integer work.  Rounding: each offset is within 2^-23 of its value (at
    // most 5 cells), which moves r^2 by less than 1e-5 r^2, inside the FP64
    // re-test band.  The centre needs no precision.
    const bool fstage = staged && bw + 3 <= nx && bh + 3 <= ny && bd + 3 <= nz;
    const uint32_t refx = (uint32_t)__float2ull_rz((x0 - 1 + 0.5f * (bw + 2)) / (float)nx * 4294967296.0f);
    const uint32_t refy = (uint32_t)__float2ull_rz((y0 - 1 + 0.5f * (bh + 2)) / (float)ny * 4294967296.0f);
    const uint32_t refz = (uint32_t)__float2ull_rz((z0 - 1 + 0.5f * (bd + 2)) / (float)nz * 4294967296.0f);
    const float sx = S.sx[0], sy = S.sx[1], sz = S.sx[2];
    if (staged) {
        for (int32_t t = tid; t < T; t += blockDim.x) {
            int r = 0, rh = nrow - 1;  // the last row starting at or before t
            while (r < rh) {
                const int mid = (r + rh + 1) >> 1;
                if (s_cell[mid][0] <= t) r = mid;
                else rh = mid - 1;
            }
            if (t >= s_cell[r][bw + 2]) {  // a row's sentinel slot
                if (fstage) pair_put(P, t, 1e18f, 1e18f, 1e18f, -1);
                continue;
            }
            const int32_t j = t + (t < s_sw[r] ? s_da[r] : s_db[r]);
            const int4 q = xq[j];
            if (fstage)
                pair_put(P, t, (float)(int32_t)((uint32_t)q.x - refx) * sx, (float)(int32_t)((uint32_t)q.y - refy) * sy,
                         (float)(int32_t)((uint32_t)q.z - refz) * sz, j);
            else
                s_x[t] = q;
        }
    }
    __syncthreads();
    const float lo = S.rl2_lo, hi = S.rl2_hi;
    if (fstage) {
        const f2 lolo = pk(lo, lo), hihi = pk(hi, hi);
        const float rwin = sqrtf((float)S.rl2) * 1.00001f + 1e-5f;
        const ulonglong2 *P2 = reinterpret_cast<const ulonglong2 *>(P);
        int32_t *const ring = s_ring + tid;
        const int32_t Hw = (H + 31) & ~31;  // whole warps walk the rows together
        for (int32_t h = tid; h < Hw; h += blockDim.x) {
            const bool act = h < H;
            const int32_t hh = act ? h : H - 1;  // idle lanes shadow the last home atom
            int hr = 0;  // the last home row starting at or before hh
            while (hr + 1 < nhome && s_hoff[hr + 1] <= hh) ++hr;
            const int32_t i = s_home[hr][0] + (hh - s_hoff[hr]);
            const int32_t hy = hr % bh, hz = hr / bh;
            int t = 0;
            while (t + 1 < bw && i >= s_home[hr][t + 1]) ++t;
            const int32_t sself = s_cell[(hz + 1) * nyr + hy + 1][t + 1] + (i - s_home[hr][t]);
            float xi, yi, zi;
            {
                const float4 a = P[sself & ~1], b = P[sself | 1];
                const bool odd = sself & 1;
                xi = odd ? a.y : a.x;
                yi = odd ? a.w : a.z;
                zi = odd ? b.y : b.x;
            }
            const f2 xii = pk(xi, xi), yii = pk(yi, yi), zii = pk(zi, zi);
            const float xlo = xi - rwin, xhi = xi + rwin;
            int32_t *wp = ring;  // next free ring entry
            int32_t nout = 0;    // entries written out
            // writes out the ring's complete groups of four (all, padded
            // with -1, when last); warp-wide
            auto flush = [&](bool last) {
                const int32_t n = (int32_t)(wp - ring) / BRICK_THREADS;
                const int32_t g = last ? (n + 3) >> 2 : n >> 2;
                const int32_t gmax = __reduce_max_sync(0xffffffffu, g);
                for (int32_t x = 0; x < gmax; ++x) {
                    if (x >= g) continue;
                    int32_t v[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) v[q] = 4 * x + q < n ? ring[(4 * x + q) * BRICK_THREADS] : -1;
                    const int32_t e = nout + 4 * x;
                    if (!act || e >= max_nbr) continue;
                    if (VEC4) {
                        reinterpret_cast<int4 *>(W)[(int64_t)(e >> 2) * ld + i] = make_int4(v[0], v[1], v[2], v[3]);
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (4 * x + q < n && e + q < max_nbr) W[(int64_t)(e + q) * ld + i] = v[q];
                    }
                }
                if (last) {
                    nout += n;
                } else {
                    const int32_t rest = n - 4 * g;  // 0 .. 3 entries move to the front
                    for (int q = 0; q < rest; ++q) ring[q * BRICK_THREADS] = ring[(4 * g + q) * BRICK_THREADS];
                    wp = ring + rest * BRICK_THREADS;
                    nout += 4 * g;
                }
            };
            for (int q = 0; q < 9; ++q) {
                const int r = (hz + q / 3) * nyr + hy + q % 3;
                int32_t a = s_cell[r][t], e = s_cell[r][t + 3];
                {  // the window: first candidate with x >= xlo, first with x > xhi
                    int32_t u = a, v = e;
                    while (u < v) {
                        const int32_t mid = (u + v) >> 1;
                        if (pair_x(P, mid) < xlo) u = mid + 1;
                        else v = mid;
                    }
                    a = u;
                    v = e;
                    while (u < v) {
                        const int32_t mid = (u + v) >> 1;
                        if (pair_x(P, mid) <= xhi) u = mid + 1;
                        else v = mid;
                    }
                    e = u;
                }
                a &= ~1;  // rows start on even slots: a stays in the row
                if (!act) e = a;
                const int32_t nstep = __reduce_max_sync(0xffffffffu, (e - a + 3) >> 2);
                const int32_t rs = (s_cell[r][bw + 2] + 1) & ~1;  // four of the row's sentinels
                // center: true for the row of the atom's own cell, the only
                // one that holds the atom itself (excluded by its stage slot)
                auto walk = [&](auto center) {
                    for (int32_t s = 0; s < nstep; ++s) {
                        const int32_t k = a + 4 * s;
                        // Reads run at most three slots past the window:
                        // candidates with x beyond the window (never within
                        // r_list), atoms two cells away, or the row's
                        // sentinels; a lane past its window reads sentinels.
                        const int32_t kk = k < e ? k : rs;
                        const ulonglong2 A = P2[kk], Bv = P2[kk + 1], C = P2[kk + 2], D = P2[kk + 3];
                        // sign bits of r^2 - lo (a hit) and of r^2 - hi (below
                        // the band's top): the sign of a rounded difference is
                        // exact
                        uint32_t l[4], h[4];
                        {
                            const f2 dx = sub2(xii, A.x), dy = sub2(yii, A.y), dz = sub2(zii, Bv.x);
                            const f2 r2a = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
                            const f2 ex = sub2(xii, C.x), ey = sub2(yii, C.y), ez = sub2(zii, D.x);
                            const f2 r2b = fma2(ex, ex, fma2(ey, ey, mul2(ez, ez)));
                            float t0, t1;
                            upk(sub2(r2a, lolo), t0, t1);
                            l[0] = __float_as_uint(t0), l[1] = __float_as_uint(t1);
                            upk(sub2(r2b, lolo), t0, t1);
                            l[2] = __float_as_uint(t0), l[3] = __float_as_uint(t1);
                            upk(sub2(r2a, hihi), t0, t1);
                            h[0] = __float_as_uint(t0), h[1] = __float_as_uint(t1);
                            upk(sub2(r2b, hihi), t0, t1);
                            h[2] = __float_as_uint(t0), h[3] = __float_as_uint(t1);
                        }
                        const int32_t jv[4] = {(int32_t)(uint32_t)Bv.y, (int32_t)(uint32_t)(Bv.y >> 32),
                                               (int32_t)(uint32_t)D.y, (int32_t)(uint32_t)(D.y >> 32)};
                        uint32_t hit[4];
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            hit[c] = l[c] >> 31;
                            if (decltype(center)::value) hit[c] &= (uint32_t)(kk + c != sself);
                        }
                        if (((h[0] & ~l[0]) | (h[1] & ~l[1]) | (h[2] & ~l[2]) | (h[3] & ~l[3])) >> 31) {
                            // rare: within the FP32 decision band of r_list
                            // (FP64 decides; never the atom itself, r^2 = 0)
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                if ((h[c] & ~l[c]) >> 31) {
                                    double dr[3];
                                    hit[c] = min_image_r2(pos64 + 3 * (int64_t)i, pos64 + 3 * (int64_t)jv[c], S, dr) < S.rl2;
                                }
                            }
                        }
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            *wp = jv[c];
                            wp += hit[c] * BRICK_THREADS;
                        }
                        if (__any_sync(0xffffffffu, wp >= ring + (RING - 4) * BRICK_THREADS)) flush(false);
                    }
                };
                if (q == 4) walk(Flag<true>());
                else walk(Flag<false>());
            }
            flush(true);
            if (act) {
                cnt[i] = nout;
                if (nout > max_nbr) {
                    latch_status(status, PPMD_ERR_CAPACITY);
                    latch_needed(needed, (unsigned long long)nout);
                }
            }
        }
        return;
    }
    // Small grids (the neighbourhood wraps onto itself) and neighbourhoods
    // too large to stage: a thread per home atom, fixed-point differences,
    // hits stored as they are found (same order).
    const f2 sxx = pk(sx, sx), syy = pk(sy, sy), szz = pk(sz, sz);
    for (int32_t h = tid; h < H; h += blockDim.x) {
        int hr = 0;
        while (hr + 1 < nhome && s_hoff[hr + 1] <= h) ++hr;
        const int32_t i = s_home[hr][0] + (h - s_hoff[hr]);
        const int32_t hy = hr % bh, hz = hr / bh;
        const int4 xi = xq[i];
        int t = 0;
        while (t + 1 < bw && i >= s_home[hr][t + 1]) ++t;
        int32_t count = 0;
        auto hit = [&](int32_t j) {
            if (count < max_nbr) put_entry<VEC4>(W, ld, i, count, j);
            ++count;
        };
        for (int dz = 0; dz < 3; ++dz)
            for (int dy = 0; dy < 3; ++dy) {
                const int r = (hz + dz) * nyr + hy + dy;
                const int32_t a = s_cell[r][t], b = s_cell[r][t + 3];
                const int32_t sw = s_sw[r], da = s_da[r], db = s_db[r];
                for (int32_t k = a; k < b; k += 2) {
                    const bool v1 = k + 1 < b;
                    const int32_t kb = v1 ? k + 1 : k;
                    const int4 xa = staged ? s_x[k] : xq[k + (k < sw ? da : db)];
                    const int4 xb = staged ? s_x[kb] : xq[kb + (kb < sw ? da : db)];
                    const f2 dx = mul2(pk(fdiff(xi.x, xa.x), fdiff(xi.x, xb.x)), sxx);
                    const f2 dy_ = mul2(pk(fdiff(xi.y, xa.y), fdiff(xi.y, xb.y)), syy);
                    const f2 dz_ = mul2(pk(fdiff(xi.z, xa.z), fdiff(xi.z, xb.z)), szz);
                    const f2 r2 = fma2(dx, dx, fma2(dy_, dy_, mul2(dz_, dz_)));
                    float ra, rb2;
                    upk(r2, ra, rb2);
                    const int32_t ja = k + (k < sw ? da : db);
                    const int32_t jb = k + 1 + (k + 1 < sw ? da : db);
                    if (ra < hi && ja != i) {
                        double dr[3];
                        if (ra < lo || min_image_r2(pos64 + 3 * (int64_t)i, pos64 + 3 * (int64_t)ja, S, dr) < S.rl2) hit(ja);
                    }
                    if (v1 && rb2 < hi && jb != i) {
                        double dr[3];
                        if (rb2 < lo || min_image_r2(pos64 + 3 * (int64_t)i, pos64 + 3 * (int64_t)jb, S, dr) < S.rl2) hit(jb);
                    }
                }
            }
        // the last, partial group, padded with -1
        if (VEC4)
            for (int32_t e = count; e < ((count + 3) & ~3) && e < max_nbr; ++e) put_entry<VEC4>(W, ld, i, e, -1);
        cnt[i] = count;
        if (count > max_nbr) {
            latch_status(status, PPMD_ERR_CAPACITY);
            latch_needed(needed, (unsigned long long)count);
        }
    }
}

int neigh_brick_setup(ppmd_ctx *ctx, int32_t max_nbr) {
    int rc = PPMD_OK;
    for (const void *f : {(const void *)k_neigh_brick<false>, (const void *)k_neigh_brick<true>})
        if (rc == PPMD_OK)
            rc = cuda_check(ctx, cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      (int)neigh_brick_smem(max_nbr)),
                            "cudaFuncSetAttribute");
    return rc;
}

int build_list_bricks(ppmd_ctx *ctx, int64_t nbricks, const Brick *bricks, BrickShape shape, const int4 *xq,
                      const double *pos64, const SegTable &st, const int32_t *cell_start, int32_t *W, int64_t ld,
                      int32_t *cnt, int32_t max_nbr, int32_t stage_cap, bool vec4) {
    if (stage_cap <= 0 || stage_cap > NB_MAX) stage_cap = NB_MAX;
    if (vec4 && (max_nbr & 3)) return set_error(ctx, PPMD_ERR_INVALID, "grouped list needs a capacity divisible by 4");
    if (nbricks > 0) {
        auto kern = vec4 ? k_neigh_brick<true> : k_neigh_brick<false>;
        PPMD_LAUNCH(ctx, kern, nbricks, BRICK_THREADS, (size_t)stage_cap * sizeof(int4), bricks, shape, xq, pos64, st,
                    cell_start, W, ld, cnt, max_nbr, stage_cap, ctx->d_status, ctx->d_needed);
    }
    return check_launch(ctx, "build_list_bricks");
}

__device__ __forceinline__ void block_sum3(double a, double b, double c, double *partials) {
    __shared__ double sh[3][32];
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][w] = a;
        sh[1][w] = b;
        sh[2][w] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double u = 0, v = 0, k = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            u += sh[0][q];
            v += sh[1][q];
            k += sh[2][q];
        }
        partials[3 * blockIdx.x] = u;
        partials[3 * blockIdx.x + 1] = v;
        partials[3 * blockIdx.x + 2] = k;
    }
}

// As block_sum3, with the warp sums taken on FP32 pairs (hi, lo) by
// error-free transformations (about 48 significant bits) instead of FP64
// additions on every lane, which are slow on this part.
__device__ __forceinline__ void pair_add(float &s, float &e, float s2, float e2) {
    const float t = s + s2, bb = t - s, err = (s - (t - bb)) + (s2 - bb);
    const float lo = err + (e + e2);
    s = t + lo;
    e = lo - (s - t);
}

__device__ __forceinline__ void block_sum3_pairs(double a, double b, double c, double *partials) {
    __shared__ double sh[3][32];
    float hs[3], ls[3];
    const double v[3] = {a, b, c};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        hs[k] = (float)v[k];
        ls[k] = (float)(v[k] - (double)hs[k]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float h2 = __shfl_xor_sync(0xffffffffu, hs[k], o), l2 = __shfl_xor_sync(0xffffffffu, ls[k], o);
            pair_add(hs[k], ls[k], h2, l2);
        }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 3; ++k) sh[k][w] = (double)hs[k] + (double)ls[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        double u = 0, vv = 0, kk = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            u += sh[0][q];
            vv += sh[1][q];
            kk += sh[2][q];
        }
        partials[3 * blockIdx.x] = u;
        partials[3 * blockIdx.x + 1] = vv;
        partials[3 * blockIdx.x + 2] = kk;
    }
}

constexpr int COL_BLOCK = 256;

// One thread per atom; a launch with fewer blocks than atoms / BLOCK (a
// persistent grid) walks the atoms block by block (grid stride), each
// thread summing the energy and the largest displacement over its atoms.
// Registers: 1024 threads per SM (64 registers; a few words of the
// epilogue spill, which measured faster than 72 registers at 896 threads)
// for the steps without energies, 768 (80) for the energy steps.
template <bool ENERGY, bool DRIFT, int BLOCK>
__global__ void __launch_bounds__(BLOCK, (ENERGY ? 768 : 1024) / BLOCK) k_lj_col32(int64_t n, int64_t ld, const int4 *__restrict__ xq,
                                                        const double *__restrict__ pos64, SegTable st, LJConst c,
                                                        const int32_t *__restrict__ W, const int32_t *__restrict__ cnt,
                                                        int32_t max_nbr, float4 *__restrict__ f4,
                                                        double *__restrict__ vel, double h, double half_m,
                                                        double *__restrict__ partials, Drift dr) {
    double u_i = 0.0, w_i = 0.0, k_i = 0.0;
    float d2 = 0.0f;
    for (int64_t i0 = (int64_t)blockIdx.x * BLOCK; i0 < n; i0 += (int64_t)gridDim.x * BLOCK) {
    const int64_t i = i0 + threadIdx.x;
    if (i < n) {
        const int4 xi = xq[i];
        const Seg &S = seg_ref(st, xi.w);
        const f2 sxx = pk(S.sx[0], S.sx[0]), syy = pk(S.sx[1], S.sx[1]), szz = pk(S.sx[2], S.sx[2]);
        const f2 two = pk(2.0f, 2.0f), half = pk(0.5f, 0.5f), one = pk(1.0f, 1.0f);
        const f2 s2 = pk(c.s2, c.s2), f48 = pk(c.f48, c.f48), e2 = pk(c.e2, c.e2), shift = pk(c.shift, c.shift);
        const int32_t m = min(cnt[i], max_nbr);
        Kahan2 fx, fy, fz, ea, vir;
        fx.init();
        fy.init();
        fz.init();
        if (ENERGY) {
            ea.init();
            vir.init();
        }
        const int4 *col4 = reinterpret_cast<const int4 *>(W) + i;  // groups of four entries
        // Two neighbours per packed step; the list entries of the next four
        // neighbours are loaded one iteration ahead of their use.
        // Two neighbours per packed step: their force terms fm dr (fm = 0
        // outside the cutoff) are returned; energy and virial are added here.
        auto step = [&](int32_t j0, int32_t j1, const int4 &a, const int4 &b, f2 &tx, f2 &ty, f2 &tz) {
            const bool v0 = j0 >= 0, v1 = j1 >= 0;
            const f2 dx = mul2(pk(fdiff(xi.x, a.x), fdiff(xi.x, b.x)), sxx);
            const f2 dy = mul2(pk(fdiff(xi.y, a.y), fdiff(xi.y, b.y)), syy);
            const f2 dz = mul2(pk(fdiff(xi.z, a.z), fdiff(xi.z, b.z)), szz);
            const f2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
            float r2a, r2b;
            upk(r2, r2a, r2b);
            bool in0 = v0 && r2a < c.rc2_lo, in1 = v1 && r2b < c.rc2_lo;
            if (v0 && !in0 && r2a < c.rc2_hi) {
                double dr[3];
                in0 = min_image_r2(pos64 + 3 * i, pos64 + 3 * (int64_t)j0, S, dr) < c.rc2;
            }
            if (v1 && !in1 && r2b < c.rc2_hi) {
                double dr[3];
                in1 = min_image_r2(pos64 + 3 * i, pos64 + 3 * (int64_t)j1, S, dr) < c.rc2;
            }
            // 1/r^2: hardware estimate refined by one Newton-Raphson step r (2 - x r)
            f2 ir = pk(rcp_approx(r2a), rcp_approx(r2b));
            ir = mul2(ir, fma2(pk(-r2a, -r2b), ir, two));
            const f2 sr2 = mul2(s2, ir);
            const f2 sr6 = mul2(mul2(sr2, sr2), sr2);
            f2 fm = mul2(mul2(f48, sub2(sr6, half)), mul2(sr6, ir));
            float fa, fb;
            upk(fm, fa, fb);
            fm = pk(in0 ? fa : 0.0f, in1 ? fb : 0.0f);
            tx = mul2(fm, dx);
            ty = mul2(fm, dy);
            tz = mul2(fm, dz);
            if (ENERGY) {
                f2 v = mul2(e2, fma2(sr6, sub2(sr6, one), shift));
                float va, vb;
                upk(v, va, vb);
                ea.add_prod(pk(in0 ? va : 0.0f, in1 ? vb : 0.0f), one);
                vir.add_prod(fm, r2);
            }
        };
        // one 16-byte list word per four neighbours (entries past the row
        // are -1), loaded one group ahead of its use
        auto group = [&](int32_t k) { return k < m ? ld_stream4(col4 + (int64_t)(k >> 2) * ld) : make_int4(-1, -1, -1, -1); };
        int4 g = group(0);
        for (int32_t k = 0; k < m; k += 4) {
            const int4 nx = group(k + 4);
            const int32_t j0 = g.x, j1 = g.y, j2 = g.z, j3 = g.w;
            const int4 a0 = __ldg(&xq[j0 >= 0 ? j0 : i]), a1 = __ldg(&xq[j1 >= 0 ? j1 : i]);
            const int4 a2 = __ldg(&xq[j2 >= 0 ? j2 : i]), a3 = __ldg(&xq[j3 >= 0 ? j3 : i]);
            // the four terms of each component enter the compensated sum as
            // one plain FP32 partial (two terms per stream)
            f2 tx0, ty0, tz0, tx1, ty1, tz1;
            step(j0, j1, a0, a1, tx0, ty0, tz0);
            step(j2, j3, a2, a3, tx1, ty1, tz1);
            fx.add(add2(tx0, tx1));
            fy.add(add2(ty0, ty1));
            fz.add(add2(tz0, tz1));
            g = nx;
        }
        float hx, lx, hy, ly, hz, lz;
        fx.merged(hx, lx);
        fy.merged(hy, ly);
        fz.merged(hz, lz);
        // The force word is hx + lx rounded once to FP32.  The FP32 sum gives
        // the same float as the FP64 sum rounded to FP32: rounding a sum of
        // two floats first to 53 bits and then to 24 equals rounding it to 24
        // bits directly, since 53 >= 2 x 24 + 2 (double rounding is then
        // innocuous), so no FP64 operation is needed here.
        const float Fx = hx + lx, Fy = hy + ly, Fz = hz + lz;
        float he = 0.f, le = 0.f;
        if (ENERGY) {
            ea.merged(he, le);
            float hv, lv;
            vir.merged(hv, lv);
            u_i += (double)he + (double)le;
            w_i += 0.5 * ((double)hv + (double)lv);
        }
        f4[i] = make_float4(Fx, Fy, Fz, he + le);
        if (vel) {
            // second kick of Algorithm 6 with the forces just computed
            const float4 fq = f4[i];
            const double f[3] = {(double)fq.x, (double)fq.y, (double)fq.z};
            double v[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) v[d] = fma(h, f[d], vel[3 * i + d]);
            if (ENERGY) k_i += half_m * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            if (DRIFT) {
                // the next step's kick and drift, in the same arithmetic as
                // k_kick_drift2 (the atom's segment is looked up again, so
                // that nothing of the pair loop stays live until here)
                const int4 ref = dr.xq_ref[i];
                const Seg &Sd = seg_ref(st, ref.w);
                uint32_t q[3];
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    v[d] = fma(h, f[d], v[d]);
                    const double r = fma(dr.dt, v[d], pos64[3 * i + d]);
                    dr.pos_next[3 * i + d] = r;
                    q[d] = (uint32_t)(unsigned long long)__double2ll_rn(r * Sd.fxs[d]);
                }
                dr.xq_next[i] = make_int4((int)q[0], (int)q[1], (int)q[2], ref.w);
                const float ex = fixed_delta(q[0], (uint32_t)ref.x, Sd.sx[0]);
                const float ey = fixed_delta(q[1], (uint32_t)ref.y, Sd.sx[1]);
                const float ez = fixed_delta(q[2], (uint32_t)ref.z, Sd.sx[2]);
                d2 = fmaxf(d2, fmaf(ex, ex, fmaf(ey, ey, ez * ez)));
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) vel[3 * i + d] = v[d];
        }
    }
    }
    if (DRIFT) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d2 = fmaxf(d2, __shfl_xor_sync(0xffffffffu, d2, o));
        if ((threadIdx.x & 31) == 0 && d2 > 0.0f) atomicMax(dr.max_disp_bits, __float_as_uint(d2));
    }
    if (ENERGY) block_sum3_pairs(u_i, w_i, k_i, partials);
}

// G lanes per atom (a power of two up to 32): lane l takes the list entries
// k = l, l + G, ...; the lanes' sums are combined by a butterfly of
// shuffles (every lane ends with the same bits), and lane 0 writes the
// force and makes the kick.  G = 1 for systems that fill the GPU; small
// systems take more lanes, since FP64 issues slowly and a thread per atom
// would leave most SMs idle.
template <bool ENERGY, int G>
__global__ void __launch_bounds__(COL_BLOCK) k_lj_col64(int64_t n, int64_t ld, const int4 *__restrict__ xq,
                                                        const double *__restrict__ pos64, SegTable st, LJConst c,
                                                        const int32_t *__restrict__ W, const int32_t *__restrict__ cnt,
                                                        int32_t max_nbr, double *__restrict__ f64,
                                                        double *__restrict__ vel, double h, double half_m,
                                                        double *__restrict__ partials) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = t / G;
    const int l = (int)(t % G);
    double u_i = 0.0, w_i = 0.0, k_i = 0.0;
    double fx = 0.0, fy = 0.0, fz = 0.0;
    if (i < n) {
        const Seg &S = seg_ref(st, xq[i].w);
        const int32_t m = min(cnt[i], max_nbr);
        const double *pi = pos64 + 3 * i;
        for (int32_t k = l; k < m; k += G) {
            const int32_t j = __ldg(W + (((int64_t)(k >> 2) * ld + i) << 2) + (k & 3));  // grouped by four
            double dr[3];
            const double r2 = min_image_r2(pi, pos64 + 3 * (int64_t)j, S, dr);
            if (r2 < c.rc2) {
                const double sr2 = c.s2d / r2;
                const double sr6 = sr2 * sr2 * sr2;
                const double sr8 = sr6 * sr2;
                const double sr12 = sr6 * sr6;
                const double fmag = c.f48d * (sr12 * sr2 - 0.5 * sr8);
                fx += fmag * dr[0];
                fy += fmag * dr[1];
                fz += fmag * dr[2];
                if (ENERGY) {
                    u_i += c.e2d * (sr12 - sr6 + c.shiftd);
                    w_i += 0.5 * fmag * r2;
                }
            }
        }
    }
    if (G > 1) {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            fx += __shfl_xor_sync(0xffffffffu, fx, o);
            fy += __shfl_xor_sync(0xffffffffu, fy, o);
            fz += __shfl_xor_sync(0xffffffffu, fz, o);
            if (ENERGY) {
                u_i += __shfl_xor_sync(0xffffffffu, u_i, o);
                w_i += __shfl_xor_sync(0xffffffffu, w_i, o);
            }
        }
        if (l != 0) u_i = w_i = 0.0;  // the atom counted once
    }
    if (i < n && l == 0) {
        f64[3 * i] = fx;
        f64[3 * i + 1] = fy;
        f64[3 * i + 2] = fz;
        if (vel) {
            const double vx = fma(h, fx, vel[3 * i]);
            const double vy = fma(h, fy, vel[3 * i + 1]);
            const double vz = fma(h, fz, vel[3 * i + 2]);
            vel[3 * i] = vx;
            vel[3 * i + 1] = vy;
            vel[3 * i + 2] = vz;
            if (ENERGY) k_i = half_m * (vx * vx + vy * vy + vz * vz);
        }
    }
    if (ENERGY) block_sum3(u_i, w_i, k_i, partials);
}

// FP64 runs at a small fraction of the FP32 rate on this part: a system of
// fewer atoms than 148 x 256 takes G lanes per atom (the power of two that
// brings the threads to at least 148 x 256, at most 16) on 128-thread
// blocks, so that its pair terms spread over the SMs.
int lj_col64_lanes(int64_t n) {
    int g = 1;
    while (g < 16 && n * g < (int64_t)148 * COL_BLOCK) g *= 2;
    return g;
}
int lj_col64_atoms_per_block(int64_t n) {
    const int g = lj_col64_lanes(n);
    return g == 1 ? COL_BLOCK : 128 / g;
}

template <bool ENERGY>
void launch_col64(ppmd_ctx *ctx, int64_t n, int64_t ld, const int4 *xq, const double *pos64, const SegTable &st,
                  const LJConst &c, const int32_t *W, const int32_t *cnt, int32_t max_nbr, double *f64, double *vel,
                  double h, double half_m, double *partials) {
    const int g = lj_col64_lanes(n);
    const int64_t nb = div_up(n, lj_col64_atoms_per_block(n));
    const int block = g == 1 ? COL_BLOCK : 128;
    auto kern = g == 1 ? k_lj_col64<ENERGY, 1>
                       : g == 2 ? k_lj_col64<ENERGY, 2>
                                : g == 4 ? k_lj_col64<ENERGY, 4> : g == 8 ? k_lj_col64<ENERGY, 8> : k_lj_col64<ENERGY, 16>;
    PPMD_LAUNCH(ctx, kern, nb, block, 0, n, ld, xq, pos64, st, c, W, cnt, max_nbr, f64, vel, h, half_m, partials);
}

int64_t lj_columns_blocks(int64_t n, const ColShape &shape) {
    const int64_t nb = div_up(n, shape.block);
    return shape.grid_cap > 0 ? std::min<int64_t>(nb, shape.grid_cap) : nb;
}

int lj_columns(ppmd_ctx *ctx, int64_t n, int64_t ld, const int4 *xq, const double *pos64, const SegTable &st,
               const LJConst &c, const int32_t *W, const int32_t *cnt, int32_t max_nbr, int prec, float4 *f4,
               double *f64, double *vel, double h, double half_m, double *partials, const Drift &drift,
               const ColShape &shape) {
    if (n <= 0) return PPMD_OK;
    if (drift.pos_next && (prec != PPMD_FP32 || !vel)) return set_error(ctx, PPMD_ERR_INVALID, "lj_columns: drift needs FP32 and a kick");
    if (prec == PPMD_FP32) {
        if (shape.block != 128 && shape.block != 256) return set_error(ctx, PPMD_ERR_INVALID, "lj_columns: block %d", shape.block);
        const int64_t nb = lj_columns_blocks(n, shape);
        const bool e = partials != nullptr, d = drift.pos_next != nullptr;
        if (shape.block == 256) {
            auto kern = e ? (d ? k_lj_col32<true, true, 256> : k_lj_col32<true, false, 256>)
                          : (d ? k_lj_col32<false, true, 256> : k_lj_col32<false, false, 256>);
            PPMD_LAUNCH(ctx, kern, nb, 256, 0, n, ld, xq, pos64, st, c, W, cnt, max_nbr, f4, vel, h, half_m, partials,
                        drift);
        } else {
            auto kern = e ? (d ? k_lj_col32<true, true, 128> : k_lj_col32<true, false, 128>)
                          : (d ? k_lj_col32<false, true, 128> : k_lj_col32<false, false, 128>);
            PPMD_LAUNCH(ctx, kern, nb, 128, 0, n, ld, xq, pos64, st, c, W, cnt, max_nbr, f4, vel, h, half_m, partials,
                        drift);
        }
    } else {
        if (partials) launch_col64<true>(ctx, n, ld, xq, pos64, st, c, W, cnt, max_nbr, f64, vel, h, half_m, partials);
        else launch_col64<false>(ctx, n, ld, xq, pos64, st, c, W, cnt, max_nbr, f64, vel, h, half_m, partials);
    }
    return check_launch(ctx, "lj_columns");
}

// ---------------------------------------------------------------------
// Kick + drift (the first half kick and the drift of Algorithm 6).
// ---------------------------------------------------------------------
template <class F>
__device__ __forceinline__ void load_f(const F *f, int64_t i, double out[3]);
template <>
__device__ __forceinline__ void load_f<float4>(const float4 *f, int64_t i, double out[3]) {
    const float4 v = f[i];
    out[0] = v.x;
    out[1] = v.y;
    out[2] = v.z;
}
template <>
__device__ __forceinline__ void load_f<double>(const double *f, int64_t i, double out[3]) {
    out[0] = f[3 * i];
    out[1] = f[3 * i + 1];
    out[2] = f[3 * i + 2];
}

template <class F>
__global__ void __launch_bounds__(256) k_kick_drift2(int64_t n, double *__restrict__ pos, double *__restrict__ vel,
                                                     const F *__restrict__ force, int4 *__restrict__ xq,
                                                     const int4 *__restrict__ xq_ref, SegTable st, double h, double dt,
                                                     unsigned int *max_disp_bits) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float d2 = 0.0f;
    if (i < n) {
        double f[3];
        load_f<F>(force, i, f);
        const int32_t sid = xq_ref[i].w;
        const Seg &S = seg_ref(st, sid);
        uint32_t q[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double v = fma(h, f[d], vel[3 * i + d]);
            vel[3 * i + d] = v;
            const double r = fma(dt, v, pos[3 * i + d]);
            pos[3 * i + d] = r;
            // r may leave [0, L) until the next list build; the fixed-point
            // word wraps modulo 2^32, i.e. modulo L
            q[d] = (uint32_t)(unsigned long long)__double2ll_rn(r * S.fxs[d]);
        }
        xq[i] = make_int4((int)q[0], (int)q[1], (int)q[2], sid);
        const int4 ref = xq_ref[i];
        const float ex = fixed_delta(q[0], (uint32_t)ref.x, S.sx[0]);
        const float ey = fixed_delta(q[1], (uint32_t)ref.y, S.sx[1]);
        const float ez = fixed_delta(q[2], (uint32_t)ref.z, S.sx[2]);
        d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d2 = fmaxf(d2, __shfl_xor_sync(0xffffffffu, d2, o));
    if ((threadIdx.x & 31) == 0 && d2 > 0.0f) atomicMax(max_disp_bits, __float_as_uint(d2));
}

int md_kick_drift2(ppmd_ctx *ctx, int64_t n, double *pos, double *vel, const float4 *f4, const double *f64, int4 *xq,
                   const int4 *xq_ref, const SegTable &st, double h, double dt, unsigned int *max_disp_bits) {
    if (n <= 0) return PPMD_OK;
    if (f4)
        PPMD_LAUNCH(ctx, k_kick_drift2<float4>, div_up(n, 256), 256, 0, n, pos, vel, f4, xq, xq_ref, st, h, dt, max_disp_bits);
    else
        PPMD_LAUNCH(ctx, k_kick_drift2<double>, div_up(n, 256), 256, 0, n, pos, vel, f64, xq, xq_ref, st, h, dt, max_disp_bits);
    return check_launch(ctx, "md_kick_drift2");
}

// With xq (the current fixed-point words, modulo 2^32 already those of the
// wrapped positions to within a quantum) the words are gathered; without,
// they are made from the wrapped positions.  The in-box test runs on the
// FP64 bit patterns (for x >= 0 their order is that of the values; -0.0
// counts as inside, as in the comparison x >= 0.0), so an atom that stays
// in the box takes no FP64 operation.
__global__ void k_md_gather(int64_t n, const int32_t *__restrict__ perm, SegTable st, const double *__restrict__ pos,
                            const double *__restrict__ vel, const int32_t *__restrict__ orig,
                            const int32_t *__restrict__ seg_of, const int4 *__restrict__ xq, double *__restrict__ pos_o,
                            double *__restrict__ vel_o, int4 *__restrict__ xq_o, int4 *__restrict__ xq_o2,
                            int32_t *__restrict__ orig_o, int32_t *__restrict__ seg_o) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t j = perm[k];
    const int32_t sid = seg_of[j];
    const Seg &S = seg_ref(st, sid);
    uint32_t q[3];
    int4 qj = make_int4(0, 0, 0, 0);
    if (xq) qj = xq[j];
    const uint32_t qin[3] = {(uint32_t)qj.x, (uint32_t)qj.y, (uint32_t)qj.z};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double x = pos[3 * j + d];
        const long long b = __double_as_longlong(x);
        const bool inside = b >= 0 ? b < __double_as_longlong(S.L[d]) : b == (long long)0x8000000000000000ull;
        if (!inside) x = wrap_exact(x, S.L[d]);
        pos_o[3 * k + d] = x;
        vel_o[3 * k + d] = vel[3 * j + d];
        q[d] = xq ? qin[d] : to_fixed(x, S.fxs[d]);
    }
    const int4 w = make_int4((int)q[0], (int)q[1], (int)q[2], sid);
    xq_o[k] = w;
    if (xq_o2) xq_o2[k] = w;
    orig_o[k] = orig[j];
    seg_o[k] = sid;
}

int md_gather(ppmd_ctx *ctx, int64_t n, const int32_t *perm, const SegTable &st, const double *pos, const double *vel,
              const int32_t *orig, const int32_t *seg_of, const int4 *xq, double *pos_o, double *vel_o, int4 *xq_o,
              int4 *xq_o2, int32_t *orig_o, int32_t *seg_o) {
    if (n > 0)
        PPMD_LAUNCH(ctx, k_md_gather, div_up(n, 256), 256, 0, n, perm, st, pos, vel, orig, seg_of, xq, pos_o, vel_o, xq_o,
                    xq_o2, orig_o, seg_o);
    return check_launch(ctx, "md_gather");
}

}  // namespace ppmd
