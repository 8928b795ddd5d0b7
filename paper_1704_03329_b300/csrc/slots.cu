// Brick-staged integrator path (FP32 pair arithmetic).
//
// The paper's neighbour matrix W (Sec. 3.5.1) holds, for each atom, the
// atoms within the extended cutoff of Eq. (3).  Here the atoms are sorted by
// cell and the grid is cut into bricks of cells; the neighbourhood of a
// brick (its cells and one layer of cells around it) is a fixed list of
// contiguous runs of the sorted atoms between two list builds.  A list entry
// is therefore stored as the neighbour's slot in that staged neighbourhood
// (16 bits) instead of its atom index:
//  - the list build stages the neighbourhood once per brick, each home atom
//    is tested against its 27 cells by a group of eight lanes (the candidate
//    windows |dx| < r_list of the nine rows, split evenly over the lanes),
//    and the slots of the hits are written column-major in groups of eight
//    (one 16-byte word per eight neighbours);
//  - the pair loop of every step copies the brick's neighbourhood into
//    shared memory with bulk asynchronous copies (one per contiguous run,
//    completion on an mbarrier), then each thread walks the slot list of
//    one home atom with every neighbour position read from shared memory.
// Pair arithmetic, compensated sums and the fused integration are those of
// the column-major loop in md_kernels.cu, entry for entry in the same order,
// so the two paths give the same forces bit for bit.
#include "md_kernels.cuh"
#include "pair32.cuh"

namespace ppmd {

namespace {

constexpr int NROW = (BH_MAX + 2) * (BD_MAX + 2);
constexpr int NHOME = BH_MAX * BD_MAX;
constexpr int GROUP = 8;                          // lanes per home atom in the list build
constexpr int NGROUP = SLOT_THREADS / GROUP;      // home atoms in flight per list-build block
constexpr uint32_t STAGE_WAIT_LIMIT = 1u << 22;   // polls of the staging mbarrier

// Where a brick's neighbourhood sits in the stage, and where its home atoms
// are.  Stage row r (r = dy + (bh + 2) dz for the rows y0-1+dy, planes
// z0-1+dz) holds the cells x0-1 .. x1 of that row one after the other; rows
// follow each other with no gap.  Slot s of row r is atom
// s + (s < sw[r] ? da[r] : db[r]) of the sorted order (two runs where the
// row wraps around the periodic x edge).
//
// The layout is one flat array of words in shared memory, written once per
// entry and read through volatile accessors (every access a real load or
// store at an explicitly computed offset).
constexpr int LW_CELL = BW_MAX + 3;  // cell starts of a row: t = 0 .. bw + 1, then the row's end
constexpr int LW_HOME = BW_MAX + 1;
constexpr int LO_CELL = 0;
constexpr int LO_DA = LO_CELL + NROW * LW_CELL;
constexpr int LO_DB = LO_DA + NROW;
constexpr int LO_SW = LO_DB + NROW;
constexpr int LO_HOME = LO_SW + NROW;  // first atom of home cell t of home row l; [bw] = end
constexpr int LO_HOFF = LO_HOME + NHOME * LW_HOME;  // first home index of home row l (then the number of home atoms)
constexpr int LO_TOTAL = LO_HOFF + 32;               // slots of the neighbourhood
constexpr int LAYOUT_WORDS = LO_TOTAL + 1;

struct Lay {
    volatile int32_t *w;
    __device__ __forceinline__ int32_t cell(int r, int t) const { return w[LO_CELL + r * LW_CELL + t]; }
    __device__ __forceinline__ int32_t da(int r) const { return w[LO_DA + r]; }
    __device__ __forceinline__ int32_t db(int r) const { return w[LO_DB + r]; }
    __device__ __forceinline__ int32_t sw(int r) const { return w[LO_SW + r]; }
    __device__ __forceinline__ int32_t home(int l, int t) const { return w[LO_HOME + l * LW_HOME + t]; }
    __device__ __forceinline__ int32_t hoff(int l) const { return w[LO_HOFF + l]; }
    __device__ __forceinline__ int32_t total() const { return w[LO_TOTAL]; }
};

struct BrickDims {
    int32_t x0, x1, y0, y1, z0, z1, bw, bh, bd, nyr, nrow, nhome;
};

__device__ __forceinline__ BrickDims brick_dims(const Brick &B) {
    BrickDims d;
    d.x0 = B.x01 & 0xffff;
    d.x1 = B.x01 >> 16;
    d.y0 = B.y01 & 0xffff;
    d.y1 = B.y01 >> 16;
    d.z0 = B.z01 & 0xffff;
    d.z1 = B.z01 >> 16;
    d.bw = d.x1 - d.x0;
    d.bh = d.y1 - d.y0;
    d.bd = d.z1 - d.z0;
    d.nyr = d.bh + 2;
    d.nrow = d.nyr * (d.bd + 2);
    d.nhome = d.bh * d.bd;
    return d;
}

__device__ __forceinline__ int32_t wrapc(int32_t v, int32_t n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Staging request of the pair loop: warp 0 issues the bulk copies of the
// rows (one or two contiguous runs each) from the values it computes, and
// arms the mbarrier with the bytes it copies.
struct StageCopy {
    uint32_t smem_base;  // shared address of slot 0
    uint32_t bar;        // shared address of the mbarrier (initialised, visible to warp 0)
    const int4 *xq;
    int64_t n;  // atoms in xq
    int32_t *status;
};

__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Fills the layout (warps 0 and 1; the caller synchronises the block).
// Every entry is written once, from values held in registers.  With cp,
// warp 0 also stages the neighbourhood when it fits cap slots; a run that
// would fall outside the stage or the atoms is not copied (and latches
// PPMD_ERR_INVALID: it cannot happen for a consistent cell list).
__device__ __forceinline__ void brick_layout(const BrickDims d, const Seg &S, const int32_t *__restrict__ cs, Lay L,
                                             const StageCopy *cp = nullptr, int32_t cap = 0) {
    const int tid = threadIdx.x, lane = tid & 31;
    const int32_t nx = S.nc[0], ny = S.nc[1], nz = S.nc[2];
    if (tid < 32) {
        const bool mine = tid < d.nrow;
        int32_t rb = 0, tot = 0;
        if (mine) {
            const int32_t yy = wrapc(d.y0 - 1 + tid % d.nyr, ny), zz = wrapc(d.z0 - 1 + tid / d.nyr, nz);
            rb = S.cell0 + (zz * ny + yy) * nx;
            for (int t = 0; t <= d.bw + 1; ++t) {
                const int32_t x = wrapc(d.x0 - 1 + t, nx);
                tot += cs[rb + x + 1] - cs[rb + x];
            }
        }
        int32_t inc = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        const int32_t base = inc - tot, total = __shfl_sync(0xffffffffu, inc, 31);
        int32_t da = 0, db = 0, sw = base + tot;
        if (mine) {
            int32_t acc = base;
            for (int t = 0; t <= d.bw + 1; ++t) {
                const int32_t x = wrapc(d.x0 - 1 + t, nx);
                L.w[LO_CELL + tid * LW_CELL + t] = acc;
                acc += cs[rb + x + 1] - cs[rb + x];
            }
            L.w[LO_CELL + tid * LW_CELL + d.bw + 2] = acc;
            const int32_t xa = d.x0 - 1, xb = d.x1;  // inclusive cell range of the row
            if (xa < 0) {  // cell nx-1 first, then cells 0 .. xb
                const int32_t len1 = cs[rb + nx] - cs[rb + nx - 1];
                da = cs[rb + nx - 1] - base;
                sw = base + len1;
                db = cs[rb] - (base + len1);
            } else if (xb >= nx) {  // cells xa .. nx-1, then cell 0
                const int32_t len1 = cs[rb + nx] - cs[rb + xa];
                da = cs[rb + xa] - base;
                sw = base + len1;
                db = cs[rb] - (base + len1);
            } else {
                da = cs[rb + xa] - base;
                db = da;
            }
            L.w[LO_DA + tid] = da;
            L.w[LO_DB + tid] = db;
            L.w[LO_SW + tid] = sw;
        }
        if (lane == 0) L.w[LO_TOTAL] = total;
        if (cp && total <= cap) {
            const int32_t a1 = base + tot;
            uint32_t b1 = 0, b2 = 0;
            if (mine) {
                const bool good = base >= 0 && base <= sw && sw <= a1 && a1 <= total &&
                                  (sw == base || ((int64_t)base + da >= 0 && (int64_t)sw - 1 + da < cp->n)) &&
                                  (a1 == sw || ((int64_t)sw + db >= 0 && (int64_t)a1 - 1 + db < cp->n));
                if (good) {
                    b1 = 16u * (uint32_t)(sw - base);
                    b2 = 16u * (uint32_t)(a1 - sw);
                } else {
                    latch_status(cp->status, PPMD_ERR_INVALID);
                }
            }
            const uint32_t bytes = __reduce_add_sync(0xffffffffu, b1 + b2);
            if (lane == 0)
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(cp->bar), "r"(bytes)
                             : "memory");
            __syncwarp();
            if (b1) bulk_copy_g2s(cp->smem_base + 16u * (uint32_t)base, cp->xq + (base + da), b1, cp->bar);
            if (b2) bulk_copy_g2s(cp->smem_base + 16u * (uint32_t)sw, cp->xq + (sw + db), b2, cp->bar);
        }
    } else if (tid < 64) {
        int32_t c = 0;
        if (lane < d.nhome) {
            const int32_t rm = S.cell0 + ((d.z0 + lane / d.bh) * ny + d.y0 + lane % d.bh) * nx;
            for (int t = 0; t <= d.bw; ++t) L.w[LO_HOME + lane * LW_HOME + t] = cs[rm + d.x0 + t];
            c = cs[rm + d.x0 + d.bw] - cs[rm + d.x0];
        }
        int32_t inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        L.w[LO_HOFF + lane] = inc - c;  // rows past nhome hold the number of home atoms
    }
}

// Stage row of slot s (the last row starting at or before s).
__device__ __forceinline__ int row_of(const Lay &L, int32_t nrow, int32_t s) {
    int r = 0, rh = nrow - 1;
    while (r < rh) {
        const int mid = (r + rh + 1) >> 1;
        if (L.cell(mid, 0) <= s) r = mid;
        else rh = mid - 1;
    }
    return r;
}

// Sorted atom index of slot s.
__device__ __forceinline__ int32_t slot_atom(const Lay &L, int32_t nrow, int32_t s) {
    const int r = row_of(L, nrow, s);
    return s + (s < L.sw(r) ? L.da(r) : L.db(r));
}

// Home atom h of the brick: its sorted index, home row and home cell.
struct HomeAtom {
    int32_t i, hr, t;
};
__device__ __forceinline__ HomeAtom home_atom(const Lay &L, const BrickDims &d, int32_t h) {
    HomeAtom a;
    a.hr = 0;
    while (a.hr + 1 < d.nhome && L.hoff(a.hr + 1) <= h) ++a.hr;
    a.i = L.home(a.hr, 0) + (h - L.hoff(a.hr));
    a.t = 0;
    while (a.t + 1 < d.bw && a.i >= L.home(a.hr, a.t + 1)) ++a.t;
    return a;
}

// Slot of a home atom in its own stage row.
__device__ __forceinline__ int32_t home_slot(const Lay &L, const BrickDims &d, const HomeAtom &a) {
    const int32_t r = (a.hr / d.bh + 1) * d.nyr + (a.hr % d.bh + 1);
    return L.cell(r, a.t + 1) + (a.i - L.home(a.hr, a.t));
}


// ---------------------------------------------------------------------
// List build.
// ---------------------------------------------------------------------
__global__ void __launch_bounds__(SLOT_THREADS) k_slot_list(const Brick *__restrict__ bricks, const int4 *__restrict__ xq,
                                                            const double *__restrict__ pos64, SegTable st,
                                                            const int32_t *__restrict__ cs, uint16_t *__restrict__ W16,
                                                            int64_t ld, int32_t *__restrict__ cnt, int32_t max_nbr,
                                                            int32_t stage_cap, int32_t *status,
                                                            unsigned long long *needed, int32_t *stage_need,
                                                            int64_t n) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int32_t lay_w[LAYOUT_WORDS];
    const Lay L{lay_w};
    const Brick B = bricks[blockIdx.x];
    const Seg &S = seg_ref(st, B.seg);
    const BrickDims d = brick_dims(B);
    brick_layout(d, S, cs, L);
    __syncthreads();
    const int32_t T = L.total(), H = L.hoff(d.nhome);
    const int tid = threadIdx.x;
    if (T > stage_cap) {
        // the neighbourhood does not fit the stage: no list for these atoms
        for (int32_t h = tid; h < H; h += blockDim.x) cnt[home_atom(L, d, h).i] = 0;
        if (tid == 0) {
            atomicMax(stage_need, T);
            latch_status(status, PPMD_ERR_CAPACITY);
        }
        return;
    }
    // Where the neighbourhood leaves at least one cell of the periodic grid
    // outside it in every direction, positions are staged as FP32 offsets
    // from its centre (the periodic image seen from the brick) and ordered
    // by x within each row, so each row's candidates are a window in x;
    // otherwise the fixed-point words are staged and every candidate of the
    // 27 cells is tested.
    const bool FSTAGE = d.bw + 3 <= S.nc[0] && d.bh + 3 <= S.nc[1] && d.bd + 3 <= S.nc[2];
    float4 *s_f = reinterpret_cast<float4 *>(smem);
    int4 *s_x = reinterpret_cast<int4 *>(smem);
    uint16_t *rowbuf = reinterpret_cast<uint16_t *>(smem + (size_t)stage_cap * 16);
    // FP32 offsets from the neighbourhood's centre, exact to 2^-23 of at most
    // five cells: r^2 moves by less than 1e-5 r^2, inside the FP64 re-test band
    const uint32_t refx = (uint32_t)__float2ull_rz((d.x0 - 1 + 0.5f * (d.bw + 2)) / (float)S.nc[0] * 4294967296.0f);
    const uint32_t refy = (uint32_t)__float2ull_rz((d.y0 - 1 + 0.5f * (d.bh + 2)) / (float)S.nc[1] * 4294967296.0f);
    const uint32_t refz = (uint32_t)__float2ull_rz((d.z0 - 1 + 0.5f * (d.bd + 2)) / (float)S.nc[2] * 4294967296.0f);
    const float sx = S.sx[0], sy = S.sx[1], sz = S.sx[2];
    for (int32_t s = tid; s < T; s += blockDim.x) {
        const int32_t j = slot_atom(L, d.nrow, s);
        if (j < 0 || j >= n) {  // cannot happen for a consistent cell list
            latch_status(status, PPMD_ERR_INVALID);
            continue;
        }
        const int4 q = xq[j];
        if (FSTAGE)
            s_f[s] = make_float4((float)(int32_t)((uint32_t)q.x - refx) * sx, (float)(int32_t)((uint32_t)q.y - refy) * sy,
                                 (float)(int32_t)((uint32_t)q.z - refz) * sz, 0.0f);
        else
            s_x[s] = q;
    }
    __syncthreads();
    const int g = tid / GROUP, l8 = tid % GROUP;
    const unsigned gmask = 0xffu << (GROUP * (g % (32 / GROUP)));
    const unsigned lt = (1u << l8) - 1u;
    uint16_t *rb = rowbuf + (size_t)g * max_nbr;
    const float lo = S.rl2_lo, hi = S.rl2_hi;
    const float rwin = sqrtf((float)S.rl2) * 1.00001f + 1e-5f;
    for (int32_t h = g; h < H; h += NGROUP) {
        const HomeAtom a = home_atom(L, d, h);
        const int32_t self = home_slot(L, d, a);
        if (a.i < 0 || a.i >= n || self < 0 || self >= T) {  // cannot happen for a consistent cell list
            if (l8 == 0) latch_status(status, PPMD_ERR_INVALID);
            continue;
        }
        const int32_t hy = a.hr % d.bh, hz = a.hr / d.bh;
        const double *pi = pos64 + 3 * (int64_t)a.i;
        const float4 fi = s_f[self];  // one of the two, as staged
        const int4 qi = s_x[self];
        // candidate window of each of the nine rows: lane q finds row q's
        // (rows 0 .. 7), every lane row 8's
        auto window = [&](int q, int32_t &wa, int32_t &wb) {
            const int r = (hz + q / 3) * d.nyr + hy + q % 3;
            wa = max(L.cell(r, a.t), 0);
            wb = min(L.cell(r, a.t + 3), T);
            if (FSTAGE) {
                const float xlo = fi.x - rwin, xhi = fi.x + rwin;
                int32_t lo_ = wa, hi_ = wb;
                while (lo_ < hi_) {  // first slot with x >= xlo
                    const int32_t mid = (lo_ + hi_) >> 1;
                    if (s_f[mid].x < xlo) lo_ = mid + 1;
                    else hi_ = mid;
                }
                int32_t lo2 = lo_, hi2 = wb;
                while (lo2 < hi2) {  // first slot with x > xhi
                    const int32_t mid = (lo2 + hi2) >> 1;
                    if (s_f[mid].x <= xhi) lo2 = mid + 1;
                    else hi2 = mid;
                }
                wa = lo_;
                wb = lo2;
            }
        };
        int32_t wa_l, wb_l, wa8, wb8;
        window(l8, wa_l, wb_l);
        window(8, wa8, wb8);
        int32_t count = 0;
        for (int q = 0; q < 9; ++q) {
            const int32_t wa = q < 8 ? __shfl_sync(gmask, wa_l, q, GROUP) : wa8;
            const int32_t wb = q < 8 ? __shfl_sync(gmask, wb_l, q, GROUP) : wb8;
            const int r = (hz + q / 3) * d.nyr + hy + q % 3;
            for (int32_t k0 = wa; k0 < wb; k0 += GROUP) {
                const int32_t k = k0 + l8;
                bool hit = false;
                if (k < wb && k != self) {
                    float r2;
                    if (FSTAGE) {
                        const float4 f = s_f[k];
                        const float dx = fi.x - f.x, dy = fi.y - f.y, dz = fi.z - f.z;
                        r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    } else {
                        const int4 x = s_x[k];
                        const float dx = fdiff(qi.x, x.x) * sx, dy = fdiff(qi.y, x.y) * sy, dz = fdiff(qi.z, x.z) * sz;
                        r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    }
                    if (r2 < hi) {
                        if (r2 < lo) {
                            hit = true;
                        } else {
                            const int32_t j = k + (k < L.sw(r) ? L.da(r) : L.db(r));
                            double dr[3];
                            hit = j >= 0 && j < n && min_image_r2(pi, pos64 + 3 * (int64_t)j, S, dr) < S.rl2;
                        }
                    }
                }
                const unsigned m = __ballot_sync(gmask, hit) >> (GROUP * (g % (32 / GROUP)));
                const int32_t at = count + __popc(m & lt);
                if (hit && at < max_nbr) rb[at] = (uint16_t)k;
                count += __popc(m);
            }
        }
        // pad the last group of eight with the sentinel slot (T, far away)
        const int32_t kept = min(count, max_nbr);
        const int32_t words = (kept + 7) >> 3;
        for (int32_t e = kept + l8; e < words * 8; e += GROUP) rb[e] = (uint16_t)T;
        __syncwarp(gmask);
        uint4 *col = reinterpret_cast<uint4 *>(W16) + a.i;
        for (int32_t w = l8; w < words; w += GROUP) col[(int64_t)w * ld] = reinterpret_cast<const uint4 *>(rb)[w];
        if (l8 == 0) {
            cnt[a.i] = count;
            if (count > max_nbr) {
                latch_status(status, PPMD_ERR_CAPACITY);
                latch_needed(needed, (unsigned long long)count);
            }
        }
        __syncwarp(gmask);
    }
}

// ---------------------------------------------------------------------
// Pair loop.
// ---------------------------------------------------------------------
__device__ __forceinline__ uint4 ld_stream16(const uint4 *p) {
    uint4 v;
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}
__device__ __forceinline__ void pair_add(float &s, float &e, float s2, float e2) {
    const float t = s + s2, bb = t - s, err = (s - (t - bb)) + (s2 - bb);
    const float lo = err + (e + e2);
    s = t + lo;
    e = lo - (s - t);
}

// Per-block (U, W, K) sums as the column-major loop takes them: FP32 pairs
// (hi, lo) reduced over the warp by error-free transformations, FP64 over
// the warps in a fixed order.
__device__ __forceinline__ void block_sum3_pairs(double a, double b, double c, double *partials) {
    __shared__ double sh[3][SLOT_THREADS / 32];
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

__device__ __forceinline__ bool stage_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t it = 0; it < STAGE_WAIT_LIMIT; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n"
            ".reg .pred p;\n"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n"
            "}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

template <bool ENERGY, bool DRIFT>
__global__ void __launch_bounds__(SLOT_THREADS, 6) k_lj_slots32(const Brick *__restrict__ bricks,
                                                                const int4 *__restrict__ xq,
                                                                const double *__restrict__ pos64, SegTable st,
                                                                const int32_t *__restrict__ cs, LJConst c,
                                                                const uint16_t *__restrict__ W16, int64_t ld,
                                                                const int32_t *__restrict__ cnt, int32_t max_nbr,
                                                                int32_t stage_cap, float4 *__restrict__ f4,
                                                                double *__restrict__ vel, double h, double half_m,
                                                                double *__restrict__ partials, Drift dr,
                                                                int32_t *status, int64_t n) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int32_t lay_w[LAYOUT_WORDS];
    __shared__ __align__(8) unsigned long long bar_word;
    const Lay L{lay_w};
    int4 *s_x = reinterpret_cast<int4 *>(smem);
    const Brick B = bricks[blockIdx.x];
    const Seg &S = seg_ref(st, B.seg);
    const BrickDims d = brick_dims(B);
    const int tid = threadIdx.x;
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&bar_word);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    // the layout; warp 0 also copies the neighbourhood into the stage (the
    // row's one or two contiguous runs of the sorted positions per lane)
    const StageCopy cp{(uint32_t)__cvta_generic_to_shared(s_x), bar, xq, n, status};
    brick_layout(d, S, cs, L, &cp, stage_cap);
    __syncthreads();
    const int32_t T = L.total(), H = L.hoff(d.nhome);
    const bool staged = T <= stage_cap;  // else the list build left no entries (and latched the error)
    bool ok = true;
    if (staged) {
        if (tid == 32) {
            // sentinel slot T: half a box away from the neighbourhood's
            // centre in every direction, beyond every cutoff from a home atom
            const uint32_t rx = (uint32_t)__float2ull_rz((d.x0 - 1 + 0.5f * (d.bw + 2)) / (float)S.nc[0] * 4294967296.0f);
            const uint32_t ry = (uint32_t)__float2ull_rz((d.y0 - 1 + 0.5f * (d.bh + 2)) / (float)S.nc[1] * 4294967296.0f);
            const uint32_t rz = (uint32_t)__float2ull_rz((d.z0 - 1 + 0.5f * (d.bd + 2)) / (float)S.nc[2] * 4294967296.0f);
            s_x[T] = make_int4((int)(rx + 0x80000000u), (int)(ry + 0x80000000u), (int)(rz + 0x80000000u), B.seg);
        }
        __syncthreads();  // the sentinel
        ok = stage_wait(bar, 0);
        if (!ok) {
            // give the copies in flight a second bounded wait before the
            // block (and its shared memory) ends
            latch_status(status, PPMD_ERR_TIMEOUT);
            stage_wait(bar, 0);
        }
    }
    double u_sum = 0.0, w_sum = 0.0, k_sum = 0.0;
    float d2max = 0.0f;
    const f2 sxx = pk(S.sx[0], S.sx[0]), syy = pk(S.sx[1], S.sx[1]), szz = pk(S.sx[2], S.sx[2]);
    for (int32_t hh = tid; ok && hh < H; hh += blockDim.x) {
        const int64_t i = home_atom(L, d, hh).i;
        if (i < 0 || i >= n) {  // cannot happen for a consistent cell list
            latch_status(status, PPMD_ERR_INVALID);
            continue;
        }
        const int4 xi = xq[i];
        const f2 two = pk(2.0f, 2.0f), half = pk(0.5f, 0.5f), one = pk(1.0f, 1.0f);
        const f2 s2 = pk(c.s2, c.s2), f48 = pk(c.f48, c.f48), e2 = pk(c.e2, c.e2), shift = pk(c.shift, c.shift);
        const int32_t m = staged ? min(cnt[i], max_nbr) : 0;
        Kahan2 fx, fy, fz, ea, vir;
        fx.init();
        fy.init();
        fz.init();
        if (ENERGY) {
            ea.init();
            vir.init();
        }
        // two neighbours per packed step; fm = 0 outside the cutoff (the
        // sentinel is always outside)
        auto step = [&](int32_t s0, int32_t s1, const int4 &a, const int4 &b, f2 &tx, f2 &ty, f2 &tz) {
            const f2 dx = mul2(pk(fdiff(xi.x, a.x), fdiff(xi.x, b.x)), sxx);
            const f2 dy = mul2(pk(fdiff(xi.y, a.y), fdiff(xi.y, b.y)), syy);
            const f2 dz = mul2(pk(fdiff(xi.z, a.z), fdiff(xi.z, b.z)), szz);
            const f2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
            float r2a, r2b;
            upk(r2, r2a, r2b);
            bool in0 = r2a < c.rc2_lo, in1 = r2b < c.rc2_lo;
            if (!in0 && r2a < c.rc2_hi) {
                const int32_t j = slot_atom(L, d.nrow, s0);
                double drr[3];
                in0 = j >= 0 && j < n && min_image_r2(pos64 + 3 * i, pos64 + 3 * (int64_t)j, S, drr) < c.rc2;
            }
            if (!in1 && r2b < c.rc2_hi) {
                const int32_t j = slot_atom(L, d.nrow, s1);
                double drr[3];
                in1 = j >= 0 && j < n && min_image_r2(pos64 + 3 * i, pos64 + 3 * (int64_t)j, S, drr) < c.rc2;
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
        // four neighbours: the four terms of each component enter the
        // compensated sum as one plain FP32 partial (two per stream)
        auto quad = [&](uint32_t w01, uint32_t w23) {
            // slots past the sentinel cannot come from the list build; the
            // clamp keeps every read inside the stage whatever the list holds
            const int32_t s0 = min((int32_t)(w01 & 0xffffu), T), s1 = min((int32_t)(w01 >> 16), T);
            const int32_t s2_ = min((int32_t)(w23 & 0xffffu), T), s3 = min((int32_t)(w23 >> 16), T);
            const int4 a0 = s_x[s0], a1 = s_x[s1], a2 = s_x[s2_], a3 = s_x[s3];
            f2 tx0, ty0, tz0, tx1, ty1, tz1;
            step(s0, s1, a0, a1, tx0, ty0, tz0);
            step(s2_, s3, a2, a3, tx1, ty1, tz1);
            fx.add(add2(tx0, tx1));
            fy.add(add2(ty0, ty1));
            fz.add(add2(tz0, tz1));
        };
        const uint4 *col = reinterpret_cast<const uint4 *>(W16) + i;  // eight entries per word
        const int32_t nw = (m + 7) >> 3;
        uint4 g = nw > 0 ? ld_stream16(col) : make_uint4(0u, 0u, 0u, 0u);
        for (int32_t w = 0; w < nw; ++w) {
            const uint4 nx = w + 1 < nw ? ld_stream16(col + (int64_t)(w + 1) * ld) : g;
            quad(g.x, g.y);
            if (8 * w + 4 < m) quad(g.z, g.w);  // the second half holds entries (or only sentinels)
            g = nx;
        }
        float hx, lx, hy, ly, hz, lz;
        fx.merged(hx, lx);
        fy.merged(hy, ly);
        fz.merged(hz, lz);
        // hx + lx rounded once to FP32 (the same float as through FP64: the
        // double rounding of a sum of two floats is innocuous at 53 bits)
        const float Fx = hx + lx, Fy = hy + ly, Fz = hz + lz;
        float he = 0.f, le = 0.f;
        if (ENERGY) {
            ea.merged(he, le);
            float hv, lv;
            vir.merged(hv, lv);
            u_sum += (double)he + (double)le;
            w_sum += 0.5 * ((double)hv + (double)lv);
        }
        f4[i] = make_float4(Fx, Fy, Fz, he + le);
        if (vel) {
            // second kick of Algorithm 6 with the forces just computed
            const float4 fq = make_float4(Fx, Fy, Fz, 0.0f);
            const double f[3] = {(double)fq.x, (double)fq.y, (double)fq.z};
            double v[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) v[k] = fma(h, f[k], vel[3 * i + k]);
            if (ENERGY) k_sum += half_m * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            if (DRIFT) {
                // the next step's kick and drift, as k_kick_drift2
                const int4 ref = dr.xq_ref[i];
                const Seg &Sd = seg_ref(st, ref.w);
                uint32_t q[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    v[k] = fma(h, f[k], v[k]);
                    const double r = fma(dr.dt, v[k], pos64[3 * i + k]);
                    dr.pos_next[3 * i + k] = r;
                    q[k] = (uint32_t)(unsigned long long)__double2ll_rn(r * Sd.fxs[k]);
                }
                dr.xq_next[i] = make_int4((int)q[0], (int)q[1], (int)q[2], ref.w);
                const float ex = fixed_delta(q[0], (uint32_t)ref.x, Sd.sx[0]);
                const float ey = fixed_delta(q[1], (uint32_t)ref.y, Sd.sx[1]);
                const float ez = fixed_delta(q[2], (uint32_t)ref.z, Sd.sx[2]);
                d2max = fmaxf(d2max, fmaf(ex, ex, fmaf(ey, ey, ez * ez)));
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) vel[3 * i + k] = v[k];
        }
    }
    if (DRIFT) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d2max = fmaxf(d2max, __shfl_xor_sync(0xffffffffu, d2max, o));
        if ((tid & 31) == 0 && d2max > 0.0f) atomicMax(dr.max_disp_bits, __float_as_uint(d2max));
    }
    if (ENERGY) block_sum3_pairs(u_sum, w_sum, k_sum, partials);
}

// Slot lists to the column-major atom-index list (entries grouped by four,
// as build_list_bricks writes them), same entries in the same order.
__global__ void __launch_bounds__(SLOT_THREADS) k_slots_to_atoms(const Brick *__restrict__ bricks, SegTable st,
                                                                 const int32_t *__restrict__ cs,
                                                                 const uint16_t *__restrict__ W16, int64_t ld,
                                                                 const int32_t *__restrict__ cnt, int32_t max_nbr,
                                                                 int32_t stage_cap, int32_t *__restrict__ W,
                                                                 int64_t n) {
    __shared__ int32_t lay_w[LAYOUT_WORDS];
    const Lay L{lay_w};
    const Brick B = bricks[blockIdx.x];
    const Seg &S = seg_ref(st, B.seg);
    const BrickDims d = brick_dims(B);
    brick_layout(d, S, cs, L);
    __syncthreads();
    const int32_t H = L.hoff(d.nhome), T = L.total();
    if (T > stage_cap) return;
    for (int32_t hh = threadIdx.x; hh < H; hh += blockDim.x) {
        const int64_t i = home_atom(L, d, hh).i;
        if (i < 0 || i >= n) continue;  // cannot happen for a consistent cell list
        const int32_t m = min(cnt[i], max_nbr);
        for (int32_t e = 0; e < ((m + 3) & ~3); ++e) {
            int32_t j = -1;
            if (e < m) j = slot_atom(L, d.nrow, min((int32_t)W16[(((int64_t)(e >> 3) * ld + i) << 3) + (e & 7)], T - 1));
            if (j >= n) j = -1;
            W[(((int64_t)(e >> 2) * ld + i) << 2) + (e & 3)] = j;
        }
    }
}

}  // namespace

size_t slot_list_smem(int32_t stage_cap, int32_t max_nbr) {
    return (size_t)stage_cap * 16 + (size_t)NGROUP * (size_t)((max_nbr + 7) & ~7) * sizeof(uint16_t);
}

size_t slot_pair_smem(int32_t stage_cap) { return (size_t)(stage_cap + 1) * 16; }

int slots_setup(ppmd_ctx *ctx, int32_t stage_cap, int32_t max_nbr) {
    const int ls = (int)slot_list_smem(stage_cap, max_nbr), ps = (int)slot_pair_smem(stage_cap);
    int rc = cuda_check(ctx, cudaFuncSetAttribute(k_slot_list, cudaFuncAttributeMaxDynamicSharedMemorySize, ls),
                        "cudaFuncSetAttribute");
    auto set = [&](const void *f) {
        if (rc == PPMD_OK)
            rc = cuda_check(ctx, cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, ps),
                            "cudaFuncSetAttribute");
    };
    set((const void *)k_lj_slots32<false, false>);
    set((const void *)k_lj_slots32<false, true>);
    set((const void *)k_lj_slots32<true, false>);
    set((const void *)k_lj_slots32<true, true>);
    return rc;
}

int build_slot_list(ppmd_ctx *ctx, int64_t nbricks, const Brick *bricks, const int4 *xq,
                    const double *pos64, const SegTable &st, const int32_t *cell_start, uint16_t *W16, int64_t ld,
                    int32_t *cnt, int32_t max_nbr, int32_t stage_cap, int32_t *stage_need, int64_t n_atoms) {
    if ((max_nbr & 7) || max_nbr <= 0) return set_error(ctx, PPMD_ERR_INVALID, "slot list needs a capacity divisible by 8");
    if (nbricks > 0) {
        PPMD_LAUNCH(ctx, k_slot_list, nbricks, SLOT_THREADS, slot_list_smem(stage_cap, max_nbr), bricks, xq, pos64, st,
                    cell_start, W16, ld, cnt, max_nbr, stage_cap, ctx->d_status, ctx->d_needed, stage_need, n_atoms);
    }
    return check_launch(ctx, "build_slot_list");
}

int lj_slots(ppmd_ctx *ctx, int64_t nbricks, const Brick *bricks, const int4 *xq, const double *pos64,
             const SegTable &st, const int32_t *cell_start, const LJConst &c, const uint16_t *W16, int64_t ld,
             const int32_t *cnt, int32_t max_nbr, int32_t stage_cap, float4 *f4, double *vel, double h,
             double half_m, double *partials, const Drift &drift, int64_t n_atoms) {
    if (nbricks <= 0) return PPMD_OK;
    if (drift.pos_next && !vel) return set_error(ctx, PPMD_ERR_INVALID, "lj_slots: drift needs a kick");
    const bool e = partials != nullptr, dd = drift.pos_next != nullptr;
    auto kern = e ? (dd ? k_lj_slots32<true, true> : k_lj_slots32<true, false>)
                  : (dd ? k_lj_slots32<false, true> : k_lj_slots32<false, false>);
    PPMD_LAUNCH(ctx, kern, nbricks, SLOT_THREADS, slot_pair_smem(stage_cap), bricks, xq, pos64, st, cell_start, c, W16,
                ld, cnt, max_nbr, stage_cap, f4, vel, h, half_m, partials, drift, ctx->d_status, n_atoms);
    return check_launch(ctx, "lj_slots");
}

int slots_to_atoms(ppmd_ctx *ctx, int64_t nbricks, const Brick *bricks, const SegTable &st, const int32_t *cell_start,
                   const uint16_t *W16, int64_t ld, const int32_t *cnt, int32_t max_nbr, int32_t stage_cap, int32_t *W,
                   int64_t n_atoms) {
    if (nbricks > 0)
        PPMD_LAUNCH(ctx, k_slots_to_atoms, nbricks, SLOT_THREADS, 0, bricks, st, cell_start, W16, ld, cnt, max_nbr,
                    stage_cap, W, n_atoms);
    return check_launch(ctx, "slots_to_atoms");
}

}  // namespace ppmd
