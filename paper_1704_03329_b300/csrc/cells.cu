// Cell binning by counting sort (Sec. 3.5): histogram -> exclusive scan ->
// scatter -> per-cell ordering by atom index (or by x coordinate, for the
// sorted layouts whose list build searches each row of cells by x).
#include "cells.cuh"

namespace ppmd {

template <bool EXACT>
__global__ void k_bin(const double *__restrict__ pos, int64_t n, SegTable st, const int32_t *__restrict__ seg_of,
                      int32_t *__restrict__ cell_of, int32_t *__restrict__ count, int32_t *status) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t sid = seg_of ? seg_of[i] : 0;
    const Seg &S = seg_ref(st, sid);
    int32_t c[3];
    bool bad = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double x = pos[3 * i + d];
        if (!isfinite(x)) {
            bad = true;
            x = 0.0;
        }
        int32_t cd;
        if (EXACT) {
            double xw = wrap_exact(x, S.L[d]);
            cd = (int32_t)floor(__ddiv_rn(xw, S.w[d]));
        } else {
            cd = (int32_t)floor(x * S.inv_w[d]);
            if (x < 0.0 || x >= S.L[d]) cd = (int32_t)floor(wrap_exact(x, S.L[d]) * S.inv_w[d]);
        }
        cd = cd < 0 ? 0 : (cd > S.nc[d] - 1 ? S.nc[d] - 1 : cd);
        c[d] = cd;
    }
    if (bad) latch_status(status, PPMD_ERR_NONFINITE);
    int32_t cell = S.cell0 + (c[2] * S.nc[1] + c[1]) * S.nc[0] + c[0];
    cell_of[i] = cell;
    atomicAdd(&count[cell], 1);
}

__global__ void k_scatter(int64_t n, const int32_t *__restrict__ cell_of, const int32_t *__restrict__ cell_start,
                          int32_t *__restrict__ cursor, int32_t *__restrict__ cell_atoms) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t c = cell_of[i];
    int32_t slot = atomicAdd(&cursor[c], 1);
    cell_atoms[cell_start[c] + slot] = (int32_t)i;
}

// As k_scatter, also writing the sort key of each slot: the atom's x
// coordinate wrapped into its box (FP32; monotone in the fixed-point word).
__global__ void k_scatter_x(int64_t n, const double *__restrict__ pos, SegTable st, const int32_t *__restrict__ seg_of,
                            const int32_t *__restrict__ cell_of, const int32_t *__restrict__ cell_start,
                            int32_t *__restrict__ cursor, int32_t *__restrict__ cell_atoms, float *__restrict__ key) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Seg &S = seg_ref(st, seg_of ? seg_of[i] : 0);
    double x = pos[3 * i];
    if (!(x >= 0.0 && x < S.L[0])) x = isfinite(x) ? wrap_exact(x, S.L[0]) : 0.0;
    int32_t c = cell_of[i];
    int32_t slot = cell_start[c] + atomicAdd(&cursor[c], 1);
    cell_atoms[slot] = (int32_t)i;
    key[slot] = (float)x;
}

// Order every cell's atoms by (x, index): one thread per slot counts the
// members of its cell that come first (cells are small) and writes its atom
// at that rank.  The key is the x coordinate (FP32) or its fixed-point word.
template <class Key>
__global__ void k_rank_cells_x(int64_t n, const int32_t *__restrict__ cell_of, const int32_t *__restrict__ cell_start,
                               const int32_t *__restrict__ tmp_atoms, const Key *__restrict__ key,
                               int32_t *__restrict__ cell_atoms) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int32_t v = tmp_atoms[s];
    const Key kv = key[s];
    const int32_t c = cell_of[v], a = cell_start[c], b = cell_start[c + 1];
    int32_t rank = 0;
    for (int32_t t = a; t < b; ++t) {
        const Key kt = key[t];
        rank += (kt < kv) || (kt == kv && tmp_atoms[t] < v);
    }
    cell_atoms[a + rank] = v;
}

// Cell of a fixed-point coordinate word q on a grid of nc cells: the c with
// c 2^32 <= q nc < (c + 1) 2^32 (cells of the box's edge L / nc, in exact
// integer arithmetic).
__device__ __forceinline__ int32_t fixed_cell(uint32_t q, int32_t nc) {
    return (int32_t)(((unsigned long long)q * (unsigned long long)(uint32_t)nc) >> 32);
}

__global__ void k_bin_fixed(const int4 *__restrict__ xq, int64_t n, SegTable st, int32_t *__restrict__ cell_of,
                            int32_t *__restrict__ count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int4 x = xq[i];
    const Seg &S = seg_ref(st, x.w);
    const int32_t cell = S.cell0 + (fixed_cell((uint32_t)x.z, S.nc[2]) * S.nc[1] + fixed_cell((uint32_t)x.y, S.nc[1])) *
                                       S.nc[0] +
                         fixed_cell((uint32_t)x.x, S.nc[0]);
    cell_of[i] = cell;
    atomicAdd(&count[cell], 1);
}

// As k_scatter, the sort key of each slot being the atom's fixed-point x word.
__global__ void k_scatter_fx(int64_t n, const int4 *__restrict__ xq, const int32_t *__restrict__ cell_of,
                             const int32_t *__restrict__ cell_start, int32_t *__restrict__ cursor,
                             int32_t *__restrict__ cell_atoms, uint32_t *__restrict__ key) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t c = cell_of[i];
    const int32_t slot = cell_start[c] + atomicAdd(&cursor[c], 1);
    cell_atoms[slot] = (int32_t)i;
    key[slot] = (uint32_t)xq[i].x;
}

// Order every cell's atoms by index (insertion sort; cells are small).
__global__ void k_sort_cells(int64_t ncell, const int32_t *__restrict__ cell_start, int32_t *__restrict__ cell_atoms) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    int32_t a = cell_start[c], b = cell_start[c + 1];
    for (int32_t k = a + 1; k < b; ++k) {
        int32_t v = cell_atoms[k];
        int32_t m = k - 1;
        while (m >= a && cell_atoms[m] > v) {
            cell_atoms[m + 1] = cell_atoms[m];
            --m;
        }
        cell_atoms[m + 1] = v;
    }
}

int bin_atoms(ppmd_ctx *ctx, const double *pos, int64_t n, const SegTable &st, const int32_t *seg_of, int64_t ncell,
              bool exact, int32_t *cell_of, int32_t *cell_start, int32_t *cell_atoms, bool order_x) {
    cudaStream_t s = ctx->stream;
    PPMD_TRY(cuda_check(ctx, cudaMemsetAsync(cell_start, 0, sizeof(int32_t) * (size_t)(ncell + 1), s), "memset"));
    if (n > 0) {
        if (exact)
            PPMD_LAUNCH(ctx, k_bin<true>, div_up(n, 256), 256, 0, pos, n, st, seg_of, cell_of, cell_start, ctx->d_status);
        else
            PPMD_LAUNCH(ctx, k_bin<false>, div_up(n, 256), 256, 0, pos, n, st, seg_of, cell_of, cell_start, ctx->d_status);
    }
    PPMD_TRY(exclusive_scan(ctx, cell_start, cell_start, ncell));
    if (n > 0) {
        int32_t *cursor = (int32_t *)scratch(ctx, S_COUNT, sizeof(int32_t) * (size_t)ncell);
        if (!cursor) return PPMD_ERR_NOMEM;
        PPMD_TRY(cuda_check(ctx, cudaMemsetAsync(cursor, 0, sizeof(int32_t) * (size_t)ncell, s), "memset"));
        if (order_x) {
            float *key = (float *)scratch(ctx, S_CELLKEY, sizeof(float) * (size_t)n);
            int32_t *tmp = (int32_t *)scratch(ctx, S_CELLTMP, sizeof(int32_t) * (size_t)n);
            if (!key || !tmp) return PPMD_ERR_NOMEM;
            PPMD_LAUNCH(ctx, k_scatter_x, div_up(n, 256), 256, 0, n, pos, st, seg_of, cell_of, cell_start, cursor, tmp,
                        key);
            PPMD_LAUNCH(ctx, k_rank_cells_x<float>, div_up(n, 256), 256, 0, n, cell_of, cell_start, tmp, key, cell_atoms);
        } else {
            PPMD_LAUNCH(ctx, k_scatter, div_up(n, 256), 256, 0, n, cell_of, cell_start, cursor, cell_atoms);
            PPMD_LAUNCH(ctx, k_sort_cells, div_up(ncell, 128), 128, 0, ncell, cell_start, cell_atoms);
        }
    }
    return check_launch(ctx, "bin_atoms");
}

// Words of a cell fraction (2^-32 of a cell edge) within which a word is
// taken to lie on a cell face.
constexpr uint32_t FACE_MARGIN = 1u << 22;

// The cells of k_bin<false> (FP64 positions, reciprocal of the cell edge)
// found from the fixed-point words instead.  The word of an axis is the
// position to within a quantum L 2^-32 (nc units of the cell fraction), and
// the FP64 product x / w is exact to 2^-52 relative, so away from a cell face
// (FACE_MARGIN >> nc) the cell c = floor(q nc / 2^32) is the FP64 formula's
// cell; within the margin (about one atom in 500 per axis) and for
// non-finite positions the FP64 formula itself decides.  Integer work for
// almost every atom: FP64 runs at a small fraction of the integer rate here.
__global__ void k_bin_xq(const int4 *__restrict__ xq, const double *__restrict__ pos, int64_t n, SegTable st,
                         const int32_t *__restrict__ seg_of, int32_t *__restrict__ cell_of, int32_t *__restrict__ count,
                         int32_t *status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int4 q = xq[i];
    const Seg &S = seg_ref(st, seg_of ? seg_of[i] : 0);
    const uint32_t qw[3] = {(uint32_t)q.x, (uint32_t)q.y, (uint32_t)q.z};
    int32_t c[3];
    bool bad = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double x = pos[3 * i + d];
        const bool finite = ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;  // exponent not all ones
        const unsigned long long prod = (unsigned long long)qw[d] * (unsigned long long)(uint32_t)S.nc[d];
        const uint32_t frac = (uint32_t)prod;
        int32_t cd = (int32_t)(prod >> 32);
        if (!finite || frac < FACE_MARGIN || frac > 0xffffffffu - FACE_MARGIN) {
            if (!finite) {
                bad = true;
                x = 0.0;
            }
            cd = (int32_t)floor(x * S.inv_w[d]);
            if (x < 0.0 || x >= S.L[d]) cd = (int32_t)floor(wrap_exact(x, S.L[d]) * S.inv_w[d]);
            cd = cd < 0 ? 0 : (cd > S.nc[d] - 1 ? S.nc[d] - 1 : cd);
        }
        c[d] = cd;
    }
    if (bad) latch_status(status, PPMD_ERR_NONFINITE);
    const int32_t cell = S.cell0 + (c[2] * S.nc[1] + c[1]) * S.nc[0] + c[0];
    cell_of[i] = cell;
    atomicAdd(&count[cell], 1);
}

// As k_scatter, the sort key of each slot being the atom's x word relative
// to the centre of its cell (signed: monotone in x across the cell even
// where the cell touches the periodic face at x = 0).
__global__ void k_scatter_xq(int64_t n, const int4 *__restrict__ xq, SegTable st, const int32_t *__restrict__ seg_of,
                             const int32_t *__restrict__ cell_of, const int32_t *__restrict__ cell_start,
                             int32_t *__restrict__ cursor, int32_t *__restrict__ cell_atoms, int32_t *__restrict__ key) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Seg &S = seg_ref(st, seg_of ? seg_of[i] : 0);
    const int32_t c = cell_of[i];
    const int32_t cx = (c - S.cell0) % S.nc[0];
    const uint32_t mid = (uint32_t)((((unsigned long long)(2 * cx + 1)) << 31) / (unsigned long long)(uint32_t)S.nc[0]);
    const int32_t slot = cell_start[c] + atomicAdd(&cursor[c], 1);
    cell_atoms[slot] = (int32_t)i;
    key[slot] = (int32_t)((uint32_t)xq[i].x - mid);
}

int bin_atoms_md(ppmd_ctx *ctx, const int4 *xq, const double *pos, int64_t n, const SegTable &st, const int32_t *seg_of,
                 int64_t ncell, int32_t *cell_of, int32_t *cell_start, int32_t *cell_atoms) {
    cudaStream_t s = ctx->stream;
    PPMD_TRY(cuda_check(ctx, cudaMemsetAsync(cell_start, 0, sizeof(int32_t) * (size_t)(ncell + 1), s), "memset"));
    if (n > 0)
        PPMD_LAUNCH(ctx, k_bin_xq, div_up(n, 256), 256, 0, xq, pos, n, st, seg_of, cell_of, cell_start, ctx->d_status);
    PPMD_TRY(exclusive_scan(ctx, cell_start, cell_start, ncell));
    if (n > 0) {
        int32_t *cursor = (int32_t *)scratch(ctx, S_COUNT, sizeof(int32_t) * (size_t)ncell);
        int32_t *key = (int32_t *)scratch(ctx, S_CELLKEY, sizeof(int32_t) * (size_t)n);
        int32_t *tmp = (int32_t *)scratch(ctx, S_CELLTMP, sizeof(int32_t) * (size_t)n);
        if (!cursor || !key || !tmp) return PPMD_ERR_NOMEM;
        PPMD_TRY(cuda_check(ctx, cudaMemsetAsync(cursor, 0, sizeof(int32_t) * (size_t)ncell, s), "memset"));
        PPMD_LAUNCH(ctx, k_scatter_xq, div_up(n, 256), 256, 0, n, xq, st, seg_of, cell_of, cell_start, cursor, tmp, key);
        PPMD_LAUNCH(ctx, k_rank_cells_x<int32_t>, div_up(n, 256), 256, 0, n, cell_of, cell_start, tmp, key, cell_atoms);
    }
    return check_launch(ctx, "bin_atoms_md");
}

int bin_atoms_fixed(ppmd_ctx *ctx, const int4 *xq, int64_t n, const SegTable &st, int64_t ncell, int32_t *cell_of,
                    int32_t *cell_start, int32_t *cell_atoms) {
    cudaStream_t s = ctx->stream;
    PPMD_TRY(cuda_check(ctx, cudaMemsetAsync(cell_start, 0, sizeof(int32_t) * (size_t)(ncell + 1), s), "memset"));
    if (n > 0) PPMD_LAUNCH(ctx, k_bin_fixed, div_up(n, 256), 256, 0, xq, n, st, cell_of, cell_start);
    PPMD_TRY(exclusive_scan(ctx, cell_start, cell_start, ncell));
    if (n > 0) {
        int32_t *cursor = (int32_t *)scratch(ctx, S_COUNT, sizeof(int32_t) * (size_t)ncell);
        uint32_t *key = (uint32_t *)scratch(ctx, S_CELLKEY, sizeof(uint32_t) * (size_t)n);
        int32_t *tmp = (int32_t *)scratch(ctx, S_CELLTMP, sizeof(int32_t) * (size_t)n);
        if (!cursor || !key || !tmp) return PPMD_ERR_NOMEM;
        PPMD_TRY(cuda_check(ctx, cudaMemsetAsync(cursor, 0, sizeof(int32_t) * (size_t)ncell, s), "memset"));
        PPMD_LAUNCH(ctx, k_scatter_fx, div_up(n, 256), 256, 0, n, xq, cell_of, cell_start, cursor, tmp, key);
        PPMD_LAUNCH(ctx, k_rank_cells_x<uint32_t>, div_up(n, 256), 256, 0, n, cell_of, cell_start, tmp, key, cell_atoms);
    }
    return check_launch(ctx, "bin_atoms_fixed");
}

}  // namespace ppmd

using namespace ppmd;

extern "C" int ppmd_build_cells(ppmd_ctx *ctx, const double *pos, int64_t n, const ppmd_box *box, double min_cell_width,
                                int32_t *cell_of, int32_t *cell_start, int32_t *cell_atoms, int32_t ncell_out[3],
                                int64_t cell_capacity) {
    if (!ctx || !box || n < 0 || !(min_cell_width > 0)) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_build_cells: bad argument");
    if (n > 0 && (!pos || !cell_of || !cell_atoms)) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_build_cells: null array");
    if (!cell_start) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_build_cells: null cell_start");
    if (n >= (int64_t)1 << 31) return set_error(ctx, PPMD_ERR_INVALID, "ppmd_build_cells: n too large");
    cudaSetDevice(ctx->device);
    SegTable st;
    st.d = nullptr;
    st.nseg = 1;
    PPMD_TRY(make_seg(ctx, st.one, box->L, min_cell_width, 0.0));
    int64_t ncell = (int64_t)st.one.nc[0] * st.one.nc[1] * st.one.nc[2];
    if (ncell_out)
        for (int d = 0; d < 3; ++d) ncell_out[d] = st.one.nc[d];
    if (ncell + 1 > cell_capacity) {
        ctx->host_needed = ncell + 1;
        return set_error(ctx, PPMD_ERR_CAPACITY, "cell_start needs %lld entries", (long long)(ncell + 1));
    }
    return bin_atoms(ctx, pos, n, st, nullptr, ncell, true, cell_of, cell_start, cell_atoms);
}
