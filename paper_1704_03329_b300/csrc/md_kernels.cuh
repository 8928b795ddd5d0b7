// Kernels of the time-stepping driver (atoms kept in cell order).
#pragma once
#include "common.cuh"
#include "lj.cuh"

namespace ppmd {

// A brick: the cells x0 <= x < x1, y0 <= y < y1, z0 <= z < z1 of one
// segment (at most BW_MAX x BH_MAX x BD_MAX).  Its neighbourhood is the
// cells x0-1 .. x1 of the rows y0-1 .. y1 of the planes z0-1 .. z1.
struct Brick {
    int32_t seg, x01, y01, z01;  // x01 = x0 | x1 << 16, and so on
};
struct BrickShape {
    int32_t bw, bh, bd;  // cells of a brick along x, y, z
};

constexpr int NB_MAX = 2048;        // largest neighbourhood staged in shared memory
constexpr int BRICK_THREADS = 128;  // home atoms handled per pass of a brick block
constexpr int BW_MAX = 8, BH_MAX = 4, BD_MAX = 2;
constexpr int ROW_GAP = 4;  // stage slots after each row (candidates are read in fours from even slots)

// Brick shape for a segment: the most home atoms up to one per thread whose
// neighbourhood (with a margin for density fluctuations) fits the stage.
// home_max (at most BRICK_THREADS) bounds the expected home atoms of a brick.
BrickShape brick_shape(const Seg &S, int32_t home_max = BRICK_THREADS);
// Bricks of the cell grids of several segments (host).
// Returns the stage capacity covering every segment.
int32_t make_bricks(const std::vector<Seg> &segs, std::vector<Brick> &out, int32_t home_max = BRICK_THREADS);
int64_t brick_count(const Seg &S, BrickShape b);
// Shared-memory stage (atoms) of a brick of that shape.
int32_t brick_stage_cap(const Seg &S, BrickShape b);
size_t neigh_brick_smem(int32_t max_nbr);
int neigh_brick_setup(ppmd_ctx *ctx, int32_t max_nbr);

// Column-major neighbour list W[m * ld + i] (the paper's neighbour matrix)
// of atoms stored in cell order, one block per brick.  With vec4 the
// entries are grouped by four: entry m of atom i at W[((m/4) ld + i) 4 + m%4],
// the last group padded with -1 (max_nbr must be divisible by 4).  With bricks == null
// the grid is one segment's (st.nseg == 1) cut into bricks of `shape`, in
// x-fastest order.
int build_list_bricks(ppmd_ctx *ctx, int64_t nbricks, const Brick *bricks, BrickShape shape, const int4 *xq,
                      const double *pos64, const SegTable &st, const int32_t *cell_start, int32_t *W, int64_t ld,
                      int32_t *cnt, int32_t max_nbr, int32_t stage_cap, bool vec4 = false);

// Pair loop over the grouped column-major list (vec4 layout above), one
// thread per atom, followed by the second kick of Algorithm 6
// (v += dt/(2m) F) when vel != null.
// partials (energy steps): per-block rows (U, W, K).
// The next step's first kick and drift (Algorithm 6) fused into the FP32
// pair loop: after the second kick, v += dt/(2m) F once more and
// x' = x + dt v is written to the other position buffers (the pair loop is
// still reading x), with the displacement guard against xq_ref.
struct Drift {
    double *pos_next = nullptr;
    int4 *xq_next = nullptr;
    const int4 *xq_ref = nullptr;
    double dt = 0.0;
    unsigned int *max_disp_bits = nullptr;
};
// Launch shape of the FP32 pair loop: threads per block (128 or 256) and,
// with grid_cap > 0, at most grid_cap blocks, each walking its share of the
// atoms (a persistent grid); else one thread per atom.  The per-atom
// arithmetic, and so the trajectory, is the same for every shape; the
// per-block energy sums (partials) follow the shape.  The FP64 loop takes
// lj_col64_lanes lanes per atom.
struct ColShape {
    int32_t block = 128;
    int64_t grid_cap = 0;
};
int lj_columns(ppmd_ctx *ctx, int64_t n, int64_t ld, const int4 *xq, const double *pos64, const SegTable &st,
               const LJConst &c, const int32_t *W, const int32_t *cnt, int32_t max_nbr, int prec, float4 *f4,
               double *f64, double *vel, double h, double half_m, double *partials, const Drift &drift = Drift(),
               const ColShape &shape = ColShape());
// blocks (and partial rows) of a launch of that shape
int64_t lj_columns_blocks(int64_t n, const ColShape &shape = ColShape());
// lanes per atom of the FP64 loop for n atoms (1 to 16) and atoms per block
// (its partial rows: div_up(n, atoms per block), at most div_up(n, 8))
int lj_col64_lanes(int64_t n);
int lj_col64_atoms_per_block(int64_t n);

// Brick-staged FP32 path (slots.cu).  A list entry is the neighbour's slot
// (16 bits) in its brick's staged neighbourhood: the cells of the brick's
// neighbourhood row by row, each row the cells x0-1 .. x1 of one (y, z) row
// of the sorted atoms, rows back to back; slot T (the neighbourhood's size)
// is a sentinel far from every home atom and pads the last group of eight.
// Entry m of atom i: W16[((m / 8) ld + i) 8 + m % 8]; max_nbr divisible by 8.
constexpr int SLOT_THREADS = 128;
size_t slot_list_smem(int32_t stage_cap, int32_t max_nbr);
size_t slot_pair_smem(int32_t stage_cap);
int slots_setup(ppmd_ctx *ctx, int32_t stage_cap, int32_t max_nbr);
// List build over the bricks; a neighbourhood larger than stage_cap leaves
// its home atoms without entries, raises *stage_need to its size and latches
// PPMD_ERR_CAPACITY.
int build_slot_list(ppmd_ctx *ctx, int64_t nbricks, const Brick *bricks, const int4 *xq, const double *pos64,
                    const SegTable &st, const int32_t *cell_start, uint16_t *W16, int64_t ld, int32_t *cnt,
                    int32_t max_nbr, int32_t stage_cap, int32_t *stage_need, int64_t n_atoms);
// Pair loop of the slot lists (one block per brick, its neighbourhood copied
// into shared memory by bulk asynchronous copies); kick, drift and partials
// as lj_columns (partials: one row per brick).
int lj_slots(ppmd_ctx *ctx, int64_t nbricks, const Brick *bricks, const int4 *xq, const double *pos64,
             const SegTable &st, const int32_t *cell_start, const LJConst &c, const uint16_t *W16, int64_t ld,
             const int32_t *cnt, int32_t max_nbr, int32_t stage_cap, float4 *f4, double *vel, double h,
             double half_m, double *partials, const Drift &drift, int64_t n_atoms);
// The slot lists as the grouped column-major atom-index list of
// build_list_bricks (vec4 layout), same entries in the same order.
int slots_to_atoms(ppmd_ctx *ctx, int64_t nbricks, const Brick *bricks, const SegTable &st, const int32_t *cell_start,
                   const uint16_t *W16, int64_t ld, const int32_t *cnt, int32_t max_nbr, int32_t stage_cap, int32_t *W,
                   int64_t n_atoms);

// Kick + drift without wrapping (coordinates stay continuous between list
// builds), fixed-point refresh, displacement guard.
int md_kick_drift2(ppmd_ctx *ctx, int64_t n, double *pos, double *vel, const float4 *f4, const double *f64, int4 *xq,
                   const int4 *xq_ref, const SegTable &st, double h, double dt, unsigned int *max_disp_bits);

// Gather through perm into cell order, wrapping positions into the box.
// With xq the fixed-point words are gathered (else made from the wrapped
// positions); xq_o2 (may be null) receives a second copy of them.
int md_gather(ppmd_ctx *ctx, int64_t n, const int32_t *perm, const SegTable &st, const double *pos, const double *vel,
              const int32_t *orig, const int32_t *seg_of, const int4 *xq, double *pos_o, double *vel_o, int4 *xq_o,
              int4 *xq_o2, int32_t *orig_o, int32_t *seg_o);

}  // namespace ppmd
