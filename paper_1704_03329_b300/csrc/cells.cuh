// Cell binning shared by the cell-list entry point, the integrator and the
// analysis pipeline.
#pragma once
#include "common.cuh"

namespace ppmd {
// Bin n atoms into the global cell index space of the segment table (ncell
// cells in total).  exact = true evaluates the cell coordinate with the
// same IEEE operations as the documented formula (division by the cell
// edge); exact = false multiplies by the reciprocal (positions already in
// the box).  Writes cell_of[n], cell_start[ncell+1], cell_atoms[n] (atoms
// of a cell in increasing index).
int bin_atoms(ppmd_ctx *ctx, const double *pos, int64_t n, const SegTable &st, const int32_t *seg_of, int64_t ncell,
              bool exact, int32_t *cell_of, int32_t *cell_start, int32_t *cell_atoms, bool order_x = false);
// The same from fixed-point coordinates xq (their .w the segment): cell c
// along an axis of nc cells holds the words q with c 2^32 <= q nc <
// (c + 1) 2^32 (integer arithmetic), atoms of a cell ordered by (x word,
// index).  For pipelines that convert to fixed point first.
int bin_atoms_fixed(ppmd_ctx *ctx, const int4 *xq, int64_t n, const SegTable &st, int64_t ncell, int32_t *cell_of,
                    int32_t *cell_start, int32_t *cell_atoms);
// The integrator's binning: the cells of bin_atoms(exact = false) for FP64
// positions pos whose fixed-point words xq (modulo 2^32) are current, found
// by integer arithmetic except within a hair of a cell face; atoms of a cell
// ordered by (x word relative to the cell centre, index).
int bin_atoms_md(ppmd_ctx *ctx, const int4 *xq, const double *pos, int64_t n, const SegTable &st, const int32_t *seg_of,
                 int64_t ncell, int32_t *cell_of, int32_t *cell_start, int32_t *cell_atoms);
}  // namespace ppmd
