// Neighbour-list build shared by the list entry point, the integrator and
// the analysis pipeline.
#pragma once
#include "common.cuh"

namespace ppmd {
// Fixed-point positions (x 2^32 / L, segment id in .w) and, if cell_of is
// not null, the exact cell of every atom.
int prep_fixed(ppmd_ctx *ctx, const double *pos, int64_t n, const SegTable &st, const int32_t *seg_of, int4 *xq,
               int32_t *cell_of);
// Full neighbour list with the segment's list cutoff: nbr[i * max_nbr + m],
// cnt[i].  cell_atoms == nullptr: atoms are stored in cell order.
int build_list(ppmd_ctx *ctx, int64_t n, const int4 *xq, const double *pos64, const SegTable &st, const int32_t *cell_of,
               const int32_t *cell_start, const int32_t *cell_atoms, int32_t *nbr, int32_t *cnt, int32_t max_nbr);
}  // namespace ppmd
