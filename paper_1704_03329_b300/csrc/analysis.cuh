// Structure analysis kernels (bond order parameters, common neighbour
// analysis) and the sorted-snapshot pipeline shared with the classifier.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace ppmd {
// Atoms of one box binned and sorted by cell, with their neighbour list
// (column-major, built by bricks).
struct Snapshot {
    int64_t n = 0;
    SegTable st{};
    double Lmax = 0;
    double *pos = nullptr;      // [n][3] sorted
    int4 *xq = nullptr;         // fixed-point, sorted
    int32_t *perm = nullptr;    // sorted index -> caller index
    int32_t *cell_of = nullptr, *cell_start = nullptr;
    int32_t *nbr = nullptr, *cnt = nullptr;
    int32_t max_nbr = 0;
    int64_t ld = 0;  // column-major list: entry m of atom i at nbr[m * ld + i]
};
// Bin/sort the caller's atoms with cells of edge >= r_list and build the
// list at r_list with max_nbr entries per atom (no synchronisation: an
// overflow is latched in the context's status).
// List capacity of the analysis pipelines for n atoms in box at r_list.
int32_t snapshot_capacity(int64_t n, const ppmd_box *box, double r_list);
// End of a pipeline: wait and read the status (and the aux result word).
// Returns PIPELINE_RETRY when the list overflowed on the first attempt, with
// max_nbr raised to what was needed (the caller runs the pipeline again),
// else the status.
constexpr int PIPELINE_RETRY = 1;
int end_pipeline(ppmd_ctx *ctx, int attempt, int32_t &max_nbr, int32_t *aux = nullptr);
// Q4, Q5, Q6 over the integrator's column-major list (see analysis.cu).
int boa_otf_launch(ppmd_ctx *ctx, int64_t n, const int4 *xq, const double *pos64, const SegTable &st, const int32_t *W,
                   const int32_t *cnt, int32_t max_nbr, int64_t ld, double r_cut, double Lmax, const int32_t *out_idx,
                   float *q3, double *partials);
int64_t boa_otf_blocks(int64_t n);
int sorted_snapshot(ppmd_ctx *ctx, const double *pos, int64_t n, const ppmd_box *box, double r_list, int32_t max_nbr,
                    Snapshot &s);
// The same over nbox independent boxes (box b holds the caller's atoms
// atom_off[b] .. atom_off[b + 1] - 1; atom_off and boxes in host memory),
// one segment per box: the atoms stay grouped by box in the sorted order.
int sorted_snapshot_boxes(ppmd_ctx *ctx, const double *pos, int64_t nbox, const int64_t *atom_off,
                          const ppmd_box *boxes, double r_list, int32_t max_nbr, Snapshot &s);
// Largest snapshot_capacity over the boxes.
int32_t snapshot_capacity_boxes(int64_t nbox, const int64_t *atom_off, const ppmd_box *boxes, double r_list);
// Checks a box set: 1 <= nbox < 2^31, atom_off[0] = 0, non-decreasing, total < 2^31.
int check_boxes(ppmd_ctx *ctx, int64_t nbox, const int64_t *atom_off, const ppmd_box *boxes, const char *who);
int boa_launch(ppmd_ctx *ctx, int64_t n, const int4 *xq, const double *pos64, const SegTable &st, const int32_t *nbr,
               const int32_t *cnt, int32_t max_nbr, int64_t ld, double r_cut, double Lmax, const int32_t *out_idx, float *q4,
               float *q6, int32_t *nnb);
// Labels from (Q4, Q6) by the nearest perfect-lattice value within tol
// (k_boa_tolerance in analysis.cu); dist (may be null) the nearest distance.
int boa_tolerance_launch(ppmd_ctx *ctx, int64_t n, const float *q4, const float *q6, float tol, int8_t *label,
                         float *dist);
int cna_launch(ppmd_ctx *ctx, int64_t n, const int4 *xq, const double *pos64, const SegTable &st, const int32_t *nbr,
               const int32_t *cnt, int32_t max_nbr, int64_t ld, double r_cut, double Lmax, const int32_t *out_idx, uint32_t *trip,
               int8_t *label);
// CNA labels of the snapshot atoms listed in `which` (m of them), written
// at label[out_idx[which[k]]] (label[which[k]] when out_idx is null).
int cna_subset_launch(ppmd_ctx *ctx, int64_t m_max, const int32_t *m_dev, const int32_t *which, const int4 *xq, const double *pos64,
                      const SegTable &st, const int32_t *nbr, const int32_t *cnt, int32_t max_nbr, int64_t ld, double r_cut,
                      double Lmax, const int32_t *out_idx, int8_t *label);
// Classifier features (30 per atom) of the snapshot atoms, written at out_idx.
int features_launch(ppmd_ctx *ctx, int64_t n, const int4 *xq, const double *pos64, const SegTable &st,
                    const int32_t *nbr, const int32_t *cnt, int32_t max_nbr, int64_t ld, double r_feat, double r_ref, double Lmax,
                    const int32_t *out_idx, float *f32, __nv_bfloat16 *fb16);
}  // namespace ppmd
