/*
 * ppmd.h -- C ABI of the B300 (sm_103a) implementation of the data-parallel
 * hot path of Saunders, Grant & Mueller, "A Domain Specific Language for
 * Performance Portable Molecular Dynamics Algorithms" (arXiv:1704.03329):
 * the cell-list / neighbour-list Lennard-Jones pair loop under periodic
 * boundaries, the Velocity Verlet particle loops that feed it, and the two
 * per-atom structure analyses (bond order Q4/Q6 and common neighbour
 * analysis) plus a learned structure classifier that falls back to CNA.
 *
 * Conventions (every entry point):
 *  - Pointers to particle data are DEVICE pointers owned by the caller; the
 *    library never frees or retains them past the call.  Arrays of 3-vectors
 *    are row-major [n][3] FP64 (the paper's ParticleDat with ncomp = 3).
 *    Scalar outputs marked "device" are device pointers too.  Arguments
 *    marked "host" are ordinary host memory read or written during the call.
 *  - The library owns its scratch memory (allocated on first use and grown
 *    as needed, freed by ppmd_destroy) and runs everything on the stream
 *    bound to the context.  Calls are asynchronous on that stream unless a
 *    host output is requested.
 *  - Boxes are orthorhombic [0, L0) x [0, L1) x [0, L2), periodic in x, y, z
 *    (the paper's BoundaryTypePeriodic domain, Sec. 3.5).  Minimum-image
 *    separations r_i - r_j are used; every cutoff must be below L/2 and the
 *    cell grid needs at least three cells per edge (else PPMD_ERR_BOX).
 *  - Cutoff tests are strict (r < r_cut), as in the paper's kernels.
 *    Neighbour and cutoff decisions are exact: a single-precision test with
 *    a double-precision re-test of every pair within a small band of the
 *    cutoff, the double-precision test computing
 *        d = r_i - r_j;  d = d - L * rint(d / L);  r^2 = dx*dx + dy*dy + dz*dz
 *    with IEEE round-to-nearest operations and no fused multiply-add.
 *  - Return value: 0 = PPMD_OK, < 0 an error, > 0 a warning.  Conditions
 *    found by a kernel (capacity overflow, non-finite data, a bounded wait
 *    that ran out) are latched in the context and returned by the next
 *    synchronising call (ppmd_sync / ppmd_status, or any call with a host
 *    output).  No C++ exception crosses this interface.
 */
#ifndef PPMD_H
#define PPMD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PPMD_OK 0
#define PPMD_ERR_INVALID (-1)   /* bad argument (null pointer, negative size, ...) */
#define PPMD_ERR_BOX (-2)       /* fewer than 3 cells per edge, or a cutoff >= L/2 */
#define PPMD_ERR_CAPACITY (-3)  /* an output array is too small; ppmd_status reports the size needed */
#define PPMD_ERR_NONFINITE (-4) /* NaN or infinite coordinate met */
#define PPMD_ERR_CUDA (-5)      /* CUDA runtime error; ppmd_last_error has the text */
#define PPMD_ERR_TIMEOUT (-6)   /* a bounded device-side wait ran out */
#define PPMD_ERR_NOMEM (-7)     /* scratch allocation failed */
#define PPMD_WARN_SKIN 1        /* an atom moved more than half the list skin between rebuilds */

/* Structure codes written by ppmd_cna and ppmd_classify. */
#define PPMD_OTHER 0
#define PPMD_FCC 1
#define PPMD_HCP 2
#define PPMD_BCC 3

typedef struct ppmd_ctx ppmd_ctx;
typedef struct ppmd_md ppmd_md;

/* Orthorhombic periodic domain (Sec. 3.5, Listing "state-example"). */
typedef struct {
    double L[3];
} ppmd_box;

/* Arithmetic of the pair loop.  PPMD_FP64: double precision throughout.
 * PPMD_FP32: single-precision pair arithmetic with compensated (Kahan)
 * per-atom sums; positions enter as exact 32-bit fixed-point box
 * coordinates, integration and global reductions stay in double. */
typedef enum { PPMD_FP64 = 0, PPMD_FP32 = 1 } ppmd_prec;

/* Truncated Lennard-Jones, Eq. (9) and Eq. (12):
 *   V(r) = 4 eps ((sigma/r)^12 - (sigma/r)^6 + shift)   for r < rc, else 0
 *   F_i  = sum_j 48 eps / sigma^2 (r_i - r_j) ((sigma/r)^14 - (sigma/r)^8 / 2)
 * shift = 0 gives the truncated, unshifted potential; shift = 0.25 is the
 * form printed as Eq. (9).  Forces do not depend on shift. */
typedef struct {
    double eps, sigma, rc, shift;
} ppmd_lj_params;

/* ------------------------------------------------------------------ */
/* Context                                                            */
/* ------------------------------------------------------------------ */

/* Create a context on CUDA device `device`, bound to `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream).  *ctx receives the
 * handle; free it with ppmd_destroy. */
int ppmd_create(ppmd_ctx **ctx, int device, void *cuda_stream);
int ppmd_destroy(ppmd_ctx *ctx);
/* Rebind the context to another stream of the same device. */
int ppmd_set_stream(ppmd_ctx *ctx, void *cuda_stream);
/* Wait for the stream; return (and clear) the latched status. */
int ppmd_sync(ppmd_ctx *ctx);
/* As ppmd_sync; *needed (host, may be NULL) receives the capacity that the
 * last PPMD_ERR_CAPACITY asked for (atoms, cells or neighbours). */
int ppmd_status(ppmd_ctx *ctx, int64_t *needed);
/* Text of the last error (static storage owned by the context). */
const char *ppmd_last_error(const ppmd_ctx *ctx);
/* Number of kernels this context has launched so far (host counter;
 * graph replays count every kernel node). */
int64_t ppmd_kernel_count(const ppmd_ctx *ctx);

/* ------------------------------------------------------------------ */
/* Cell list, Sec. 3.5 (cell width >= cutoff, every particle in exactly one
 * cell; the paper's cell-occupancy matrix H in compressed-row form).
 *   n_d = floor(L_d / min_cell_width), w_d = L_d / n_d (>= min_cell_width),
 *   x' = x - L floor(x / L) (the wrapped coordinate),
 *   c_d = min(floor(x'_d / w_d), n_d - 1),  c = (c_z n_y + c_y) n_x + c_x.
 * Outputs (device): cell_of[n]; cell_start[ncell + 1] (exclusive prefix of
 * the occupancies); cell_atoms[n] (atom indices grouped by cell, increasing
 * within a cell).  ncell_out (host, 3 ints) receives n_x, n_y, n_z.
 * PPMD_ERR_BOX if some n_d < 3; PPMD_ERR_CAPACITY if ncell + 1 >
 * cell_capacity (ppmd_status then reports ncell + 1). */
int ppmd_build_cells(ppmd_ctx *ctx, const double *pos, int64_t n, const ppmd_box *box, double min_cell_width,
                     int32_t *cell_of, int32_t *cell_start, int32_t *cell_atoms, int32_t ncell_out[3],
                     int64_t cell_capacity);

/* Neighbour list, Sec. 3.5 and Eq. (3): for every atom i all j != i with
 * |r_i - r_j| < r_list (minimum image), found through the 27 cells around
 * the cell of i.  This is the paper's neighbour matrix W (W_{m,i} = m-th
 * neighbour of i), stored transposed as nbr[i * max_nbr + m] so that the
 * neighbours of one atom are contiguous; the order within a row is
 * unspecified.  nbr_count[i] (device) receives the full count even when it
 * exceeds max_nbr (entries past max_nbr are not written, and the call
 * latches PPMD_ERR_CAPACITY with the largest count as the needed size).
 * The cell arrays are those of ppmd_build_cells with min_cell_width >=
 * r_list.  needed_max_nbr (host, may be NULL): if given, the call
 * synchronises and stores the largest count. */
int ppmd_build_neighbours(ppmd_ctx *ctx, const double *pos, int64_t n, const ppmd_box *box, double r_list,
                          const int32_t *cell_start, const int32_t *cell_atoms, const int32_t ncell[3],
                          int32_t *nbr, int32_t *nbr_count, int32_t max_nbr, int32_t *needed_max_nbr);

/* Lennard-Jones pair loop over a neighbour list (Eqs. (9) and (12), Listing
 * "LJ-kernel"): every listed ordered pair (i, j) with r < rc adds its force
 * to i only (Sec. 2, no Newton's-third-law symmetry).  force[n][3] has
 * INC_ZERO semantics (set, not accumulated).  e_atom[n] (device, may be
 * NULL) receives 1/2 sum_j V(r_ij), e_total[1] and virial[1] (device, may
 * be NULL) receive U = sum_i e_atom[i] and W = 1/2 sum_{i != j} r_ij . f_ij.
 * The list must have been built with r_list >= rc. */
int ppmd_lj_forces(ppmd_ctx *ctx, const double *pos, int64_t n, const ppmd_box *box, const ppmd_lj_params *lj,
                   const int32_t *nbr, const int32_t *nbr_count, int32_t max_nbr, ppmd_prec prec, double *force,
                   double *e_atom, double *e_total, double *virial);

/* The same forces, per-atom energies, U and W as ppmd_lj_forces, without a
 * neighbour list: the cell structure of Sec. 3.5 is swept directly and no
 * neighbour matrix W is built or read (the role of the layer algorithm that
 * Sec. 3.5 cites for cell-based codes).  The call bins pos into cells of
 * edge >= rc (at least three per axis, rc < L/2: else PPMD_ERR_BOX), sorts
 * the atoms by cell in scratch memory, and every atom sweeps the 27 cells
 * around its own (8 lanes per atom).  Cutoff decisions are exact (FP32 test,
 * FP64 re-test inside the band), as in ppmd_lj_forces; prec, outputs
 * (caller order, device memory), INC_ZERO semantics and NULL options as
 * there.  Asynchronous. */
int ppmd_lj_forces_cells(ppmd_ctx *ctx, const double *pos, int64_t n, const ppmd_box *box, const ppmd_lj_params *lj,
                         ppmd_prec prec, double *force, double *e_atom, double *e_total, double *virial);

/* Half neighbour list (Newton's third law; Sec. 2 on write conflicts):
 * half[i][0..half_count[i]) = the entries j of row i of the full row-major
 * list nbr [n][max_nbr] (as ppmd_build_neighbours writes it, for the same
 * pos and box) whose minimum-image displacement r_j - r_i, in the 32-bit
 * fixed-point box coordinates, is positive in the order (z, y, x): the
 * first non-zero component decides.  These integer differences are exactly
 * antisymmetric, so every listed pair is kept by exactly one of its atoms,
 * and rows hold about half of the full length in any atom order (a pair of
 * coincident atoms is dropped).  half: device int32 [n][max_half]; a row
 * with more than max_half entries latches PPMD_ERR_CAPACITY with the length
 * needed (reported by the next synchronising call, e.g. ppmd_status).
 * Asynchronous. */
int ppmd_half_list(ppmd_ctx *ctx, const double *pos, int64_t n, const ppmd_box *box, const int32_t *nbr,
                   const int32_t *nbr_count, int32_t max_nbr, int32_t *half, int32_t *half_count, int32_t max_half);

/* The forces, per-atom energies, U and W of ppmd_lj_forces from a half
 * list (ppmd_half_list): each unordered pair is evaluated once, by the atom
 * whose row holds it, and its force and half of its energy go to both
 * atoms (the other through atomic adds).  Same arguments, outputs and exact
 * cutoff decisions as ppmd_lj_forces.  PPMD_FP32: single-precision pair
 * terms, each atom's own share in compensated sums and the shares from its
 * neighbours through FP32 atomic adds, so the last bits of F and e_i vary
 * with the order in which the GPU performs those adds; PPMD_FP64: double
 * precision with double atomic adds.  Asynchronous. */
int ppmd_lj_forces_newton3(ppmd_ctx *ctx, const double *pos, int64_t n, const ppmd_box *box, const ppmd_lj_params *lj,
                           const int32_t *half, const int32_t *half_count, int32_t max_half, ppmd_prec prec,
                           double *force, double *e_atom, double *e_total, double *virial);

/* Velocity Verlet particle loops, Algorithm 6 and Listings
 * "position_update" / "velocity_update":
 *   phase 1 (first half kick, drift): v += dt/(2m) F;  r += dt v;  r wrapped
 *   phase 2 (second half kick, after the forces): v += dt/(2m) F
 * pos and vel are updated in place (pos is not touched in phase 2). */
int ppmd_verlet_step(ppmd_ctx *ctx, int phase, double *pos, double *vel, const double *force, int64_t n,
                     const ppmd_box *box, double mass, double dt);

/* Kinetic energy K = sum_i m |v_i|^2 / 2 (Sec. 2, Example 1) into ke[1] (device). */
int ppmd_kinetic_energy(ppmd_ctx *ctx, const double *vel, int64_t n, double mass, double *ke);

/* ------------------------------------------------------------------ */
/* Structure analysis (Sec. 4).                                          */
/* ------------------------------------------------------------------ */

/* Bond order parameters, Eqs. (4)-(5) with Algorithms 1 and 2: for every
 * atom i, nu_i = number of list neighbours j with |r_i - r_j| < r_cut and
 *   Q_l(i) = sqrt(4 pi / (2l+1) sum_{m=-l..l} |q_lm(i)|^2),
 *   q_lm(i) = (1/nu_i) sum_j Y_l^m(r_ij / |r_ij|),
 * for l = 4 and l = 6 (orthonormal spherical harmonics; Q_l = 0 when
 * nu_i = 0).  The list (as from ppmd_build_neighbours, cutoff >= r_cut)
 * is read, not changed.  Outputs (device, any may be NULL): q4[n], q6[n]
 * single precision, n_nb[n]. */
int ppmd_boa_q46(ppmd_ctx *ctx, const double *pos, int64_t n, const ppmd_box *box, double r_cut, const int32_t *nbr,
                 const int32_t *nbr_count, int32_t max_nbr, float *q4, float *q6, int32_t *n_nb);

/* Common neighbour analysis, Eqs. (6)-(8) with Algorithms 3, 4, 5 and 7:
 * atoms closer than r_cut are bonded; for each bonded pair (i, j) the
 * common neighbours C = N(i) n N(j), the bonds E among them and the
 * number of bonds in the largest connected part of (C, E) give the triplet
 * (n_cn, n_b, n_lcb), stored as n_cn << 16 | n_b << 8 | n_lcb in
 * triplets[i * max_nbr + m] for list slot m (0xFFFFFFFF where nbr[i][m] is
 * not bonded; triplets may be NULL).  label[n] (device, may be NULL): 1 fcc
 * (12 bonds, all (4,2,1)), 2 hcp (12 bonds, 6 (4,2,1) + 6 (4,2,2)), 3 bcc
 * (14 bonds, 8 (6,6,6) + 6 (4,4,4)), else 0.  At most 64 bonds per atom
 * (more latches PPMD_ERR_CAPACITY and labels the atom 0). */
int ppmd_cna(ppmd_ctx *ctx, const double *pos, int64_t n, const ppmd_box *box, double r_cut, const int32_t *nbr,
             const int32_t *nbr_count, int32_t max_nbr, uint32_t *triplets, int8_t *label);

/* Both analyses straight from positions: the atoms are binned and sorted by
 * cell internally, the list is built at max(r_boa, r_cna) and the results
 * are returned in caller order.  Bond order is computed when any of q4, q6,
 * n_nb is given (cutoff r_boa), CNA labels when label is given (cutoff
 * r_cna).  Asynchronous: the list capacity is set from the box density
 * (1.6 times the mean neighbour count plus 16, at least 48); an overflow
 * (PPMD_ERR_CAPACITY, results invalid) is reported by the next
 * synchronising call. */
int ppmd_analyze(ppmd_ctx *ctx, const double *pos, int64_t n, const ppmd_box *box, double r_boa, double r_cna,
                 float *q4, float *q6, int32_t *n_nb, int8_t *label);

/* ppmd_analyze over nbox independent periodic boxes in one pipeline (one
 * binning, one list build and one launch per analysis for all of them):
 * box b (boxes[b], host array) holds atoms atom_off[b] .. atom_off[b+1]-1
 * of pos (atom_off: host int64 array of nbox + 1 offsets, atom_off[0] = 0,
 * non-decreasing; 1 <= nbox < 2^31; n = atom_off[nbox] < 2^31).  Atoms of different boxes
 * never interact.  Outputs and their layout as ppmd_analyze over the n
 * atoms (caller order); every box must hold at least 3 cells of edge
 * max(r_boa, r_cna) along each axis.  List capacity: the largest over the
 * boxes.  Asynchronous, as ppmd_analyze: with nbox > 1 the box tables go
 * through a pinned buffer of the context (reused once the copies of the
 * previous call have run; allocated, or grown, on first use). */
int ppmd_analyze_boxes(ppmd_ctx *ctx, const double *pos, int64_t nbox, const int64_t *atom_off, const ppmd_box *boxes,
                       double r_boa, double r_cna, float *q4, float *q6, int32_t *n_nb, int8_t *label);

/* Adaptive CNA (the extension of CNA that Sec. 4.2 cites, Stukowski 2012):
 * every atom sets its own bond cutoff from its N nearest neighbours
 * (distances d_1 <= ... <= d_N over the list at r_list, ties by index):
 *   fcc/hcp test, N = 12:  r = f (d_1 + ... + d_12) / 12,
 *   bcc test,     N = 14:  r = f (c (d_1 + ... + d_8) + d_9 + ... + d_14) / 14,
 * f = (1 + sqrt 2)/2, c = 2/sqrt 3.  Only those N neighbours take part (all
 * bonded to the atom, two of them bonded when closer than r) and each bond
 * gets the triplet of Eqs. (6)-(8) over its common neighbours among them.
 * Labels (caller order, label[n] device int8): 1 fcc (12 x (4,2,1)), 2 hcp
 * (6 x (4,2,1) + 6 x (4,2,2)), else 3 bcc (8 x (6,6,6) + 6 x (4,4,4) in the
 * 14-neighbour test), else 0.  rcut (device FP64 [n][2], may be NULL): the
 * two cutoffs, 0 when not computed (the bcc one only after the fcc/hcp test
 * failed).  Decisions and cutoffs equal the FP64 evaluation bit for bit.
 * r_list must reach the 14th neighbour (e.g. 1.8 at density 0.8442); a test
 * that needs more neighbours than the list holds fails.  At most 64 list
 * entries per atom (more: PPMD_ERR_CAPACITY, latched).  Asynchronous, as
 * ppmd_analyze. */
int ppmd_acna(ppmd_ctx *ctx, const double *pos, int64_t n, const ppmd_box *box, double r_list, int8_t *label,
              double *rcut);

/* ------------------------------------------------------------------ */
/* Learned structure classifier (not in the paper): an MLP 30 -> 64 -> 64
 * -> 4 (ReLU, softmax over 0 other, 1 fcc, 2 hcp, 3 bcc) on local-
 * environment features, trained on labels from ppmd_cna, with exact CNA as
 * the fallback for low-confidence atoms.  Parameters are one FP32 device
 * vector of PPMD_MLP_NPARAM values, laid out
 *   mu[30] | isd[30] | W1[30][64] | b1[64] | W2[64][64] | b2[64] | W3[64][4] | b3[4]
 * with x' = (x - mu) isd (input standardisation, set by
 * ppmd_mlp_fit_input_norm, never trained) and y = x' W + b.
 * Arithmetic: BF16 inputs, weights and activations, FP32 accumulation
 * (tensor cores).                                                       */
/* ------------------------------------------------------------------ */
#define PPMD_MLP_NPARAM 6464

/* Features of every atom from its bonds (r < r_feat, the BOA cutoff):
 * [0] Q4, [1] Q6 (Eqs. (4)-(5)); [2..15] the 14 smallest bond lengths d,
 * ascending, as (d - r_ref) / (r_feat - r_ref) with r_ref < r_feat a
 * reference length (the CNA cutoff: values change sign where CNA's bond
 * test does), missing ones 1; [16..29] a histogram of the chords
 * |r_ij - r_ik| of the bond angles between bonded neighbours (closer than
 * r_ref), 14 bins of width 0.05 centred on r_ref - 0.35 + 0.05 (b + 1/2),
 * linear weights between centres, clamped at both ends, divided by 24.
 * Outputs (device, at
 * least one given): feat[n][30] FP32, feat_bf16[n][32] BF16 (last two 0),
 * caller order.  Synchronises once at the end to check the list capacity
 * (set as for ppmd_analyze); if the list overflowed, the features are
 * computed again with the capacity that was needed. */
int ppmd_features(ppmd_ctx *ctx, const double *pos, int64_t n, const ppmd_box *box, double r_feat, double r_ref,
                  float *feat, uint16_t *feat_bf16);
/* Sets mu and isd of params to the mean and 1/standard deviation of each of
 * the 30 features over the n rows of x [n][32] (BF16); isd = 1 for a
 * constant feature. */
int ppmd_mlp_fit_input_norm(ppmd_ctx *ctx, float *params, const uint16_t *x, int64_t n);
/* Logits [n][4] (FP32) of the BF16 feature rows x [n][32]. */
int ppmd_mlp_forward(ppmd_ctx *ctx, const float *params, const uint16_t *x, int64_t n, float *logits);
/* Gradient (FP32 [PPMD_MLP_NPARAM], device) of the mean cross entropy of
 * the batch x [batch][32] (BF16), labels y [batch] (int8 class codes), and
 * the loss (device float, may be NULL). */
int ppmd_mlp_grad(ppmd_ctx *ctx, const float *params, const uint16_t *x, const int8_t *y, int64_t batch, float *grad,
                  float *loss);
/* One AdamW update (Loshchilov & Hutter; decay on the weight matrices only)
 * of params with moments m, v (device, PPMD_MLP_NPARAM each), step >= 1. */
int ppmd_mlp_adamw(ppmd_ctx *ctx, float *params, float *m, float *v, const float *grad, int64_t step, float lr,
                   float wd, float beta1, float beta2, float eps);
/* ppmd_mlp_grad followed by ppmd_mlp_adamw with beta = (0.9, 0.999), eps = 1e-8. */
int ppmd_mlp_train_step(ppmd_ctx *ctx, float *params, float *m, float *v, int64_t step, const uint16_t *x,
                        const int8_t *y, int64_t batch, float lr, float wd, float *loss);
/* Structure labels of every atom (caller order, label[n] device int8).
 * mode 2: bond order within a tolerance (Sec. 4.1, compared with the table
 * of Q4, Q5, Q6 of perfect lattices): Q4 and Q6 over neighbours within
 * r_feat (Eqs. (4)-(5)); the label is the lattice whose (Q4, Q6) in that
 * table (fcc 0.191, 0.575; hcp 0.097, 0.485; bcc 0.036, 0.511) is nearest in
 * the (Q4, Q6) plane, fcc before hcp before bcc on ties, when that distance
 * is below threshold (the tolerance, >= 0), else other; confidence (may be
 * NULL) receives that distance; params and r_cna are not used; n_fallback
 * (may be NULL) receives 0 and makes the call synchronise as in mode 1.
 * mode 0: exact CNA (cutoff r_cna).  mode 1: features (cutoff r_feat >
 * r_cna, reference length r_cna) -> MLP -> class and confidence (max softmax probability, device
 * float [n], may be NULL); atoms with confidence < threshold are labelled
 * by exact CNA instead (the device keeps the count: no synchronisation
 * between the MLP and CNA).  n_fallback (host, may be NULL) receives the
 * number of atoms labelled by CNA; when it is given the call synchronises
 * once at the end (list capacity check and rerun, as ppmd_features),
 * otherwise it is asynchronous (an overflow is reported by the next
 * synchronising call). */
int ppmd_classify(ppmd_ctx *ctx, int mode, const double *pos, int64_t n, const ppmd_box *box, double r_feat, double r_cna,
                  const float *params, float threshold, int8_t *label, float *confidence, int64_t *n_fallback);
/* ppmd_classify over nbox independent boxes in one pipeline (box set as
 * for ppmd_analyze_boxes); labels and confidences of all n = atom_off[nbox]
 * atoms in the caller's order, n_fallback the total over the boxes. */
int ppmd_classify_boxes(ppmd_ctx *ctx, int mode, const double *pos, int64_t nbox, const int64_t *atom_off,
                        const ppmd_box *boxes, double r_feat, double r_cna, const float *params, float threshold,
                        int8_t *label, float *confidence, int64_t *n_fallback);

/* ------------------------------------------------------------------ */
/* Time stepping (Algorithm 6 driven by the list-reuse policy of Sec. 3.5,
 * the paper's IntegratorRange), for one box or a batch of independent boxes
 * (replicas) advanced together.  The integrator keeps its own copy of the
 * particles, sorted by cell at every list rebuild, in device memory.      */
/* ------------------------------------------------------------------ */
typedef struct {
    ppmd_lj_params lj;
    double r_list;         /* list cutoff r_c + delta (Eq. (3)); per box min(r_list, box_r_list[b]) */
    double mass, dt;
    int32_t rebuild_every; /* list rebuilt when step % rebuild_every == 0 (and at set-up) */
    int32_t max_nbr;       /* row capacity of the neighbour list (rounded up to a multiple of 8 for
                              PPMD_FP32, of 4 for PPMD_FP64) */
    int32_t prec;          /* ppmd_prec of the pair loop */
    int32_t energy_every;  /* potential/kinetic energy recorded every k steps (0 = never) */
} ppmd_md_params;

/* nbox boxes; atoms of box b are [atom_off[b], atom_off[b+1]) of the arrays
 * given to ppmd_md_set_state (atom_off, boxes and box_r_list are host
 * arrays; box_r_list may be NULL: r_list for every box). */
int ppmd_md_create(ppmd_ctx *ctx, ppmd_md **md, int64_t nbox, const int64_t *atom_off, const ppmd_box *boxes,
                   const double *box_r_list, const ppmd_md_params *params);
int ppmd_md_destroy(ppmd_md *md);
/* Load positions and velocities (device, [n][3], caller order), wrap, sort,
 * build the list and compute the initial forces F(r_0).
 * With the PPMD_PAIR_BRICKS mechanism (ppmd_md_set_pair_loop) the list (the
 * paper's neighbour matrix, Sec. 3.5.1) is kept per brick of cells: the
 * grid is cut into bricks, each brick's neighbourhood (its cells and one
 * layer around them) is copied into shared memory by the pair loop of every
 * step, and a list entry is the neighbour's place in that copy.  At set-up
 * the call then reads one device word
 * (it synchronises) to check that every neighbourhood fits the copy; a
 * larger one makes it grow the copy and build again, or fail with
 * PPMD_ERR_CAPACITY when it would exceed what one block may hold.  A
 * neighbourhood that outgrows the copy at a later rebuild latches
 * PPMD_ERR_CAPACITY (its atoms get no forces), reported by the next
 * synchronising call. */
int ppmd_md_set_state(ppmd_md *md, const double *pos, const double *vel);
/* Advance nsteps steps of Algorithm 6.  energies (device, may be NULL):
 * [nsteps][2] receives (kinetic, potential) energy summed over all boxes
 * on every step s with s % energy_every == 0 (other rows untouched).
 * use_graph != 0 replays CUDA graphs of whole rebuild periods.  Inside a
 * run, the FP32 pair loop of each step but the last also applies the next
 * step's first kick and drift (same arithmetic, so the same bits as separate
 * kernels); a run always ends with full-step velocities. */
int ppmd_md_run(ppmd_md *md, int32_t nsteps, double *energies, int use_graph);
/* The on-the-fly analysis run of Sec. 5.2: the time-stepping loop extended
 * by an Andersen thermostat and by the bond order parameters.
 *
 * Andersen thermostat (nu = 0: off): at the end of step s (after the second
 * kick and the energies) atom id (caller index) collides with probability
 * p = nu dt: the first word of Philox4x32-10 (Salmon et al., SC'11) at
 * counter (id, s mod 2^32, s / 2^32, 0) and key (seed mod 2^32, seed / 2^32)
 * is compared with floor(p 2^32) (every atom when p >= 1); a colliding atom
 * gets velocities from N(0, T/m) by Box-Muller on U(u) = (u + 1/2) 2^-32:
 * (v_x, v_y) = sqrt(-2 ln U1) (cos, sin)(2 pi U2), v_z = sqrt(-2 ln U3)
 * cos(2 pi U4), U1..U3 from words 1..3, U4 from word 0 of the draw at
 * counter word 3 = 1 (FP64).  Steps count from ppmd_md_set_state. */
int ppmd_md_set_thermostat(ppmd_md *md, double T, double nu, uint64_t seed);
/* Q4, Q5, Q6 (Eqs. (4)-(5)) of every atom over the integrator's own list,
 * bonds r < r_boa (0 < r_boa <= rc), after every step s with
 * s % every == 0 (every = 0: off), on the positions of step s. */
int ppmd_md_set_boa(ppmd_md *md, int32_t every, double r_boa);
/* ppmd_md_run, also writing (mean Q4, mean Q5, mean Q6) over all atoms to
 * qrows (device [nsteps][3], may be NULL) on analysis steps.  Steps with the
 * thermostat or an analysis are not fused with the next step's drift. */
int ppmd_md_run_analysed(ppmd_md *md, int32_t nsteps, double *energies, double *qrows, int use_graph);
/* Pair-loop mechanism of the integrator (Sec. 3.4: different pair-looping
 * mechanisms give the same result at different cost), chosen before
 * ppmd_md_set_state (PPMD_ERR_INVALID after it):
 *   PPMD_PAIR_COLUMNS (default): the neighbour matrix W of Sec. 3.5.1 as
 *     atom indices, column-major in groups of four, one thread per atom
 *     gathering its neighbours' positions from global memory;
 *   PPMD_PAIR_BRICKS (PPMD_FP32, no on-the-fly analysis): the grid cut into
 *     bricks of cells; each brick's neighbourhood is copied into shared
 *     memory by bulk asynchronous copies in every pair loop and W holds each
 *     neighbour's 16-bit place in that copy (see ppmd_md_set_state).
 * Both give the same forces bit for bit (same pairs in the same order). */
#define PPMD_PAIR_COLUMNS 0
#define PPMD_PAIR_BRICKS 1
int ppmd_md_set_pair_loop(ppmd_md *md, int mechanism);
/* Launch shapes of the atom-index mechanism (PPMD_PAIR_COLUMNS, PPMD_FP32):
 * shape k of PPMD_MD_SHAPES sets the pair loop's threads per block (128 or
 * 256), whether it runs one thread per atom or as a persistent grid (a few
 * blocks per SM, each walking its share of the atoms), and the list build's
 * brick size (up to 128 or 64 expected atoms per brick):
 *   k  block  blocks per SM  brick atoms      k  block  blocks per SM  brick atoms
 *   0  128    one per atom   128              4  128    one per atom   64
 *   1  256    one per atom   128              5  256    one per atom   64
 *   2  128    8 (persistent) 128              6  128    8 (persistent) 64
 *   3  256    4 (persistent) 128              7  256    4 (persistent) 64
 * Every shape gives the same list (same pairs in the same order) and the
 * same positions, velocities and forces bit for bit; only the grouping of
 * the energy and virial sums follows the shape (last bits of the totals).
 * Shape 0 is the default.  ppmd_md_set_shape may be called at any time
 * (PPMD_ERR_INVALID for k != 0 with PPMD_FP64 or PPMD_PAIR_BRICKS);
 * ppmd_md_get_shape reads the shape and its three parameters (any output
 * may be NULL).
 * ppmd_md_tune (after ppmd_md_set_state): with cache_path (a text file, may
 * be NULL) holding an entry for this workload (atoms, boxes, cells,
 * cutoffs, list capacity and policy, device name and SM count), applies
 * the cached shape without timing anything; otherwise runs each shape from
 * the present state for `steps` steps (rounded up to whole graph units,
 * after one unit of warm-up), keeps the fastest, starts again from the
 * present state (as ppmd_md_set_state: the step counters restart at 0) and
 * appends the entry "key TAB shape TAB ms_per_step" to cache_path.
 * shape (host, may be NULL) receives the choice; ms_per_step (host, may be
 * NULL, PPMD_MD_SHAPES doubles) the measured time per step of each shape
 * (-1 where nothing was timed); timed (host, may be NULL) 1 if shapes were
 * timed, 0 if the cache (or a PPMD_FP64 / PPMD_PAIR_BRICKS run, which has
 * one shape) decided.  Uses 48 bytes of device memory per atom once. */
#define PPMD_MD_SHAPES 8
int ppmd_md_set_shape(ppmd_md *md, int32_t shape);
int ppmd_md_get_shape(ppmd_md *md, int32_t *shape, int32_t *block, int32_t *per_sm, int32_t *brick_home);
int ppmd_md_tune(ppmd_md *md, int32_t steps, const char *cache_path, int32_t *shape, double *ms_per_step, int *timed);
/* List-age check (Sec. 3.5, Eq. (3): a list built with the extended cutoff
 * r_list = r_c + delta holds every pair that can come within r_c before the
 * next build only while no atom moves more than delta / 2).  With on != 0
 * every later rebuild counts the pairs that are within r_c at that rebuild
 * but were at least r_list apart at the previous build, i.e. missing from
 * the list the pair loop used until then (FP32 tests, FP64 near both
 * cutoffs, positions to the fixed-point quantum L 2^-32).  It changes no
 * state: a checked run gives the same trajectory bit for bit.  Pairs that
 * came within r_c and left again between two builds are not seen, so the
 * count is a lower bound on the pairs the list missed.  The count restarts
 * at ppmd_md_set_state; ppmd_md_missed_pairs (host int64) reads it
 * (synchronises).  Uses 16 extra bytes of device memory per atom. */
int ppmd_md_set_check(ppmd_md *md, int on);
int ppmd_md_missed_pairs(ppmd_md *md, int64_t *missed);
/* Measurement aid: with on != 0, the last whole graph unit of each later run
 * replays a second graph that records a CUDA event before and after every
 * pair-loop launch (event-record graph nodes, on the integrator's stream;
 * the other units replay the graph without them, so the events cost the
 * run one unit's worth of nodes); ppmd_md_pair_loop_times then returns the
 * average duration (ms) of the pair loops of the last timed unit, those
 * that also made the next step's kick and drift (fused, FP32) and the
 * others, with their counts (host outputs, any may be NULL).  Synchronises.
 * PPMD_ERR_INVALID when no timed unit has run.  A run of several units
 * captures both graphs on first use. */
int ppmd_md_time_pair_loops(ppmd_md *md, int on);
int ppmd_md_pair_loop_times(ppmd_md *md, double *ms_fused, int32_t *n_fused, double *ms_other, int32_t *n_other);
/* Per-atom Q4, Q5, Q6 of the last analysis step (device float [n] each,
 * caller order; any may be NULL).  PPMD_ERR_INVALID before the first. */
int ppmd_md_get_q(ppmd_md *md, float *q4, float *q5, float *q6);
/* Copy positions, velocities and forces back in caller order (device,
 * [n][3] each; any may be NULL). */
int ppmd_md_get_state(ppmd_md *md, double *pos, double *vel, double *force);
/* Counters (host, any may be NULL): steps taken, list rebuilds, and the
 * largest displacement since a rebuild seen so far.  Synchronises; returns
 * PPMD_WARN_SKIN when that displacement exceeded half the list skin. */
int ppmd_md_info(ppmd_md *md, int64_t *steps, int64_t *rebuilds, double *max_disp);
/* Recompute the forces of the current state (the pair loop alone, the force
 * step of Algorithm 6), e.g. to time it; the state is otherwise unchanged. */
int ppmd_md_forces(ppmd_md *md);
/* Current neighbour list (host outputs, may be NULL): total listed pairs and
 * the largest row.  Synchronises. */
int ppmd_md_list_stats(ppmd_md *md, int64_t *pairs, int32_t *max_row);
/* The list of the last build (Sec. 3.5: pairs within the list cutoff r_list
 * of Eq. (3) at that build) in the caller's order: nbr_count[i] (device
 * int32 [n]) the number of neighbours of caller atom i, nbr (device int32
 * [n][max_nbr], row-major) the caller indices of its first max_nbr
 * neighbours in list order (entries past the count untouched).  Uses context
 * scratch of 4 bytes per atom and row entry. */
int ppmd_md_get_list(ppmd_md *md, int32_t *nbr, int32_t *nbr_count, int32_t max_nbr);

/* ------------------------------------------------------------------ */
/* Forces without any allocation.  The paper has no counterpart: this entry
 * point exists for callers that may not allocate device memory -- programs
 * whose device memory is owned by a host framework (a fixed pool or a
 * caching allocator that must see every byte), or latency-critical loops
 * that may not pay the device synchronisation cudaMalloc/cudaFree can imply.
 * It computes exactly what ppmd_lj_forces computes, with the same arguments
 * except that a CUDA stream (cudaStream_t, NULL = legacy default stream of
 * the current device) replaces the context.  It never calls cudaMalloc,
 * cudaFree or any allocating routine: its working memory is one statically
 * sized device array inside the library (about 4.2 MB, held by every GPU
 * that loads the library until the process exits).
 *  - n may not exceed PPMD_NOALLOC_MAX_ATOMS; larger n returns
 *    PPMD_ERR_CAPACITY at once (with a message on stderr), nothing launched.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.  The address is kept for the process: a
 *    device reset (cudaDeviceReset, which destroys the primary context and
 *    the module) invalidates it, so no call may follow a reset of that
 *    device.
 *  - All calls share the one array, which keeps the last call's contents:
 *    calls whose work overlaps on the GPU (different streams, or different
 *    host threads without ordering) race and give wrong results.
 *  - There is no context, so device-detected conditions (a non-finite
 *    coordinate) are not reported; argument and CUDA launch errors are. */
#define PPMD_NOALLOC_MAX_ATOMS 262144
int ppmd_lj_forces_noalloc(void *cuda_stream, const double *pos, int64_t n, const ppmd_box *box,
                           const ppmd_lj_params *lj, const int32_t *nbr, const int32_t *nbr_count, int32_t max_nbr,
                           ppmd_prec prec, double *force, double *e_atom, double *e_total, double *virial);

#ifdef __cplusplus
}
#endif
#endif /* PPMD_H */
