/*
 * Plain FP64 CPU oracle for the particle method of Saunders, Grant & Mueller,
 * "A Domain Specific Language for Performance Portable Molecular Dynamics
 * Algorithms" (arXiv:1704.03329).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the CUDA path is compared against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it.  It
 * shares no code, header, table or helper with the CUDA library.
 *
 * Every routine is a direct transcription of a definition in the paper:
 *   - periodic domain, cell list and neighbour list: Sec. 3.5 and Eq. (3)
 *     (extended cutoff), with the O(N^2) loop of Sec. 3.4 as brute force;
 *   - Lennard-Jones potential and force: Eq. (9) and Eq. (12) (appendix A.1);
 *   - Velocity Verlet: Algorithm 6 with the access descriptors of Table 5;
 *   - bond order parameters: Eqs. (4)-(5), Algorithms 1 and 2;
 *   - common neighbour analysis: Eqs. (6)-(8), Algorithms 3-5 and the
 *     largest-cluster Algorithm 7 (appendix D);
 *   - adaptive CNA (the extension the CNA section cites): per-atom cutoffs
 *     from the 12 or 14 nearest neighbours, then Eqs. (6)-(8).
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *   - all cutoff tests are strict (r < rc), as in the printed kernels;
 *   - the pair energy is V(r) = 4 eps ((s/r)^12 - (s/r)^6 + shift) with
 *     shift = 0 (truncated, unshifted) by default and 1/4 for Eq. (9);
 *   - the force follows Eq. (12) (repulsive at short range);
 *   - every ordered pair (i,j) is visited and only i is written (Sec. 2,
 *     "Comment on Newton's third law"), so the per-atom energy takes half of
 *     each pair term and the total energy is U = 1/2 sum_{i != j} V(r_ij);
 *   - periodic wrap x <- x - L floor(x/L) (an exact L maps to 0) and the
 *     minimum-image convention dr <- dr - L rint(dr/L).
 *
 * Built with -O2 -ffp-contract=off (no fused multiply-add) so that every
 * floating-point decision is the plain IEEE sequence written below.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_PI 3.14159265358979323846

/* Threads of the per-atom loops of the integrator (neighbour search, pair
 * loop, particle loops): 1 by default.  Every reduction over atoms is taken
 * afterwards in atom order, so the results do not depend on the count.   */
static int ora_nthreads = 1;
void ora_set_threads(int k) { ora_nthreads = k > 0 ? k : 1; }

/* ------------------------------------------------------------------ */
/* Periodic domain (Sec. 3.5)                                          */
/* ------------------------------------------------------------------ */

static double wrap1(double x, double L) {
    double y = x - L * floor(x / L);
    if (y >= L) y = 0.0;
    if (y < 0.0) y = 0.0;
    return y;
}

void ora_wrap(int64_t n, double *pos, const double *L) {
    for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d) pos[3 * i + d] = wrap1(pos[3 * i + d], L[d]);
}

/* Minimum-image separation r_i - r_j and its square. */
static double min_image(const double *pi, const double *pj, const double *L, double dr[3]) {
    for (int d = 0; d < 3; ++d) {
        double t = pi[d] - pj[d];
        t = t - L[d] * rint(t / L[d]);
        dr[d] = t;
    }
    return dr[0] * dr[0] + dr[1] * dr[1] + dr[2] * dr[2];
}

/* ------------------------------------------------------------------ */
/* Cell list (Sec. 3.5): cells of edge w_d = L_d / n_d >= r, n_d = floor(L_d / r).
 * Linear cell index c = (cz * ny + cy) * nx + cx.  The CSR arrays list the
 * atoms of every cell in increasing atom index.                         */
/* ------------------------------------------------------------------ */

void ora_cell_grid(const double *L, double r, int32_t *nc) {
    for (int d = 0; d < 3; ++d) nc[d] = (int32_t)floor(L[d] / r);
}

static int32_t cell_coord(double x, double L, int32_t n) {
    double w = L / n;
    double xw = wrap1(x, L);
    int32_t c = (int32_t)floor(xw / w);
    if (c > n - 1) c = n - 1;
    if (c < 0) c = 0;
    return c;
}

void ora_cells(int64_t n, const double *pos, const double *L, const int32_t *nc, int32_t *cell_of,
               int32_t *cell_start, int32_t *cell_atoms) {
    int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    for (int64_t c = 0; c <= ncell; ++c) cell_start[c] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int32_t cx = cell_coord(pos[3 * i + 0], L[0], nc[0]);
        int32_t cy = cell_coord(pos[3 * i + 1], L[1], nc[1]);
        int32_t cz = cell_coord(pos[3 * i + 2], L[2], nc[2]);
        cell_of[i] = (cz * nc[1] + cy) * nc[0] + cx;
        cell_start[cell_of[i] + 1] += 1;
    }
    for (int64_t c = 0; c < ncell; ++c) cell_start[c + 1] += cell_start[c];
    int32_t *fill = (int32_t *)calloc((size_t)(ncell > 0 ? ncell : 1), sizeof(int32_t));
    for (int64_t i = 0; i < n; ++i) {
        int32_t c = cell_of[i];
        cell_atoms[cell_start[c] + fill[c]] = (int32_t)i;
        fill[c] += 1;
    }
    free(fill);
}

/* ------------------------------------------------------------------ */
/* Neighbour lists: all j != i with |r_i - r_j| < r (minimum image), as CSR
 * (offs[n+1], nbr[offs[n]]), every row sorted by j.  Called once with
 * nbr == NULL to size the list.                                        */
/* ------------------------------------------------------------------ */

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* O(N^2) loop of Sec. 3.4. */
int64_t ora_neigh_brute(int64_t n, const double *pos, const double *L, double r, int64_t *offs, int32_t *nbr) {
    double r2 = r * r, dr[3];
    int64_t tot = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (offs) offs[i] = tot;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            if (min_image(&pos[3 * i], &pos[3 * j], L, dr) < r2) {
                if (nbr) nbr[tot] = (int32_t)j;
                ++tot;
            }
        }
    }
    if (offs) offs[n] = tot;
    return tot;
}

/* Cell-based loop of Sec. 3.5: the 27 cells around the cell of i.  Needs at
 * least three cells per edge so that the 27 cells are distinct.
 * Row of atom i: the number of its neighbours, written (sorted) to out when
 * out is not NULL. */
static int64_t neigh_cells_row(int64_t i, const double *pos, const double *L, double r2, const int32_t *nc,
                               const int32_t *cell_of, const int32_t *cell_start, const int32_t *cell_atoms,
                               int32_t *out) {
    double dr[3];
    int64_t cnt = 0;
    int32_t c = cell_of[i];
    int32_t cx = c % nc[0], cy = (c / nc[0]) % nc[1], cz = c / (nc[0] * nc[1]);
    for (int oz = -1; oz <= 1; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
                int32_t x = (cx + ox + nc[0]) % nc[0];
                int32_t y = (cy + oy + nc[1]) % nc[1];
                int32_t z = (cz + oz + nc[2]) % nc[2];
                int32_t cc = (z * nc[1] + y) * nc[0] + x;
                for (int32_t k = cell_start[cc]; k < cell_start[cc + 1]; ++k) {
                    int32_t j = cell_atoms[k];
                    if (j == i) continue;
                    if (min_image(&pos[3 * i], &pos[3 * j], L, dr) < r2) {
                        if (out) out[cnt] = j;
                        ++cnt;
                    }
                }
            }
    if (out) qsort(out, (size_t)cnt, sizeof(int32_t), cmp_i32);
    return cnt;
}

/* All rows: the counts first, their running sum as the row offsets, then
 * the rows (each atom's row depends on that atom alone). */
int64_t ora_neigh_cells(int64_t n, const double *pos, const double *L, double r, const int32_t *nc,
                        const int32_t *cell_of, const int32_t *cell_start, const int32_t *cell_atoms,
                        int64_t *offs, int32_t *nbr) {
    double r2 = r * r;
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for num_threads(ora_nthreads) schedule(static)
    for (int64_t i = 0; i < n; ++i) cnt[i] = neigh_cells_row(i, pos, L, r2, nc, cell_of, cell_start, cell_atoms, NULL);
    int64_t tot = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (offs) offs[i] = tot;
        tot += cnt[i];
    }
    if (offs) offs[n] = tot;
    if (nbr && offs) {
#pragma omp parallel for num_threads(ora_nthreads) schedule(static)
        for (int64_t i = 0; i < n; ++i)
            neigh_cells_row(i, pos, L, r2, nc, cell_of, cell_start, cell_atoms, nbr + offs[i]);
    }
    free(cnt);
    return tot;
}

/* ------------------------------------------------------------------ */
/* Lennard-Jones pair loop: Eq. (9) potential, Eq. (12) force.
 * For every ordered pair (i,j) in the list with r^2 < rc^2:
 *   F_i += 48 eps / sigma^2 * dr * ((sigma/r)^14 - 1/2 (sigma/r)^8)
 *   e_i += 1/2 * 4 eps ((sigma/r)^12 - (sigma/r)^6 + shift)
 * U = sum_i e_i; virial W = 1/2 sum_{i != j} dr_ij . f_ij (= sum_{i<j}).  */
/* ------------------------------------------------------------------ */

void ora_lj(int64_t n, const double *pos, const double *L, double eps, double sigma, double rc, double shift,
            const int64_t *offs, const int32_t *nbr, double *F, double *e_atom, double *U, double *W) {
    double rc2 = rc * rc, s2 = sigma * sigma;
    /* per-atom energy and virial terms, summed over the atoms in atom order below */
    double *ew = (double *)malloc(sizeof(double) * (size_t)(2 * (n > 0 ? n : 1)));
#pragma omp parallel for num_threads(ora_nthreads) schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double dr[3];
        double fx = 0.0, fy = 0.0, fz = 0.0, ei = 0.0, wsum = 0.0;
        for (int64_t k = offs[i]; k < offs[i + 1]; ++k) {
            int32_t j = nbr[k];
            double r2 = min_image(&pos[3 * i], &pos[3 * j], L, dr);
            if (!(r2 < rc2)) continue;
            double sr2 = s2 / r2;
            double sr6 = sr2 * sr2 * sr2;
            double sr8 = sr6 * sr2;
            double sr12 = sr6 * sr6;
            double sr14 = sr12 * sr2;
            double fmag = 48.0 * eps / s2 * (sr14 - 0.5 * sr8);
            fx += fmag * dr[0];
            fy += fmag * dr[1];
            fz += fmag * dr[2];
            ei += 0.5 * 4.0 * eps * (sr12 - sr6 + shift);
            wsum += 0.5 * fmag * r2;
        }
        F[3 * i + 0] = fx;
        F[3 * i + 1] = fy;
        F[3 * i + 2] = fz;
        if (e_atom) e_atom[i] = ei;
        ew[2 * i] = ei;
        ew[2 * i + 1] = wsum;
    }
    double usum = 0.0, wtot = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        usum += ew[2 * i];
        wtot += ew[2 * i + 1];
    }
    free(ew);
    if (U) *U = usum;
    if (W) *W = wtot;
}

/* ------------------------------------------------------------------ */
/* Velocity Verlet, Algorithm 6.
 *   phase 1 (first half kick, drift): v += dt/(2m) F ; r += dt v ; then wrap
 *   phase 2 (second half kick, after the forces): v += dt/(2m) F        */
/* ------------------------------------------------------------------ */

void ora_vv(int phase, int64_t n, double *pos, double *vel, const double *F, const double *L, double mass,
            double dt) {
    double h = dt / (2.0 * mass);
    for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d) {
            vel[3 * i + d] += h * F[3 * i + d];
            if (phase == 1) pos[3 * i + d] = wrap1(pos[3 * i + d] + dt * vel[3 * i + d], L[d]);
        }
}

double ora_kinetic(int64_t n, const double *vel, double mass) {
    double k = 0.0;
    for (int64_t i = 0; i < n; ++i)
        k += 0.5 * mass * (vel[3 * i] * vel[3 * i] + vel[3 * i + 1] * vel[3 * i + 1] + vel[3 * i + 2] * vel[3 * i + 2]);
    return k;
}

/* Full time-stepping loop (Algorithm 6 driven by the list-reuse policy of
 * Sec. 3.5 / Eq. (3)): the list with cutoff r_list is built from the
 * initial positions, F(r_0) is computed once, and for s = 1..nsteps:
 * kick+drift, rebuild the list if s % rebuild_every == 0, forces, kick.
 * energies (if not NULL) receives [KE, PE] after every step (2*nsteps).
 * Returns the largest displacement seen between rebuilds (the skin guard).
 */
static int64_t build_list_cells(int64_t n, const double *pos, const double *L, double r_list, int64_t *offs,
                                int32_t **nbr, int64_t *cap) {
    int32_t nc[3];
    ora_cell_grid(L, r_list, nc);
    if (nc[0] < 3 || nc[1] < 3 || nc[2] < 3) {
        /* fewer than three cells per edge: the 27 cells would repeat, so use
         * the O(N^2) loop instead */
        int64_t tot = ora_neigh_brute(n, pos, L, r_list, offs, NULL);
        if (tot > *cap) {
            free(*nbr);
            *nbr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(tot > 0 ? tot : 1));
            *cap = tot;
        }
        ora_neigh_brute(n, pos, L, r_list, offs, *nbr);
        return tot;
    }
    int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    int32_t *cell_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *cell_start = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ncell + 1));
    int32_t *cell_atoms = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    ora_cells(n, pos, L, nc, cell_of, cell_start, cell_atoms);
    int64_t tot = ora_neigh_cells(n, pos, L, r_list, nc, cell_of, cell_start, cell_atoms, offs, NULL);
    if (tot > *cap) {
        free(*nbr);
        *nbr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(tot > 0 ? tot : 1));
        *cap = tot;
    }
    ora_neigh_cells(n, pos, L, r_list, nc, cell_of, cell_start, cell_atoms, offs, *nbr);
    free(cell_of);
    free(cell_start);
    free(cell_atoms);
    return tot;
}

void ora_boa_direct(int64_t n, const double *pos, const double *L, double r_cut, const int64_t *offs,
                    const int32_t *nbr, int l, double *Q, int32_t *nnb);

/* Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers:
 * as easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplications
 * by 0xD2511F53 and 0xCD9E8D57, the counter words permuted and mixed with
 * the key, the key advanced by the Weyl constants 0x9E3779B9 and 0xBB67AE85
 * before every round but the first. */
static uint32_t mulhilo32(uint32_t a, uint32_t b, uint32_t *lo) {
    const uint64_t p = (uint64_t)a * (uint64_t)b;
    *lo = (uint32_t)p;
    return (uint32_t)(p >> 32);
}

void ora_philox4x32(const uint32_t *ctr, const uint32_t *key, uint32_t *out) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3], k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t lo0, lo1;
        const uint32_t hi0 = mulhilo32(0xD2511F53u, c0, &lo0);
        const uint32_t hi1 = mulhilo32(0xCD9E8D57u, c2, &lo1);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* Andersen thermostat (the on-the-fly analysis run of Sec. 5.2 couples the
 * system to one): at the end of step s, atom id collides with the heat bath
 * with probability p = nu dt, decided by the first word u0 of Philox at
 * counter (id, s mod 2^32, s / 2^32, 0) and key (seed mod 2^32, seed / 2^32):
 * u0 < thr = floor(p 2^32) (every atom when p >= 1).  Its new velocity is
 * drawn from N(0, T/m) per component by the Box-Muller transform of the
 * uniforms U(u) = (u + 1/2) 2^-32: (v_x, v_y) from (u1, u2), v_z from u3 and
 * the first word of the draw at counter word 3 = 1. */
static int andersen_draw(uint64_t seed, int64_t id, int64_t step, uint64_t thr, double sd, double v[3]) {
    const double two_pi = 6.283185307179586, inv32 = 2.3283064365386962890625e-10;
    uint32_t ctr[4] = {(uint32_t)id, (uint32_t)step, (uint32_t)((uint64_t)step >> 32), 0u};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t u[4], w[4];
    ora_philox4x32(ctr, key, u);
    if ((uint64_t)u[0] >= thr) return 0;
    ctr[3] = 1u;
    ora_philox4x32(ctr, key, w);
    const double U1 = ((double)u[1] + 0.5) * inv32, U2 = ((double)u[2] + 0.5) * inv32;
    const double U3 = ((double)u[3] + 0.5) * inv32, U4 = ((double)w[0] + 0.5) * inv32;
    const double r1 = sqrt(-2.0 * log(U1)), t1 = two_pi * U2;
    const double r2 = sqrt(-2.0 * log(U3)), t2 = two_pi * U4;
    v[0] = sd * (r1 * cos(t1));
    v[1] = sd * (r1 * sin(t1));
    v[2] = sd * (r2 * cos(t2));
    return 1;
}

uint64_t ora_andersen_threshold(double nu, double dt) {
    const double p = nu * dt;
    if (!(p > 0.0)) return 0;
    if (p >= 1.0) return (uint64_t)1 << 32;
    return (uint64_t)floor(p * 4294967296.0);
}

/* Algorithm 6 as ora_md_run, with the additions of the on-the-fly analysis
 * run (Sec. 5.2): after the kick of step s (and the energies) the Andersen
 * thermostat (thr = 0: none; T, seed as above); then, when boa_every > 0
 * and s % boa_every == 0, Q4, Q5, Q6 of every atom over the current list
 * with cutoff r_boa (Eqs. (4)-(5)), their means written to
 * qrows[3 (s - 1) .. +2] and the per-atom values of the last such step to
 * qlast [3][n] (either may be NULL).  Returns the number of collisions. */
int64_t ora_md_run_otf(int64_t n, double *pos, double *vel, double *F, const double *L, double eps, double sigma,
                       double rc, double shift, double r_list, int32_t rebuild_every, double mass, double dt,
                       int32_t nsteps, double *energies, uint64_t thr, double T, uint64_t seed, int32_t boa_every,
                       double r_boa, double *qrows, double *qlast, double *maxdisp_out) {
    int64_t *offs = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int32_t *nbr = NULL;
    int64_t cap = 0, ncoll = 0;
    double *ref = (double *)malloc(sizeof(double) * (size_t)(3 * n));
    double *Q = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    const double sd = sqrt(T / mass);
    double maxdisp = 0.0;
    ora_wrap(n, pos, L);
    build_list_cells(n, pos, L, r_list, offs, &nbr, &cap);
    memcpy(ref, pos, sizeof(double) * (size_t)(3 * n));
    double U;
    ora_lj(n, pos, L, eps, sigma, rc, shift, offs, nbr, F, NULL, &U, NULL);
    for (int32_t s = 1; s <= nsteps; ++s) {
        ora_vv(1, n, pos, vel, F, L, mass, dt);
        double md2 = maxdisp * maxdisp;
#pragma omp parallel for num_threads(ora_nthreads) schedule(static) reduction(max : md2)
        for (int64_t i = 0; i < n; ++i) {
            double dr[3];
            double d2 = min_image(&pos[3 * i], &ref[3 * i], L, dr);
            if (d2 > md2) md2 = d2;
        }
        maxdisp = sqrt(md2);
        if (rebuild_every > 0 && s % rebuild_every == 0) {
            build_list_cells(n, pos, L, r_list, offs, &nbr, &cap);
            memcpy(ref, pos, sizeof(double) * (size_t)(3 * n));
        }
        ora_lj(n, pos, L, eps, sigma, rc, shift, offs, nbr, F, NULL, &U, NULL);
        ora_vv(2, n, pos, vel, F, L, mass, dt);
        if (energies) {
            energies[2 * (s - 1)] = ora_kinetic(n, vel, mass);
            energies[2 * (s - 1) + 1] = U;
        }
        if (thr > 0)
            for (int64_t i = 0; i < n; ++i) ncoll += andersen_draw(seed, i, s, thr, sd, &vel[3 * i]);
        if (boa_every > 0 && s % boa_every == 0) {
            for (int l = 4; l <= 6; ++l) {
                ora_boa_direct(n, pos, L, r_boa, offs, nbr, l, Q, NULL);
                double sum = 0.0;
                for (int64_t i = 0; i < n; ++i) sum += Q[i];
                if (qrows) qrows[3 * (s - 1) + (l - 4)] = sum / (double)(n > 0 ? n : 1);
                if (qlast) memcpy(&qlast[(l - 4) * n], Q, sizeof(double) * (size_t)n);
            }
        }
    }
    free(offs);
    free(nbr);
    free(ref);
    free(Q);
    if (maxdisp_out) *maxdisp_out = maxdisp;
    return ncoll;
}

double ora_md_run(int64_t n, double *pos, double *vel, double *F, const double *L, double eps, double sigma,
                  double rc, double shift, double r_list, int32_t rebuild_every, double mass, double dt,
                  int32_t nsteps, double *energies) {
    int64_t *offs = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int32_t *nbr = NULL;
    int64_t cap = 0;
    double *ref = (double *)malloc(sizeof(double) * (size_t)(3 * n));
    double maxdisp = 0.0;
    ora_wrap(n, pos, L);
    build_list_cells(n, pos, L, r_list, offs, &nbr, &cap);
    memcpy(ref, pos, sizeof(double) * (size_t)(3 * n));
    double U;
    ora_lj(n, pos, L, eps, sigma, rc, shift, offs, nbr, F, NULL, &U, NULL);
    for (int32_t s = 1; s <= nsteps; ++s) {
        ora_vv(1, n, pos, vel, F, L, mass, dt);
        double md2 = maxdisp * maxdisp;
#pragma omp parallel for num_threads(ora_nthreads) schedule(static) reduction(max : md2)
        for (int64_t i = 0; i < n; ++i) {
            double dr[3];
            double d2 = min_image(&pos[3 * i], &ref[3 * i], L, dr);
            if (d2 > md2) md2 = d2;
        }
        maxdisp = sqrt(md2);
        if (rebuild_every > 0 && s % rebuild_every == 0) {
            build_list_cells(n, pos, L, r_list, offs, &nbr, &cap);
            memcpy(ref, pos, sizeof(double) * (size_t)(3 * n));
        }
        ora_lj(n, pos, L, eps, sigma, rc, shift, offs, nbr, F, NULL, &U, NULL);
        ora_vv(2, n, pos, vel, F, L, mass, dt);
        if (energies) {
            energies[2 * (s - 1)] = ora_kinetic(n, vel, mass);
            energies[2 * (s - 1) + 1] = U;
        }
    }
    free(offs);
    free(nbr);
    free(ref);
    return maxdisp;
}

/* ------------------------------------------------------------------ */
/* Bond order analysis, Eqs. (4)-(5), Algorithms 1-2.
 * Two independent evaluations of Q_l for l = 4 and l = 6:
 *  (a) direct: q~_lm = sum_j Y_l^m(r^_ij) with orthonormal spherical
 *      harmonics built from the associated Legendre three-term recurrence
 *      (Abramowitz & Stegun 8.5.3 / 8.6.x), every m = -l..l evaluated;
 *  (b) addition theorem: sum_m Y_l^m(u) conj(Y_l^m(v)) = (2l+1)/(4 pi) P_l(u.v),
 *      so Q_l = sqrt(sum_j sum_k P_l(u_j . u_k)) / nu, with P_l from Bonnet's
 *      recurrence (l+1) P_{l+1} = (2l+1) x P_l - l P_{l-1}.
 * Neighbours: every j in the given list with |r_i - r_j| < r_cut.
 * Q_l = 0 when an atom has no neighbour.                                */
/* ------------------------------------------------------------------ */

/* Associated Legendre P_l^m(x), m >= 0, with the Condon-Shortley phase. */
static double assoc_legendre(int l, int m, double x) {
    double pmm = 1.0;
    double s = sqrt((1.0 - x) * (1.0 + x));
    double fact = 1.0;
    for (int k = 1; k <= m; ++k) {
        pmm *= -fact * s;
        fact += 2.0;
    }
    if (l == m) return pmm;
    double pmmp1 = x * (2.0 * m + 1.0) * pmm;
    if (l == m + 1) return pmmp1;
    double pll = 0.0;
    for (int ll = m + 2; ll <= l; ++ll) {
        pll = ((2.0 * ll - 1.0) * x * pmmp1 - (ll + m - 1.0) * pmm) / (ll - m);
        pmm = pmmp1;
        pmmp1 = pll;
    }
    return pll;
}

static double factorial(int k) {
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= i;
    return f;
}

/* Y_l^m(theta, phi) for any m in [-l, l], orthonormal on the unit sphere;
 * Y_l^{-m} = (-1)^m conj(Y_l^m). */
static void sph_harm(int l, int m, double ct, double phi, double *re, double *im) {
    int am = m < 0 ? -m : m;
    double norm = sqrt((2.0 * l + 1.0) / (4.0 * ORA_PI) * factorial(l - am) / factorial(l + am));
    double p = norm * assoc_legendre(l, am, ct);
    double yr = p * cos(am * phi), yi = p * sin(am * phi);
    if (m < 0) {
        double sgn = (am % 2) ? -1.0 : 1.0;
        yr = sgn * yr;
        yi = -sgn * yi;
    }
    *re = yr;
    *im = yi;
}

void ora_boa_direct(int64_t n, const double *pos, const double *L, double r_cut, const int64_t *offs,
                    const int32_t *nbr, int l, double *Q, int32_t *nnb) {
    double rc2 = r_cut * r_cut, dr[3];
    double qre[32], qim[32];
    for (int64_t i = 0; i < n; ++i) {
        int nu = 0;
        for (int m = -l; m <= l; ++m) qre[m + l] = qim[m + l] = 0.0;
        for (int64_t k = offs[i]; k < offs[i + 1]; ++k) {
            int32_t j = nbr[k];
            double r2 = min_image(&pos[3 * i], &pos[3 * j], L, dr);
            if (!(r2 < rc2)) continue;
            double r = sqrt(r2);
            double ct = dr[2] / r;
            if (ct > 1.0) ct = 1.0;
            if (ct < -1.0) ct = -1.0;
            double phi = atan2(dr[1], dr[0]);
            for (int m = -l; m <= l; ++m) {
                double yr, yi;
                sph_harm(l, m, ct, phi, &yr, &yi);
                qre[m + l] += yr;
                qim[m + l] += yi;
            }
            ++nu;
        }
        if (nnb) nnb[i] = nu;
        if (nu == 0) {
            Q[i] = 0.0;
            continue;
        }
        double s = 0.0;
        for (int m = -l; m <= l; ++m) {
            double a = qre[m + l] / nu, b = qim[m + l] / nu;
            s += a * a + b * b;
        }
        Q[i] = sqrt(4.0 * ORA_PI / (2.0 * l + 1.0) * s);
    }
}

static double legendre_p(int l, double x) {
    double p0 = 1.0, p1 = x;
    if (l == 0) return p0;
    for (int k = 1; k < l; ++k) {
        double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

void ora_boa_addition(int64_t n, const double *pos, const double *L, double r_cut, const int64_t *offs,
                      const int32_t *nbr, int l, double *Q) {
    double rc2 = r_cut * r_cut, dr[3];
    double *u = NULL;
    int64_t ucap = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t deg = offs[i + 1] - offs[i];
        if (deg > ucap) {
            free(u);
            u = (double *)malloc(sizeof(double) * (size_t)(3 * deg));
            ucap = deg;
        }
        int nu = 0;
        for (int64_t k = offs[i]; k < offs[i + 1]; ++k) {
            double r2 = min_image(&pos[3 * i], &pos[3 * nbr[k]], L, dr);
            if (!(r2 < rc2)) continue;
            double r = sqrt(r2);
            u[3 * nu] = dr[0] / r;
            u[3 * nu + 1] = dr[1] / r;
            u[3 * nu + 2] = dr[2] / r;
            ++nu;
        }
        if (nu == 0) {
            Q[i] = 0.0;
            continue;
        }
        double s = 0.0;
        for (int a = 0; a < nu; ++a)
            for (int b = 0; b < nu; ++b) {
                double c = u[3 * a] * u[3 * b] + u[3 * a + 1] * u[3 * b + 1] + u[3 * a + 2] * u[3 * b + 2];
                s += legendre_p(l, c);
            }
        if (s < 0.0) s = 0.0;
        Q[i] = sqrt(s) / nu;
    }
    free(u);
}

/* ------------------------------------------------------------------ */
/* Common neighbour analysis, Eqs. (6)-(8), Algorithms 3, 4, 5 and 7.
 * Bonded: |r_i - r_j| < r_cut.  For every atom i the bond array E^(i)
 * (pairs of global ids) is filled by loop I (direct bonds (i, j)) and loop
 * II (indirect bonds (j, w) of every bonded j, w != i); loop III then forms
 * for each bonded pair (i, j) the common-neighbour set C, the set E of bonds
 * among C (canonical (min, max), no duplicates) and the triplet
 * (|C|, |E|, largest cluster of E counted in edges).
 * Output: nbond[i] = nu_nb(i); trip[i*max_bond + t] = ncn<<16 | nb<<8 | nlcb
 * and partner[i*max_bond + t] = j for the t-th bonded neighbour (list order).
 * Returns the largest nu_nb seen; when it exceeds max_bond nothing past
 * max_bond is written for that atom.                                   */
/* ------------------------------------------------------------------ */

typedef struct {
    int32_t a, b;
} ora_edge;

/* Algorithm 7: edges of the largest connected component of the edge set. */
static int max_cluster_size(const ora_edge *edges_in, int ne) {
    ora_edge *E = (ora_edge *)malloc(sizeof(ora_edge) * (size_t)(ne > 0 ? ne : 1));
    int32_t *Q = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * ne + 2));
    memcpy(E, edges_in, sizeof(ora_edge) * (size_t)ne);
    int left = ne, smax = 0;
    while (left > 0) {
        int S = 0, qn = 0;
        Q[qn++] = E[0].a; /* pick some edge (v1, v2); Q = {v1} */
        while (qn > 0) {
            int32_t v = Q[--qn]; /* pick some v in Q and remove it */
            /* P = remaining edges incident to v (edges are undirected) */
            int k = 0;
            while (k < left) {
                if (E[k].a == v || E[k].b == v) {
                    int32_t w = (E[k].a == v) ? E[k].b : E[k].a;
                    int seen = 0;
                    for (int q = 0; q < qn; ++q) seen |= (Q[q] == w);
                    if (!seen) Q[qn++] = w;
                    S += 1;
                    E[k] = E[left - 1]; /* remove the edge from the set */
                    --left;
                } else {
                    ++k;
                }
            }
        }
        if (S > smax) smax = S;
    }
    free(E);
    free(Q);
    return smax;
}

static int in_set(const int32_t *s, int n, int32_t v) {
    for (int k = 0; k < n; ++k)
        if (s[k] == v) return 1;
    return 0;
}

int32_t ora_cna(int64_t n, const double *pos, const double *L, double r_cut, const int64_t *offs,
                const int32_t *nbr, int32_t max_bond, int32_t *nbond, uint32_t *trip, int32_t *partner) {
    double rc2 = r_cut * r_cut, dr[3];
    /* Loop I: direct bonds. */
    int32_t *nu_nb = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    int64_t *eoff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t tot = 0;
    for (int64_t i = 0; i < n; ++i) {
        eoff[i] = tot;
        for (int64_t k = offs[i]; k < offs[i + 1]; ++k)
            if (min_image(&pos[3 * i], &pos[3 * nbr[k]], L, dr) < rc2) ++tot;
    }
    eoff[n] = tot;
    int32_t *direct = (int32_t *)malloc(sizeof(int32_t) * (size_t)(tot > 0 ? tot : 1));
    int32_t numax = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t t = eoff[i];
        for (int64_t k = offs[i]; k < offs[i + 1]; ++k)
            if (min_image(&pos[3 * i], &pos[3 * nbr[k]], L, dr) < rc2) direct[t++] = nbr[k];
        nu_nb[i] = (int32_t)(t - eoff[i]);
        if (nu_nb[i] > numax) numax = nu_nb[i];
    }
    /* Loop II: indirect bonds of atom i, E^(i) = direct part followed by the
     * bonds (j, w) of every bonded j with w != i. */
    for (int64_t i = 0; i < n; ++i) {
        int ni = nu_nb[i];
        int64_t cap = ni;
        for (int a = 0; a < ni; ++a) cap += nu_nb[direct[eoff[i] + a]];
        ora_edge *Ei = (ora_edge *)malloc(sizeof(ora_edge) * (size_t)(cap > 0 ? cap : 1));
        int nb_i = 0;
        for (int a = 0; a < ni; ++a) {
            Ei[nb_i].a = (int32_t)i;
            Ei[nb_i].b = direct[eoff[i] + a];
            ++nb_i;
        }
        for (int a = 0; a < ni; ++a) {
            int32_t j = direct[eoff[i] + a];
            for (int b = 0; b < nu_nb[j]; ++b) {
                int32_t w = direct[eoff[j] + b];
                if (w != (int32_t)i) {
                    Ei[nb_i].a = j;
                    Ei[nb_i].b = w;
                    ++nb_i;
                }
            }
        }
        /* Loop III: one triplet per bonded pair (i, j). */
        int32_t *C = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ni > 0 ? ni : 1));
        ora_edge *Ec = (ora_edge *)malloc(sizeof(ora_edge) * (size_t)(nb_i > 0 ? nb_i : 1));
        for (int a = 0; a < ni; ++a) {
            int32_t j = direct[eoff[i] + a];
            int nc = 0;
            for (int b = 0; b < ni; ++b) {
                int32_t v = direct[eoff[i] + b];
                if (in_set(&direct[eoff[j]], nu_nb[j], v)) C[nc++] = v;
            }
            int ne = 0;
            for (int k = ni; k < nb_i; ++k) {
                int32_t v = Ei[k].a, w = Ei[k].b;
                if (!in_set(C, nc, v) || !in_set(C, nc, w)) continue;
                if (v > w) {
                    int32_t t = v;
                    v = w;
                    w = t;
                }
                int dup = 0;
                for (int e = 0; e < ne; ++e) dup |= (Ec[e].a == v && Ec[e].b == w);
                if (!dup) {
                    Ec[ne].a = v;
                    Ec[ne].b = w;
                    ++ne;
                }
            }
            int nl = max_cluster_size(Ec, ne);
            if (a < max_bond) {
                trip[i * max_bond + a] = ((uint32_t)nc << 16) | ((uint32_t)ne << 8) | (uint32_t)nl;
                if (partner) partner[i * max_bond + a] = j;
            }
        }
        nbond[i] = ni;
        free(C);
        free(Ec);
        free(Ei);
    }
    free(nu_nb);
    free(eoff);
    free(direct);
    return numax;
}

/* Structure label from the multiset of triplets of one atom (Sec. 4.2 and
 * the reference signatures it cites):
 *   fcc: 12 bonds, all (4,2,1);  hcp: 12 bonds, 6 x (4,2,1) + 6 x (4,2,2);
 *   bcc: 14 bonds, 8 x (6,6,6) + 6 x (4,4,4);  anything else: other.
 * Codes: 0 other, 1 fcc, 2 hcp, 3 bcc. */
void ora_cna_label(int64_t n, const int32_t *nbond, const uint32_t *trip, int32_t max_bond, int8_t *label) {
    const uint32_t t421 = (4u << 16) | (2u << 8) | 1u;
    const uint32_t t422 = (4u << 16) | (2u << 8) | 2u;
    const uint32_t t444 = (4u << 16) | (4u << 8) | 4u;
    const uint32_t t666 = (6u << 16) | (6u << 8) | 6u;
    for (int64_t i = 0; i < n; ++i) {
        int nb = nbond[i];
        int c421 = 0, c422 = 0, c444 = 0, c666 = 0;
        if (nb <= max_bond)
            for (int a = 0; a < nb; ++a) {
                uint32_t t = trip[i * max_bond + a];
                c421 += (t == t421);
                c422 += (t == t422);
                c444 += (t == t444);
                c666 += (t == t666);
            }
        int8_t lab = 0;
        if (nb == 12 && c421 == 12) lab = 1;
        else if (nb == 12 && c421 == 6 && c422 == 6) lab = 2;
        else if (nb == 14 && c666 == 8 && c444 == 6) lab = 3;
        label[i] = lab;
    }
}

/* ------------------------------------------------------------------ */
/* Local-environment features for the learned classifier (30 per atom):
 *   [0] Q4, [1] Q6 over neighbours within r_feat (Eqs. (4)-(5), computed by
 *       the direct route above);
 *   [2..15]  the 14 smallest neighbour distances d within r_feat, ascending,
 *            as (d - r_ref) / (r_feat - r_ref) (r_ref: a reference length
 *            inside the shell, the CNA cutoff), missing ones set to 1;
 *   [16..29] a 14-bin histogram of the chord |r_ij - r_ik| of every bond
 *            angle theta_jik between two bonded neighbours j, k of i (bonded:
 *            closer than r_ref), bins of width 0.05 centred on
 *            r_ref - 0.35 + 0.05 (b + 1/2), linear (tent) weights between
 *            adjacent centres, clamped at both ends, divided by 24 (the number
 *            of such pairs a perfect fcc or hcp site has at 60 degrees).
 */
/* ------------------------------------------------------------------ */

static int cmp_f64(const void *a, const void *b) {
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

void ora_features(int64_t n, const double *pos, const double *L, double r_feat, double r_ref, const int64_t *offs,
                  const int32_t *nbr, double *feat) {
    double rc2 = r_feat * r_feat, dr[3];
    double *q4 = (double *)malloc(sizeof(double) * (size_t)n);
    double *q6 = (double *)malloc(sizeof(double) * (size_t)n);
    ora_boa_direct(n, pos, L, r_feat, offs, nbr, 4, q4, NULL);
    ora_boa_direct(n, pos, L, r_feat, offs, nbr, 6, q6, NULL);
    double *d = NULL, *u = NULL;
    int64_t cap = 0;
    for (int64_t i = 0; i < n; ++i) {
        double *f = &feat[30 * i];
        f[0] = q4[i];
        f[1] = q6[i];
        int64_t deg = offs[i + 1] - offs[i];
        if (deg > cap) {
            free(d);
            free(u);
            d = (double *)malloc(sizeof(double) * (size_t)deg);
            u = (double *)malloc(sizeof(double) * (size_t)(3 * deg));
            cap = deg;
        }
        int nu = 0;
        for (int64_t k = offs[i]; k < offs[i + 1]; ++k) {
            double r2 = min_image(&pos[3 * i], &pos[3 * nbr[k]], L, dr);
            if (!(r2 < rc2)) continue;
            double r = sqrt(r2);
            d[nu] = r;
            u[3 * nu] = dr[0] / r;
            u[3 * nu + 1] = dr[1] / r;
            u[3 * nu + 2] = dr[2] / r;
            ++nu;
        }
        qsort(d, (size_t)nu, sizeof(double), cmp_f64);
        for (int k = 0; k < 14; ++k) f[2 + k] = (k < nu) ? (d[k] - r_ref) / (r_feat - r_ref) : 1.0;
        for (int b = 0; b < 14; ++b) f[16 + b] = 0.0;
        /* bonded neighbours: the vectors r_i - r_j with |r_i - r_j| < r_ref */
        int nb_ = 0;
        for (int64_t k = offs[i]; k < offs[i + 1]; ++k) {
            double r2 = min_image(&pos[3 * i], &pos[3 * nbr[k]], L, dr);
            if (!(r2 < r_ref * r_ref)) continue;
            u[3 * nb_] = dr[0];
            u[3 * nb_ + 1] = dr[1];
            u[3 * nb_ + 2] = dr[2];
            ++nb_;
        }
        double lo = r_ref - 0.35;
        for (int a = 0; a < nb_; ++a)
            for (int b = a + 1; b < nb_; ++b) {
                double cx = u[3 * a] - u[3 * b], cy = u[3 * a + 1] - u[3 * b + 1], cz = u[3 * a + 2] - u[3 * b + 2];
                double chord = sqrt(cx * cx + cy * cy + cz * cz);
                double x = (chord - lo) / 0.05 - 0.5;
                int b0 = (int)floor(x);
                double t = x - b0;
                if (b0 < 0) {
                    f[16 + 0] += 1.0;
                } else if (b0 >= 13) {
                    f[16 + 13] += 1.0;
                } else {
                    f[16 + b0] += 1.0 - t;
                    f[16 + b0 + 1] += t;
                }
            }
        for (int b = 0; b < 14; ++b) f[16 + b] /= 24.0;
    }
    free(d);
    free(u);
    free(q4);
    free(q6);
}

/* ------------------------------------------------------------------ */
/* Adaptive CNA: the extension of CNA that the CNA section cites
 * (Stukowski 2012) to remove the choice of the cutoff.  Each atom i sets its
 * own bond cutoff from its N nearest neighbours (distances d_1 <= ... <= d_N
 * over its list, ties by index; N = 12 for the fcc/hcp test, 14 for bcc):
 *   fcc/hcp  r_i = f (d_1 + ... + d_12) / 12,
 *   bcc      r_i = f (c (d_1 + ... + d_8) + d_9 + ... + d_14) / 14,
 * with f = (1 + sqrt 2) / 2 (midway between the first and second shells of
 * fcc in units of the nearest-neighbour distance) and c = 2 / sqrt 3 (the
 * first bcc shell scaled to the second).  Only those N neighbours take part:
 * all are bonded to i, and two of them are bonded when closer than r_i
 * (strict, as everywhere).  The bond i-j then gets the CNA triplet of
 * Eqs. (6)-(8) over the common neighbours among the N, with Algorithm 7 for
 * the largest cluster.  fcc: 12 x (4,2,1); hcp: 6 x (4,2,1) + 6 x (4,2,2)
 * (12-neighbour test); failing both, bcc: 8 x (6,6,6) + 6 x (4,4,4)
 * (14-neighbour test); else other.  A test that needs more neighbours than
 * the list holds fails.  rcut (may be NULL): [n][2], the two cutoffs, 0 when
 * not computed (the bcc one only when the fcc/hcp test failed).
 * ------------------------------------------------------------------ */
typedef struct {
    double r2;
    int32_t j;
} ora_nb;

static int cmp_nb(const void *a, const void *b) {
    const ora_nb *x = (const ora_nb *)a, *y = (const ora_nb *)b;
    if (x->r2 < y->r2) return -1;
    if (x->r2 > y->r2) return 1;
    return (x->j > y->j) - (x->j < y->j);
}

/* Triplet of the bond between the centre and sel[a] among the N selected. */
static uint32_t acna_triplet(const double *pos, const double *L, const int32_t *sel, int N, int a, double rc2) {
    int32_t cn[16];
    int ncn = 0;
    double dr[3];
    for (int b = 0; b < N; ++b)
        if (b != a && min_image(&pos[3 * sel[a]], &pos[3 * sel[b]], L, dr) < rc2) cn[ncn++] = sel[b];
    ora_edge E[16 * 15 / 2];
    int ne = 0;
    for (int p = 0; p < ncn; ++p)
        for (int q = p + 1; q < ncn; ++q)
            if (min_image(&pos[3 * cn[p]], &pos[3 * cn[q]], L, dr) < rc2) {
                E[ne].a = cn[p];
                E[ne].b = cn[q];
                ++ne;
            }
    const int nlcb = ne > 0 ? max_cluster_size(E, ne) : 0;
    return ((uint32_t)ncn << 16) | ((uint32_t)ne << 8) | (uint32_t)nlcb;
}

void ora_acna(int64_t n, const double *pos, const double *L, const int64_t *offs, const int32_t *nbr, int8_t *label,
              double *rcut) {
    const double f = (1.0 + sqrt(2.0)) * 0.5;
    const double c = 2.0 / sqrt(3.0);
    const uint32_t t421 = (4u << 16) | (2u << 8) | 1u, t422 = (4u << 16) | (2u << 8) | 2u;
    const uint32_t t444 = (4u << 16) | (4u << 8) | 4u, t666 = (6u << 16) | (6u << 8) | 6u;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t deg = offs[i + 1] - offs[i];
        ora_nb *cand = (ora_nb *)malloc(sizeof(ora_nb) * (size_t)(deg > 0 ? deg : 1));
        double dr[3];
        for (int64_t k = 0; k < deg; ++k) {
            cand[k].j = nbr[offs[i] + k];
            cand[k].r2 = min_image(&pos[3 * i], &pos[3 * cand[k].j], L, dr);
        }
        qsort(cand, (size_t)deg, sizeof(ora_nb), cmp_nb);
        int8_t lab = 0;
        double rc12 = 0.0, rc14 = 0.0;
        int32_t sel[14];
        if (deg >= 12) {
            double s = 0.0;
            for (int a = 0; a < 12; ++a) {
                s += sqrt(cand[a].r2);
                sel[a] = cand[a].j;
            }
            rc12 = f * (s / 12.0);
            const double rc2 = rc12 * rc12;
            int c421 = 0, c422 = 0;
            for (int a = 0; a < 12; ++a) {
                const uint32_t t = acna_triplet(pos, L, sel, 12, a, rc2);
                c421 += (t == t421);
                c422 += (t == t422);
            }
            if (c421 == 12) lab = 1;
            else if (c421 == 6 && c422 == 6) lab = 2;
        }
        if (lab == 0 && deg >= 14) {
            double s8 = 0.0, s6 = 0.0;
            for (int a = 0; a < 14; ++a) {
                if (a < 8) s8 += sqrt(cand[a].r2);
                else s6 += sqrt(cand[a].r2);
                sel[a] = cand[a].j;
            }
            rc14 = f * ((c * s8 + s6) / 14.0);
            const double rc2 = rc14 * rc14;
            int c444 = 0, c666 = 0;
            for (int a = 0; a < 14; ++a) {
                const uint32_t t = acna_triplet(pos, L, sel, 14, a, rc2);
                c444 += (t == t444);
                c666 += (t == t666);
            }
            if (c666 == 8 && c444 == 6) lab = 3;
        }
        label[i] = lab;
        if (rcut) {
            rcut[2 * i] = rc12;
            rcut[2 * i + 1] = rc14;
        }
        free(cand);
    }
}
