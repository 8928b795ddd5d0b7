"""The five seeded workloads (plus small variants used by tests).

Each builder returns plain NumPy arrays (float64 positions/velocities, box
edges) and a dict of run parameters.  Nothing here evaluates the method.

Workloads (LJ units, sigma = epsilon = m = 1, density 0.8442 unless stated):
  lj_small    1000 atoms, sc 10^3, uniform noise +-0.05, T = 1.0, rc = 2.5
  lj_solid    fcc 63^3 cells = 1,000,188 atoms, Gaussian noise 0.02, T = 0.8,
              rc = 2.5, list cutoff 2.8, list rebuilt every 10 steps
  structure   four 512,000-atom periodic boxes (fcc, bcc, hcp, LJ liquid)
              per noise level sigma in {0.02, 0.05, 0.1} x nearest-neighbour distance
  replicas    256 independent boxes, N log-uniform in [500, 32000],
              density U[0.7, 1.0], T U[0.7, 1.5], jittered sc
  classifier  training and inference sets of structure-style boxes
"""
from __future__ import annotations

import math
import os

import numpy as np

from .lattices import (cell_edges, jittered, make_lattice, maxwell_boltzmann, rng_stream, wrap)

RHO = 0.8442
RC = 2.5
R_BOA = 1.5
# CNA cutoff: midway between the first (a/sqrt2) and second (a) shells of fcc at RHO.
_A_FCC = (4.0 / RHO) ** (1.0 / 3.0)
R_CNA = 0.5 * (_A_FCC / math.sqrt(2.0) + _A_FCC)
DT = 0.005


def lj_small(seed: int = 1, n_side: int = 10, temperature: float = 1.0):
    """Plain method, small, FP64 (1000 atoms on a 10^3 simple-cubic lattice)."""
    lat = make_lattice("sc", n_side, RHO)
    pos, box = jittered(lat, rng_stream(seed, 0), "uniform", 0.05, cutoffs=(RC,),
                        resample_rng=rng_stream(seed, 1))
    vel = maxwell_boltzmann(rng_stream(seed, 2), len(pos), temperature)
    return dict(pos=pos, vel=vel, box=box, rc=RC, r_list=RC, rebuild_every=1, dt=DT,
                steps=100, mass=1.0, name=f"lj_small_sc{n_side}^3")


def lj_solid(seed: int = 2, n_cells: int = 63, temperature: float = 0.8, skin: float = 0.3,
             noise: float = 0.02):
    """Large LJ solid: fcc n_cells^3 (63^3 -> 1,000,188 atoms)."""
    lat = make_lattice("fcc", n_cells, RHO)
    r_list = RC + skin
    pos, box = jittered(lat, rng_stream(seed, 0), "gauss", noise, cutoffs=(RC, r_list),
                        resample_rng=rng_stream(seed, 1))
    vel = maxwell_boltzmann(rng_stream(seed, 2), len(pos), temperature)
    return dict(pos=pos, vel=vel, box=box, rc=RC, r_list=r_list, rebuild_every=10, dt=DT,
                steps=1000, mass=1.0, name=f"lj_solid_fcc{n_cells}^3")


def otf_box(seed: int = 6, n: int = 524288, temperature: float = 1.0):
    """The on-the-fly analysis workload at the size of the paper's weak-scaling
    table for it (524,288 atoms per node, rho 0.8442, rc 3.0, list 3.3,
    rebuild every 18): particles on a periodic cubic lattice (the first n of
    ceil(n^(1/3))^3 simple-cubic sites, box (n/rho)^(1/3)), +-0.05 uniform
    jitter, Maxwell-Boltzmann velocities."""
    side = int(math.ceil(round(n ** (1.0 / 3.0), 9)))
    box_l = (n / RHO) ** (1.0 / 3.0)
    lat = make_lattice("sc", side, 1.0)
    lat.edges = np.full(3, box_l / side)
    lat.box = lat.edges * side
    pos, box = jittered(lat, rng_stream(seed, 0), "uniform", 0.05, cutoffs=(3.0, 3.3, R_BOA), n_active=n,
                        resample_rng=rng_stream(seed, 1))
    vel = maxwell_boltzmann(rng_stream(seed, 2), n, temperature)
    return dict(pos=pos, vel=vel, box=box, rc=3.0, r_list=3.3, rebuild_every=18, dt=DT, mass=1.0)


def nn_distance(kind: str, rho: float = RHO) -> float:
    e = cell_edges(kind, rho)
    if kind == "fcc":
        return e[0] / math.sqrt(2.0)
    if kind == "bcc":
        return e[0] * math.sqrt(3.0) / 2.0
    if kind in ("hcp", "sc"):
        return e[0]
    raise ValueError(kind)


# Cell counts giving 512,000 atoms for each structure box (for the liquid:
# simple-cubic sites, i.e. atoms per edge).
STRUCTURE_CELLS = {"fcc": (80, 80, 20), "bcc": (80, 80, 40), "hcp": (80, 40, 40), "liquid": (80, 80, 80)}

# LJ liquid snapshots (density 0.8442, T = 1.5 after 2000 steps), written by
# the oracle's integrator (oracle/make_liquid.py) and stored with the
# package: periodic cubes of side^3 atoms, tiled here into larger boxes.
_DATA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")
_LIQUID_CACHE = {}


def liquid_snapshot(side: int, variant: int):
    """(positions float64 [side^3, 3], box[3]) of snapshot `variant` of a
    cube of side^3 atoms."""
    key = (side, variant)
    if key not in _LIQUID_CACHE:
        with np.load(os.path.join(_DATA, f"liquid_sc{side}_v{variant}.npz")) as z:
            _LIQUID_CACHE[key] = (z["pos"].astype(np.float64), np.asarray(z["box"], dtype=np.float64))
    pos, box = _LIQUID_CACHE[key]
    return pos.copy(), box.copy()


def _away_from_cutoffs(pos, box, cutoffs, rng, margin=1e-6, step=1e-4, max_rounds=50):
    """Moves, by seeded uniform steps of at most `step` per component, every
    atom in a pair whose minimum-image distance lies within `margin` of a
    cutoff, until none is left (pairs found with a periodic k-d tree)."""
    from scipy.spatial import cKDTree
    pos = wrap(pos, box)
    for _ in range(max_rounds):
        pairs = cKDTree(pos, boxsize=box).query_pairs(max(cutoffs) + margin, output_type="ndarray")
        if len(pairs) == 0:
            return pos
        d = pos[pairs[:, 0]] - pos[pairs[:, 1]]
        d -= box * np.rint(d / box)
        r = np.sqrt((d * d).sum(1))
        bad = np.zeros(len(r), dtype=bool)
        for c in cutoffs:
            bad |= np.abs(r - c) < margin
        if not bad.any():
            return pos
        idx = np.unique(pairs[bad].ravel())
        pos[idx] = wrap(pos[idx] + rng.uniform(-step, step, (len(idx), 3)), box)
    raise RuntimeError("could not move all pairs away from the cutoffs")


def liquid_box(cells, seed: int, cutoffs=()):
    """An LJ liquid box of cells[0] x cells[1] x cells[2] atoms: copies of a
    snapshot cube (side 40 when every count is a multiple of 40, else side
    12), the snapshot chosen by the seed (side 40: (seed // 1000) % 2, so
    the classifier's training set, seed 50, and its inference set, seed 51,
    see different liquids; side 12: seed % 4), moved off the cutoffs."""
    side = 40 if all(c % 40 == 0 for c in cells) else 12
    if any(c % side for c in cells):
        raise ValueError(f"liquid box of {cells} atoms per edge is not a tiling of a {side}^3 snapshot")
    variant = (seed // 1000) % 2 if side == 40 else seed % 4
    base, edge = liquid_snapshot(side, variant)
    if cutoffs:
        base = _away_from_cutoffs(base, edge, cutoffs, rng_stream(seed, 7))
    reps = [c // side for c in cells]
    shifts = np.stack(np.meshgrid(*[np.arange(r) for r in reps], indexing="ij"), -1).reshape(-1, 3) * edge
    pos = (shifts[:, None, :] + base[None, :, :]).reshape(-1, 3)
    return np.ascontiguousarray(pos), edge * np.asarray(reps, dtype=np.float64)


def structure_box(kind: str, sigma_frac: float, seed: int, cells=None):
    """One structure-analysis box.  `kind` in fcc, bcc, hcp, liquid.  The
    crystals carry Gaussian noise of sigma_frac times their nearest-neighbour
    distance; the liquid is an equilibrated LJ liquid (liquid_box; its
    disorder is thermal, sigma_frac does not apply)."""
    cells = cells if cells is not None else STRUCTURE_CELLS[kind]
    if kind == "liquid":
        pos, box = liquid_box(cells, seed, cutoffs=(R_BOA, R_CNA))
        return dict(pos=pos, box=box, kind=kind, sigma=0.0)
    stream0 = {"fcc": 0, "bcc": 2, "hcp": 4}[kind]
    lat = make_lattice(kind, cells, RHO)
    amp = sigma_frac * nn_distance(kind)
    pos, box = jittered(lat, rng_stream(seed, stream0), "gauss", amp, cutoffs=(R_BOA, R_CNA),
                        resample_rng=rng_stream(seed, stream0 + 1))
    return dict(pos=pos, box=box, kind=kind, sigma=amp)


def structure(sigma_frac: float = 0.02, seed: int = 30, cells=None):
    """The four boxes of one noise level, in the order fcc, bcc, hcp, liquid."""
    out = []
    for kind in ("fcc", "bcc", "hcp", "liquid"):
        c = None if cells is None else cells[kind]
        out.append(structure_box(kind, sigma_frac, seed, c))
    return out


def replicas(seed: int = 4, nrep: int = 256, n_min: int = 500, n_max: int = 32000, skin: float = 0.3):
    """Batched replicas: per replica N, density, temperature, box, positions, velocities.

    N = round(exp(U(ln n_min, ln n_max))); sc lattice with ceil(N^(1/3)) sites per
    edge scaled to the box L = (N/rho)^(1/3); the first N sites in index order are
    used; uniform +-0.05 jitter.  The list cutoff is min(rc + skin, L/3) so that
    every box has at least three cells per edge.
    """
    g = rng_stream(seed, 0)
    ns = np.rint(np.exp(g.uniform(math.log(n_min), math.log(n_max), nrep))).astype(np.int64)
    rhos = g.uniform(0.7, 1.0, nrep)
    temps = g.uniform(0.7, 1.5, nrep)
    reps = []
    for r in range(nrep):
        n = int(ns[r])
        side = int(math.ceil(round(n ** (1.0 / 3.0), 9)))
        box_l = (n / rhos[r]) ** (1.0 / 3.0)
        lat = make_lattice("sc", side, 1.0)
        lat.edges = np.full(3, box_l / side)
        lat.box = lat.edges * side
        r_list = min(RC + skin, math.floor(box_l / 3.0 * 1e6) / 1e6)
        pos, box = jittered(lat, rng_stream(seed, 10 + 3 * r), "uniform", 0.05, cutoffs=(RC, r_list),
                            n_active=n, resample_rng=rng_stream(seed, 11 + 3 * r))
        vel = maxwell_boltzmann(rng_stream(seed, 12 + 3 * r), n, float(temps[r]))
        reps.append(dict(pos=pos, vel=vel, box=box, rho=float(rhos[r]), T=float(temps[r]), r_list=r_list))
    return reps


def random_box(n: int, box, seed: int, cutoffs=(), margin: float = 1e-6, min_dist: float = 0.0):
    """n atoms placed one after another uniformly in a box (random sequential
    addition; small n).  A candidate closer than min_dist to a placed atom, or
    at a distance within `margin` of a cutoff, is drawn again."""
    box = np.asarray(box, dtype=np.float64)
    g = rng_stream(seed, 0)
    pos = np.zeros((n, 3))
    for k in range(n):
        for _ in range(100000):
            x = g.uniform(0.0, 1.0, 3) * box
            if k == 0:
                break
            dr = pos[:k] - x
            dr -= box * np.rint(dr / box)
            r = np.sqrt((dr ** 2).sum(-1))
            ok = (r >= min_dist).all()
            for c in cutoffs:
                ok = ok and not (np.abs(r - c) < margin).any()
            if ok:
                break
        else:
            raise RuntimeError("random_box: could not place an atom")
        pos[k] = x
    return wrap(pos, box), box


CLASSIFIER_CELLS = {"fcc": (40, 40, 20), "bcc": (40, 40, 40), "hcp": (40, 20, 40), "liquid": (40, 40, 80)}


def classifier_box(seed: int, k: int, nbox: int = 32, sigma_lo: float = 0.01, sigma_hi: float = 0.12, cells=None):
    """Box k of classifier_boxes(seed, nbox, ...), built on its own (the noise
    draws of boxes 0..k are repeated, so the result is the same)."""
    g = rng_stream(seed, 99)
    kinds = ("fcc", "bcc", "hcp", "liquid")
    per_kind = max(1, nbox // 4)
    for j in range(k + 1):
        u = g.uniform()
    kind = kinds[k % 4]
    stratum = (k // 4) % per_kind
    sig = sigma_lo + (sigma_hi - sigma_lo) * (stratum + u) / per_kind
    c = (cells or CLASSIFIER_CELLS)[kind]
    b = structure_box(kind, float(sig), seed * 1000 + k, c)
    b["sigma_frac"] = float(sig)
    return b


def classifier_boxes(seed: int, nbox: int = 32, sigma_lo: float = 0.01, sigma_hi: float = 0.12, cells=None):
    """Structure boxes for the learned classifier (32 boxes of 128,000 atoms =
    4,096,000 atoms by default).  Box k is fcc, bcc, hcp or liquid-like
    (k mod 4); the noise levels of each structure are stratified over
    [sigma_lo, sigma_hi] x d_nn (one draw in each of nbox/4 equal strata), so
    that every structure is seen across the whole noise range."""
    return [classifier_box(seed, k, nbox, sigma_lo, sigma_hi, cells) for k in range(nbox)]
