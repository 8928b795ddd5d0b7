"""Seeded synthetic particle configurations (input generation only).

This module is shared by the CUDA path's tests/benchmarks and by the CPU
oracle's tests.  It holds no arithmetic of the method itself (no cell lists,
neighbour lists, forces, integrators or structure analysis): it only places
atoms on lattices, adds seeded noise, draws Maxwell-Boltzmann velocities and
re-jitters atoms whose pair distance would sit within a small margin of a
cutoff, so that every later cutoff decision is well conditioned.

Every random draw comes from a NumPy PCG64 stream keyed by (seed, stream id).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Lattice bases in fractional coordinates of the conventional (orthorhombic)
# cell.  hcp uses the 4-atom orthorhombic cell with edges (a, sqrt(3) a,
# sqrt(8/3) a), so that every lattice here is an orthorhombic tiling.
_BASIS = {
    "sc": np.array([[0.5, 0.5, 0.5]]),
    "fcc": np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]]),
    "bcc": np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]]),
    "hcp": np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 5.0 / 6.0, 0.5], [0.0, 1.0 / 3.0, 0.5]]),
}


def rng_stream(seed: int, stream: int) -> np.random.Generator:
    """Independent PCG64 stream number `stream` of experiment seed `seed`."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed, spawn_key=(stream,))))


def cell_edges(kind: str, rho: float) -> np.ndarray:
    """Edges of the conventional cell of lattice `kind` at number density rho."""
    if kind == "sc":
        a = rho ** (-1.0 / 3.0)
        return np.array([a, a, a])
    if kind == "fcc":
        a = (4.0 / rho) ** (1.0 / 3.0)
        return np.array([a, a, a])
    if kind == "bcc":
        a = (2.0 / rho) ** (1.0 / 3.0)
        return np.array([a, a, a])
    if kind == "hcp":
        a = (math.sqrt(2.0) / rho) ** (1.0 / 3.0)  # nearest-neighbour distance
        return np.array([a, math.sqrt(3.0) * a, math.sqrt(8.0 / 3.0) * a])
    raise ValueError(kind)


@dataclass
class Lattice:
    """A perfect orthorhombic lattice; site index = ((c0*n1 + c1)*n2 + c2)*B + k."""

    kind: str
    ncell: tuple
    edges: np.ndarray
    basis: np.ndarray
    box: np.ndarray = field(init=False)

    def __post_init__(self):
        self.box = self.edges * np.asarray(self.ncell, dtype=np.float64)

    @property
    def nsite(self) -> int:
        return int(np.prod(self.ncell)) * len(self.basis)

    def sites(self) -> np.ndarray:
        n0, n1, n2 = self.ncell
        g = np.stack(np.meshgrid(np.arange(n0), np.arange(n1), np.arange(n2), indexing="ij"), -1)
        g = g.reshape(-1, 1, 3).astype(np.float64)
        return ((g + self.basis[None]) * self.edges).reshape(-1, 3)


def make_lattice(kind: str, ncell, rho: float) -> Lattice:
    if np.isscalar(ncell):
        ncell = (int(ncell),) * 3
    return Lattice(kind, tuple(int(c) for c in ncell), cell_edges(kind, rho), _BASIS[kind].copy())


def wrap(pos: np.ndarray, box: np.ndarray) -> np.ndarray:
    """Map coordinates into [0, L) per axis (x - L floor(x/L); an exact L maps to 0)."""
    out = pos - box * np.floor(pos / box)
    out[out >= box] = 0.0
    return out


def _near_cutoff_atoms(lat: Lattice, pos: np.ndarray, disp_max: float, cutoffs, margin: float,
                       n_active=None) -> np.ndarray:
    """Atoms in some pair whose minimum-image distance lies within `margin` of a cutoff.

    Pairs are enumerated through lattice offsets: a pair whose true distance is
    near a cutoff c has an ideal lattice separation within c +- (2*disp_max +
    margin), so only those (cell offset, basis pair) combinations are visited.
    """
    n = np.asarray(lat.ncell)
    nb = len(lat.basis)
    box = lat.box
    ncell_tot = int(np.prod(n))
    cidx = np.stack(np.meshgrid(np.arange(n[0]), np.arange(n[1]), np.arange(n[2]), indexing="ij"), -1).reshape(-1, 3)
    slack = 2.0 * disp_max + margin
    rmax = max(cutoffs) + slack
    dmax = np.ceil(rmax / lat.edges).astype(int) + 1
    flagged = np.zeros(len(pos), dtype=bool)
    nsite = ncell_tot * nb
    for d0 in range(-dmax[0], dmax[0] + 1):
        for d1 in range(-dmax[1], dmax[1] + 1):
            for d2 in range(-dmax[2], dmax[2] + 1):
                d = np.array([d0, d1, d2], dtype=np.float64)
                for k in range(nb):
                    for kp in range(nb):
                        v = (d + lat.basis[kp] - lat.basis[k]) * lat.edges
                        r0 = math.sqrt(float(v @ v))
                        if not any(abs(r0 - c) <= slack for c in cutoffs):
                            continue
                        cj = (cidx + np.array([d0, d1, d2])) % n
                        i = np.arange(ncell_tot) * nb + k
                        j = ((cj[:, 0] * n[1] + cj[:, 1]) * n[2] + cj[:, 2]) * nb + kp
                        if n_active is not None and n_active < nsite:
                            keep = (i < n_active) & (j < n_active)
                            i, j = i[keep], j[keep]
                        keep = i != j
                        i, j = i[keep], j[keep]
                        dr = pos[i] - pos[j]
                        dr -= box * np.rint(dr / box)
                        r = np.sqrt(np.einsum("ij,ij->i", dr, dr))
                        bad = np.zeros(len(r), dtype=bool)
                        for c in cutoffs:
                            bad |= np.abs(r - c) < margin
                        if bad.any():
                            flagged[i[bad]] = True
                            flagged[j[bad]] = True
    return flagged


def jittered(lat: Lattice, rng: np.random.Generator, noise: str, amp: float, cutoffs=(),
             margin: float = 1e-6, n_active=None, resample_rng=None, max_rounds: int = 50):
    """Lattice sites plus seeded noise, wrapped into the box.

    noise = "uniform": each component uniform in [-amp, amp];
    noise = "gauss":   each component normal with standard deviation amp.
    Atoms found in a pair within `margin` of any cutoff in `cutoffs` get fresh
    noise (from `resample_rng`, in increasing atom order) until none is left.
    Returns (positions[n_active or nsite, 3], box[3]).
    """
    sites = lat.sites()
    nsite = len(sites)

    def draw(g, k):
        if noise == "uniform":
            return g.uniform(-amp, amp, size=(k, 3))
        if noise == "gauss":
            return g.normal(0.0, amp, size=(k, 3))
        raise ValueError(noise)

    disp = draw(rng, nsite)
    if n_active is not None and n_active < nsite:
        disp[n_active:] = 0.0
    rs = resample_rng if resample_rng is not None else rng
    for _ in range(max_rounds):
        pos = wrap(sites + disp, lat.box)
        if not cutoffs:
            break
        dm = float(np.sqrt((disp ** 2).sum(1)).max())
        bad = _near_cutoff_atoms(lat, pos, dm, cutoffs, margin, n_active)
        if not bad.any():
            break
        idx = np.nonzero(bad)[0]
        disp[idx] = draw(rs, len(idx))
    else:
        raise RuntimeError("could not move all pairs away from the cutoffs")
    if n_active is not None:
        pos = pos[:n_active]
    return np.ascontiguousarray(pos), lat.box.copy()


def maxwell_boltzmann(rng: np.random.Generator, n: int, temperature: float, mass: float = 1.0) -> np.ndarray:
    """Velocities v ~ N(0, T/m) per component, zero total momentum, rescaled so that
    sum(m v^2) / (3N - 3) equals T exactly."""
    v = rng.normal(0.0, math.sqrt(temperature / mass), size=(n, 3))
    v -= v.mean(axis=0)
    t_now = mass * float((v * v).sum()) / (3 * n - 3)
    if t_now > 0:
        v *= math.sqrt(temperature / t_now)
    return np.ascontiguousarray(v)


def min_pair_margin(pos: np.ndarray, box: np.ndarray, cutoffs) -> float:
    """Smallest |r_ij - c| over all pairs and cutoffs (brute force; small inputs only)."""
    dr = pos[:, None, :] - pos[None, :, :]
    dr -= box * np.rint(dr / box)
    r = np.sqrt((dr ** 2).sum(-1))
    iu = np.triu_indices(len(pos), 1)
    r = r[iu]
    return float(min(np.abs(r - c).min() for c in cutoffs)) if len(r) else float("inf")
