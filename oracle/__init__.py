"""FP64 CPU oracle for the particle method of arXiv:1704.03329.

TEST INFRASTRUCTURE ONLY: the slow, plain reference that the CUDA library is
checked against.  Only the tests, the smoke check and the benchmark's CPU
baseline may import this package.  It shares no code with the CUDA library
(`paper_1704_03329_b300`) and never imports it.

The arithmetic lives in `ppmd_oracle.c` (plain C, built with gcc -O2 and
-ffp-contract=off) and, for the learned classifier, in `mlp.py` (NumPy FP64).
This module only marshals NumPy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ppmd_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None


def compile_source(src: str, out: str) -> None:
    """gcc -O2 with FP contraction off: the one way every build of the oracle's C source is made."""
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
                           "-fno-fast-math", "-fopenmp", "-o", out, src, "-lm"])


def build(force: bool = False) -> str:
    """Compile the oracle if it is missing or stale."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        compile_source(_SRC, tmp)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    # PPMD_ORACLE_LIB names another build of ppmd_oracle.c: the tests that
    # plant a mistake in a copy of the oracle's source (test_oracle_mutants)
    # run the pins against that copy's build through it
    lib = C.CDLL(os.environ.get("PPMD_ORACLE_LIB") or build())
    i64, i32, f64 = C.c_int64, C.c_int32, C.c_double
    P = C.c_void_p
    sig = {
        "ora_wrap": (None, [i64, P, P]),
        "ora_set_threads": (None, [C.c_int]),
        "ora_cell_grid": (None, [P, f64, P]),
        "ora_cells": (None, [i64, P, P, P, P, P, P]),
        "ora_neigh_brute": (i64, [i64, P, P, f64, P, P]),
        "ora_neigh_cells": (i64, [i64, P, P, f64, P, P, P, P, P, P]),
        "ora_lj": (None, [i64, P, P, f64, f64, f64, f64, P, P, P, P, P, P]),
        "ora_vv": (None, [C.c_int, i64, P, P, P, P, f64, f64]),
        "ora_kinetic": (f64, [i64, P, f64]),
        "ora_md_run": (f64, [i64, P, P, P, P, f64, f64, f64, f64, f64, i32, f64, f64, i32, P]),
        "ora_boa_direct": (None, [i64, P, P, f64, P, P, C.c_int, P, P]),
        "ora_boa_addition": (None, [i64, P, P, f64, P, P, C.c_int, P]),
        "ora_cna": (i32, [i64, P, P, f64, P, P, i32, P, P, P]),
        "ora_cna_label": (None, [i64, P, P, i32, P]),
        "ora_features": (None, [i64, P, P, f64, f64, P, P, P]),
        "ora_acna": (None, [i64, P, P, P, P, P, P]),
        "ora_philox4x32": (None, [P, P, P]),
        "ora_andersen_threshold": (C.c_uint64, [f64, f64]),
        "ora_md_run_otf": (i64, [i64, P, P, P, P, f64, f64, f64, f64, f64, i32, f64, f64, i32, P, C.c_uint64, f64,
                                 C.c_uint64, i32, f64, P, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _p(a):
    return C.c_void_p(a.ctypes.data) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(k: int) -> None:
    """Threads of the integrator's per-atom loops (neighbour search, pair
    loop, particle loops; 1 by default).  Results do not depend on it."""
    _load().ora_set_threads(int(k))


def wrap(pos, box):
    pos = _f64(pos).copy()
    _load().ora_wrap(len(pos), _p(pos), _p(_f64(box)))
    return pos


def cell_grid(box, r):
    nc = np.zeros(3, np.int32)
    _load().ora_cell_grid(_p(_f64(box)), float(r), _p(nc))
    return nc


def cells(pos, box, r):
    """Cell list with cells of edge >= r.  Returns (ncell[3], cell_of, cell_start, cell_atoms)."""
    pos, box = _f64(pos), _f64(box)
    nc = cell_grid(box, r)
    n = len(pos)
    cell_of = np.zeros(n, np.int32)
    cell_start = np.zeros(int(np.prod(nc)) + 1, np.int32)
    cell_atoms = np.zeros(n, np.int32)
    _load().ora_cells(n, _p(pos), _p(box), _p(nc), _p(cell_of), _p(cell_start), _p(cell_atoms))
    return nc, cell_of, cell_start, cell_atoms


def neighbours_brute(pos, box, r):
    """O(N^2) full neighbour list as CSR (offs[n+1] int64, nbr int32), rows sorted."""
    pos, box = _f64(pos), _f64(box)
    n = len(pos)
    lib = _load()
    offs = np.zeros(n + 1, np.int64)
    tot = lib.ora_neigh_brute(n, _p(pos), _p(box), float(r), _p(offs), None)
    nbr = np.zeros(max(tot, 1), np.int32)
    lib.ora_neigh_brute(n, _p(pos), _p(box), float(r), _p(offs), _p(nbr))
    return offs, nbr[:tot]


def neighbours_cells(pos, box, r, cell_r=None):
    """Cell-list neighbour list (cells of edge >= cell_r, default r) as sorted CSR."""
    pos, box = _f64(pos), _f64(box)
    n = len(pos)
    nc, cell_of, cell_start, cell_atoms = cells(pos, box, r if cell_r is None else cell_r)
    if (nc < 3).any():
        raise ValueError("cell list needs at least three cells per edge")
    lib = _load()
    offs = np.zeros(n + 1, np.int64)
    args = (n, _p(pos), _p(box), float(r), _p(nc), _p(cell_of), _p(cell_start), _p(cell_atoms), _p(offs))
    tot = lib.ora_neigh_cells(*args, None)
    nbr = np.zeros(max(tot, 1), np.int32)
    lib.ora_neigh_cells(*args, _p(nbr))
    return offs, nbr[:tot]


def lj(pos, box, offs, nbr, rc=2.5, eps=1.0, sigma=1.0, shift=0.0):
    """Forces, per-atom energies, total energy U and virial W (Eqs. (9) and (12))."""
    pos, box = _f64(pos), _f64(box)
    n = len(pos)
    F = np.zeros((n, 3))
    e = np.zeros(n)
    U = C.c_double()
    W = C.c_double()
    offs = np.ascontiguousarray(offs, np.int64)
    nbr = np.ascontiguousarray(nbr, np.int32)
    _load().ora_lj(n, _p(pos), _p(box), eps, sigma, rc, shift, _p(offs), _p(nbr), _p(F), _p(e),
                   C.byref(U), C.byref(W))
    return F, e, U.value, W.value


def vv(phase, pos, vel, F, box, mass=1.0, dt=0.005):
    """One Velocity Verlet particle loop (phase 1: kick+drift+wrap, phase 2: kick); returns copies."""
    pos, vel = _f64(pos).copy(), _f64(vel).copy()
    _load().ora_vv(int(phase), len(pos), _p(pos), _p(vel), _p(_f64(F)), _p(_f64(box)), mass, dt)
    return pos, vel


def kinetic(vel, mass=1.0):
    vel = _f64(vel)
    return _load().ora_kinetic(len(vel), _p(vel), mass)


def md_run(pos, vel, box, nsteps, rc=2.5, r_list=2.5, rebuild_every=1, dt=0.005, mass=1.0, eps=1.0,
           sigma=1.0, shift=0.0):
    """Algorithm 6 with list reuse.  Returns (pos, vel, F, energies[nsteps, 2] = (KE, PE), max_disp)."""
    pos, vel = _f64(pos).copy(), _f64(vel).copy()
    n = len(pos)
    F = np.zeros((n, 3))
    en = np.zeros((max(nsteps, 1), 2))
    md = _load().ora_md_run(n, _p(pos), _p(vel), _p(F), _p(_f64(box)), eps, sigma, rc, shift, r_list,
                            int(rebuild_every), mass, dt, int(nsteps), _p(en))
    return pos, vel, F, en[:nsteps], md


def philox4x32(ctr, key):
    """Philox4x32-10 of a 4-word counter and a 2-word key (uint32 arrays)."""
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    _load().ora_philox4x32(_p(c), _p(k), _p(out))
    return out


def andersen_threshold(nu, dt):
    return int(_load().ora_andersen_threshold(float(nu), float(dt)))


def md_run_otf(pos, vel, box, nsteps, rc=2.5, r_list=2.5, rebuild_every=1, dt=0.005, mass=1.0, eps=1.0,
               sigma=1.0, shift=0.0, thermostat=None, boa=None):
    """md_run with the on-the-fly analysis run's additions: thermostat =
    (T, nu, seed) for Andersen collisions, boa = (every, r_boa) for Q4, Q5,
    Q6.  Returns (pos, vel, F, energies, qrows [nsteps, 3] of means (0 on
    other steps), qlast [3, n] of the last analysis step, collisions)."""
    pos, vel = _f64(pos).copy(), _f64(vel).copy()
    n = len(pos)
    F = np.zeros((n, 3))
    en = np.zeros((max(nsteps, 1), 2))
    qrows = np.zeros((max(nsteps, 1), 3))
    qlast = np.zeros((3, n))
    md = np.zeros(1)
    T, nu, seed = thermostat if thermostat else (0.0, 0.0, 0)
    thr = andersen_threshold(nu, dt) if thermostat else 0
    every, r_boa = boa if boa else (0, 0.0)
    ncoll = _load().ora_md_run_otf(n, _p(pos), _p(vel), _p(F), _p(_f64(box)), eps, sigma, rc, shift, r_list,
                                   int(rebuild_every), mass, dt, int(nsteps), _p(en), thr, float(T), int(seed),
                                   int(every), float(r_boa), _p(qrows), _p(qlast), _p(md))
    return pos, vel, F, en[:nsteps], qrows[:nsteps], qlast, int(ncoll)


def boa(pos, box, offs, nbr, r_cut=1.5, l=6, method="direct"):
    """Q_l per atom (Eqs. (4)-(5)); method 'direct' (Y_lm sums) or 'addition' (Legendre)."""
    pos, box = _f64(pos), _f64(box)
    n = len(pos)
    Q = np.zeros(n)
    nnb = np.zeros(n, np.int32)
    offs = np.ascontiguousarray(offs, np.int64)
    nbr = np.ascontiguousarray(nbr, np.int32)
    lib = _load()
    if method == "direct":
        lib.ora_boa_direct(n, _p(pos), _p(box), float(r_cut), _p(offs), _p(nbr), int(l), _p(Q), _p(nnb))
        return Q, nnb
    lib.ora_boa_addition(n, _p(pos), _p(box), float(r_cut), _p(offs), _p(nbr), int(l), _p(Q))
    return Q


def cna(pos, box, offs, nbr, r_cut, max_bond=64):
    """CNA triplets (Algorithms 3-5, 7).  Returns (nbond[n], trip[n, max_bond] uint32,
    partner[n, max_bond] int32, numax); triplet = ncn<<16 | nb<<8 | nlcb."""
    pos, box = _f64(pos), _f64(box)
    n = len(pos)
    nbond = np.zeros(n, np.int32)
    trip = np.zeros((n, max_bond), np.uint32)
    partner = np.full((n, max_bond), -1, np.int32)
    offs = np.ascontiguousarray(offs, np.int64)
    nbr = np.ascontiguousarray(nbr, np.int32)
    numax = _load().ora_cna(n, _p(pos), _p(box), float(r_cut), _p(offs), _p(nbr), int(max_bond), _p(nbond),
                            _p(trip), _p(partner))
    return nbond, trip, partner, numax


def cna_label(nbond, trip):
    """Structure codes 0 other, 1 fcc, 2 hcp, 3 bcc from the triplets of each atom."""
    nbond = np.ascontiguousarray(nbond, np.int32)
    trip = np.ascontiguousarray(trip, np.uint32)
    n, mb = trip.shape
    lab = np.zeros(n, np.int8)
    _load().ora_cna_label(n, _p(nbond), _p(trip), int(mb), _p(lab))
    return lab


def acna(pos, box, offs, nbr):
    """Adaptive CNA over a neighbour list that holds at least the 14 nearest
    neighbours of every atom (see ppmd_oracle.c).  Returns (label int8 [n],
    rcut [n, 2]: the fcc/hcp and bcc local cutoffs, 0 when not computed)."""
    pos, box = _f64(pos), _f64(box)
    n = len(pos)
    lab = np.zeros(n, np.int8)
    rc = np.zeros((n, 2))
    offs = np.ascontiguousarray(offs, np.int64)
    nbr = np.ascontiguousarray(nbr, np.int32)
    _load().ora_acna(n, _p(pos), _p(box), _p(offs), _p(nbr), _p(lab), _p(rc))
    return lab, rc


def features(pos, box, offs, nbr, r_feat=1.5, r_ref=1.433625):
    """30 local-environment features per atom (see ppmd_oracle.c)."""
    pos, box = _f64(pos), _f64(box)
    n = len(pos)
    f = np.zeros((n, 30))
    offs = np.ascontiguousarray(offs, np.int64)
    nbr = np.ascontiguousarray(nbr, np.int32)
    _load().ora_features(n, _p(pos), _p(box), float(r_feat), float(r_ref), _p(offs), _p(nbr), _p(f))
    return f


# (Q4, Q6) of perfect fcc, hcp and bcc lattices as printed in the table of
# Q4, Q5, Q6 of Sec. 4.1, with the structure codes of cna_label.
BOA_TABLE = ((1, 0.191, 0.575), (2, 0.097, 0.485), (3, 0.036, 0.511))


def boa_tolerance_labels(q4, q6, tol):
    """Sec. 4.1: the local structure is that of the lattice whose Q_l agree
    with the atom's within a tolerance.  Reading: the lattice of BOA_TABLE
    nearest to (Q4, Q6) in the plane (the first in table order on ties),
    when its distance is below tol; otherwise 0 (other).  Returns (labels
    int8, that nearest distance)."""
    q4 = np.asarray(q4, dtype=np.float64)
    q6 = np.asarray(q6, dtype=np.float64)
    best = np.full(q4.shape, np.inf)
    lab = np.zeros(q4.shape, np.int8)
    for code, r4, r6 in BOA_TABLE:
        d = np.sqrt((q4 - r4) ** 2 + (q6 - r6) ** 2)
        closer = d < best
        best = np.where(closer, d, best)
        lab = np.where(closer, np.int8(code), lab)
    return np.where(best < tol, lab, np.int8(0)).astype(np.int8), best


def triplet(ncn, nb, nlcb):
    return (ncn << 16) | (nb << 8) | nlcb


LABELS = {0: "other", 1: "fcc", 2: "hcp", 3: "bcc"}
