"""Writes the Lennard-Jones liquid snapshots used as the "liquid" structure
boxes (test infrastructure: run once, the files are committed).

An equilibrated LJ liquid at density 0.8442 and T = 1.5: a simple-cubic
lattice of side^3 sites with +-0.05 uniform jitter and Maxwell-Boltzmann
velocities at T = 1.5 (synth), then 2000 steps of the oracle's Velocity
Verlet (Algorithm 6; rc 2.5, list 2.8 rebuilt every 10 steps, dt 0.005)
with the velocities rescaled to T = 1.5 every 10 steps (centre-of-mass
velocity removed, sum m v^2 / (3N - 3) = T).  Every number comes from the
oracle and the seeded generators; nothing from the CUDA library.

Files: synth/data/liquid_sc{side}_v{variant}.npz with the final positions
(float32, wrapped into the box), the box edges and the run's parameters.

    python -m oracle.make_liquid            # all snapshots
"""
from __future__ import annotations

import os
import sys

import numpy as np

import oracle
from synth.lattices import jittered, make_lattice, maxwell_boltzmann, rng_stream

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(os.path.dirname(HERE), "synth", "data")
RHO, T, STEPS, EVERY = 0.8442, 1.5, 2000, 10
# (side, variant, seed): side 40 for the 512,000- and 128,000-atom boxes
# (variant 0: the classifier's training set, 1: every other box), side 12
# for test-sized boxes (four independent variants)
SNAPSHOTS = [(40, 0, 7001), (40, 1, 7002), (12, 0, 7101), (12, 1, 7102), (12, 2, 7103), (12, 3, 7104)]


def rescale(v, temperature, mass=1.0):
    v = v - v.mean(axis=0)
    t_now = mass * float((v * v).sum()) / (3 * len(v) - 3)
    return v * np.sqrt(temperature / t_now)


def make(side: int, seed: int):
    lat = make_lattice("sc", side, RHO)
    pos, box = jittered(lat, rng_stream(seed, 0), "uniform", 0.05)
    vel = maxwell_boltzmann(rng_stream(seed, 1), len(pos), T)
    for _ in range(STEPS // EVERY):
        pos, vel, _, _, _ = oracle.md_run(pos, vel, box, EVERY, rc=2.5, r_list=2.8, rebuild_every=EVERY)
        vel = rescale(vel, T)
    return oracle.wrap(pos, box), box


def main(threads: int = os.cpu_count() or 1):
    oracle.set_threads(threads)
    os.makedirs(OUT, exist_ok=True)
    for side, variant, seed in SNAPSHOTS:
        path = os.path.join(OUT, f"liquid_sc{side}_v{variant}.npz")
        pos, box = make(side, seed)
        np.savez_compressed(path, pos=pos.astype(np.float32), box=box, rho=RHO, temperature=T, steps=STEPS,
                            rescale_every=EVERY, seed=seed, side=side)
        print(path, len(pos), flush=True)
    oracle.set_threads(1)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else os.cpu_count() or 1)
