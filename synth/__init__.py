"""Seeded synthetic inputs shared by tests and benchmarks (no method arithmetic)."""
from .lattices import (Lattice, make_lattice, jittered, maxwell_boltzmann, rng_stream, wrap,
                       min_pair_margin, cell_edges)
from . import configs

__all__ = ["Lattice", "make_lattice", "jittered", "maxwell_boltzmann", "rng_stream", "wrap",
           "min_pair_margin", "cell_edges", "configs"]
