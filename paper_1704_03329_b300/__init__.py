"""B300 (sm_103a) implementation of the data-parallel hot path of
arXiv:1704.03329: cell and neighbour lists, the Lennard-Jones pair loop,
Velocity Verlet, bond order analysis, common neighbour analysis and a learned
structure classifier, behind the C ABI of include/ppmd.h.

The CUDA library is loaded on first use of `lib` (no CPU fallback).
"""
import importlib

__all__ = ["lib", "build"]


def __getattr__(name):
    if name == "lib":
        return importlib.import_module("._lib", __name__)
    if name == "build":
        return importlib.import_module(".build", __name__)
    raise AttributeError(name)
