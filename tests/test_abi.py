"""The C ABI library loads and exports every entry point declared in include/*.h
(no compute call: runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(ppmd_[a-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_1704_03329_b300 import build
    return build.build()


def test_header_declares_entry_points():
    names = _declared()
    for required in ("ppmd_build_cells", "ppmd_build_neighbours", "ppmd_lj_forces", "ppmd_verlet_step"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_declared_symbols(libpath):
    from paper_1704_03329_b300 import lib as L
    assert set(L.exported_symbols()) == _declared()


def test_oracle_and_library_share_no_sources():
    lib_src = glob.glob(os.path.join(ROOT, "paper_1704_03329_b300", "csrc", "*"))
    ora = open(os.path.join(ROOT, "oracle", "ppmd_oracle.c")).read()
    assert "ppmd.h" not in ora and "common.cuh" not in ora
    for f in lib_src:
        assert "oracle" not in open(f).read().lower() or f.endswith(".md")
