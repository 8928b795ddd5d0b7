"""The allocation-free force entry point (ppmd_lj_forces_noalloc).

It serves callers that may not allocate device memory themselves or through
a library (memory owned by a host framework's pool, or loops that may not
pay the synchronisation of cudaMalloc/cudaFree).  These tests call it
through the C ABI, with outputs allocated by the test, and compare it with
ppmd_lj_forces on two calls in a row (the second on a different, smaller
configuration, so that anything left in the shared static array from the
first call would show).  The file is named so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

import oracle
from synth import configs

pytestmark = pytest.mark.gpu


def cu(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _reference(L, ctx, pos, box, prec):
    nc, cell_of, start, atoms = L.ppmd_build_cells(ctx, pos, box, 2.8)
    nbr, cnt = L.ppmd_build_neighbours(ctx, pos, box, 2.8, start, atoms, nc, 128)
    F, e, tot = L.ppmd_lj_forces(ctx, pos, box, nbr, cnt, prec=prec)
    return nbr, cnt, F, e, tot


@pytest.mark.parametrize("prec_name", ["FP32", "FP64"])
def test_noalloc_matches_lj_forces_on_two_calls(prec_name):
    from paper_1704_03329_b300 import lib as L
    prec = getattr(L, prec_name)
    ctx = L.Context(0)
    tol = 1e-5 if prec_name == "FP32" else 1e-12
    for n_cells in (10, 7):  # 4000 atoms, then 1372 atoms
        c = configs.lj_solid(n_cells=n_cells, seed=40 + n_cells)
        pos = cu(c["pos"])
        box = c["box"]
        nbr, cnt, F_ref, e_ref, tot_ref = _reference(L, ctx, pos, box, prec)
        n = pos.shape[0]
        F = torch.full((n, 3), np.nan, dtype=torch.float64, device="cuda")
        e = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
        tot = torch.full((2,), np.nan, dtype=torch.float64, device="cuda")
        rc = L.ppmd_lj_forces_noalloc(pos, box, nbr, cnt, F, e, tot, prec=prec)
        assert rc == L.OK
        torch.cuda.synchronize()
        F, e, tot = F.cpu().numpy(), e.cpu().numpy(), tot.cpu().numpy()
        Fr, er, tr = F_ref.cpu().numpy(), e_ref.cpu().numpy(), tot_ref.cpu().numpy()
        rms = np.sqrt((Fr ** 2).sum(1).mean())
        assert np.sqrt(((F - Fr) ** 2).sum(1)).max() <= tol * rms
        assert np.abs(e - er).max() <= (1e-6 if prec_name == "FP32" else 1e-12) * np.abs(er).mean()
        assert abs(tot[0] - tr[0]) <= tol * abs(tr[0]) and abs(tot[1] - tr[1]) <= tol * max(abs(tr[1]), 1.0)
        # and against the oracle directly
        offs, nb_o = oracle.neighbours_cells(c["pos"], box, 2.8)
        Fo = oracle.lj(c["pos"], box, offs, nb_o)[0]
        assert np.sqrt(((F - Fo) ** 2).sum(1)).max() <= tol * np.sqrt((Fo ** 2).sum(1).mean())
    ctx.close()


def test_noalloc_rejects_too_many_atoms():
    from paper_1704_03329_b300 import lib as L
    pos = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    nbr = torch.zeros((4, 8), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(4, dtype=torch.int32, device="cuda")
    F = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    rc = L.ppmd_lj_forces_noalloc(pos, [20.0, 20.0, 20.0], nbr, cnt, F, None, None, n=L.NOALLOC_MAX_ATOMS + 1)
    assert rc == L.ERR_CAPACITY
