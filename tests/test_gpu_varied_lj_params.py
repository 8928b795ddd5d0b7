"""GPU parity of the pair loop at epsilon and sigma other than 1 (every other
parity test runs in LJ units, eps = sigma = 1, where a constant folded the
wrong way would not show), with the paper's shift 1/4: the granular call in
both precisions and the integrator's set-up forces, against the FP64 oracle
at the tolerances of the unit-parameter tests (FP32: forces only, since
some pairs of this box lie below sigma)."""
import numpy as np
import pytest
import torch

import oracle
from synth import configs

pytestmark = pytest.mark.gpu

EPS, SIGMA, SHIFT = 1.7, 1.1, 0.25


@pytest.fixture(scope="module")
def L():
    from paper_1704_03329_b300 import lib
    return lib


@pytest.fixture(scope="module")
def ctx(L):
    return L.Context(0)


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=torch.float64)


def force_err(F, Fo):
    return np.sqrt(((F - Fo) ** 2).sum(1)).max() / np.sqrt((Fo ** 2).sum(1).mean())


@pytest.fixture(scope="module")
def case():
    c = configs.lj_solid(n_cells=7)
    offs, nb = oracle.neighbours_cells(c["pos"], c["box"], 2.8)
    return c, oracle.lj(c["pos"], c["box"], offs, nb, rc=2.5, eps=EPS, sigma=SIGMA, shift=SHIFT)


@pytest.mark.parametrize("prec", ["FP64", "FP32"])
def test_lj_forces_at_other_eps_and_sigma(L, ctx, case, prec):
    c, (Fo, eo, Uo, Wo) = case
    p = cu(c["pos"])
    nc, _, start, atoms = L.ppmd_build_cells(ctx, p, c["box"], 2.8)
    nbr, cnt = L.ppmd_build_neighbours(ctx, p, c["box"], 2.8, start, atoms, nc, 128)
    F, e, tot = L.ppmd_lj_forces(ctx, p, c["box"], nbr, cnt, rc=2.5, eps=EPS, sigma=SIGMA, shift=SHIFT,
                                 prec=getattr(L, prec))
    F, e, tot = F.cpu().numpy(), e.cpu().numpy(), tot.cpu().numpy()
    if prec == "FP64":
        assert force_err(F, Fo) <= 1e-12
        assert np.abs(e - eo).max() <= 1e-12 * np.abs(eo).mean()
        assert abs(tot[0] - Uo) <= 1e-12 * abs(Uo) and abs(tot[1] - Wo) <= 1e-12 * abs(Wo)
    else:
        assert force_err(F, Fo) <= 1e-5


def test_integrator_forces_at_other_eps_and_sigma(L, ctx, case):
    c, (Fo, _, _, _) = case
    n = len(c["pos"])
    md = L.MD(ctx, [0, n], [c["box"]], r_list=2.8, rc=2.5, eps=EPS, sigma=SIGMA, shift=SHIFT, rebuild_every=10,
              max_nbr=128, prec=L.FP32)
    md.set_state(cu(c["pos"]), cu(c["vel"]))
    F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    md.get_state(None, None, F)
    md.close()
    assert force_err(F.cpu().numpy(), Fo) <= 1e-5
