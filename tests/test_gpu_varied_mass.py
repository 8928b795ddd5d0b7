"""GPU parity at a particle mass other than 1 (every other parity test runs in
LJ units, m = 1, where a dropped mass factor would not show): the Verlet
kicks (dt / 2m), the kinetic energy (m |v|^2 / 2) and the thermostat's
draws (variance T / m), against the FP64 oracle at m = 2 with the
tolerances of the m = 1 tests."""
import numpy as np
import pytest
import torch

import oracle
from synth import configs

pytestmark = pytest.mark.gpu

MASS = 2.0


@pytest.fixture(scope="module")
def L():
    from paper_1704_03329_b300 import lib
    return lib


@pytest.fixture(scope="module")
def ctx(L):
    return L.Context(0)


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=torch.float64)


@pytest.mark.parametrize("phase", [1, 2])
def test_verlet_step_bit_exact_at_mass_2(L, ctx, phase):
    c = configs.lj_small()
    F = np.random.default_rng(4).normal(0, 3, c["pos"].shape)
    po, vo = oracle.vv(phase, c["pos"], c["vel"], F, c["box"], MASS, 0.005)
    p, v = cu(c["pos"]), cu(c["vel"])
    L.ppmd_verlet_step(ctx, phase, p, v, cu(F), c["box"], MASS, 0.005)
    assert np.array_equal(p.cpu().numpy(), po)
    assert np.array_equal(v.cpu().numpy(), vo)
    ke = L.ppmd_kinetic_energy(ctx, v, MASS)
    assert abs(float(ke) - oracle.kinetic(vo, MASS)) <= 1e-12 * oracle.kinetic(vo, MASS)


def test_md_fp64_small_at_mass_2(L, ctx):
    """The 1000-atom FP64 run of the m = 1 test, 50 steps, list at r_c
    rebuilt every step, energies every step."""
    c = configs.lj_small()
    n = len(c["pos"])
    po, vo, Fo, eno, _ = oracle.md_run(c["pos"], c["vel"], c["box"], 50, r_list=2.5, rebuild_every=1, mass=MASS)
    md = L.MD(ctx, [0, n], [c["box"]], r_list=2.5, rebuild_every=1, max_nbr=128, prec=L.FP64, energy_every=1,
              mass=MASS)
    md.set_state(cu(c["pos"]), cu(c["vel"]))
    en = torch.zeros((50, 2), dtype=torch.float64, device="cuda")
    md.run(50, en)
    p = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    v = torch.empty_like(p)
    md.get_state(p, v)
    md.close()
    d = p.cpu().numpy() - po
    d -= c["box"] * np.rint(d / c["box"])
    assert np.abs(d).max() <= 1e-10
    assert np.abs(v.cpu().numpy() - vo).max() <= 1e-9
    eno_ = np.asarray(eno)
    assert np.abs(en.cpu().numpy() - eno_).max() <= 1e-10 * np.abs(eno_).max()


def test_thermostat_draws_at_mass_2(L, ctx):
    """Every atom collides on every step (nu dt >= 1): the final velocities
    are the last step's draws, with spread sqrt(T / m), as the oracle's."""
    c = configs.lj_solid(n_cells=6)
    n = len(c["pos"])
    T, seed = 0.7, 12345678901
    _, vo, _, _, _, _, ncoll = oracle.md_run_otf(c["pos"], c["vel"], c["box"], 3, r_list=2.8, rebuild_every=10,
                                                 mass=MASS, thermostat=(T, 1000.0, seed))
    assert ncoll == 3 * n
    md = L.MD(ctx, [0, n], [c["box"]], r_list=2.8, rebuild_every=10, max_nbr=128, prec=L.FP32, mass=MASS)
    md.set_thermostat(T, 1000.0, seed)
    md.set_state(cu(c["pos"]), cu(c["vel"]))
    md.run_analysed(3, None, None, use_graph=False)
    v = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    md.get_state(None, v)
    md.close()
    assert np.abs(v.cpu().numpy() - vo).max() <= 1e-12
