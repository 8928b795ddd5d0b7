"""GPU parity of the cell list, neighbour list, Lennard-Jones pair loop,
Velocity Verlet and the time-stepping driver against the FP64 oracle.

Tolerances (floating point, relative to the oracle):
  FP64 forces   max_i |dF_i| / rms|F| <= 1e-12, |dU| / |U| <= 1e-12
  FP32 forces   max_i |dF_i| / rms|F| <= 1e-5,  max_i |de_i| <= 1e-6 mean|e_i|
                (the energy bound assumes no pair closer than sigma: single-precision
                pair energies carry ~2^-19 V(r) error, which grows fast below sigma)
  FP32 trajectories: positions within the displacement a 1e-5 rms|F| force error
                gives over the run, (k dt)^2 1e-5 rms|F|.
Integer results (cells, neighbour sets) are compared bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle
from synth import configs, make_lattice
from synth.configs import random_box

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1704_03329_b300 import lib
    return lib


@pytest.fixture(scope="module")
def ctx(L):
    return L.Context(0)


def cu(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def rows_as_sets(nbr, cnt):
    nbr = nbr.cpu().numpy()
    cnt = cnt.cpu().numpy()
    return [np.sort(nbr[i, :cnt[i]]) for i in range(len(cnt))]


def force_err(F, Fo):
    rms = np.sqrt((Fo ** 2).sum(1).mean())
    return np.sqrt(((F - Fo) ** 2).sum(1)).max() / rms


CASES = {
    "fcc10_r2.8": lambda: (configs.lj_solid(n_cells=10), 2.8),
    "sc10_r2.5": lambda: (configs.lj_small(), 2.5),
    "random_ragged": lambda: (dict(zip(("pos", "box"), random_box(997, [12.1, 11.3, 13.7], 3, cutoffs=(2.5, 2.8),
                                                                   margin=1e-6, min_dist=1.0))), 2.8),
}


@pytest.mark.parametrize("case", list(CASES))
def test_cells_bit_exact(L, ctx, case):
    c, r = CASES[case]()
    pos, box = c["pos"], c["box"]
    nc_o, cell_of_o, start_o, atoms_o = oracle.cells(pos, box, r)
    nc, cell_of, start, atoms = L.ppmd_build_cells(ctx, cu(pos), box, r)
    ctx.sync()
    assert list(nc) == list(nc_o)
    assert np.array_equal(cell_of.cpu().numpy(), cell_of_o)
    assert np.array_equal(start.cpu().numpy(), start_o)
    assert np.array_equal(atoms.cpu().numpy(), atoms_o)


@pytest.mark.parametrize("case", list(CASES))
def test_neighbour_sets_bit_exact(L, ctx, case):
    c, r = CASES[case]()
    pos, box = c["pos"], c["box"]
    offs, nbr_o = oracle.neighbours_cells(pos, box, r)
    p = cu(pos)
    nc, cell_of, start, atoms = L.ppmd_build_cells(ctx, p, box, r)
    nbr, cnt, needed = L.ppmd_build_neighbours(ctx, p, box, r, start, atoms, nc, 128, want_needed=True)
    assert needed == int(np.diff(offs).max())
    assert np.array_equal(cnt.cpu().numpy(), np.diff(offs))
    got = rows_as_sets(nbr, cnt)
    for i in range(len(pos)):
        assert np.array_equal(got[i], nbr_o[offs[i]:offs[i + 1]])


def test_neighbour_capacity_overflow_reports_needed(L, ctx):
    c = configs.lj_solid(n_cells=6)
    p = cu(c["pos"])
    nc, cell_of, start, atoms = L.ppmd_build_cells(ctx, p, c["box"], 2.8)
    with pytest.raises(L.PPMDError) as ei:
        L.ppmd_build_neighbours(ctx, p, c["box"], 2.8, start, atoms, nc, 40, want_needed=True)
    assert ei.value.code == L.ERR_CAPACITY
    rc, needed = ctx.status()
    assert rc == 0  # the status was consumed by the failing call
    nbr, cnt, needed = L.ppmd_build_neighbours(ctx, p, c["box"], 2.8, start, atoms, nc, 128, want_needed=True)
    assert needed == 78 or needed > 40


def test_box_too_small_is_rejected(L, ctx):
    pos = cu(np.zeros((4, 3)))
    with pytest.raises(L.PPMDError) as ei:
        L.ppmd_build_cells(ctx, pos, [7.0, 9.0, 9.0], 2.8)
    assert ei.value.code == L.ERR_BOX


def test_nonfinite_position_is_reported(L, ctx):
    c = configs.lj_small()
    pos = c["pos"].copy()
    pos[17, 1] = np.nan
    nc, cell_of, start, atoms = L.ppmd_build_cells(ctx, cu(pos), c["box"], 2.5)
    rc, _ = ctx.status()
    assert rc == L.ERR_NONFINITE


def _lists(L, ctx, pos, box, r, max_nbr=128):
    p = cu(pos)
    nc, cell_of, start, atoms = L.ppmd_build_cells(ctx, p, box, r)
    nbr, cnt = L.ppmd_build_neighbours(ctx, p, box, r, start, atoms, nc, max_nbr)
    return p, nbr, cnt


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("shift", [0.0, 0.25])
def test_lj_fp64_parity(L, ctx, case, shift):
    c, r = CASES[case]()
    pos, box = c["pos"], c["box"]
    offs, nbr_o = oracle.neighbours_cells(pos, box, r)
    Fo, eo, Uo, Wo = oracle.lj(pos, box, offs, nbr_o, shift=shift)
    p, nbr, cnt = _lists(L, ctx, pos, box, r)
    F, e, tot = L.ppmd_lj_forces(ctx, p, box, nbr, cnt, shift=shift, prec=L.FP64)
    F, e, tot = F.cpu().numpy(), e.cpu().numpy(), tot.cpu().numpy()
    assert force_err(F, Fo) <= 1e-12
    assert np.abs(e - eo).max() <= 1e-12 * np.abs(eo).mean()
    assert abs(tot[0] - Uo) <= 1e-12 * abs(Uo)
    assert abs(tot[1] - Wo) <= 1e-12 * max(abs(Wo), 1.0)


@pytest.mark.parametrize("case", list(CASES))
def test_lj_fp32_parity(L, ctx, case):
    c, r = CASES[case]()
    pos, box = c["pos"], c["box"]
    offs, nbr_o = oracle.neighbours_cells(pos, box, r)
    Fo, eo, Uo, Wo = oracle.lj(pos, box, offs, nbr_o)
    p, nbr, cnt = _lists(L, ctx, pos, box, r)
    F, e, tot = L.ppmd_lj_forces(ctx, p, box, nbr, cnt, prec=L.FP32)
    F, e, tot = F.cpu().numpy(), e.cpu().numpy(), tot.cpu().numpy()
    assert force_err(F, Fo) <= 1e-5
    assert np.abs(e - eo).max() <= 1e-6 * np.abs(eo).mean()
    assert abs(tot[0] - Uo) / len(pos) <= 1e-6 * abs(Uo) / len(pos)


def test_lj_fp32_forces_with_pairs_below_sigma(L, ctx):
    """FP32 force parity where pairs come as close as 0.7 sigma (random
    sequential addition with a 0.7 minimum distance): forces only, through
    the granular call and through the integrator's pair loop (set-up forces
    of ppmd_md_set_state).  The FP32 energy bound of the other tests assumes
    no pair below sigma: single-precision pair energies carry ~2^-19 V(r),
    and V grows as r^-12 there."""
    pos, box = random_box(997, [12.1, 11.3, 13.7], 7, cutoffs=(2.5, 2.8), margin=1e-6, min_dist=0.7)
    offs, nbr_o = oracle.neighbours_cells(pos, box, 2.8)
    dr = pos[np.repeat(np.arange(len(pos)), np.diff(offs))] - pos[nbr_o]
    dr -= box * np.rint(dr / box)
    assert np.sqrt((dr ** 2).sum(1)).min() < 0.8  # pairs well inside sigma
    Fo = oracle.lj(pos, box, offs, nbr_o)[0]
    p, nbr, cnt = _lists(L, ctx, pos, box, 2.8)
    F = L.ppmd_lj_forces(ctx, p, box, nbr, cnt, prec=L.FP32, want_energy=False)[0].cpu().numpy()
    assert force_err(F, Fo) <= 1e-5
    n = len(pos)
    md = L.MD(ctx, [0, n], [box], r_list=2.8, rebuild_every=10, max_nbr=128, prec=L.FP32)
    md.set_state(p, cu(np.zeros((n, 3))))
    F2 = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    md.get_state(None, None, F2)
    ctx.sync()
    assert force_err(F2.cpu().numpy(), Fo) <= 1e-5
    md.close()


CELL_CASES = dict(CASES, three_cells=lambda: (dict(zip(("pos", "box"), random_box(300, [7.6, 8.1, 9.9], 5, cutoffs=(2.5,),
                                                                                  margin=1e-6, min_dist=1.0))), 2.5))


@pytest.mark.parametrize("case", list(CELL_CASES))
@pytest.mark.parametrize("prec", ["FP32", "FP64"])
def test_lj_cells_parity(L, ctx, case, prec):
    """List-free pair loop: the oracle's forces, energies and totals at the
    tolerances of the list-based loop of the same precision (three cells per
    axis: every row of the sweep wraps)."""
    c, r = CELL_CASES[case]()
    pos, box = c["pos"], c["box"]
    offs, nbr_o = oracle.neighbours_cells(pos, box, r)
    Fo, eo, Uo, Wo = oracle.lj(pos, box, offs, nbr_o)
    F, e, tot = L.ppmd_lj_forces_cells(ctx, cu(pos), box, prec=getattr(L, prec))
    F, e, tot = F.cpu().numpy(), e.cpu().numpy(), tot.cpu().numpy()
    if prec == "FP64":
        assert force_err(F, Fo) <= 1e-12
        assert np.abs(e - eo).max() <= 1e-12 * np.abs(eo).mean()
        assert abs(tot[0] - Uo) <= 1e-12 * abs(Uo)
        assert abs(tot[1] - Wo) <= 1e-12 * max(abs(Wo), 1.0)
    else:
        assert force_err(F, Fo) <= 1e-5
        assert np.abs(e - eo).max() <= 1e-6 * np.abs(eo).mean()
        assert abs(tot[0] - Uo) <= 1e-6 * abs(Uo)


def test_lj_cells_empty_single_and_small_box(L, ctx):
    box = [9.0, 9.0, 9.0]
    for n in (0, 1):
        F, e, tot = L.ppmd_lj_forces_cells(ctx, cu(np.full((n, 3), 1.0)), box, prec=L.FP32)
        ctx.sync()
        assert F.shape == (n, 3) and (F.cpu() == 0).all() and float(tot[0]) == 0.0
    with pytest.raises(L.PPMDError) as ei:  # fewer than three cells of edge rc
        L.ppmd_lj_forces_cells(ctx, cu(np.full((4, 3), 1.0)), [7.4, 9.0, 9.0], prec=L.FP32)
    assert ei.value.code == L.ERR_BOX


@pytest.mark.parametrize("case", list(CASES))
def test_half_list_keeps_every_pair_once(L, ctx, case):
    """Every pair of the full list is in exactly one of its two atoms' half
    rows, each half row is a subset of the full row, and no row is far from
    half of the full length (the kept side is the upper half space)."""
    c, r = CASES[case]()
    p, nbr, cnt = _lists(L, ctx, c["pos"], c["box"], r)
    half, hcnt = L.ppmd_half_list(ctx, p, c["box"], nbr, cnt)
    full = rows_as_sets(nbr, cnt)
    got = rows_as_sets(half, hcnt)
    kept = set()
    for i in range(len(full)):
        assert np.isin(got[i], full[i]).all()
        for j in got[i]:
            key = (min(i, int(j)), max(i, int(j)))
            assert key not in kept
            kept.add(key)
    assert 2 * len(kept) == int(cnt.sum())
    hc, fc = hcnt.cpu().numpy(), cnt.cpu().numpy()
    assert (np.abs(2 * hc - fc) <= 0.5 * fc + 8).all()


def test_half_list_capacity_reports_needed(L, ctx):
    c, r = CASES["fcc10_r2.8"]()
    p, nbr, cnt = _lists(L, ctx, c["pos"], c["box"], r)
    L.ppmd_half_list(ctx, p, c["box"], nbr, cnt, max_half=8)
    code, needed = ctx.status()
    assert code == L.ERR_CAPACITY and needed > 8


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", ["FP32", "FP64"])
def test_lj_newton3_parity(L, ctx, case, prec):
    """Half-list pair loop: the oracle's forces, energies and totals at the
    tolerances of the full-list loop of the same precision, except the FP32
    per-atom energies: the partner halves arrive by FP32 atomics, without
    compensation and in any order, so an atom's energy can carry up to
    (partner terms) x 2^-24 x sum_j |V_ij| / 2 on top of the compensated own
    sum's error; on these cases that worst case is 1.5-2.0e-6 of the mean
    per-atom energy (at most 30 partner terms), so the bound is 3e-6 of it
    (1e-6 for the own sums plus 2e-6)."""
    c, r = CASES[case]()
    pos, box = c["pos"], c["box"]
    offs, nbr_o = oracle.neighbours_cells(pos, box, r)
    Fo, eo, Uo, Wo = oracle.lj(pos, box, offs, nbr_o)
    p, nbr, cnt = _lists(L, ctx, pos, box, r)
    half, hcnt = L.ppmd_half_list(ctx, p, box, nbr, cnt)
    F, e, tot = L.ppmd_lj_forces_newton3(ctx, p, box, half, hcnt, prec=getattr(L, prec))
    F, e, tot = F.cpu().numpy(), e.cpu().numpy(), tot.cpu().numpy()
    if prec == "FP64":
        assert force_err(F, Fo) <= 1e-12
        assert np.abs(e - eo).max() <= 1e-12 * np.abs(eo).mean()
        assert abs(tot[0] - Uo) <= 1e-12 * abs(Uo)
        assert abs(tot[1] - Wo) <= 1e-12 * max(abs(Wo), 1.0)
    else:
        assert force_err(F, Fo) <= 1e-5
        assert np.abs(e - eo).max() <= 3e-6 * np.abs(eo).mean()
        assert abs(tot[0] - Uo) <= 1e-6 * abs(Uo)
    # Newton's third law: the forces sum to zero (up to the arithmetic)
    assert np.abs(F.sum(0)).max() <= (1e-9 if prec == "FP64" else 1e-4) * np.abs(Fo).sum(0).max()


def test_lj_empty_and_single_atom(L, ctx):
    box = [9.0, 9.0, 9.0]
    for n in (0, 1):
        pos = cu(np.full((n, 3), 1.0))
        nc, cell_of, start, atoms = L.ppmd_build_cells(ctx, pos, box, 2.5)
        nbr, cnt = L.ppmd_build_neighbours(ctx, pos, box, 2.5, start, atoms, nc, 8)
        F, e, tot = L.ppmd_lj_forces(ctx, pos, box, nbr, cnt, prec=L.FP32)
        ctx.sync()
        assert F.shape == (n, 3) and (F.cpu() == 0).all() and float(tot[0]) == 0.0


@pytest.mark.parametrize("phase", [1, 2])
def test_verlet_step_bit_exact(L, ctx, phase):
    c = configs.lj_small()
    rng = np.random.default_rng(4)
    F = rng.normal(0, 3, c["pos"].shape)
    po, vo = oracle.vv(phase, c["pos"], c["vel"], F, c["box"], 1.0, 0.005)
    p, v = cu(c["pos"]), cu(c["vel"])
    L.ppmd_verlet_step(ctx, phase, p, v, cu(F), c["box"], 1.0, 0.005)
    assert np.array_equal(p.cpu().numpy(), po)
    assert np.array_equal(v.cpu().numpy(), vo)


def test_kinetic_energy(L, ctx):
    c = configs.lj_small()
    ke = L.ppmd_kinetic_energy(ctx, cu(c["vel"]), 1.0)
    assert abs(float(ke[0]) - oracle.kinetic(c["vel"])) <= 1e-13 * oracle.kinetic(c["vel"])


def _md(L, ctx, c, prec, nsteps, use_graph, energy_every=0, max_nbr=128):
    n = len(c["pos"])
    md = L.MD(ctx, [0, n], [c["box"]], r_list=c["r_list"], rebuild_every=c["rebuild_every"], max_nbr=max_nbr,
              prec=prec, energy_every=energy_every)
    md.set_state(cu(c["pos"]), cu(c["vel"]))
    en = torch.zeros((max(nsteps, 1), 2), dtype=torch.float64, device="cuda")
    md.run(nsteps, en if energy_every else None, use_graph=use_graph)
    pos = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    vel = torch.empty_like(pos)
    F = torch.empty_like(pos)
    md.get_state(pos, vel, F)
    info = md.info()
    return pos.cpu().numpy(), vel.cpu().numpy(), F.cpu().numpy(), en.cpu().numpy(), info


def _pos_err(p, po, box):
    d = p - po
    d -= box * np.rint(d / box)
    return np.abs(d).max()


@pytest.mark.parametrize("use_graph", [False, True])
def test_md_fp64_small_100_steps(L, ctx, use_graph):
    """Plain method, small, FP64: 1000 atoms, rebuild every step, 100 steps."""
    c = configs.lj_small()
    po, vo, Fo, eno, _ = oracle.md_run(c["pos"], c["vel"], c["box"], 100, r_list=2.5, rebuild_every=1)
    p, v, F, en, info = _md(L, ctx, c, L.FP64, 100, use_graph, energy_every=1)
    assert info["steps"] == 100 and info["rebuilds"] == 101
    assert _pos_err(p, po, c["box"]) <= 1e-10
    assert np.abs(v - vo).max() <= 1e-9
    assert force_err(F, Fo) <= 1e-9
    assert np.abs(en - eno).max() <= 1e-10 * np.abs(eno).max()


@pytest.mark.parametrize("use_graph", [False, True])
def test_md_fp32_solid_10_steps(L, ctx, use_graph):
    """FP32 pair forces with FP64 integration against the FP64 oracle over 10
    steps (one rebuild at step 10), fcc solid with skin 0.3."""
    c = configs.lj_solid(n_cells=10)
    po, vo, Fo, eno, _ = oracle.md_run(c["pos"], c["vel"], c["box"], 10, r_list=2.8, rebuild_every=10)
    p, v, F, en, info = _md(L, ctx, c, L.FP32, 10, use_graph, energy_every=10)
    assert force_err(F, Fo) <= 1e-5
    assert _pos_err(p, po, c["box"]) / c["box"][0] <= 1e-8
    assert abs(en[9, 1] - eno[9, 1]) <= 1e-6 * abs(eno[9, 1])
    assert abs(en[9, 0] - eno[9, 0]) <= 1e-6 * abs(eno[9, 0])


def test_md_fp32_full_size_sampled(L, ctx):
    """The 1,000,188-atom solid in the launch configuration the bench times
    (FP32 pair loop, graph replay, list 2.8 rebuilt every 10, 128 list
    slots): after 10 steps, the forces of a seeded sample of 400 atoms
    against the oracle on the same positions (the oracle's neighbour rows
    restricted to the sample, so it only works on those atoms)."""
    c = configs.lj_solid()
    assert len(c["pos"]) == 1000188
    p, v, F, en, info = _md(L, ctx, c, L.FP32, 10, True, energy_every=10)
    assert info["steps"] == 10
    sample = np.sort(np.random.default_rng(5).choice(len(p), 400, replace=False))
    offs, nb = oracle.neighbours_cells(p, c["box"], 2.8)
    deg = np.zeros(len(p), np.int64)
    deg[sample] = np.diff(offs)[sample]
    offs_s = np.concatenate([[0], np.cumsum(deg)])
    nb_s = np.concatenate([nb[offs[i]:offs[i + 1]] for i in sample])
    Fo, _, _, _ = oracle.lj(p, c["box"], offs_s, nb_s)
    rms = np.sqrt((Fo[sample] ** 2).sum(1).mean())
    assert np.sqrt(((F[sample] - Fo[sample]) ** 2).sum(1)).max() <= 1e-5 * rms
    assert np.isfinite(en[9]).all()


def test_md_fp64_solid_10_steps_is_exact(L, ctx):
    c = configs.lj_solid(n_cells=8)
    po, vo, Fo, eno, _ = oracle.md_run(c["pos"], c["vel"], c["box"], 10, r_list=2.8, rebuild_every=10)
    p, v, F, en, info = _md(L, ctx, c, L.FP64, 10, True, energy_every=10)
    assert force_err(F, Fo) <= 1e-11
    assert _pos_err(p, po, c["box"]) <= 1e-12 * c["box"][0]


def test_md_skin_violation_is_flagged(L, ctx):
    """Atoms moving more than half the skin between list builds: the run goes
    on (the guard never acts) and the state reports PPMD_WARN_SKIN with the
    largest displacement; with a wide skin and frequent builds it stays clear."""
    c = configs.lj_small()
    n = len(c["pos"])
    for r_list, every, max_nbr, flagged in ((2.55, 50, 128, True), (3.5, 10, 192, False)):
        md = L.MD(ctx, [0, n], [c["box"]], r_list=r_list, rc=2.5, rebuild_every=every, max_nbr=max_nbr, prec=L.FP32)
        md.set_state(cu(c["pos"]), cu(c["vel"]))
        md.run(2 * every)
        info = md.info()
        md.close()
        assert info["steps"] == 2 * every
        assert (info["status"] == L.WARN_SKIN) == flagged, (r_list, info)
        if flagged:
            assert info["max_disp"] > 0.5 * (r_list - 2.5)


@pytest.mark.parametrize("prec", ["FP32", "FP64"])
def test_md_list_capacity_overflow_reports_exact_need(L, ctx, prec):
    """A list capacity below the true neighbour count (LJ liquid, ragged
    counts): the integrator's list build latches PPMD_ERR_CAPACITY and
    reports the largest count exactly (the oracle's); with that capacity the
    build is clean."""
    c = configs.structure_box("liquid", 0.0, 3, cells=(40, 40, 40))
    pos, box = oracle.wrap(c["pos"], c["box"]), np.asarray(c["box"], float)
    offs, _ = oracle.neighbours_cells(pos, box, 2.8)
    need = int(np.diff(offs).max())
    n = len(pos)
    for max_nbr, fits in ((40, False), (need, True)):
        ctx.status()  # clear
        md = L.MD(ctx, [0, n], [box], r_list=2.8, rc=2.5, rebuild_every=10, max_nbr=max_nbr, prec=getattr(L, prec))
        md.set_state(cu(pos), cu(np.zeros((n, 3))))
        code, needed = ctx.status()  # synchronises and consumes the status
        md.close()
        if fits:
            assert code == 0, (code, needed)
        else:
            assert code == L.ERR_CAPACITY and needed == need, (code, needed, need)


def test_md_momentum_conserved(L, ctx):
    c = configs.lj_solid(n_cells=8)
    p, v, F, en, info = _md(L, ctx, c, L.FP32, 50, True)
    assert np.abs(v.sum(0)).max() <= 1e-9 * np.abs(v).sum()


def test_md_batched_boxes_equal_single_runs(L, ctx):
    """Several independent boxes advanced together give the single-box results."""
    reps = configs.replicas(seed=4, nrep=3, n_min=600, n_max=3000)
    pos = np.concatenate([r["pos"] for r in reps])
    vel = np.concatenate([r["vel"] for r in reps])
    off = np.cumsum([0] + [len(r["pos"]) for r in reps])
    md = L.MD(ctx, off, [r["box"] for r in reps], r_list=2.8, rebuild_every=10, max_nbr=128, prec=L.FP32,
              box_r_list=[r["r_list"] for r in reps])
    md.set_state(cu(pos), cu(vel))
    md.run(20)
    P = torch.empty((off[-1], 3), dtype=torch.float64, device="cuda")
    md.get_state(P)
    P = P.cpu().numpy()
    for k, r in enumerate(reps):
        po, _, Fo, _, _ = oracle.md_run(r["pos"], r["vel"], r["box"], 20, r_list=r["r_list"], rebuild_every=10)
        # displacement that a force error of 1e-5 rms|F| produces over 20 steps
        bound = (20 * 0.005) ** 2 * 1e-5 * np.sqrt((Fo ** 2).sum(1).mean())
        assert _pos_err(P[off[k]:off[k + 1]], po, r["box"]) <= bound


def test_md_replicas_full_size_sampled(L, ctx):
    """The 256-replica workload (2,034,923 atoms) in the launch configuration
    the bench times (one launch per kernel for all boxes, graph replay, 160
    list slots): after 10 steps, the forces of eight seeded boxes against the
    oracle on the same positions."""
    reps = configs.replicas()
    pos = np.concatenate([r["pos"] for r in reps])
    vel = np.concatenate([r["vel"] for r in reps])
    off = np.cumsum([0] + [len(r["pos"]) for r in reps])
    assert len(reps) == 256 and off[-1] == 2034923
    md = L.MD(ctx, off, [r["box"] for r in reps], r_list=2.8, rc=2.5, rebuild_every=10, max_nbr=160, prec=L.FP32,
              box_r_list=[r["r_list"] for r in reps])
    md.set_state(cu(pos), cu(vel))
    md.run(10)
    P = torch.empty((off[-1], 3), dtype=torch.float64, device="cuda")
    F = torch.empty_like(P)
    md.get_state(P, None, F)
    P, F = P.cpu().numpy(), F.cpu().numpy()
    md.close()
    for k in np.random.default_rng(6).choice(256, 8, replace=False):
        r, lo, hi = reps[k], off[k], off[k + 1]
        offs, nb = oracle.neighbours_cells(P[lo:hi], r["box"], r["r_list"])
        Fo, _, _, _ = oracle.lj(P[lo:hi], r["box"], offs, nb)
        assert force_err(F[lo:hi], Fo) <= 1e-5, k


def test_md_fused_kick_drift_is_bit_identical(L, ctx):
    """Inside a run the FP32 pair loop also makes the next step's kick and
    drift (the same arithmetic as the separate kernel): one run of 23 steps
    (graph replays plus single steps, or single steps only) and 23 runs of one
    step (no fusion) give identical bits."""
    c = configs.lj_solid(n_cells=8)
    n = len(c["pos"])

    def state(runs, use_graph):
        md = L.MD(ctx, [0, n], [c["box"]], r_list=c["r_list"], rebuild_every=c["rebuild_every"], max_nbr=128,
                  prec=L.FP32, energy_every=5)
        md.set_state(cu(c["pos"]), cu(c["vel"]))
        en = torch.zeros((23, 2), dtype=torch.float64, device="cuda")
        done = 0
        for r in runs:
            md.run(r, en[done:done + r], use_graph=use_graph)
            done += r
        p = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        v = torch.empty_like(p)
        md.get_state(p, v)
        return p.cpu().numpy(), v.cpu().numpy(), en.cpu().numpy()

    ref = state([1] * 23, False)
    for runs, g in (([23], True), ([23], False), ([7, 16], True)):
        got = state(runs, g)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b), (runs, g)


def _otf_md(L, ctx, c, nsteps, use_graph, thermo, boa):
    n = len(c["pos"])
    md = L.MD(ctx, [0, n], [c["box"]], r_list=c["r_list"], rebuild_every=c["rebuild_every"], max_nbr=128,
              prec=L.FP32, energy_every=5)
    if thermo:
        md.set_thermostat(*thermo)
    if boa:
        md.set_boa(*boa)
    md.set_state(cu(c["pos"]), cu(c["vel"]))
    en = torch.zeros((nsteps, 2), dtype=torch.float64, device="cuda")
    q = torch.zeros((nsteps, 3), dtype=torch.float64, device="cuda")
    md.run_analysed(nsteps, en, q, use_graph=use_graph)
    p = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    v = torch.empty_like(p)
    md.get_state(p, v)
    ql = md.get_q().cpu().numpy() if boa else None
    return p.cpu().numpy(), v.cpu().numpy(), en.cpu().numpy(), q.cpu().numpy(), ql


@pytest.mark.parametrize("use_graph", [False, True])
def test_otf_run_matches_oracle(L, ctx, use_graph):
    """The on-the-fly analysis run: Andersen collisions (p = 0.05 per step,
    decided by integer counters, so the same atoms collide on both sides)
    and Q4/Q5/Q6 every second step, 20 steps of the fcc solid, against the
    FP64 oracle with the FP32-force tolerances."""
    c = configs.lj_solid(n_cells=8)
    thermo, boa = (0.5, 10.0, 987654321), (2, 1.5)
    po, vo, Fo, eno, qo, qlo, ncoll = oracle.md_run_otf(c["pos"], c["vel"], c["box"], 20, r_list=2.8,
                                                        rebuild_every=10, thermostat=thermo, boa=boa)
    assert ncoll > 0
    p, v, en, q, ql = _otf_md(L, ctx, c, 20, use_graph, thermo, boa)
    assert _pos_err(p, po, c["box"]) / c["box"][0] <= 1e-8
    # velocity change a 1e-5 rms|F| force error makes over 20 steps (twice)
    assert np.abs(v - vo).max() <= 2 * 20 * 0.005 * 1e-5 * np.sqrt((Fo ** 2).sum(1).mean())
    rows = np.arange(1, 20, 2)
    assert np.abs(q[rows] - qo[rows]).max() <= 1e-5
    assert (q[np.arange(0, 20, 2)] == 0).all()
    assert np.abs(ql - qlo).max() <= 1e-5
    assert np.abs(en[4::5, 0] - eno[4::5, 0]).max() <= 1e-6 * np.abs(eno[4::5, 0]).max()


def test_otf_full_size_q_against_oracle(L, ctx):
    """The on-the-fly analysis workload at full size (524,288 atoms, r_c 3.0,
    list 3.3, rebuild every 18, thermostat and Q4/Q5/Q6 every step) in the
    bench's launch configuration (one 18-step graph replay): every atom's
    Q4, Q5, Q6 of the last step against the oracle on the final positions."""
    c = configs.otf_box()
    n = len(c["pos"])
    assert n == 524288
    md = L.MD(ctx, [0, n], [c["box"]], r_list=3.3, rc=3.0, rebuild_every=18, max_nbr=192, prec=L.FP32,
              energy_every=18)
    md.set_thermostat(0.1, 1.0, 20170410)
    md.set_boa(1, 1.5)
    md.set_state(cu(c["pos"]), cu(c["vel"]))
    md.run_analysed(18, None, None, use_graph=True)
    p = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    md.get_state(p)
    q = md.get_q().cpu().numpy()
    md.close()
    p = p.cpu().numpy()
    offs, nb = oracle.neighbours_cells(p, c["box"], 1.5)
    for row, l in enumerate((4, 5, 6)):
        Qo, _ = oracle.boa(p, c["box"], offs, nb, 1.5, l)
        assert np.abs(q[row] - Qo).max() <= 1e-5, l


def test_otf_graph_and_single_steps_are_bit_identical(L, ctx):
    """Graph replays take the thermostat's step numbers from the device: the
    same bits as single steps."""
    c = configs.lj_solid(n_cells=8)
    a = _otf_md(L, ctx, c, 23, True, (0.5, 10.0, 5), (1, 1.5))
    b = _otf_md(L, ctx, c, 23, False, (0.5, 10.0, 5), (1, 1.5))
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_otf_q_rows_of_a_crystal_at_rest(L, ctx, golden):
    lat = make_lattice("fcc", (8, 8, 8), 0.8442)
    c = {"pos": lat.sites(), "vel": np.zeros((len(lat.sites()), 3)), "box": lat.box, "r_list": 2.8,
         "rebuild_every": 10}
    _, _, _, q, ql = _otf_md(L, ctx, c, 10, True, None, (5, 1.5))
    tab = golden["Q_table"]["fcc"]
    assert np.allclose(q[[4, 9]], [tab["Q4"], tab["Q5"], tab["Q6"]], atol=5e-4)
    assert np.allclose(ql.mean(1), q[9], atol=1e-6)


def _oracle_missed(p_old, p_new, box, rc, r_list):
    """Pairs within rc at p_new that were at least r_list apart at p_old."""
    offs, nb = oracle.neighbours_cells(p_new, box, rc)
    i = np.repeat(np.arange(len(p_new)), np.diff(offs))
    d = p_old[i] - p_old[nb]
    d -= box * np.rint(d / box)
    return int((np.sqrt((d ** 2).sum(1)) >= r_list).sum())


def test_md_missed_pairs_count_matches_oracle(L, ctx):
    """A thin skin (list 2.55, rebuilt every 50 steps) on the small sc box:
    the list-age check counts, at the rebuilds of steps 50 and 100, the
    pairs within rc that were beyond the list cutoff at the previous build
    (FP64 run, so the GPU and oracle trajectories agree to ~1e-12)."""
    c = configs.lj_small()
    n = len(c["pos"])
    md = L.MD(ctx, [0, n], [c["box"]], r_list=2.55, rc=2.5, rebuild_every=50, max_nbr=128, prec=L.FP64)
    md.set_check(True)
    md.set_state(cu(c["pos"]), cu(c["vel"]))
    md.run(100)
    got = md.missed_pairs()
    md.close()
    box = c["box"]
    p0 = oracle.wrap(c["pos"], box)
    p50, v50, _, _, _ = oracle.md_run(c["pos"], c["vel"], box, 50, r_list=2.55, rebuild_every=50)
    p100, _, _, _, _ = oracle.md_run(p50, v50, box, 50, r_list=2.55, rebuild_every=50)
    want = _oracle_missed(p0, p50, box, 2.5, 2.55) + _oracle_missed(p50, p100, box, 2.5, 2.55)
    assert want > 0 and got == want, (got, want)


def test_md_check_leaves_the_trajectory_unchanged(L, ctx):
    c = configs.lj_solid(n_cells=8)
    n = len(c["pos"])
    out = []
    for check in (False, True):
        md = L.MD(ctx, [0, n], [c["box"]], r_list=2.8, rc=2.5, rebuild_every=10, max_nbr=128, prec=L.FP32)
        md.set_check(check)
        md.set_state(cu(c["pos"]), cu(c["vel"]))
        md.run(30)
        p = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        md.get_state(p)
        out.append((p.cpu().numpy(), md.missed_pairs()))
        md.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == 0  # no count without the check


def test_md_lists_with_atoms_on_cell_faces(L, ctx):
    """Atoms on the faces of the list cells: a simple-cubic lattice of
    spacing half the cell edge (every coordinate an exact binary fraction,
    pairs at exactly r_list), some atoms moved 2^-40 off a face, some just
    below the box face.  The integrator's lists at set-up and at the rebuild
    after 10 steps (the lattice at rest stays on the faces) are the oracle's
    sets; pairs at exactly r_list are not listed (strict cutoff)."""
    a, m = 1.375, 12
    edge = a * m  # 16.5: six cells of 2.75 = r_list
    g = np.arange(m) * a
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    rng = np.random.default_rng(5)
    k = rng.choice(len(pos), 200, replace=False)
    pos[k[:100], 0] += np.where(rng.random(100) < 0.5, 1.0, -1.0) * 2.0 ** -40
    pos[k[100:150], 1] -= 2.0 ** -40
    pos[pos < 0] += edge  # just below the box face
    box = np.array([edge] * 3)
    n = len(pos)
    md = L.MD(ctx, [0, n], [box], r_list=2.75, rc=2.5, rebuild_every=10, max_nbr=128, prec=L.FP32)
    md.set_state(cu(pos), cu(np.zeros_like(pos)))
    for steps in (0, 10):
        md.run(steps)
        p = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        md.get_state(p)
        P = p.cpu().numpy()
        nbr, cnt = md.get_list()
        offs, nb = oracle.neighbours_brute(P, box, 2.75)
        assert np.array_equal(cnt.cpu().numpy(), np.diff(offs)), steps
        got = rows_as_sets(nbr, cnt)
        for i in range(n):
            assert np.array_equal(got[i], nb[offs[i]:offs[i + 1]]), (steps, i)
    md.close()


def test_md_without_atoms(L, ctx):
    """A system of no atoms: set-up, graph units and single steps, energy
    rows, state and list reads all succeed; the energies are zero."""
    box = np.array([9.0, 9.5, 10.0])
    md = L.MD(ctx, [0, 0], [box], r_list=2.8, rc=2.5, rebuild_every=10, max_nbr=64, prec=L.FP32, energy_every=10)
    md.set_state(cu(np.zeros((0, 3))), cu(np.zeros((0, 3))))
    en = torch.ones((23, 2), dtype=torch.float64, device="cuda")
    md.run(23, en)
    p = torch.empty((0, 3), dtype=torch.float64, device="cuda")
    md.get_state(p, p, p)
    nbr, cnt = md.get_list()
    info = md.info()
    md.close()
    assert nbr.shape[0] == 0 and cnt.shape[0] == 0 and info["steps"] == 23
    e = en.cpu().numpy()
    assert (e[[9, 19]] == 0).all()


def test_md_empty_box_among_replicas(L, ctx):
    """An empty box between replicas changes nothing: positions and
    velocities of the others are those of the run without it, bit for bit."""
    reps = configs.replicas(seed=4, nrep=3, n_min=600, n_max=3000)
    pos = np.concatenate([r["pos"] for r in reps])
    vel = np.concatenate([r["vel"] for r in reps])
    sizes = [len(r["pos"]) for r in reps]
    out = []
    for with_empty in (False, True):
        boxes = [r["box"] for r in reps]
        rl = [r["r_list"] for r in reps]
        sz = list(sizes)
        if with_empty:
            boxes.insert(1, np.array([9.0, 9.0, 9.0]))
            rl.insert(1, 2.8)
            sz.insert(1, 0)
        off = np.cumsum([0] + sz)
        md = L.MD(ctx, off, boxes, r_list=2.8, rebuild_every=10, max_nbr=128, prec=L.FP32, box_r_list=rl)
        md.set_state(cu(pos), cu(vel))
        md.run(23)
        P = torch.empty((off[-1], 3), dtype=torch.float64, device="cuda")
        V = torch.empty_like(P)
        md.get_state(P, V)
        md.close()
        out.append((P.cpu().numpy(), V.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
