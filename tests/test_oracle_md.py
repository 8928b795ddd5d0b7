"""Pins of the FP64 oracle's cell list, neighbour list, LJ pair loop and
Velocity Verlet against facts fixed by the paper and by mathematics (no GPU)."""
import itertools
import math

import numpy as np
import pytest

import oracle
from synth import configs, make_lattice, maxwell_boltzmann, rng_stream
from synth.configs import random_box

RHO = 0.8442


def _lattice_energy_per_atom(kind, rc, shift=0.0):
    """Closed-form lattice sum by integer enumeration (independent of the oracle):
    fcc sites are (i, j, k) a/2 with i + j + k even; sc sites are (i, j, k) a."""
    if kind == "fcc":
        a = (4.0 / RHO) ** (1.0 / 3.0)
        scale, parity = a / 2.0, True
    else:
        a = RHO ** (-1.0 / 3.0)
        scale, parity = a, False
    R = int(rc / scale) + 1
    s = 0.0
    for i, j, k in itertools.product(range(-R, R + 1), repeat=3):
        if parity and (i + j + k) % 2:
            continue
        r = math.sqrt(i * i + j * j + k * k) * scale
        if 0 < r < rc:
            s += 2.0 * (r ** -12 - r ** -6 + shift)
    return s


@pytest.mark.parametrize("kind,ncell", [("fcc", 6), ("sc", 8)])
@pytest.mark.parametrize("shift", [0.0, 0.25])
def test_lattice_energy_closed_form(kind, ncell, shift):
    lat = make_lattice(kind, ncell, RHO)
    pos, box = lat.sites(), lat.box
    offs, nbr = oracle.neighbours_cells(pos, box, 2.5)
    F, e, U, W = oracle.lj(pos, box, offs, nbr, shift=shift)
    ref = _lattice_energy_per_atom(kind, 2.5, shift)
    assert abs(U / len(pos) - ref) < 1e-11 * abs(ref)
    assert np.allclose(e, ref, rtol=1e-11, atol=0)
    assert np.abs(F).max() < 1e-11  # every atom is a centre of inversion
    # neighbour counts within 2.5: 54 for fcc, 56 for sc; within 2.8 fcc has 78
    assert (np.diff(offs) == (54 if kind == "fcc" else 56)).all()
    if kind == "fcc":
        o28, _ = oracle.neighbours_cells(pos, box, 2.8)
        assert (np.diff(o28) == 78).all()


def test_fcc_closed_form_values():
    # fixed decimal values of the two lattice sums at rho = 0.8442, rc = 2.5
    assert abs(_lattice_energy_per_atom("fcc", 2.5) - (-6.773368053253)) < 1e-11
    assert abs(_lattice_energy_per_atom("fcc", 2.5, 0.25) - 20.226631946747) < 1e-11
    assert abs(_lattice_energy_per_atom("sc", 2.5) - (-5.220218519441)) < 1e-11


def _tiny_box(seed, n=60, L=7.3, margin=1e-3):
    return random_box(n, [L, L * 1.1, L * 0.95], seed, cutoffs=(2.5, 2.8), margin=margin, min_dist=0.85)


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_neighbour_list_cells_equal_brute_force(seed):
    pos, box = _tiny_box(seed, n=140, L=9.0)
    for r in (2.5, 2.8):
        o1, n1 = oracle.neighbours_brute(pos, box, r)
        o2, n2 = oracle.neighbours_cells(pos, box, r)
        assert np.array_equal(o1, o2) and np.array_equal(n1, n2)
        # symmetric: j in N(i) iff i in N(j)
        pairs = {(i, int(j)) for i in range(len(pos)) for j in n1[o1[i]:o1[i + 1]]}
        assert all((j, i) in pairs for (i, j) in pairs)


@pytest.mark.parametrize("seed", [14, 15])
def test_cells_and_lists_on_an_uneven_grid(seed):
    """A box of 3 x 4 x 5 (r 2.8) and 3 x 4 x 6 (r 2.5) cells: every cell
    index, its decoding and the stencil's wrap use the edge's own count
    (on an n x n x n grid the axes could be swapped unseen)."""
    box = np.array([9.0, 12.0, 15.3])
    pos, box = random_box(320, box, seed, cutoffs=(2.5, 2.8), margin=1e-3, min_dist=0.85)
    for r, grid in ((2.8, [3, 4, 5]), (2.5, [3, 4, 6])):
        nc, cell_of, start, atoms = oracle.cells(pos, box, r)
        assert list(nc) == grid
        w = box / nc
        cz, rem = np.divmod(cell_of, nc[0] * nc[1])
        cy, cx = np.divmod(rem, nc[0])
        cc = np.stack([cx, cy, cz], 1)
        assert (cc * w <= pos + 1e-12).all() and (pos < (cc + 1) * w + 1e-12).all()
        o1, n1 = oracle.neighbours_brute(pos, box, r)
        o2, n2 = oracle.neighbours_cells(pos, box, r)
        assert np.array_equal(o1, o2) and np.array_equal(n1, n2)
        # periodic images of the positions (whole box lengths added or taken
        # away) fall in the same cells: coordinates are wrapped first
        shift = np.random.default_rng(seed).integers(-2, 3, pos.shape) * box
        assert np.array_equal(oracle.cells(pos + shift, box, r)[1], cell_of)


def test_cells_contain_their_atoms():
    c = configs.lj_solid(n_cells=6)
    pos, box = c["pos"], c["box"]
    # and atoms a hair below each box face, whose x / w can round up to n
    edge = np.array([np.nextafter(box, 0.0), [np.nextafter(box[0], 0.0), 0.0, 0.0],
                     [0.0, np.nextafter(box[1], 0.0), 0.0], [0.0, 0.0, np.nextafter(box[2], 0.0)]])
    pos = np.concatenate([pos, edge])
    nc, cell_of, start, atoms = oracle.cells(pos, box, 2.8)
    assert (nc == np.floor(box / 2.8)).all()
    w = box / nc
    cz, rem = np.divmod(cell_of, nc[0] * nc[1])
    cy, cx = np.divmod(rem, nc[0])
    cc = np.stack([cx, cy, cz], 1)
    assert (cc * w <= pos + 1e-12).all() and (pos < (cc + 1) * w + 1e-12).all()
    assert (cc[-4:] == np.array([nc - 1, [nc[0] - 1, 0, 0], [0, nc[1] - 1, 0], [0, 0, nc[2] - 1]])).all()
    assert start[0] == 0 and start[-1] == len(pos) and (np.diff(start) >= 0).all()
    for c_ in range(len(start) - 1):
        members = atoms[start[c_]:start[c_ + 1]]
        assert (cell_of[members] == c_).all() and (np.diff(members) > 0).all()


@pytest.mark.parametrize("seed", [21, 22])
def test_force_is_minus_energy_gradient(seed):
    """F = -grad U (Eq. (12) from Eq. (9)) by central differences of the total energy;
    pins the force's sign, exponents and prefactor."""
    pos, box = _tiny_box(seed)
    offs, nbr = oracle.neighbours_brute(pos, box, 2.5)
    F, e, U, W = oracle.lj(pos, box, offs, nbr)
    h = 1e-6
    rng = np.random.default_rng(seed)
    for i in rng.choice(len(pos), 8, replace=False):
        for d in range(3):
            pp = pos.copy(); pp[i, d] += h
            pm = pos.copy(); pm[i, d] -= h
            Up = oracle.lj(pp, box, offs, nbr)[2]
            Um = oracle.lj(pm, box, offs, nbr)[2]
            fd = -(Up - Um) / (2 * h)
            assert abs(fd - F[i, d]) < 1e-6 * max(1.0, abs(F[i, d]))


@pytest.mark.parametrize("seed", [31])
def test_virial_is_volume_derivative(seed):
    """W = sum_{i<j} r_ij . f_ij equals -dU/dlambda under uniform scaling r -> lambda r."""
    pos, box = _tiny_box(seed)
    offs, nbr = oracle.neighbours_brute(pos, box, 2.5)
    F, e, U, W = oracle.lj(pos, box, offs, nbr)
    h = 1e-7
    Up = oracle.lj(pos * (1 + h), box * (1 + h), offs, nbr)[2]
    Um = oracle.lj(pos * (1 - h), box * (1 - h), offs, nbr)[2]
    assert abs(-(Up - Um) / (2 * h) - W) < 1e-5 * max(1.0, abs(W))


def test_newton_third_law_and_energy_sum():
    c = configs.lj_solid(n_cells=6)
    offs, nbr = oracle.neighbours_cells(c["pos"], c["box"], 2.8)
    F, e, U, W = oracle.lj(c["pos"], c["box"], offs, nbr)
    rmsF = np.sqrt((F ** 2).sum(1).mean())
    assert np.abs(F.sum(0)).max() < 1e-12 * len(F) * rmsF
    assert abs(e.sum() - U) < 1e-12 * abs(U)
    # the list at 2.8 gives the same forces as the list at exactly 2.5
    o2, n2 = oracle.neighbours_cells(c["pos"], c["box"], 2.5)
    F2 = oracle.lj(c["pos"], c["box"], o2, n2)[0]
    assert np.abs(F - F2).max() < 1e-12 * rmsF


def test_lj_scales_with_epsilon_and_sigma():
    """Eqs. (9) and (12) in reduced units: stretching every length (positions,
    box, cutoff) by sigma and every energy by epsilon leaves the reduced
    problem unchanged, so the per-atom energies, U and W scale by epsilon
    and the forces by epsilon / sigma (the paper's 1/4 shift included)."""
    c = configs.lj_solid(n_cells=6)
    pos, box = c["pos"], c["box"]
    offs, nb = oracle.neighbours_cells(pos, box, 2.8)
    F1, e1, U1, W1 = oracle.lj(pos, box, offs, nb, rc=2.5, eps=1.0, sigma=1.0, shift=0.25)
    eps, sigma = 1.7, 1.3
    F, e, U, W = oracle.lj(pos * sigma, box * sigma, offs, nb, rc=2.5 * sigma, eps=eps, sigma=sigma, shift=0.25)
    assert np.allclose(e, eps * e1, rtol=1e-12, atol=1e-12 * np.abs(e1).max())
    assert abs(U - eps * U1) <= 1e-12 * abs(U1) and abs(W - eps * W1) <= 1e-12 * abs(W1)
    assert np.allclose(F, eps / sigma * F1, rtol=0, atol=1e-12 * np.abs(F1).max())


def test_shift_changes_energy_not_force():
    c = configs.lj_small()
    offs, nbr = oracle.neighbours_cells(c["pos"], c["box"], 2.5)
    F0, e0, U0, _ = oracle.lj(c["pos"], c["box"], offs, nbr, shift=0.0)
    F1, e1, U1, _ = oracle.lj(c["pos"], c["box"], offs, nbr, shift=0.25)
    assert np.array_equal(F0, F1)
    # +eps per pair term, half to each atom of the pair: e_i gains nu_i / 2
    assert np.allclose(e1 - e0, np.diff(offs) * 0.5, rtol=0, atol=1e-12)


def test_cells_of_atoms_below_the_box_face():
    """For these edges (14.0 and neighbours, cells of 2.8) the largest double
    below L divided by the cell width rounds to n itself: such an atom
    belongs to the last cell, n - 1."""
    box = np.array([14.0, 14.004, 14.008])
    nc = oracle.cell_grid(box, 2.8)
    below = np.nextafter(box, 0.0)
    assert (np.floor(below / (box / nc)) == nc).all()  # the rounding the clamp is for
    pos = np.array([[1.0, 1.0, 1.0], below, [below[0], 0.0, 7.0], [7.0, below[1], 0.0], [0.0, 7.0, below[2]]])
    _, cell_of, start, atoms = oracle.cells(pos, box, 2.8)
    cz, rem = np.divmod(cell_of, nc[0] * nc[1])
    cy, cx = np.divmod(rem, nc[0])
    assert [cx[1], cy[1], cz[1]] == list(nc - 1)
    assert cx[2] == nc[0] - 1 and cy[3] == nc[1] - 1 and cz[4] == nc[2] - 1
    assert start[-1] == len(pos) and sorted(atoms) == list(range(len(pos)))


def test_vv_constant_force_closed_form():
    """One step of Algorithm 6 under a constant force reproduces the exact
    kinematics r + v dt + F dt^2 / (2m) and v + F dt / m."""
    box = np.array([50.0, 50.0, 50.0])
    pos = np.array([[10.0, 20.0, 30.0]])
    vel = np.array([[0.3, -0.2, 0.1]])
    F = np.array([[1.5, 0.5, -2.0]])
    m, dt = 2.0, 0.01
    p1, v1 = oracle.vv(1, pos, vel, F, box, m, dt)
    p2, v2 = oracle.vv(2, p1, v1, F, box, m, dt)
    assert np.allclose(p2, pos + vel * dt + F * dt * dt / (2 * m), rtol=0, atol=1e-14)
    assert np.allclose(v2, vel + F * dt / m, rtol=0, atol=1e-14)


def test_vv_wraps_into_box():
    box = np.array([5.0, 5.0, 5.0])
    pos = np.array([[4.999, 0.0005, 2.0]])
    vel = np.array([[1.0, -1.0, 0.0]])
    p1, _ = oracle.vv(1, pos, vel, np.zeros((1, 3)), box, 1.0, 0.005)
    assert np.allclose(p1, [[0.004, 4.9955, 2.0]], atol=1e-12)
    assert ((p1 >= 0) & (p1 < box)).all()


def test_wrap_maps_into_the_half_open_box():
    """x - L floor(x / L) can round to L itself (a coordinate a hair below 0,
    a multiple of L); every wrapped coordinate lies in [0, L)."""
    box = np.array([5.0, 7.0, 3.0])
    pos = np.array([[-1e-18, -0.0, 3.0], [10.0, -7.0, -1e-300], [-5.0, 14.0, 2.9999999999999996]])
    w = oracle.wrap(pos, box)
    assert ((w >= 0) & (w < box)).all()
    assert (w[:2] == 0).all() and w[2, 0] == 0 and w[2, 1] == 0 and w[2, 2] == pos[2, 2]


def test_md_max_displacement_since_rebuild():
    """The skin guard of Sec. 3.5 (the largest displacement since the list was
    built, against half the skin of Eq. (3)), in free flight: atoms 3.2 apart
    never come within rc, feel no force and keep their velocities, so after
    25 steps with a rebuild every 10 the largest displacement since a
    rebuild is that of the fastest atom over 10 steps."""
    k = np.arange(3)
    pos = 3.2 * np.stack(np.meshgrid(k, k, k, indexing="ij"), -1).reshape(-1, 3) + 0.1
    box = np.full(3, 9.6)
    vel = np.random.default_rng(8).uniform(-1.0, 1.0, pos.shape)
    dt = 0.005
    _, v, F, _, md = oracle.md_run(pos, vel, box, 25, rc=2.5, r_list=2.8, rebuild_every=10, dt=dt)
    assert (F == 0).all() and np.array_equal(v, vel)
    expect = 10 * dt * np.sqrt((vel ** 2).sum(1)).max()
    assert abs(md - expect) < 1e-12
    # a rebuild at steps 4, 8, ... (not one step early or late): 6 steps with
    # a rebuild every 4 leave 4 steps as the longest flight since a build
    md = oracle.md_run(pos, vel, box, 6, rc=2.5, r_list=2.8, rebuild_every=4, dt=dt)[4]
    assert abs(md - 4 * dt * np.sqrt((vel ** 2).sum(1)).max()) < 1e-12


def _cold_crystal(dt, nsteps, mass=1.0):
    lat = make_lattice("fcc", 4, RHO)
    pos = lat.sites() + rng_stream(5, 0).normal(0, 0.005, (lat.nsite, 3))
    vel = maxwell_boltzmann(rng_stream(5, 1), lat.nsite, 0.01 / mass)
    return oracle.md_run(pos, vel, lat.box, nsteps, rc=2.5, r_list=2.5, rebuild_every=1, dt=dt, mass=mass)


@pytest.mark.parametrize("mass", [1.0, 2.0])
def test_vv_energy_error_is_second_order(mass):
    """Velocity Verlet conserves energy up to O(dt^2): halving dt quarters the
    energy fluctuation (cold fcc crystal: no pair crosses the cutoff).  With
    mass 2 the recorded kinetic energy must carry the mass for the total to
    be conserved."""
    _, v_a, _, en_a, _ = _cold_crystal(0.005, 200, mass)
    _, v_b, _, en_b, _ = _cold_crystal(0.0025, 400, mass)
    ea = en_a.sum(1)
    eb = en_b.sum(1)
    fa = ea.max() - ea.min()
    fb = eb.max() - eb.min()
    assert fa / abs(ea.mean()) < 1e-6
    assert 3.0 < fa / fb < 5.0
    # total momentum is conserved (it starts at zero)
    assert np.abs(v_a.sum(0)).max() < 1e-11


def test_md_time_reversible():
    c = configs.lj_small()
    p1, v1, _, _, _ = oracle.md_run(c["pos"], c["vel"], c["box"], 30)
    p0, v0, _, _, _ = oracle.md_run(p1, -v1, c["box"], 30)
    d = p0 - c["pos"]
    d -= c["box"] * np.rint(d / c["box"])
    assert np.abs(d).max() < 1e-8 and np.abs(-v0 - c["vel"]).max() < 1e-8


def test_md_rebuild_policy_matches_fresh_lists():
    """With list reuse (r_list = 2.8, rebuild every 10 steps) the trajectory equals
    the one with a fresh list at rc every step while no pair enters rc unlisted."""
    c = configs.lj_solid(n_cells=6)
    a = oracle.md_run(c["pos"], c["vel"], c["box"], 20, r_list=2.8, rebuild_every=10)
    b = oracle.md_run(c["pos"], c["vel"], c["box"], 20, r_list=2.5, rebuild_every=1)
    assert 0.0 < a[4] < 0.3  # largest displacement between rebuilds stayed below the skin
    assert np.abs(a[0] - b[0]).max() < 1e-10


# ---------------------------------------------------------------------------
# On-the-fly analysis run: Philox, Andersen thermostat, Q4/Q5/Q6 rows
# ---------------------------------------------------------------------------
def test_philox4x32_known_answers():
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.json")) as f:
        kat = json.load(f)
    for v in kat["vectors"]:
        out = oracle.philox4x32([int(x, 16) for x in v["ctr"]], [int(x, 16) for x in v["key"]])
        assert [f"{int(x):08x}" for x in out] == v["out"]


def test_andersen_threshold():
    assert oracle.andersen_threshold(0.0, 0.005) == 0
    assert oracle.andersen_threshold(1.0, 0.005) == math.floor(0.005 * 2 ** 32)
    assert oracle.andersen_threshold(400.0, 0.005) == 2 ** 32


def test_otf_run_without_additions_is_the_plain_run():
    c = configs.lj_solid(n_cells=6)
    a = oracle.md_run(c["pos"], c["vel"], c["box"], 12, r_list=2.8, rebuild_every=10)
    b = oracle.md_run_otf(c["pos"], c["vel"], c["box"], 12, r_list=2.8, rebuild_every=10)
    for x, y in zip(a[:4], b[:4]):
        assert np.array_equal(x, y)
    assert b[6] == 0


def _draws(seed, ids, step, T):
    """The thermostat's velocity draw written out with the generator above and
    numpy's transcendental functions (every atom collides)."""
    out = np.zeros((len(ids), 3))
    inv = 2.0 ** -32
    for k, i in enumerate(ids):
        c = [i & 0xffffffff, step & 0xffffffff, step >> 32, 0]
        key = [seed & 0xffffffff, seed >> 32]
        u = oracle.philox4x32(c, key).astype(np.float64)
        w = oracle.philox4x32(c[:3] + [1], key).astype(np.float64)
        r1, t1 = np.sqrt(-2.0 * np.log((u[1] + 0.5) * inv)), 2 * np.pi * (u[2] + 0.5) * inv
        r2, t2 = np.sqrt(-2.0 * np.log((u[3] + 0.5) * inv)), 2 * np.pi * (w[0] + 0.5) * inv
        out[k] = np.sqrt(T) * np.array([r1 * np.cos(t1), r1 * np.sin(t1), r2 * np.cos(t2)])
    return out


def test_andersen_every_atom_every_step():
    """With nu dt >= 1 every atom is redrawn at the end of every step: the
    final velocities are the last step's draws; their second moment is T."""
    c = configs.lj_solid(n_cells=6)
    n = len(c["pos"])
    T, seed = 0.7, 12345678901
    _, vel, _, _, _, _, ncoll = oracle.md_run_otf(c["pos"], c["vel"], c["box"], 3, r_list=2.8, rebuild_every=10,
                                                  thermostat=(T, 1000.0, seed))
    assert ncoll == 3 * n
    assert np.allclose(vel, _draws(seed, range(n), 3, T), rtol=0, atol=1e-13)
    assert abs((vel ** 2).mean() / T - 1.0) < 4 * np.sqrt(2.0 / (3 * n))


def test_andersen_draws_have_variance_t_over_m():
    """Every atom redrawn from the heat bath at mass 2 (equipartition): each
    velocity component has mean 0 and variance T/m."""
    c = configs.lj_solid(n_cells=6)
    n = len(c["pos"])
    T, m = 0.7, 2.0
    _, vel, _, _, _, _, ncoll = oracle.md_run_otf(c["pos"], c["vel"], c["box"], 2, r_list=2.8, rebuild_every=10,
                                                  mass=m, thermostat=(T, 1000.0, 99))
    assert ncoll == 2 * n
    k = 3 * n
    assert abs(vel.mean()) < 4 * np.sqrt(T / m / k)
    assert abs((vel ** 2).mean() / (T / m) - 1.0) < 4 * np.sqrt(2.0 / k)


def test_andersen_collision_rate():
    c = configs.lj_solid(n_cells=6)
    n, steps, nu, dt = len(c["pos"]), 20, 4.0, 0.005
    ncoll = oracle.md_run_otf(c["pos"], c["vel"], c["box"], steps, r_list=2.8, rebuild_every=10,
                              thermostat=(1.0, nu, 7))[6]
    p = nu * dt
    mean, sd = n * steps * p, np.sqrt(n * steps * p * (1 - p))
    assert abs(ncoll - mean) < 5 * sd


def test_otf_q_rows_of_a_crystal_at_rest(golden):
    """A perfect fcc crystal with zero velocities stays put (zero forces): every
    analysis row holds the paper's Q4, Q5, Q6 of fcc."""
    lat = make_lattice("fcc", (6, 6, 6), 0.8442)
    pos = lat.sites()
    vel = np.zeros_like(pos)
    *_, qrows, qlast, _ = oracle.md_run_otf(pos, vel, lat.box, 6, rc=2.5, r_list=2.8, rebuild_every=3,
                                            boa=(2, 1.5))
    tab = golden["Q_table"]["fcc"]
    for s in (1, 3, 5):
        assert np.allclose(qrows[s], [tab["Q4"], tab["Q5"], tab["Q6"]], atol=5e-4)
    assert (qrows[[0, 2, 4]] == 0).all()
    assert np.allclose(qlast.mean(1), qrows[5], rtol=1e-13, atol=1e-15)


def test_otf_q_rows_of_hcp_at_rest(golden):
    """hcp at rest (every site is a mirror of itself across the basal plane
    and has a threefold axis along c, so it feels no force): the analysis
    rows hold the paper's Q4, Q5, Q6 of hcp, whose Q5 is not zero."""
    lat = make_lattice("hcp", (6, 4, 4), 0.8442)
    pos = lat.sites()
    *_, qrows, qlast, _ = oracle.md_run_otf(pos, np.zeros_like(pos), lat.box, 4, rc=2.5, r_list=2.8,
                                            rebuild_every=2, boa=(1, 1.5))
    tab = golden["Q_table"]["hcp"]
    assert tab["Q5"] > 0.2
    for s in range(4):
        assert np.allclose(qrows[s], [tab["Q4"], tab["Q5"], tab["Q6"]], atol=5e-4)


def test_md_run_same_on_any_thread_count():
    """The oracle's per-atom loops on several threads (the all-core CPU
    baseline) give the one-thread run bit for bit: every reduction over atoms
    is taken in atom order."""
    c = configs.lj_solid(n_cells=7)
    runs = []
    for k in (1, 3):
        oracle.set_threads(k)
        try:
            runs.append(oracle.md_run(c["pos"], c["vel"], c["box"], 12, r_list=2.8, rebuild_every=10))
        finally:
            oracle.set_threads(1)
    for a, b in zip(runs[0][:4], runs[1][:4]):
        assert np.array_equal(a, b)
    assert runs[0][4] == runs[1][4]
