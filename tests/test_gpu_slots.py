"""GPU tests of the brick-staged FP32 pair-loop mechanism of the integrator
(PPMD_PAIR_BRICKS: lists of stage slots, pair loop reading its neighbours
from shared memory), against the oracle and against the default
atom-index mechanism.

- the list of every build holds exactly the oracle's neighbour sets (bit
  for bit), in the same order as the atom-index list of the FP64 path;
- the FP32 trajectory, forces and velocities equal those of the
  atom-index FP32 path bit for bit (same pairs, same order, same arithmetic);
- a region twice as dense as the box average outgrows the planned stage:
  set-up grows it, and lists and forces stay exact;
- switching on the on-the-fly analysis in the middle of a list period
  converts the slot list to atom indices (same entries) and the run goes on
  matching the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
from synth import configs
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


def force_err(F, Fo):
    rms = np.sqrt((Fo ** 2).sum(1).mean())
    return np.sqrt(((F - Fo) ** 2).sum(1)).max() / rms


def _dense_half():
    """Atoms at density ~1 in the half x < 12 of a 24^3 box, none in the
    other half (random sequential addition, 0.8 minimum distance)."""
    pos, _ = random_box(6912, [12.0, 24.0, 24.0], 11, cutoffs=(2.5, 2.8), margin=1e-6, min_dist=0.8)
    box = np.array([24.0, 24.0, 24.0])
    # the margin filter above saw a box periodic at 12 in x: drop pairs that
    # sit near a cutoff across x = 0 / 12 of the larger box
    keep = np.ones(len(pos), bool)
    for i in range(len(pos)):
        if not keep[i]:
            continue
        d = pos - pos[i]
        d -= box * np.rint(d / box)
        r = np.sqrt((d ** 2).sum(1))
        near = ((np.abs(r - 2.5) < 1e-6) | (np.abs(r - 2.8) < 1e-6)) & keep
        near[i] = False
        keep[np.nonzero(near)[0]] = False
    return pos[keep], box


CASES = {
    "fcc10": lambda: (configs.lj_solid(n_cells=10), 2.8, 10),
    "sc10_every_step": lambda: (configs.lj_small(), 2.5, 1),
    "random_ragged": lambda: (dict(zip(("pos", "box"), random_box(997, [12.1, 11.3, 13.7], 3, cutoffs=(2.5, 2.8),
                                                                   margin=1e-6, min_dist=1.0))), 2.8, 10),
    "dense_half": lambda: (dict(zip(("pos", "box"), _dense_half())), 2.8, 10),
}


def _make(L, ctx, pos, box, r_list, every, prec, bricks=True):
    n = len(pos)
    md = L.MD(ctx, [0, n], [box], r_list=r_list, rc=2.5, rebuild_every=every, max_nbr=128, prec=prec)
    if bricks and prec == L.FP32:
        md.set_pair_loop(L.PAIR_BRICKS)
    md.set_state(cu(pos), cu(np.zeros((n, 3))))
    return md


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("bricks", [True, False])
def test_slot_list_sets_and_forces(L, ctx, case, bricks):
    """Both mechanisms' list builds hold exactly the oracle's sets."""
    c, r_list, every = CASES[case]()
    pos, box = oracle.wrap(c["pos"], c["box"]), np.asarray(c["box"], float)
    md = _make(L, ctx, pos, box, r_list, every, L.FP32, bricks=bricks)
    nbr, cnt = md.get_list()
    F = torch.empty((len(pos), 3), dtype=torch.float64, device="cuda")
    md.get_state(None, None, F)
    ctx.sync()
    offs, nb_o = oracle.neighbours_cells(pos, box, r_list)
    cnt = cnt.cpu().numpy()
    nbr = nbr.cpu().numpy()
    assert np.array_equal(cnt, np.diff(offs))
    for i in range(len(pos)):
        assert np.array_equal(np.sort(nbr[i, :cnt[i]]), nb_o[offs[i]:offs[i + 1]]), i
    Fo = oracle.lj(pos, box, offs, nb_o)[0]
    assert force_err(F.cpu().numpy(), Fo) <= 1e-5
    md.close()


@pytest.mark.parametrize("case", ["fcc10", "random_ragged"])
def test_slot_list_order_equals_atom_index_list(L, ctx, case):
    c, r_list, every = CASES[case]()
    a = _make(L, ctx, c["pos"], c["box"], r_list, every, L.FP32)
    b = _make(L, ctx, c["pos"], c["box"], r_list, every, L.FP64)
    na, ca = a.get_list()
    nb, cb = b.get_list()
    ctx.sync()
    assert torch.equal(ca, cb) and torch.equal(na, nb)
    a.close()
    b.close()


def _run(L, ctx, c, slots, nsteps, use_graph=True):
    n = len(c["pos"])
    md = L.MD(ctx, [0, n], [c["box"]], r_list=2.8, rc=2.5, rebuild_every=10, max_nbr=128, prec=L.FP32)
    md.set_pair_loop(L.PAIR_BRICKS if slots else L.PAIR_COLUMNS)
    md.set_state(cu(c["pos"]), cu(c["vel"]))
    md.run(nsteps, use_graph=use_graph)
    out = [torch.empty((n, 3), dtype=torch.float64, device="cuda") for _ in range(3)]
    md.get_state(*out)
    md.close()
    return [o.cpu().numpy() for o in out]


@pytest.mark.parametrize("use_graph", [True, False])
def test_slot_path_bit_identical_to_atom_index_path(L, ctx, use_graph):
    """23 steps (two rebuilds, fused kick/drift inside the run) of the fcc
    solid: positions, velocities and forces equal bit for bit."""
    c = configs.lj_solid(n_cells=9)
    a = _run(L, ctx, c, True, 23, use_graph)
    b = _run(L, ctx, c, False, 23, use_graph)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_set_boa_mid_period_converts_the_list(L, ctx):
    """Five plain steps on the slot path, then Q4/Q5/Q6 on every step: the
    list of step 0 (still in use until step 10) is converted to atom indices;
    positions and the Q rows of steps 6-15 match the oracle's run with the
    analysis on from the start (the analysis does not change the dynamics)."""
    c = configs.lj_solid(n_cells=8)
    n = len(c["pos"])
    po, vo, Fo, eno, qo, qlo, _ = oracle.md_run_otf(c["pos"], c["vel"], c["box"], 15, r_list=2.8, rebuild_every=10,
                                                    boa=(1, 1.5))
    md = L.MD(ctx, [0, n], [c["box"]], r_list=2.8, rc=2.5, rebuild_every=10, max_nbr=128, prec=L.FP32)
    md.set_pair_loop(L.PAIR_BRICKS)
    md.set_state(cu(c["pos"]), cu(c["vel"]))
    md.run(5)
    md.set_boa(1, 1.5)
    q = torch.zeros((10, 3), dtype=torch.float64, device="cuda")
    md.run_analysed(10, None, q)
    p = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    md.get_state(p)
    ql = md.get_q().cpu().numpy()
    md.close()
    d = p.cpu().numpy() - po
    d -= c["box"] * np.rint(d / c["box"])
    assert np.abs(d).max() <= 1e-8 * c["box"][0]
    assert np.abs(q.cpu().numpy() - qo[5:15]).max() <= 1e-5
    assert np.abs(ql - qlo).max() <= 1e-5


def test_pair_loop_mechanism_is_chosen_before_set_state(L, ctx):
    c = configs.lj_solid(n_cells=6)
    n = len(c["pos"])
    md = L.MD(ctx, [0, n], [c["box"]], r_list=2.8, rc=2.5, rebuild_every=10, max_nbr=128, prec=L.FP64)
    with pytest.raises(L.PPMDError):  # bricks need FP32
        md.set_pair_loop(L.PAIR_BRICKS)
    md.close()
    md = L.MD(ctx, [0, n], [c["box"]], r_list=2.8, rc=2.5, rebuild_every=10, max_nbr=128, prec=L.FP32)
    md.set_state(cu(c["pos"]), cu(c["vel"]))
    with pytest.raises(L.PPMDError):
        md.set_pair_loop(L.PAIR_BRICKS)
    md.close()


def test_pair_loop_event_times(L, ctx):
    """The measurement aid: event-record nodes around the pair loops of the
    run's last replayed unit give positive durations: per 10-step unit, nine
    pair loops fused with the next step's kick and drift and one other (the
    unit's last step, here also the energy step).  The graph with the events
    and the one without give the same trajectory bit for bit."""
    c = configs.lj_solid(n_cells=10)
    n = len(c["pos"])

    def run(timed, steps):
        md = L.MD(ctx, [0, n], [c["box"]], r_list=2.8, rc=2.5, rebuild_every=10, max_nbr=128, prec=L.FP32,
                  energy_every=10)
        if timed:
            md.time_pair_loops(True)
        md.set_state(cu(c["pos"]), cu(c["vel"]))
        md.run(steps)
        times = md.pair_loop_times() if timed else None
        out = [torch.empty((n, 3), dtype=torch.float64, device="cuda") for _ in range(3)]
        md.get_state(*out)
        md.close()
        return times, [x.cpu().numpy() for x in out]

    (tf, nf, to, no), timed = run(True, 30)
    assert nf == 9 and no == 1 and tf > 0 and to > 0, (tf, nf, to, no)
    _, plain = run(False, 30)
    for a, b in zip(timed, plain):
        assert np.array_equal(a, b)
