"""GPU tests of the integrator's launch shapes (ppmd_md_set_shape) and their
tuning (ppmd_md_tune) on batched replicas.

- every shape (pair-loop block size, one thread per atom or a persistent
  grid, list-build brick size) gives the default shape's list, positions,
  velocities and forces bit for bit over 23 steps (graph replays and single
  steps), and the run matches the oracle's forces; the energies agree to
  rounding (the per-block sums are grouped by the shape);
- tuning times the shapes, keeps one, restarts from the state it was given
  (the tuned run equals an untuned run bit for bit), writes the cache, and a
  second tuning of the same workload reads the cache without timing; another
  workload does not match the entry;
- shapes other than the default are refused for FP64 runs.
"""
import numpy as np
import pytest
import torch

import oracle
from synth import configs

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


@pytest.fixture(scope="module")
def reps():
    """Twelve replicas of 500 to 8000 atoms (the batched-replica generator)."""
    return configs.replicas(seed=9, nrep=12, n_min=500, n_max=8000)


def _md(L, ctx, reps, prec=None):
    off = np.cumsum([0] + [len(r["pos"]) for r in reps])
    md = L.MD(ctx, off, [r["box"] for r in reps], r_list=2.8, rc=2.5, rebuild_every=10, max_nbr=160,
              prec=L.FP32 if prec is None else prec, energy_every=10, box_r_list=[r["r_list"] for r in reps])
    return md, off


def _state(reps):
    return cu(np.concatenate([r["pos"] for r in reps])), cu(np.concatenate([r["vel"] for r in reps]))


def _run(L, ctx, reps, shape, steps=23):
    md, off = _md(L, ctx, reps)
    md.set_shape(shape)
    p, v = _state(reps)
    md.set_state(p, v)
    nbr, cnt = md.get_list()
    md.run(steps)
    out = [torch.empty((off[-1], 3), dtype=torch.float64, device="cuda") for _ in range(3)]
    md.get_state(*out)
    info = md.get_shape()
    md.close()
    return [x.cpu().numpy() for x in out] + [nbr.cpu().numpy(), cnt.cpu().numpy()], info


def test_every_shape_gives_the_same_trajectory(L, ctx, reps):
    ref, info0 = _run(L, ctx, reps, 0)
    assert info0 == dict(shape=0, block=128, per_sm=0, brick_home=128)
    for k in range(1, L.MD_SHAPES):
        got, info = _run(L, ctx, reps, k)
        assert info["shape"] == k
        for a, b in zip(ref, got):
            assert np.array_equal(a, b), k
    # the run itself against the oracle: forces of three boxes after 23 steps
    P, _, F = ref[0], ref[1], ref[2]
    off = np.cumsum([0] + [len(r["pos"]) for r in reps])
    for k in (0, 5, 11):
        r, lo, hi = reps[k], off[k], off[k + 1]
        offs, nb = oracle.neighbours_cells(P[lo:hi], r["box"], r["r_list"])
        Fo = oracle.lj(P[lo:hi], r["box"], offs, nb)[0]
        rms = np.sqrt((Fo ** 2).sum(1).mean())
        assert np.sqrt(((F[lo:hi] - Fo) ** 2).sum(1)).max() / rms <= 1e-5, k


def test_energies_agree_across_shapes(L, ctx, reps):
    """Kinetic and potential energy of every 10th step: the shapes group the
    per-block sums differently, so the totals agree to rounding (relative
    1e-12), not bit for bit."""
    out = []
    for k in (0, 1, 2, 3):
        md, off = _md(L, ctx, reps)
        md.set_shape(k)
        md.set_state(*_state(reps))
        e = torch.zeros((30, 2), dtype=torch.float64, device="cuda")
        md.run(30, e)
        md.close()
        out.append(e.cpu().numpy())
    rows = np.arange(9, 30, 10)  # the energy steps
    for e in out[1:]:
        assert np.abs(e[rows] - out[0][rows]).max() <= 1e-12 * np.abs(out[0][rows]).max()
    assert np.abs(out[0][rows]).min() > 0


def test_tune_restarts_from_the_state_and_caches(L, ctx, reps, tmp_path):
    cache = str(tmp_path / "shapes.txt")
    ref, _ = _run(L, ctx, reps, 0)
    md, off = _md(L, ctx, reps)
    p, v = _state(reps)
    md.set_state(p, v)
    t = md.tune(steps=10, cache=cache)
    assert t["timed"] and 0 <= t["shape"] < L.MD_SHAPES
    assert all(x > 0 for x in t["ms_per_step"])
    assert t["ms_per_step"][t["shape"]] == min(t["ms_per_step"])
    md.run(23)
    out = [torch.empty((off[-1], 3), dtype=torch.float64, device="cuda") for _ in range(3)]
    md.get_state(*out)
    md.close()
    for a, b in zip(ref[:3], out):
        assert np.array_equal(a, b.cpu().numpy())
    lines = open(cache).read().splitlines()
    assert len(lines) == 1 and lines[0].split("\t")[1] == str(t["shape"])
    # the same workload: the cached shape, nothing timed
    md, _ = _md(L, ctx, reps)
    md.set_state(*_state(reps))
    t2 = md.tune(steps=10, cache=cache)
    md.close()
    assert not t2["timed"] and t2["shape"] == t["shape"] and all(x == -1 for x in t2["ms_per_step"])
    # another workload (fewer boxes) does not match the entry
    md, _ = _md(L, ctx, reps[:6])
    md.set_state(*_state(reps[:6]))
    t3 = md.tune(steps=10, cache=cache)
    md.close()
    assert t3["timed"]
    assert len(open(cache).read().splitlines()) == 2


def test_shapes_are_refused_for_fp64(L, ctx, reps):
    md, _ = _md(L, ctx, reps[:3], prec=L.FP64)
    with pytest.raises(L.PPMDError):
        md.set_shape(2)
    md.set_shape(0)
    md.set_state(*_state(reps[:3]))
    t = md.tune(steps=10)
    assert not t["timed"] and t["shape"] == 0
    md.close()
